"""CPU oracle for topological integral transforms on weighted cubical complexes.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously-correct FP64 /
int64 statement of what the GPU path computes.  Only the test-suite, the smoke
check and the CPU-baseline leg of the benchmark may import it; the product path
never does.  It shares no code with the CUDA library.

Source: Lebovici, Oudot, Passe, "Efficient computation of topological integral
transforms" (SEA 2024, arXiv 2405.02256).  Every function cites the passage it
follows (section, lemma, equation or table of the paper).

Conventions (each one a reading of the paper where it is silent or ambiguous):

* An image with n axes is a numpy array in C order; the paper's coordinate 0 is the
  FASTEST memory axis (numpy's last axis).  Appendix A's cell keys show that the
  first coordinate is ``key mod width`` (the fast axis).
* Vertex construction ("dual construction", Section 5): every pixel is a vertex with
  the pixel's value; a k-cube exists iff all of its 2^k vertices are pixels and its
  value is the minimum of its vertices' values.
* Embedding (Section 4.1): per axis, vertices are evenly spaced in [-0.5, 0.5]:
  x_k(i) = (2 i - (m_k - 1)) / (2 (m_k - 1)), one correctly rounded FP64 division.
* Orthant o in [0, 2^n): bit k set <=> eps_k = -1.  The sign vector of a direction
  is eps_k = +1 if xi_k >= 0 else -1 (Section 3 defines it for non-zero coordinates;
  a zero coordinate takes +1, and -0.0 counts as zero).
* Canonical dot product: s = fl(fl(fl(xi_0 x_0) + fl(xi_1 x_1)) + fl(xi_2 x_2)),
  left to right, every product and sum rounded separately (numpy never fuses).
* Thresholds (Appendix A.4 vectorisation): t_j = fl(a + fl(fl(j * fl(b - a)) / (T - 1))).
* Delta^-_eps(v) is the classical critical value (Section 3).  The table of
  "ordinary" values is kept as Delta_eps := Delta^-_eps - Delta^-_{-eps}, which is
  -Delta^ord_eps of Section 3 (Delta^ord = chi(UpSt) - chi(LwSt) and UpSt(eps) =
  LwSt(-eps) on a cubical complex).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from itertools import product

import numpy as np

__all__ = [
    "vertex_coords", "orthant_of", "partner", "lower_star_values", "lower_star_values_top", "delta_values",
    "CriticalTables", "critical_tables", "euler_characteristic", "thresholds",
    "dot_products", "vertex_positions", "ect_exact", "ect_eval", "ect_values",
    "radon_values", "radon_exact", "radon_exact_eval", "ect_grid", "radon_grid",
    "radon_grid_lemma", "KERNELS", "table_kernel", "hybrid_transform", "hybrid_transform_grad",
]


# ---------------------------------------------------------------------------
# Complex, embedding and sign vectors (Sections 2.1, 3, 4.1, 5)
# ---------------------------------------------------------------------------

def vertex_coords(m: int) -> np.ndarray:
    """Embedding coordinates of the m vertices along one axis (Section 4.1).

    Evenly spaced and normalised to [-0.5, 0.5]: x(i) = (2i - (m-1)) / (2(m-1)).
    Both operands are exact integers in FP64, so the result is one correctly
    rounded division and x(m-1-i) == -x(i) exactly.
    """
    if m < 2:
        raise ValueError("every axis needs at least two vertices")
    i = np.arange(m, dtype=np.float64)
    return (2.0 * i - float(m - 1)) / float(2 * (m - 1))


def orthant_of(xi) -> int:
    """Orthant index of the sign vector eps^xi (Section 3, before Lemma 3.2).

    Bit k is set iff eps_k = -1, i.e. iff xi_k < 0.  A zero coordinate (also -0.0)
    gets eps_k = +1.
    """
    o = 0
    for k, c in enumerate(xi):
        if float(c) < 0.0:
            o |= 1 << k
    return o


def partner(o: int, n: int) -> int:
    """Orthant of -eps: every sign flipped."""
    return o ^ ((1 << n) - 1)


def _axis(n: int, k: int) -> int:
    """numpy axis holding the paper's coordinate k (coordinate 0 = last numpy axis)."""
    return n - 1 - k


def _shifted(img: np.ndarray, off) -> tuple[np.ndarray, np.ndarray]:
    """Return (vals, inside) with vals[v] = img[v + off] where v + off is a pixel.

    ``off`` is indexed by the paper's coordinates.  ``inside`` marks the vertices
    for which v + off lies in the image.
    """
    n = img.ndim
    vals = np.zeros_like(img)
    inside = np.zeros(img.shape, dtype=bool)
    dst = [slice(None)] * n
    src = [slice(None)] * n
    for k in range(n):
        ax = _axis(n, k)
        m = img.shape[ax]
        o = int(off[k])
        if abs(o) >= m:
            return vals, inside
        if o >= 0:
            dst[ax] = slice(0, m - o)
            src[ax] = slice(o, m)
        else:
            dst[ax] = slice(-o, m)
            src[ax] = slice(0, m + o)
    vals[tuple(dst)] = img[tuple(src)]
    inside[tuple(dst)] = True
    return vals, inside


# ---------------------------------------------------------------------------
# Critical values (Section 3, definition of Delta^-; Section 4.2 preprocessing)
# ---------------------------------------------------------------------------

def lower_star_values(img: np.ndarray) -> np.ndarray:
    """Delta^-_eps(v) = chi(phi restricted to LwSt(eps, v)) for every orthant and vertex.

    Section 3 defines Delta^-(xi, x) as the Euler characteristic sum_P (-1)^dim P phi(P)
    over the lower star of x.  On an axis-aligned cubical complex, for a direction with
    sign vector eps, the cubes containing v whose maximum of xi is reached at v are
    exactly the boxes spanned by v and v - delta (.) eps for delta in {0,1}^n (the
    hand trace of Appendix A.1 enumerates the same cells "c - delta (.) eps").  Such a
    box has dimension |delta|, exists iff its far corner v - delta (.) eps is a pixel,
    and (vertex construction, Section 5) has value min over its 2^|delta| vertices.

    Returns an int64 array of shape (2^n,) + img.shape; entry [o] holds orthant o.
    """
    img = np.asarray(img)
    n = img.ndim
    base = img.astype(np.int64)
    out = np.zeros((1 << n,) + img.shape, dtype=np.int64)
    for o in range(1 << n):
        eps = [(-1 if (o >> k) & 1 else 1) for k in range(n)]
        acc = np.zeros(img.shape, dtype=np.int64)
        for delta in product((0, 1), repeat=n):
            far = [-delta[k] * eps[k] for k in range(n)]
            _, exists = _shifted(base, far)
            # value of the box = min over its vertices v - gamma (.) eps, gamma <= delta
            cell_min = None
            for gamma in product((0, 1), repeat=n):
                if any(g > d for g, d in zip(gamma, delta)):
                    continue
                vals, _ = _shifted(base, [-gamma[k] * eps[k] for k in range(n)])
                cell_min = vals if cell_min is None else np.minimum(cell_min, vals)
            sign = -1 if (sum(delta) % 2) else 1
            acc += sign * np.where(exists, cell_min, 0)
        out[o] = acc
    return out


def lower_star_values_top(img: np.ndarray) -> np.ndarray:
    """Delta^-_eps(v) for the top-dimensional construction (Section 4.1).

    One top-dimensional cell per pixel; every lower-dimensional cell takes the minimum
    of the values of its cofaces, i.e. of the pixels that contain it.  The vertices are
    the corners of the pixel grid, (m_k + 1) per axis.  For the sign vector eps the
    lower star of a corner v is made of the boxes spanned by v and v - delta (.) eps,
    delta in {0,1}^n, as in the vertex construction.  A box lies in the pixels p with
    p_k = v_k - 1 (eps_k = +1) or p_k = v_k (eps_k = -1) on the axes where delta_k = 1,
    and p_k in {v_k - 1, v_k} on the others; it exists iff one of those is a pixel, and
    its value is the minimum over them.

    Returns an int64 array of shape (2^n,) + (img.shape + 1); entry [o] holds orthant o.
    """
    img = np.asarray(img).astype(np.int64)
    n = img.ndim
    shape_v = tuple(s + 1 for s in img.shape)
    big = np.iinfo(np.int64).max // 4
    # padded[v + g] = pixel v + g - 1 (numpy axes), g in {0,1}^n
    padded = np.full(tuple(s + 2 for s in img.shape), big, dtype=np.int64)
    present = np.zeros(padded.shape, dtype=bool)
    inner = tuple(slice(1, s + 1) for s in img.shape)
    padded[inner] = img
    present[inner] = True
    out = np.zeros((1 << n,) + shape_v, dtype=np.int64)
    for o in range(1 << n):
        eps = [(-1 if (o >> k) & 1 else 1) for k in range(n)]     # paper coordinate k
        acc = np.zeros(shape_v, dtype=np.int64)
        for delta in product((0, 1), repeat=n):
            cell_min, cell_exists = None, None
            for g in product((0, 1), repeat=n):
                # on a spanned axis only the pixel on the side of v - eps contains the box
                if any(delta[k] and g[k] != (0 if eps[k] == 1 else 1) for k in range(n)):
                    continue
                sl = tuple(slice(g[n - 1 - ax], g[n - 1 - ax] + shape_v[ax]) for ax in range(n))
                vals, here = padded[sl], present[sl]
                cell_min = vals if cell_min is None else np.minimum(cell_min, vals)
                cell_exists = here if cell_exists is None else (cell_exists | here)
            sign = -1 if (sum(delta) % 2) else 1
            acc += sign * np.where(cell_exists, cell_min, 0)
        out[o] = acc
    return out


def delta_values(lower: np.ndarray) -> np.ndarray:
    """Delta_eps = Delta^-_eps - Delta^-_{-eps} for the representative orthants.

    Section 3: Delta^ord(xi, x) = chi(UpSt) - chi(LwSt).  The upper star for eps is the
    lower star for -eps, so Delta^ord_eps = Delta^-_{-eps} - Delta^-_eps = -Delta_eps.
    Representatives are the orthants with bit n-1 clear (o < 2^(n-1)); the partner
    table is the negation.  Returns int64 of shape (2^(n-1),) + image shape.
    """
    n = lower.ndim - 1
    half = 1 << (n - 1)
    return np.stack([lower[o] - lower[partner(o, n)] for o in range(half)])


@dataclass
class CriticalTables:
    """Critical-point tables of one image (Section 4.2: a pair of arrays per eps).

    ``lower_idx[o]``/``lower_val[o]``: vertices with Delta^-_o != 0, ascending linear
    vertex index (C order, coordinate 0 fastest), and their values.
    ``delta_idx[r]``/``delta_val[r]``: same for Delta_r, r < 2^(n-1).
    """
    shape: tuple                      # numpy shape (m_{n-1}, ..., m_0)
    lower_idx: list = field(default_factory=list)
    lower_val: list = field(default_factory=list)
    delta_idx: list = field(default_factory=list)
    delta_val: list = field(default_factory=list)
    chi: int = 0

    @property
    def n(self) -> int:
        return len(self.shape)

    @property
    def m(self) -> tuple:
        """Axis lengths in the paper's coordinate order (m_0 fastest)."""
        return tuple(reversed(self.shape))


def critical_tables(img: np.ndarray, construction: str = "vertex") -> CriticalTables:
    """Preprocessing of critical points and values (Section 4.2).

    For every sign vector the non-zero classical values Delta^-_eps and the non-zero
    Delta_eps are stored as (points, values) arrays.  Points are linear vertex
    indices in ascending order.  construction = "vertex" (pixels are vertices, Section 5)
    or "top" (pixels are top-dimensional cells, Section 4.1; the vertices are the
    (m_k + 1)^n pixel corners and the tables' shape is img.shape + 1).
    """
    img = np.asarray(img)
    if construction == "vertex":
        low = lower_star_values(img)
    elif construction == "top":
        low = lower_star_values_top(img)
    else:
        raise ValueError("construction must be 'vertex' or 'top'")
    dl = delta_values(low)
    t = CriticalTables(shape=tuple(low.shape[1:]))
    for o in range(low.shape[0]):
        flat = low[o].reshape(-1)
        idx = np.flatnonzero(flat)
        t.lower_idx.append(idx.astype(np.int64))
        t.lower_val.append(flat[idx].astype(np.int64))
    for r in range(dl.shape[0]):
        flat = dl[r].reshape(-1)
        idx = np.flatnonzero(flat)
        t.delta_idx.append(idx.astype(np.int64))
        t.delta_val.append(flat[idx].astype(np.int64))
    # Lemma 3.1 at t = +inf: ECT(xi, +inf) = chi(phi) = sum of Delta^- for any eps.
    t.chi = int(low[0].sum())
    return t


def euler_characteristic(img: np.ndarray) -> int:
    """chi(phi) = sum over cells of (-1)^dim phi(cell) (Section 2.1), cell by cell."""
    img = np.asarray(img).astype(np.int64)
    n = img.ndim
    total = 0
    # a cell = base vertex u + box spanned along the axes in S (toward +1)
    for S in product((0, 1), repeat=n):
        far = list(S)
        _, exists = _shifted(img, far)
        cell_min = None
        for gamma in product((0, 1), repeat=n):
            if any(g > s for g, s in zip(gamma, S)):
                continue
            vals, _ = _shifted(img, list(gamma))
            cell_min = vals if cell_min is None else np.minimum(cell_min, vals)
        sign = -1 if (sum(S) % 2) else 1
        total += sign * int(np.where(exists, cell_min, 0).sum())
    return total


# ---------------------------------------------------------------------------
# Directions, thresholds, dot products (Sections 3, 4.3; Appendix A.4)
# ---------------------------------------------------------------------------

def thresholds(a: float, b: float, T: int) -> np.ndarray:
    """Vectorisation grid of Appendix A.4: t_j = a + j (b - a) / (T - 1), j < T.

    Evaluated as fl(a + fl(fl(j * fl(b - a)) / (T - 1))).
    """
    if T < 2:
        raise ValueError("T must be at least 2")
    w = np.float64(b) - np.float64(a)
    j = np.arange(T, dtype=np.float64)
    return np.float64(a) + (j * w) / np.float64(T - 1)


def _vertex_multi_index(idx: np.ndarray, m: tuple) -> list:
    """Per-axis vertex indices (coordinate 0 fastest) of linear vertex indices."""
    rest = np.asarray(idx, dtype=np.int64)
    out = []
    for mk in m:
        out.append(rest % mk)
        rest = rest // mk
    return out


def dot_products(xi, idx: np.ndarray, m: tuple) -> np.ndarray:
    """<xi, x(v)> for the vertices ``idx`` of an image with axis lengths m (Section 3).

    Products are rounded one by one and summed left to right.
    """
    ii = _vertex_multi_index(idx, m)
    s = None
    for k, mk in enumerate(m):
        p = np.float64(xi[k]) * vertex_coords(mk)[ii[k]]
        s = p if s is None else s + p
    return s


def vertex_positions(idx: np.ndarray, m: tuple) -> np.ndarray:
    """Embedding x(v) of the vertices ``idx``: array [len(idx), n]."""
    ii = _vertex_multi_index(idx, m)
    return np.stack([vertex_coords(mk)[ii[k]] for k, mk in enumerate(m)], axis=1)


# ---------------------------------------------------------------------------
# ECT and Radon (Lemma 3.1, Section 4.3, Appendix A.2-A.4)
# ---------------------------------------------------------------------------

def ect_exact(tab: CriticalTables, xi):
    """Exact representation (T, E) of t -> ECT(xi, t) (Section 4.3, Appendix A.2).

    Dot products of the classical critical points of eps^xi, sorted ascending; E holds
    the cumulative sums of the sorted Delta^- with equal dot products merged.  The
    leading (-inf, 0) entry of the paper is kept implicit: ECT(xi, t) = 0 for t < T[0].
    """
    o = orthant_of(xi)
    s = dot_products(xi, tab.lower_idx[o], tab.m)
    order = np.argsort(s, kind="stable")
    s_sorted = s[order]
    v_sorted = tab.lower_val[o][order]
    Tv, first = np.unique(s_sorted, return_index=True)
    merged = np.add.reduceat(v_sorted, first) if len(first) else np.zeros(0, np.int64)
    E = np.cumsum(merged)
    return Tv, E


def ect_eval(Tv: np.ndarray, E: np.ndarray, t) -> np.ndarray:
    """ECT(xi, t) from (T, E) by binary search (Section 4.3, Appendix A.3).

    The value is E at the largest T <= t (closed sublevel set {xi <= t}), 0 if none.
    """
    t = np.asarray(t, dtype=np.float64)
    i = np.searchsorted(Tv, t, side="right")
    padded = np.concatenate([np.zeros(1, np.int64), E])
    return padded[i]


def ect_values(tab: CriticalTables, xi, t) -> np.ndarray:
    """ECT(xi, t) at arbitrary thresholds t (Lemma 3.1 through (T, E))."""
    Tv, E = ect_exact(tab, xi)
    return ect_eval(Tv, E, t)


def radon_values(tab: CriticalTables, xi, t) -> np.ndarray:
    """Radon transform R(xi, t) at arbitrary thresholds t.

    Additivity of the Euler integral (Appendix B, pushforward formulation) splits the
    level set {xi = t} as {xi <= t} + {xi >= t} - everything, so
    R(xi, t) = ECT(xi, t) + ECT(-xi, -t) - chi(phi).  Both ECT terms use Lemma 3.1
    through ect_exact; this holds for every xi, generic or not.
    """
    xi = np.asarray(xi, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    return ect_values(tab, xi, t) + ect_values(tab, -xi, -t) - tab.chi


def radon_exact(tab: CriticalTables, xi):
    """Exact representation (T', E') of the Radon transform between critical values
    (Section 4.3, Appendix A.2: the sorted "ordinary" critical values and the cumulative
    sums of their values).

    T' holds the distinct dot products of the points of the table Delta_eps, eps = eps^xi
    (for a sign vector outside the stored half, the partner's table with the sign
    flipped), ascending; E' the cumulative sums of Delta_eps with equal dot products
    merged.  For every t that is not a dot product of a critical point,
    R(xi, t) = E' at the largest T' < t (0 if none).  E' is the negative of the printed
    E' of Appendix A.2, whose values are Delta^ord = -Delta_eps.
    """
    n = tab.n
    half = 1 << (n - 1)
    o = orthant_of(xi)
    r, sg = (o, 1) if o < half else (partner(o, n), -1)
    s = dot_products(xi, tab.delta_idx[r], tab.m)
    order = np.argsort(s, kind="stable")
    s_sorted = s[order]
    v_sorted = sg * tab.delta_val[r][order]
    Tv, first = np.unique(s_sorted, return_index=True)
    merged = np.add.reduceat(v_sorted, first) if len(first) else np.zeros(0, np.int64)
    return Tv, np.cumsum(merged)


def radon_exact_eval(T_lw, E_lw, T_ord, E_ord, t) -> np.ndarray:
    """R(xi, t) at arbitrary t from the two exact representations (Appendix A.3).

    Splitting the level set as in radon_values, with sum_v Delta^-_{-eps}(v) = chi:
      R(xi, t) = sum_{s_v < t} Delta_eps(v) + sum_{s_v = t} Delta^-_eps(v),
    i.e. E' at the largest T' < t, plus the jump of E at t when t is one of the lower
    critical values T ((T, E) = ect_exact).
    """
    t = np.asarray(t, dtype=np.float64)
    i = np.searchsorted(T_ord, t, side="left")                 # number of T' < t
    below = np.concatenate([np.zeros(1, np.int64), np.asarray(E_ord, np.int64)])[i]
    T_lw = np.asarray(T_lw, dtype=np.float64)
    E0 = np.concatenate([np.zeros(1, np.int64), np.asarray(E_lw, np.int64)])   # E0[k] = E before T[k]
    k_le = np.searchsorted(T_lw, t, side="right")             # number of T <= t
    k_lt = np.searchsorted(T_lw, t, side="left")              # number of T < t
    jump = E0[k_le] - E0[k_lt]                                 # the jump at t, 0 if t is not in T
    return below + jump


def ect_grid(tab: CriticalTables, dirs, a: float, b: float, T: int) -> np.ndarray:
    """ECT(xi_d, t_j) on the vectorisation grid (Appendix A.4): int64 [D, T]."""
    t = thresholds(a, b, T)
    dirs = np.asarray(dirs, dtype=np.float64).reshape(-1, tab.n)
    return np.stack([ect_values(tab, xi, t) for xi in dirs]) if len(dirs) else \
        np.zeros((0, T), np.int64)


def radon_grid(tab: CriticalTables, dirs, a: float, b: float, T: int) -> np.ndarray:
    """R(xi_d, t_j) on the vectorisation grid: int64 [D, T]."""
    t = thresholds(a, b, T)
    dirs = np.asarray(dirs, dtype=np.float64).reshape(-1, tab.n)
    return np.stack([radon_values(tab, xi, t) for xi in dirs]) if len(dirs) else \
        np.zeros((0, T), np.int64)


def radon_grid_lemma(tab: CriticalTables, dirs, a: float, b: float, T: int) -> np.ndarray:
    """Radon transform through Lemma 3.1 directly, for GENERIC directions only.

    R(xi, .) = sum_{Crit^-} Delta^- 1_{<xi,x>} + sum_{Crit^ord} J(x) 1_{(<xi,x>, inf)}
    where J(x) is the jump R(t+) - R(t-) at x.  The proof of Lemma A.3 gives
    J = chi(LwSt) - chi(UpSt) = Delta_eps (the printed Delta^ord has the opposite
    sign; see the worked example, whose printed E' is the negation of the true one).
    Used as an independent cross-check of radon_grid.
    """
    t = thresholds(a, b, T)
    dirs = np.asarray(dirs, dtype=np.float64).reshape(-1, tab.n)
    n = tab.n
    half = 1 << (n - 1)
    out = np.zeros((dirs.shape[0], T), dtype=np.int64)
    for d, xi in enumerate(dirs):
        o = orthant_of(xi)
        r, sg = (o, 1) if o < half else (partner(o, n), -1)
        s_ord = dot_products(xi, tab.delta_idx[r], tab.m)
        j_ord = sg * tab.delta_val[r]
        s_low = dot_products(xi, tab.lower_idx[o], tab.m)
        for j, tj in enumerate(t):
            out[d, j] = int(j_ord[s_ord < tj].sum()) + int(tab.lower_val[o][s_low == tj].sum())
    return out


# ---------------------------------------------------------------------------
# Hybrid transforms (Lemma 3.1, Section 4.3) and their gradient
# ---------------------------------------------------------------------------

def _j0(x):
    from scipy.special import j0
    return j0(x)


def _j1(x):
    from scipy.special import j1
    return j1(x)


# kernel name -> (primitive kbar, kappa = kbar'), complex where needed.
#   Laplace: kbar(s) = e^s                     (Appendix A.2 uses kbar = exp)
#   Fourier: kbar(s) = sin s + i cos s          (kappa(t) = e^{-it})
#   Bessel:  kbar(s) = J0(s)                    (kappa = -J1)
KERNELS = {
    "laplace": (np.exp, np.exp),
    "fourier": (lambda s: np.sin(s) + 1j * np.cos(s), lambda s: np.cos(s) - 1j * np.sin(s)),
    "bessel": (_j0, lambda s: -_j1(s)),
    # kappa = sin, the kernel of the paper's experiments (Section 5): kbar = -cos
    "sine": (lambda s: -np.cos(s), np.sin),
}


def table_kernel(values, s_min: float, s_max: float):
    """A kernel given by samples of its primitive: (kbar, kappa) callables.

    Section 2.2 admits any locally integrable kernel kappa; Lemma 3.1 needs only its
    primitive kbar.  Here kbar is given by K >= 2 samples y_i = kbar(a + i h),
    h = (b - a) / (K - 1), i = 0 .. K - 1 (a = s_min < b = s_max), and is read as the
    piecewise-linear interpolant of the samples, constant outside [a, b]:
        u = (s - a) / h;  i = floor(u), f = u - i         (0 <= u < K - 1)
        kbar(s) = y_i + f (y_{i+1} - y_i);  y_0 for u < 0;  y_{K-1} for u >= K - 1.
    Its derivative kappa is the step function (y_{i+1} - y_i) / h on [a + i h,
    a + (i + 1) h) and zero outside [a, b) (the right derivative at the knots).
    """
    y = np.asarray(values, dtype=np.float64).ravel()
    K = y.size
    a, b = float(s_min), float(s_max)
    if K < 2 or not (a < b) or not np.all(np.isfinite(y)):
        raise ValueError("table kernel: need K >= 2 finite samples and s_min < s_max")
    h = (b - a) / (K - 1)

    def _seg(s):
        u = (np.asarray(s, dtype=np.float64) - a) / h
        inside = (u >= 0.0) & (u < K - 1)
        i = np.where(inside, np.floor(np.where(inside, u, 0.0)), 0.0).astype(np.int64)
        return u, inside, i

    def kbar(s):
        u, inside, i = _seg(s)
        f = u - i
        mid = y[i] + f * (y[i + 1] - y[i])
        return np.where(inside, mid, np.where(u < 0.0, y[0], y[K - 1]))

    def kappa(s):
        u, inside, i = _seg(s)
        return np.where(inside, (y[i + 1] - y[i]) / h, 0.0)

    return kbar, kappa


def _kernel_pair(kernel):
    return KERNELS[kernel] if isinstance(kernel, str) else kernel


def _ht_terms(tab: CriticalTables, xi):
    n = tab.n
    half = 1 << (n - 1)
    o = orthant_of(xi)
    r, sg = (o, 1) if o < half else (partner(o, n), -1)
    s = dot_products(xi, tab.delta_idx[r], tab.m)
    return r, s, sg * tab.delta_val[r]


def _fsum_complex(z: np.ndarray) -> complex:
    z = np.asarray(z)
    if np.iscomplexobj(z):
        return complex(math.fsum(z.real.tolist()), math.fsum(z.imag.tolist()))
    return math.fsum(z.tolist())


def hybrid_transform(tab: CriticalTables, kernel: str, dirs):
    """HT(xi) = -sum_{x in Crit^ord} Delta^ord(xi, x) kbar(<xi, x>) (Lemma 3.1).

    With Delta_eps = -Delta^ord_eps this is sum_v Delta_eps(v) kbar(<xi, v>); the
    sum is taken exactly (math.fsum) over the FP64 terms.  The primitive's constant
    drops out because sum_v Delta_eps(v) = 0.  ``kernel`` is a name of KERNELS or a
    real (kbar, kappa) pair such as table_kernel() returns.  Returns (values, norms): values is
    float64 [D] (complex128 for Fourier), norms[d] = sum_v |Delta kbar| (complex
    modulus for Fourier) -- the scale for relative errors.
    """
    kbar, _ = _kernel_pair(kernel)
    dirs = np.asarray(dirs, dtype=np.float64).reshape(-1, tab.n)
    cplx = isinstance(kernel, str) and kernel == "fourier"
    vals = np.zeros(dirs.shape[0], dtype=np.complex128 if cplx else np.float64)
    norms = np.zeros(dirs.shape[0], dtype=np.float64)
    for d, xi in enumerate(dirs):
        _, s, dv = _ht_terms(tab, xi)
        terms = dv.astype(np.float64) * kbar(s)
        vals[d] = _fsum_complex(terms)
        norms[d] = math.fsum(np.abs(terms).tolist())
    return vals, norms


def hybrid_transform_grad(tab: CriticalTables, kernel: str, dirs):
    """dHT/dxi = sum_v Delta_eps(v) kappa(<xi, v>) x(v), kappa = kbar'.

    Differentiates the closed form of Lemma 3.1 term by term; the critical sets do not
    move inside an orthant (Lemma 3.2).  Returns (grad, norms): grad is [D, n]
    (complex128 for Fourier: d Re / d xi + i d Im / d xi); norms[d, k] = sum |terms|.
    """
    _, kap = _kernel_pair(kernel)
    dirs = np.asarray(dirs, dtype=np.float64).reshape(-1, tab.n)
    n = tab.n
    cplx = isinstance(kernel, str) and kernel == "fourier"
    g = np.zeros((dirs.shape[0], n), dtype=np.complex128 if cplx else np.float64)
    norms = np.zeros((dirs.shape[0], n), dtype=np.float64)
    for d, xi in enumerate(dirs):
        r, s, dv = _ht_terms(tab, xi)
        pos = vertex_positions(tab.delta_idx[r], tab.m)
        base = dv.astype(np.float64) * kap(s)
        for k in range(n):
            terms = base * pos[:, k]
            g[d, k] = _fsum_complex(terms)
            norms[d, k] = math.fsum(np.abs(terms).tolist())
    return g, norms
