"""Brute-force, cell-by-cell checker for the oracle (tiny inputs only).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, never by the product path.

It enumerates every cell of the weighted cubical complex of an image (vertex
construction, Section 5; or top-dimensional construction, Section 4.1) and evaluates
the transforms from their definitions
(Section 2.2) via the per-cell formulas of Lemma 2.1 with the signs restored:

* ECT(xi, t)  = sum_P (-1)^dim P phi(P) [max_P xi <= t]
* R(xi, t)    = sum_P phi(P) c_P(t),  c_P = (-1)^dim P if P lies in {xi = t},
                (-1)^(dim P - 1) if min_P xi < t < max_P xi, 0 otherwise
* int kappa R = sum_{dim P >= 1} (-1)^(dim P - 1) phi(P) (kbar(max_P xi) - kbar(min_P xi))

(Lemma 2.1 as printed drops the (-1)^dim factors and takes min_P for the ECT; the
versions above follow from chi of the relative interiors, Appendix B.)

It also evaluates Delta^-(xi, x) straight from its definition in Section 3 -- the
Euler characteristic of the cells of the star of x whose maximum of xi is reached
at x -- for a concrete generic xi, without the box formula the oracle uses.
"""
from __future__ import annotations

from itertools import product

import numpy as np



def cells(img: np.ndarray):
    """All cells of the complex: list of (dim, phi, vertex linear indices)."""
    img = np.asarray(img).astype(np.int64)
    n = img.ndim
    m = tuple(reversed(img.shape))            # m_0 fastest
    strides = [1]
    for k in range(1, n):
        strides.append(strides[-1] * m[k - 1])
    flat = img.reshape(-1)
    out = []
    for base in product(*[range(mk) for mk in m]):      # base[k] = i_k
        for S in product((0, 1), repeat=n):
            if any(base[k] + S[k] >= m[k] for k in range(n)):
                continue
            verts = []
            for g in product((0, 1), repeat=n):
                if any(g[k] > S[k] for k in range(n)):
                    continue
                verts.append(sum((base[k] + g[k]) * strides[k] for k in range(n)))
            verts = np.array(verts, dtype=np.int64)
            out.append((sum(S), int(flat[verts].min()), verts))
    return out


def cells_top(img: np.ndarray):
    """All cells of the top-dimensional construction (Section 4.1): every face of every
    pixel, valued by the minimum over the pixels containing it; vertices are indices of
    the (m_k + 1)^n grid of pixel corners.  List of (dim, phi, vertex linear indices)."""
    img = np.asarray(img).astype(np.int64)
    n = img.ndim
    m = tuple(reversed(img.shape))            # pixels per paper axis, m_0 fastest
    mv = tuple(mk + 1 for mk in m)
    strides = [1]
    for k in range(1, n):
        strides.append(strides[-1] * mv[k - 1])
    flat = img.reshape(-1)
    pstrides = [1]
    for k in range(1, n):
        pstrides.append(pstrides[-1] * m[k - 1])
    value = {}
    for p in product(*[range(mk) for mk in m]):
        phi = int(flat[sum(p[k] * pstrides[k] for k in range(n))])
        for S in product((0, 1), repeat=n):
            for b in product((0, 1), repeat=n):
                if any(S[k] and b[k] for k in range(n)):
                    continue
                key = (tuple(p[k] + b[k] for k in range(n)), S)
                value[key] = min(value.get(key, phi), phi)
    out = []
    for (base, S), phi in value.items():
        verts = []
        for g in product((0, 1), repeat=n):
            if any(g[k] > S[k] for k in range(n)):
                continue
            verts.append(sum((base[k] + g[k]) * strides[k] for k in range(n)))
        out.append((sum(S), phi, np.array(verts, dtype=np.int64)))
    return out


def _complex(img, construction):
    """(cells, numpy shape of the vertex grid) of a construction."""
    img = np.asarray(img)
    if construction == "vertex":
        return cells(img), img.shape
    if construction == "top":
        return cells_top(img), tuple(s + 1 for s in img.shape)
    raise ValueError("construction must be 'vertex' or 'top'")


def _axis_coords(m: int) -> np.ndarray:
    """The checker's own copy of the embedding of Section 4.1: m evenly spaced points
    normalised to [-0.5, 0.5], point i at (2i - (m-1)) / (2(m-1)), each one IEEE division of
    two exact integers (so it rounds exactly as any other correct evaluation does)."""
    den = float(2 * (m - 1))
    return np.array([float(2 * i - (m - 1)) / den for i in range(m)], dtype=np.float64)


def vertex_dots(img: np.ndarray, xi, shape=None) -> np.ndarray:
    """<xi, x(v)> for every vertex, in linear order, canonical rounding.  The vertex grid
    has the numpy shape ``shape`` (default: the image's own, vertex construction)."""
    img = np.asarray(img)
    n = img.ndim
    m = tuple(reversed(shape if shape is not None else img.shape))
    N = int(np.prod(m))
    idx = np.arange(N, dtype=np.int64)
    s = None
    rest = idx.copy()
    for k in range(n):
        ik = rest % m[k]
        rest //= m[k]
        p = np.float64(xi[k]) * _axis_coords(m[k])[ik]
        s = p if s is None else s + p
    return s


def ect_brute(img, xi, t, construction: str = "vertex") -> np.ndarray:
    cl, shape = _complex(img, construction)
    s = vertex_dots(img, xi, shape)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    out = np.zeros(t.shape, dtype=np.int64)
    for dim, phi, verts in cl:
        if phi == 0:
            continue
        hi = s[verts].max()
        sgn = -1 if dim % 2 else 1
        out += sgn * phi * (hi <= t).astype(np.int64)
    return out


def radon_brute(img, xi, t, construction: str = "vertex") -> np.ndarray:
    cl, shape = _complex(img, construction)
    s = vertex_dots(img, xi, shape)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    out = np.zeros(t.shape, dtype=np.int64)
    for dim, phi, verts in cl:
        if phi == 0:
            continue
        lo, hi = s[verts].min(), s[verts].max()
        inside = (lo == t) & (hi == t)
        across = (lo < t) & (t < hi)
        sgn = -1 if dim % 2 else 1          # (-1)^dim; (-1)^(dim-1) = -sgn
        out += phi * (sgn * inside.astype(np.int64) - sgn * across.astype(np.int64))
    return out


def integral_kappa_radon(img, xi, kbar) -> complex:
    """int kappa(t) R(xi, t) dt, summed cell by cell (kbar = primitive of kappa)."""
    s = vertex_dots(img, xi)
    total = 0.0
    for dim, phi, verts in cells(img):
        if phi == 0 or dim == 0:
            continue
        lo, hi = s[verts].min(), s[verts].max()
        sgn = 1 if dim % 2 else -1          # (-1)^(dim-1)
        total = total + sgn * phi * (kbar(hi) - kbar(lo))
    return total


def lower_star_brute(img, xi) -> np.ndarray:
    """Delta^-(xi, x) for every vertex x from the definition (Section 3).

    For each cell P containing x with max_P xi attained at x (and only there, xi
    being generic), add (-1)^dim P phi(P).
    """
    img = np.asarray(img)
    N = img.size
    s = vertex_dots(img, xi)
    out = np.zeros(N, dtype=np.int64)
    for dim, phi, verts in cells(img):
        top = verts[np.argmax(s[verts])]
        if np.count_nonzero(s[verts] == s[top]) != 1:
            raise ValueError("direction is not generic on this complex")
        out[top] += (-1 if dim % 2 else 1) * phi
    return out


def ht_by_quadrature(img, xi, kappa, order: int = 12, construction: str = "vertex") -> complex:
    """HT in the paper's sign convention, -int kappa(t) R(xi, t) dt, by quadrature.

    R(xi, .) is constant on the open intervals between consecutive distinct vertex
    dot products; its value there is taken from the cell-by-cell ECT through
    R(t) = ECT(xi, t) + ECT(-xi, -t) - chi, and kappa is integrated over each interval
    with an ``order``-point Gauss-Legendre rule.  Needs no primitive of kappa.
    """
    xi = np.asarray(xi, dtype=np.float64)
    shape = _complex(img, construction)[1]
    s = np.unique(vertex_dots(img, xi, shape))
    if len(s) < 2:
        return 0.0
    mids = 0.5 * (s[:-1] + s[1:])
    chi = int(ect_brute(img, xi, np.array([np.inf]), construction)[0])
    R = ect_brute(img, xi, mids, construction) + ect_brute(img, -xi, -mids, construction) - chi
    nodes, weights = np.polynomial.legendre.leggauss(order)
    total = 0.0
    for lo, hi, r in zip(s[:-1], s[1:], R):
        if r == 0:
            continue
        half = 0.5 * (hi - lo)
        tq = lo + half * (nodes + 1.0)
        total = total + r * half * np.sum(weights * kappa(tq))
    return -total
