"""The CPU oracle against what the paper and the mathematics fix (no GPU).

Pins: the worked example of Appendix A (tests/golden/worked_example.json), the
definitions evaluated cell by cell on tiny complexes (oracle/brute.py), closed forms
for a contractible image, invariants of Lemma 3.1 / Lemma 3.2, Gauss-Legendre
quadrature of -int kappa R for the hybrid transforms, and central finite
differences for the gradient.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import brute as B
from paper_2405_02256_gb300 import synth


def _key(v, m0=4):
    # worked example: vertex (i0, i1) has cell key 2 i0 + 14 i1 on the 7x7 grid
    return 2 * (v % m0) + 14 * (v // m0)


def _orthant(eps):
    return sum(1 << k for k, e in enumerate(eps) if e == -1)


# ---------------------------------------------------------------- worked example

def test_worked_example_tables(golden):
    img = np.array(golden["image"])
    tab = O.critical_tables(img)
    for row in golden["critical_table"]["rows"]:
        o = _orthant(row["eps"])
        got_lw = {(_key(v), int(x)) for v, x in zip(tab.lower_idx[o], tab.lower_val[o])}
        assert got_lw == set(zip(row["lw_pts"], row["lw_vals"]))
        r, sg = (o, 1) if o < 2 else (O.partner(o, 2), -1)
        # printed Delta^ord = -Delta_eps
        got_ord = {(_key(v), -sg * int(x)) for v, x in zip(tab.delta_idx[r], tab.delta_val[r])}
        assert got_ord == set(zip(row["ord_pts"], row["ord_vals"]))
    assert tab.chi == 2 == O.euler_characteristic(img)


def test_worked_example_hand_trace(golden):
    img = np.array(golden["image"])
    tr = golden["hand_trace"]
    low = O.lower_star_values(img)
    o = _orthant(tr["eps"])
    v = [i for i in range(16) if _key(i) == tr["vertex_key"]][0]
    e_minus = int(low[o].reshape(-1)[v])
    e_plus = int(low[O.partner(o, 2)].reshape(-1)[v])
    assert (e_minus, e_plus) == (tr["e_minus"], tr["e_plus"])
    assert e_plus - e_minus == tr["ord_value"]


def test_worked_example_ect(golden):
    img = np.array(golden["image"])
    tab = O.critical_tables(img)
    g = golden["ect"]
    Tv, E = O.ect_exact(tab, g["xi"])
    # the two -2/3 dot products differ by one ulp under FP64 rounding: merge within 1e-12
    groups_T, groups_E = [], []
    for t, e in zip(Tv, E):
        if groups_T and abs(t - groups_T[-1]) < 1e-12:
            groups_E[-1] = e
        else:
            groups_T.append(t)
            groups_E.append(e)
    np.testing.assert_allclose(groups_T, g["T"], atol=1e-12)
    assert [int(e) for e in groups_E] == g["E"]
    for t, want in g["evaluations"]:
        assert int(O.ect_eval(Tv, E, [t])[0]) == want
    vz = golden["vectorization"]
    got = O.ect_grid(tab, [g["xi"]], vz["a"], vz["b"], vz["N"])[0]
    assert got.tolist() == vz["values"]


def test_worked_example_radon_and_ht(golden):
    img = np.array(golden["image"])
    tab = O.critical_tables(img)
    xi = np.array(golden["ect"]["xi"])
    rd = golden["radon"]
    T_ord = np.array(rd["T_ord"])
    # points just after each ordinary critical value (no vertex dot product between)
    after = T_ord + 0.1
    # true Radon on the open interval after each ordinary critical value = -E'
    want = [-e for e in rd["E_prime_printed"]]
    assert O.radon_values(tab, xi, after).tolist() == want
    assert B.radon_brute(img, xi, after).tolist() == want
    val, _ = O.hybrid_transform(tab, "laplace", [xi])
    ht = golden["hybrid_transform"]
    assert abs(val[0] - ht["value_printed"]) <= 0.5 * 10 ** (-ht["printed_digits"])
    exact = 2 * math.exp(-2 / 3) - math.exp(2 / 3) - math.exp(4 / 3)
    assert abs(val[0] - exact) < 1e-13


def test_worked_example_radon_exact(golden):
    img = np.array(golden["image"])
    tab = O.critical_tables(img)
    xi = np.array(golden["ect"]["xi"])
    rd = golden["radon"]
    Tp, Ep = O.radon_exact(tab, xi)
    # the two -2/3 dot products differ by one ulp: merge within 1e-12 as for the ECT
    gT, gE = [], []
    for t, e in zip(Tp, Ep):
        if gT and abs(t - gT[-1]) < 1e-12:
            gE[-1] = e
        else:
            gT.append(t)
            gE.append(e)
    np.testing.assert_allclose(gT, rd["T_ord"], atol=1e-12)
    assert [int(e) for e in gE] == [-e for e in rd["E_prime_printed"]]


# ---------------------------------------------------------------- brute force

def _tiny_images():
    out = []
    for seed, shape in enumerate([(5, 6), (4, 7), (6, 3), (2, 2), (3, 4, 5), (4, 3, 3), (2, 2, 2)]):
        out.append(synth.bernoulli(shape, 0.5, seed=100 + seed))
        rng = np.random.default_rng(200 + seed)
        out.append(rng.integers(0, 5, size=shape).astype(np.int64))
    out.append(np.array([[3, -2, 7], [0, 5, -1]], dtype=np.int64))   # negative values
    # n = 4 (the method holds in any dimension; the library's generic-n path)
    for seed, shape in enumerate([(2, 3, 2, 3), (3, 2, 2, 2), (2, 2, 2, 2)]):
        out.append(synth.bernoulli(shape, 0.5, seed=300 + seed))
        out.append(np.random.default_rng(400 + seed).integers(-3, 4, size=shape).astype(np.int64))
    return out


def _generic_dirs(n, rng, count=3):
    out = []
    for o in range(1 << n):
        for _ in range(count):
            mag = rng.uniform(0.2, 2.0, size=n)
            sgn = np.array([-1.0 if (o >> k) & 1 else 1.0 for k in range(n)])
            out.append(mag * sgn)
    return out


@pytest.mark.parametrize("img", _tiny_images(), ids=lambda a: "x".join(map(str, a.shape)) + a.dtype.name)
def test_lower_star_against_definition(img):
    rng = np.random.default_rng(7)
    low = O.lower_star_values(img)
    for xi in _generic_dirs(img.ndim, rng, count=2):
        o = O.orthant_of(xi)
        np.testing.assert_array_equal(low[o].reshape(-1), B.lower_star_brute(img, xi))


@pytest.mark.parametrize("img", _tiny_images(), ids=lambda a: "x".join(map(str, a.shape)) + a.dtype.name)
def test_transforms_against_cells(img):
    rng = np.random.default_rng(11)
    tab = O.critical_tables(img)
    chi = O.euler_characteristic(img)
    assert tab.chi == chi
    n = img.ndim
    dirs = _generic_dirs(n, rng, count=1)
    # non-generic directions: zero coordinates, +0.0 and -0.0
    for k in range(n):
        z = rng.uniform(0.3, 1.5, size=n) * rng.choice([-1.0, 1.0], size=n)
        z[k] = 0.0
        dirs.append(z)
        z2 = z.copy()
        z2[k] = -0.0
        dirs.append(z2)
    dirs.append(np.eye(n)[0])
    for xi in dirs:
        s = B.vertex_dots(img, xi)
        us = np.unique(s)
        # evaluate exactly at every critical value, between them and outside
        t = np.concatenate([us, (us[:-1] + us[1:]) / 2, [us[0] - 1, us[-1] + 1]])
        np.testing.assert_array_equal(O.ect_values(tab, xi, t), B.ect_brute(img, xi, t))
        np.testing.assert_array_equal(O.radon_values(tab, xi, t), B.radon_brute(img, xi, t))
        # the two exact representations (Appendix A.2 / A.3) give the same values
        Tl, El = O.ect_exact(tab, xi)
        Tp, Ep = O.radon_exact(tab, xi)
        np.testing.assert_array_equal(O.radon_exact_eval(Tl, El, Tp, Ep, t), B.radon_brute(img, xi, t))
        assert int(O.ect_values(tab, xi, [np.inf])[0]) == chi
    # grid form, with a grid built to hit vertex dot products exactly
    for xi in dirs[:4]:
        np.testing.assert_array_equal(
            O.ect_grid(tab, [xi], -1.5, 1.5, 13)[0],
            B.ect_brute(img, xi, O.thresholds(-1.5, 1.5, 13)))


@pytest.mark.parametrize("img", _tiny_images(), ids=lambda a: "x".join(map(str, a.shape)) + a.dtype.name)
def test_top_construction_against_cells(img):
    # pixels as top-dimensional cells (Section 4.1): tables on the (m_k + 1)^n corners
    rng = np.random.default_rng(17)
    tab = O.critical_tables(img, "top")
    assert tab.shape == tuple(s + 1 for s in img.shape)
    cl = B.cells_top(img)
    chi = sum((-1) ** d * phi for d, phi, _ in cl)
    assert tab.chi == chi
    low = O.lower_star_values_top(img)
    for o in range(low.shape[0]):
        assert int(low[o].sum()) == chi
    n = img.ndim
    dirs = _generic_dirs(n, rng, count=1)
    z = rng.uniform(0.3, 1.5, size=n)
    z[0] = 0.0
    dirs.append(z)
    for xi in dirs:
        s = B.vertex_dots(img, xi, tab.shape)
        us = np.unique(s)
        t = np.concatenate([us, (us[:-1] + us[1:]) / 2, [us[0] - 1, us[-1] + 1]])
        np.testing.assert_array_equal(O.ect_values(tab, xi, t), B.ect_brute(img, xi, t, "top"))
        np.testing.assert_array_equal(O.radon_values(tab, xi, t), B.radon_brute(img, xi, t, "top"))
    xi = dirs[0]
    for kernel, kappa in (("laplace", np.exp), ("fourier", lambda u: np.exp(-1j * u))):
        val, norm = O.hybrid_transform(tab, kernel, [xi])
        q = B.ht_by_quadrature(img, xi, kappa, construction="top")
        assert abs(val[0] - q) <= 1e-9 * max(1.0, norm[0])


def test_top_construction_constant_image():
    # every cell of the box [0, m]^n has the value c: the complex is contractible, so
    # ECT(xi, t) = c for t >= the smallest corner dot product and 0 below (closed form)
    for shape in [(1, 1), (3, 5), (2, 3, 4)]:
        img = np.full(shape, 7, dtype=np.int64)
        tab = O.critical_tables(img, "top")
        assert tab.chi == 7
        rng = np.random.default_rng(len(shape))
        for _ in range(4):
            xi = rng.normal(size=len(shape))
            s = B.vertex_dots(img, xi, tab.shape)
            t = np.array([s.min() - 1e-9, s.min(), s.max(), s.max() + 1])
            assert O.ect_values(tab, xi, t).tolist() == [0, 7, 7, 7]


def test_radon_lemma_form_matches_identity():
    rng = np.random.default_rng(3)
    for img in _tiny_images():
        tab = O.critical_tables(img)
        dirs = _generic_dirs(img.ndim, rng, count=1)
        for xi in dirs:
            s = np.unique(B.vertex_dots(img, xi))
            a, b = float(s[0]) - 0.1, float(s[-1]) + 0.1
            np.testing.assert_array_equal(O.radon_grid_lemma(tab, [xi], a, b, 17),
                                          O.radon_grid(tab, [xi], a, b, 17))


def test_exact_tie_grid():
    """Lattice directions whose dot products coincide with thresholds in exact arithmetic."""
    img = synth.bernoulli((5, 5), 0.5, seed=4)
    tab = O.critical_tables(img)
    t = O.thresholds(-1.0, 1.0, 9)
    for xi in ([1.0, 1.0], [1.0, -1.0], [-1.0, 1.0], [2.0, 0.0], [0.0, -1.0]):
        np.testing.assert_array_equal(O.ect_grid(tab, [xi], -1.0, 1.0, 9)[0], B.ect_brute(img, xi, t))
        np.testing.assert_array_equal(O.radon_grid(tab, [xi], -1.0, 1.0, 9)[0], B.radon_brute(img, xi, t))


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("shape", [(2, 2), (7, 5), (2, 2, 2), (4, 3, 5)])
@pytest.mark.parametrize("c", [1, 3])
def test_contractible_closed_form(shape, c):
    """A constant image is a (weighted) cube: ECT = c 1[t >= -h], R = c 1[|t| <= h]."""
    img = np.full(shape, c, dtype=np.int64)
    tab = O.critical_tables(img)
    n = img.ndim
    rng = np.random.default_rng(5)
    for xi in _generic_dirs(n, rng, count=1):
        h = float(np.sum(np.abs(xi))) / 2
        t = np.array([-h - 0.1, -h, -h / 2, 0.0, h, h + 0.1])
        ect = O.ect_values(tab, xi, t)
        rad = O.radon_values(tab, xi, t)
        # t = -h and t = h are vertex dot products up to rounding: check away from them
        for tj, e, r in zip(t, ect, rad):
            if abs(abs(tj) - h) > 1e-12:
                assert e == c * (tj >= -h)
                assert r == c * (abs(tj) <= h)
        for name, (kbar, _) in O.KERNELS.items():
            val, _ = O.hybrid_transform(tab, name, [xi])
            want = -c * (kbar(h) - kbar(-h))
            assert abs(val[0] - want) < 1e-12 * max(1.0, abs(want))


def test_invariants_sum_and_antisymmetry():
    for img in _tiny_images():
        low = O.lower_star_values(img)
        chi = O.euler_characteristic(img)
        n = img.ndim
        for o in range(1 << n):
            assert int(low[o].sum()) == chi
        dl = O.delta_values(low)
        for r in range(dl.shape[0]):
            assert int(dl[r].sum()) == 0
            np.testing.assert_array_equal(dl[r], -(low[O.partner(r, n)] - low[r]))


def test_tables_sorted_and_nonzero():
    img = synth.grf((40, 33), 4.0, seed=9)
    tab = O.critical_tables(img)
    for idx, val in zip(tab.lower_idx + tab.delta_idx, tab.lower_val + tab.delta_val):
        assert np.all(np.diff(idx) > 0)
        assert np.all(val != 0)


# ---------------------------------------------------------------- hybrid transforms

KAPPA = {
    "laplace": np.exp,
    "fourier": lambda t: np.exp(-1j * t),
    "bessel": None,   # filled below (needs scipy)
    "sine": np.sin,
}


def _kappa(name):
    if name == "bessel":
        from scipy.special import j1
        return lambda t: -j1(t)
    return KAPPA[name]


@pytest.mark.parametrize("kernel", ["laplace", "fourier", "bessel", "sine"])
def test_ht_against_cells_and_quadrature(kernel):
    rng = np.random.default_rng(21)
    kbar, _ = O.KERNELS[kernel]
    for img in _tiny_images()[::2]:
        tab = O.critical_tables(img)
        for xi in _generic_dirs(img.ndim, rng, count=1):
            xi = xi * 2.0
            val, norm = O.hybrid_transform(tab, kernel, [xi])
            cellsum = B.integral_kappa_radon(img, xi, kbar)
            assert abs(val[0] + cellsum) <= 1e-12 * max(1.0, norm[0])
            quad = B.ht_by_quadrature(img, xi, _kappa(kernel))
            assert abs(val[0] - quad) <= 1e-10 * max(1.0, norm[0])


def test_kernel_primitives():
    """kappa is the derivative of kbar for each kernel (central differences)."""
    s = np.linspace(-3, 3, 13)
    h = 1e-5
    for name, (kbar, kap) in O.KERNELS.items():
        fd = (kbar(s + h) - kbar(s - h)) / (2 * h)
        np.testing.assert_allclose(fd, kap(s), atol=1e-8)
    from scipy.special import j0
    # first zero of J0 and J0(0) = 1 (Abramowitz & Stegun, Table 9.5 / 9.1.10)
    assert abs(j0(2.404825557695773)) < 1e-15 and j0(0.0) == 1.0


@pytest.mark.parametrize("kernel", ["laplace", "fourier", "bessel", "sine"])
def test_gradient_central_differences(kernel):
    img = synth.grf((9, 11), 2.0, seed=31)
    tab = O.critical_tables(img)
    rng = np.random.default_rng(41)
    h = 1e-4
    dirs = [d for d in _generic_dirs(2, rng, count=2) if np.min(np.abs(d)) > 10 * h]
    g, _ = O.hybrid_transform_grad(tab, kernel, dirs)
    for di, xi in enumerate(dirs):
        for k in range(2):
            e = np.zeros(2)
            e[k] = h
            fp, _ = O.hybrid_transform(tab, kernel, [xi + e])
            fm, _ = O.hybrid_transform(tab, kernel, [xi - e])
            fd = (fp[0] - fm[0]) / (2 * h)
            assert abs(fd - g[di, k]) < 1e-6 * max(1.0, abs(g[di, k]))


def test_sine_kernel_is_minus_imag_fourier():
    # kappa = sin against kappa = e^{-it}: kbar_sine = -cos = -Im(sin + i cos)
    img = synth.grf((12, 13), 2.0, seed=51)
    tab = O.critical_tables(img)
    dirs = _generic_dirs(2, np.random.default_rng(52), count=2)
    vs, _ = O.hybrid_transform(tab, "sine", dirs)
    vf, _ = O.hybrid_transform(tab, "fourier", dirs)
    np.testing.assert_allclose(vs, -vf.imag, rtol=0, atol=1e-12)
    gs, _ = O.hybrid_transform_grad(tab, "sine", dirs)
    gf, _ = O.hybrid_transform_grad(tab, "fourier", dirs)
    np.testing.assert_allclose(gs, -gf.imag, rtol=0, atol=1e-12)


def test_orthant_rule():
    assert O.orthant_of([1.0, -2.0]) == 2
    assert O.orthant_of([-0.0, 0.0]) == 0
    assert O.orthant_of([-1.0, -1.0, 3.0]) == 3
    x = O.vertex_coords(7)
    np.testing.assert_array_equal(x, -x[::-1])
    assert x[0] == -0.5 and x[-1] == 0.5


# ---------------------------------------------------------------- tabulated kernels

def _table_dirs(rng, n, count):
    return [d * 1.5 for d in _generic_dirs(n, rng, count=count)]


def test_table_kernel_interpolant():
    """Samples at the knots, linear in between, constant outside, kappa = slope."""
    rng = np.random.default_rng(61)
    y = rng.normal(size=9)
    a, b = -0.7, 1.3
    kbar, kap = O.table_kernel(y, a, b)
    h = (b - a) / 8
    knots = a + h * np.arange(9)
    np.testing.assert_allclose(kbar(knots), y, rtol=0, atol=1e-14)
    mids = knots[:-1] + 0.5 * h
    np.testing.assert_allclose(kbar(mids), 0.5 * (y[:-1] + y[1:]), rtol=0, atol=1e-14)
    np.testing.assert_allclose(kap(mids), (y[1:] - y[:-1]) / h, rtol=1e-12)
    np.testing.assert_array_equal(kbar(np.array([-5.0, a - 1e-9])), [y[0], y[0]])
    np.testing.assert_array_equal(kbar(np.array([b, b + 1e-9, 7.0])), [y[-1]] * 3)
    np.testing.assert_array_equal(kap(np.array([-5.0, b, 7.0])), [0.0, 0.0, 0.0])
    # kappa is the derivative of kbar away from the knots
    s = knots[:-1] + h * rng.uniform(0.1, 0.9, size=8)
    e = 1e-7 * h
    np.testing.assert_allclose((kbar(s + e) - kbar(s - e)) / (2 * e), kap(s), rtol=1e-6)
    # samples of an affine function are reproduced everywhere on [a, b]
    lin, _ = O.table_kernel(2.0 * knots - 3.0, a, b)
    t = np.linspace(a, b, 101)
    np.testing.assert_allclose(lin(t), 2.0 * t - 3.0, rtol=0, atol=1e-13)
    with pytest.raises(ValueError):
        O.table_kernel([1.0], a, b)
    with pytest.raises(ValueError):
        O.table_kernel(y, b, a)


def test_table_ht_against_cells():
    """Lemma 3.1 with a tabulated primitive against the cell-by-cell integral (any kbar)."""
    rng = np.random.default_rng(62)
    for img in _tiny_images()[::2]:
        tab = O.critical_tables(img)
        M = 0.5 * img.ndim
        # a table that covers only part of the dot products: the constant ends count too
        kt = O.table_kernel(rng.normal(size=7), -0.4 * M, 0.5 * M)
        for xi in _table_dirs(rng, img.ndim, 1):
            val, norm = O.hybrid_transform(tab, kt, [xi])
            cellsum = B.integral_kappa_radon(img, xi, kt[0])
            assert abs(val[0] + cellsum) <= 1e-12 * max(1.0, norm[0])


def test_table_ht_outside_range_vanishes():
    # kbar constant on every dot product: HT = c * sum_v Delta_eps(v) = 0
    img = synth.grf((10, 12), 2.0, seed=63)
    tab = O.critical_tables(img)
    dirs = _table_dirs(np.random.default_rng(64), 2, 3)
    for a, b in [(5.0, 6.0), (-9.0, -5.0)]:
        val, _ = O.hybrid_transform(tab, O.table_kernel([2.5, -1.0, 4.0], a, b), dirs)
        np.testing.assert_array_equal(val, 0.0)


@pytest.mark.parametrize("n", [2, 3])
def test_table_converges_to_laplace(n):
    """Samples of e^s: |HT_table - HT_laplace| <= h^2 / 8 max e^s sum |Delta| (linear
    interpolation error); the gradient within h max e^s sum |Delta x_k|."""
    shape = (9, 11) if n == 2 else (5, 6, 7)
    img = synth.grf(shape, 2.0, seed=65)
    tab = O.critical_tables(img)
    dirs = _table_dirs(np.random.default_rng(66), n, 2)
    M = max(0.5 * float(np.sum(np.abs(d))) for d in dirs)
    for K in (65, 257):
        # strictly wider than the dot products: at s = b itself kappa is the constant
        # extension's (zero), and the extreme corners reach |s| = M exactly
        a, b = -1.01 * M, 1.01 * M
        h = (b - a) / (K - 1)
        kt = O.table_kernel(np.exp(a + h * np.arange(K)), a, b)
        got, _ = O.hybrid_transform(tab, kt, dirs)
        want, _ = O.hybrid_transform(tab, "laplace", dirs)
        gt, _ = O.hybrid_transform_grad(tab, kt, dirs)
        gw, _ = O.hybrid_transform_grad(tab, "laplace", dirs)
        for di, xi in enumerate(dirs):
            _, _, dv = O.oracle._ht_terms(tab, xi)
            l1 = float(np.sum(np.abs(dv)))
            assert abs(got[di] - want[di]) <= h * h / 8 * math.exp(b) * l1 + 1e-12
            assert np.max(np.abs(gt[di] - gw[di])) <= h * math.exp(b) * l1 * 0.5 + 1e-12


def test_table_gradient_central_differences():
    img = synth.grf((9, 11), 2.0, seed=67)
    tab = O.critical_tables(img)
    rng = np.random.default_rng(68)
    kt = O.table_kernel(np.cumsum(rng.normal(size=33)) * 0.1, -1.1, 1.2)
    h = 1e-7
    dirs = [d for d in _table_dirs(rng, 2, 3) if np.min(np.abs(d)) > 10 * h]
    g, _ = O.hybrid_transform_grad(tab, kt, dirs)
    for di, xi in enumerate(dirs):
        for k in range(2):
            e = np.zeros(2)
            e[k] = h
            fp, _ = O.hybrid_transform(tab, kt, [xi + e])
            fm, _ = O.hybrid_transform(tab, kt, [xi - e])
            assert abs((fp[0] - fm[0]) / (2 * h) - g[di, k]) < 1e-5 * max(1.0, abs(g[di, k]))


# ---------------------------------------------------------------- the oracle over processes

@pytest.mark.parametrize("parts", [1, 3, 7])
def test_row_block_tables_equal_whole_image(parts):
    """The CPU baseline's split of the tables over vertices (row blocks with a one-row halo)
    gives the whole image's tables, entry for entry."""
    from oracle import parallel as OP
    img = synth.grf((37, 29), 4.0, seed=77)
    ref = O.critical_tables(img)
    t = OP.merge_blocks(img.shape, [OP.block_tables(a) for a in OP.row_blocks(img, parts)])
    for o in range(4):
        np.testing.assert_array_equal(t.lower_idx[o], ref.lower_idx[o])
        np.testing.assert_array_equal(t.lower_val[o], ref.lower_val[o])
    for r in range(2):
        np.testing.assert_array_equal(t.delta_idx[r], ref.delta_idx[r])
        np.testing.assert_array_equal(t.delta_val[r], ref.delta_val[r])
    assert t.chi == ref.chi
