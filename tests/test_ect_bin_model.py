"""A float32 model of the ECT kernel's binning and its exactness filter (no GPU).

The kernel forms the bin coordinate u = (s - t_min) / h of a vertex from the lattice form
u = c_0 A_0 + c_1 A_1 [+ c_2 A_2] + beta (FP32 coefficients, fused multiply-adds; c_k the
integers 2 i_k - (m_k - 1)) and takes the sublevel bin ceil(u) from it only when u is at
least delta = 2^-22 M_u + 1e-12 (M_u + T + 1) away from every integer; otherwise the bin is
recomputed from the canonical FP64 dot product and the FP64 thresholds.  The model checks,
over many vertices and directions (random ones and lattice-aligned ones whose dot products
fall exactly on thresholds), that every decision taken in FP32 equals the FP64 one.
"""
import numpy as np
import pytest

import oracle as O
from paper_2405_02256_gb300 import synth

F32 = np.float32


def _fma32(a, b, c):
    # a * b exact in float64 for float32 operands; one rounding to float32 (model of fmaf)
    return (a.astype(np.float64) * np.float64(b) + np.asarray(c, dtype=np.float64)).astype(F32)


def _coef(xi, m, t_min, t_max, T):
    h = (t_max - t_min) / (T - 1)
    A = [xi[k] / (2.0 * (m[k] - 1) * h) for k in range(len(m))]
    beta = -t_min / h
    Mu = sum(abs(A[k]) * (m[k] - 1) for k in range(len(m))) + abs(beta)
    delta = (np.ldexp(Mu, -22) + 1e-12 * (Mu + T + 1.0)) * (1.0 + 1e-6)
    return [F32(a) for a in A], F32(beta), F32(delta)


def _check(shape, dirs, T, a=None, b=None, no_filter=False):
    n = len(shape)
    m = tuple(reversed(shape))                     # m_0 is the fastest axis
    if a is None:
        a, b = -synth.image_radius(n), synth.image_radius(n)
    thr = O.thresholds(a, b, T)
    idx = np.arange(int(np.prod(shape)))
    ii = O.oracle._vertex_multi_index(idx, m)
    c = [F32(2 * ii[k] - (m[k] - 1)) for k in range(n)]
    fp32_decisions = 0
    for xi in dirs:
        A, beta, delta = _coef(xi, m, a, b, T)
        u = _fma32(c[n - 1], A[n - 1], beta)
        for k in range(n - 2, -1, -1):
            u = _fma32(c[k], A[k], u)
        r = np.rint(u)
        sure = np.abs(u.astype(np.float64) - r) >= (0.0 if no_filter else delta)
        bin32 = np.clip(np.ceil(u.astype(np.float64)), 0, T).astype(np.int64)
        s = O.dot_products(xi, idx, m)
        bin64 = np.searchsorted(thr, s, side="left")   # min{j : s <= t_j}, T when none
        assert np.array_equal(bin32[sure], bin64[sure])
        fp32_decisions += int(sure.sum())
    return fp32_decisions


@pytest.mark.parametrize("shape,T", [((64, 96), 512), ((33, 40), 64), ((12, 14, 16), 256)])
def test_fp32_bins_agree_with_fp64_where_the_filter_passes(shape, T):
    n = len(shape)
    rng = np.random.default_rng(17)
    dirs = list(rng.normal(size=(300, n)) * rng.uniform(0.01, 1.0, size=(300, 1)))
    # lattice-aligned directions: dot products land on thresholds exactly
    axis = [np.eye(n)[k] for k in range(n)] + [-np.eye(n)[k] for k in range(n)]
    dirs += axis + [np.ones(n), np.ones(n) / 2, np.array([1.0, -1.0] + [0.0] * (n - 2))]
    checked = _check(shape, dirs, T)
    # the filter rejects only a small share of the decisions
    assert checked >= 0.95 * len(dirs) * int(np.prod(shape))


@pytest.mark.parametrize("shape,T,a,b", [((21, 33), 65, -0.5, 0.5), ((21, 33), 129, -1.0, 1.0),
                                         ((9, 10, 17), 33, -0.5, 0.5)])
def test_thresholds_on_the_lattice(shape, T, a, b):
    """Thresholds aligned with the vertex coordinates (t_j = a + j (b - a) / (T - 1) hits
    x_0(i) = (2 i - (m_0 - 1)) / (2 (m_0 - 1)) exactly): u lands on integers, the filter
    sends those points to FP64, and every FP32 decision still agrees."""
    n = len(shape)
    dirs = [np.eye(n)[0], -np.eye(n)[0], np.eye(n)[1], np.ones(n), np.ones(n) / 2,
            np.array([0.5, 0.25] + [0.0] * (n - 2)), np.array([1.0, -1.0] + [0.0] * (n - 2))]
    _check(shape, dirs, T, a, b)


def test_without_the_filter_some_fp32_bins_would_be_wrong():
    # random directions with every decision taken in FP32: some points lie closer to a
    # threshold than the FP32 error of u, and their FP32 bin differs from the FP64 one
    dirs = list(np.random.default_rng(17).normal(size=(100, 2)))
    with pytest.raises(AssertionError):
        _check((64, 96), dirs, 512, no_filter=True)
