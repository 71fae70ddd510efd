"""A float32 model of the tabulated kernel's lookup (no GPU).

The kernel saturates the scaled position p / K = (u + 1/2) / K to [0, 1] (NaN -> 0), rounds
p to the nearest integer j by adding 1.5 * 2^23, and reads entry j of a padded table of
K + 1 pairs: (y_0, 0), (y_r + d_r / 2, d_r) for r = 0 .. K - 2, (y_{K-1}, 0).  The model
checks that every position, inside or outside [a, b] or not finite, lands on an entry in
[0, K], and that Y + (p - j) D reproduces the oracle's interpolant and D / h its slope.
"""
import numpy as np

import oracle as O

F32 = np.float32
MAGIC = F32(12582912.0)


def _padded(y):
    K = len(y)
    t = np.zeros((K + 1, 2), dtype=F32)
    t[0] = (y[0], 0.0)
    d = np.diff(y)
    t[1:K, 0] = (y[:-1] + 0.5 * d).astype(F32)
    t[1:K, 1] = d.astype(F32)
    t[K] = (y[-1], 0.0)
    return t


def _lookup(tab, ps, K):
    ps = np.nan_to_num(np.clip(ps.astype(F32), F32(0), F32(1)), nan=0.0).astype(F32)   # fma.rn.sat
    exact = ps.astype(np.float64) * K                                                     # exact product
    t = (exact + float(MAGIC)).astype(F32)                                                # one rounding
    j = t.view(np.int32) - 0x4B400000
    g = (exact - (t - MAGIC).astype(np.float64)).astype(F32)
    return j, g


def test_every_position_lands_on_an_entry():
    for K in (2, 3, 64, 1000, 16384):
        ps = np.concatenate([np.linspace(-3, 4, 20001), [np.inf, -np.inf, np.nan, 0.0, 1.0, 0.5 / K]])
        j, g = _lookup(_padded(np.zeros(K)), ps, K)
        assert j.min() >= 0 and j.max() <= K
        assert np.all(np.abs(g) <= 0.5)


def test_interpolant_and_slope_against_the_oracle():
    rng = np.random.default_rng(0)
    for K in (2, 7, 64, 1000, 16384):
        a, b = -0.8, 1.1
        h = (b - a) / (K - 1)
        y = np.sin(3.0 * np.linspace(a, b, K))
        tab = _padded(y)
        s = np.concatenate([rng.uniform(a - 1, b + 1, 5000), a + h * np.arange(K)])
        ps = ((s - a) / h + 0.5) / K
        j, g = _lookup(tab, ps, K)
        kbar = g.astype(np.float64) * tab[j, 1] + tab[j, 0]
        kb, kap = O.table_kernel(y, a, b)
        assert np.max(np.abs(kbar - kb(s))) < 4e-7
        u = (s - a) / h
        away = np.abs(u - np.round(u)) > 1e-3          # the slope is ambiguous only next to a knot
        slope = tab[j, 1].astype(np.float64) / h
        assert np.max(np.abs(slope[away] - kap(s)[away]) / np.maximum(np.abs(kap(s)[away]), 1.0)) < 2e-7
