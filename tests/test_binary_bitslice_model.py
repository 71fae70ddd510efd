"""A bit-plane model of the binary 3-D extraction's arithmetic (no GPU).

For volumes of 0 / 1 voxels a cell's value, the minimum of its vertices, is their AND, so
the kernel forms each orthant's lower-star value from bit planes: with the lower-star
box v + g d (d_k = +1 where bit k of the orthant is set, else -1) and its bits
t0, x, y, z, xy, xz, yz, xyz,
    s1 s0 = x + y + z,   F1 F0 = xy-face + xz-face + yz-face,   c = F0 F1 xyz,
    v0 = t0 & ~(s0 ^ F0 ^ c),   v1 = t0 & s1 & (s0 ? ~F1 : ~F0),
    Delta^-_o = v0 - 2 v1,      Delta_r non-zero where the codes of r and r ^ 7 differ.
The model evaluates exactly these bitwise operations in numpy on whole volumes (outside
voxels are 0, as in the kernel's zero border) and must equal the oracle's tables, every
orthant and every Delta table, on random volumes and on constant ones.
"""
import numpy as np
import pytest

import oracle as O
from paper_2405_02256_gb300 import synth


def _shift(P, dz, dy, dx):
    # entry (z, y, x) holds the padded volume's voxel (z + dz, y + dy, x + dx)
    m2, m1, m0 = P.shape[0] - 2, P.shape[1] - 2, P.shape[2] - 2
    return P[1 + dz:1 + dz + m2, 1 + dy:1 + dy + m1, 1 + dx:1 + dx + m0]


def _codes(vol):
    P = np.pad(vol.astype(bool), 1)
    maj = lambda a, b, c: (a & b) | (a & c) | (b & c)
    t0 = _shift(P, 0, 0, 0)
    v1, v0 = [], []
    for o in range(8):
        dx = 1 if o & 1 else -1
        dy = 1 if o & 2 else -1
        dz = 1 if o & 4 else -1
        x, y, z = _shift(P, 0, 0, dx), _shift(P, 0, dy, 0), _shift(P, dz, 0, 0)
        xy, xz, yz, xyz = _shift(P, 0, dy, dx), _shift(P, dz, 0, dx), _shift(P, dz, dy, 0), _shift(P, dz, dy, dx)
        s0, s1 = x ^ y ^ z, maj(x, y, z)
        fxy, fxz, fyz = x & y & xy, x & z & xz, y & z & yz
        F0, F1 = fxy ^ fxz ^ fyz, maj(fxy, fxz, fyz)
        c = F0 & F1 & xyz
        v1.append(t0 & s1 & ((s0 & ~F1) | (~s0 & ~F0)))
        v0.append(t0 & ~(s0 ^ F0 ^ c))
    return v1, v0


def _check(vol):
    ref = O.critical_tables(vol)
    v1, v0 = _codes(vol)
    val = [(a.astype(np.int64) - 2 * b.astype(np.int64)).ravel() for a, b in zip(v0, v1)]
    for o in range(8):
        nz = np.flatnonzero(val[o])
        np.testing.assert_array_equal(nz, ref.lower_idx[o])
        np.testing.assert_array_equal(val[o][nz], ref.lower_val[o])
        assert set(np.unique(val[o])) <= {-2, -1, 0, 1}
    for r in range(4):
        d = val[r] - val[r ^ 7]
        nz = np.flatnonzero(d)
        np.testing.assert_array_equal(nz, ref.delta_idx[r])
        np.testing.assert_array_equal(d[nz], ref.delta_val[r])
        # the kernel's mask: codes differ
        mask = ((v1[r] ^ v1[r ^ 7]) | (v0[r] ^ v0[r ^ 7])).ravel()
        np.testing.assert_array_equal(np.flatnonzero(mask), ref.delta_idx[r])


@pytest.mark.parametrize("seed", range(12))
def test_random_volumes(seed):
    rng = np.random.default_rng(seed)
    shape = tuple(int(v) for v in rng.integers(2, 9, size=3))
    _check((rng.random(shape) < rng.uniform(0.15, 0.85)).astype(np.uint8))


def test_binary_grf_volume():
    _check(synth.grf((18, 20, 40), 3.0, seed=7, binary=True))


@pytest.mark.parametrize("v", [0, 1])
def test_constant_volumes(v):
    _check(np.full((4, 5, 6), v, dtype=np.uint8))
