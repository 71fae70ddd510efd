"""A float16 model of the 8-bit extraction's arithmetic (no GPU).

The kernel holds a pixel b in [0, 255] as the half-precision number 1024 + b, stages
pixels outside the image as 0 (the smallest value, so a cell leaving the image adds
nothing), and forms the lower-star value of orthant o from differences of two such
numbers, grouped as
    (phi - e_0) + (f_01 - e_1) [+ (f_02 - e_2) + (f_12 - c)]
(e_k edge minima, f_kl square minima, c the cube minimum), then Delta_o = D_o - D_{o^(2^n-1)}.
Every difference is an integer in [-255, 255], every partial sum and every Delta has
magnitude <= 2040 < 2048, so each half-precision operation is exact.  The model repeats
these operations in numpy float16 and compares with the oracle, on random images and on
the extremes (0/255 checkerboards, a 255 plateau with 0 holes) that maximise the sums.
"""
import numpy as np
import pytest

import oracle as O
from paper_2405_02256_gb300 import synth

H = np.float16


def _staged(img):
    # one pixel of zeros around the image; values as 1024 + b in half precision
    pad = np.pad(img.astype(np.int64), 1)
    return (pad + 1024).astype(H)


def _nb(S, n, shift):
    # S shifted so that entry v holds the staged value at v + shift (shift in {-1,0,1}^n)
    core = tuple(slice(1 + s, S.shape[a] - 1 + s) for a, s in enumerate(reversed(shift)))
    return S[core]


def _lower_f16(img):
    n = img.ndim
    S = _staged(img)
    out = []
    for o in range(1 << n):
        d = [1 if (o >> k) & 1 else -1 for k in range(n)]   # the lower star leaves v towards d_k on axis k

        def at(*ks):
            sh = [0] * n
            for k in ks:
                sh[k] = d[k]
            return _nb(S, n, sh)

        phi = at()
        e = [np.minimum(phi, at(k)) for k in range(n)]
        f01 = np.minimum(np.minimum(phi, at(0)), np.minimum(at(1), at(0, 1)))
        D = H(phi - e[0]) + H(f01 - e[1])
        D = D.astype(H)
        if n == 3:
            f02 = np.minimum(np.minimum(phi, at(0)), np.minimum(at(2), at(0, 2)))
            f12 = np.minimum(np.minimum(phi, at(1)), np.minimum(at(2), at(1, 2)))
            c = np.minimum(f01, np.minimum(np.minimum(at(2), at(0, 2)), np.minimum(at(1, 2), at(0, 1, 2))))
            D = (D + H(f02 - e[2])).astype(H)
            D = (D + H(f12 - c)).astype(H)
        out.append(D)
    lower = np.stack(out)
    half = 1 << (n - 1)
    full = (1 << n) - 1
    delta = np.stack([(lower[o] - lower[o ^ full]).astype(H) for o in range(half)])
    return lower, delta


def _images():
    rng = np.random.default_rng(11)
    ims = [rng.integers(0, 256, size=(9, 13)), synth.grf((17, 12), 2.0, seed=4),
           (np.indices((8, 9)).sum(0) % 2) * 255, np.where(rng.random((10, 10)) < 0.2, 0, 255),
           rng.integers(0, 256, size=(5, 6, 7)), (np.indices((5, 4, 6)).sum(0) % 2) * 255,
           np.where(rng.random((6, 6, 6)) < 0.15, 0, 255), np.full((3, 4, 2), 255)]
    return [np.asarray(im, dtype=np.uint8) for im in ims]


@pytest.mark.parametrize("img", _images(), ids=lambda a: "x".join(map(str, a.shape)) + ("_%d" % int(a.max())))
def test_half_precision_stencil_is_exact(img):
    lower, delta = _lower_f16(img)
    want_lower = O.lower_star_values(img)
    want_delta = O.delta_values(want_lower)
    np.testing.assert_array_equal(lower.astype(np.int64), want_lower)
    np.testing.assert_array_equal(delta.astype(np.int64), want_delta)
    assert np.abs(want_delta).max() <= 2040 < 2048
