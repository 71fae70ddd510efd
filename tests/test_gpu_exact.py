"""Exact representations (Section 4.3; Appendix A.2 computation, A.3 evaluation) against
the oracle: (T, E) of the ECT and (T', E') of the Radon transform bit-exact for every
image and direction, and their evaluation at arbitrary thresholds (every critical value,
points between and outside them, random points)."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2405_02256_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_02256_gb300 import binding
    binding.load()
    return binding


def _example():
    with open(os.path.join(ROOT, "tests", "golden", "worked_example.json")) as f:
        return np.array(json.load(f)["image"], dtype=np.uint8)


IMAGES = {
    "example4x4": _example(),
    "bern64": synth.bernoulli((64, 64), 0.5, seed=0),
    "grf150x211": synth.grf((150, 211), 6.0, seed=1),
    "grf512": synth.grf((512, 512), 8.0, seed=2),             # tables of ~3e4 points: several radix tiles
    "const": np.full((33, 17), 7, dtype=np.uint8),
    "i32_2d": np.random.default_rng(5).integers(-1000, 1000, size=(50, 70)).astype(np.int32),
    "grf20x33x40": synth.grf((20, 33, 40), 4.0, seed=7),
    "bin40x40x48": synth.grf((40, 40, 48), 5.0, seed=8, binary=True),
    # sum of the sides above the staged coordinate products (12288): keys from divisions
    "grf3x13000": synth.grf((3, 13000), 3.0, seed=10),
}


def _dirs(n):
    if n == 2:
        d = [synth.circle_dirs(16), synth.random_2d_dirs(8, 3, 0.01, 1.5),
             np.array([[2.0, 2.0], [0.0, 1.0], [1.0, 0.0], [-0.0, -1.0], [-1.0, -0.0], [0.0, 0.0], [1.0, -1.0]])]
    else:
        d = [synth.fibonacci_dirs(12), synth.sphere_dirs(6, 4, 0.05, 2.0),
             np.array([[0.0, 0.0, 1.0], [1.0, 0.0, -0.0], [0.5, -0.5, 0.0], [-1.0, -1.0, -1.0]])]
    return np.concatenate(d)


def _queries(reps, extra):
    t = np.concatenate([np.concatenate(reps), extra])
    t = np.unique(t)
    mids = (t[:-1] + t[1:]) / 2 if len(t) > 1 else np.zeros(0)
    return np.concatenate([t, mids, np.nextafter(t, -np.inf), [-5.0, 5.0]])


@pytest.mark.parametrize("name", list(IMAGES))
def test_exact_representation_bit_exact(tb, name):
    img = IMAGES[name]
    dt = tb.U8 if img.dtype == np.uint8 else tb.I32
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    ref = O.critical_tables(img)
    dirs = _dirs(img.ndim)
    d = torch.from_numpy(dirs).cuda()
    rep0 = tb.exact_representation(tabs, 0, d)
    rep1 = tb.exact_representation(tabs, 1, d)
    ref0 = [O.ect_exact(ref, xi) for xi in dirs]
    ref1 = [O.radon_exact(ref, xi) for xi in dirs]
    for di in range(len(dirs)):
        T, E = rep0.segment(0, di)
        np.testing.assert_array_equal(T, ref0[di][0])
        np.testing.assert_array_equal(E, ref0[di][1])
        T, E = rep1.segment(0, di)
        np.testing.assert_array_equal(T, ref1[di][0])
        np.testing.assert_array_equal(E, ref1[di][1])
    # evaluation at every critical value of a few directions, between them and outside
    sel = [0, 3, len(dirs) - 1]
    t = _queries([ref0[i][0] for i in sel] + [ref1[i][0] for i in sel],
                 np.random.default_rng(9).uniform(-1.2, 1.2, 64))
    got_e = tb.ect_exact_eval(rep0, t).cpu().numpy()[0]
    got_r = tb.radon_exact_eval(rep0, rep1, t).cpu().numpy()[0]
    for di, xi in enumerate(dirs):
        np.testing.assert_array_equal(got_e[di], O.ect_eval(*ref0[di], t))
        np.testing.assert_array_equal(got_r[di], O.radon_values(ref, xi, t))
    assert dt in (tb.U8, tb.I32)


def test_exact_ragged_batch_per_image_dirs(tb):
    shapes = synth.ragged_shapes(6, 2, 70, seed=13)
    imgs = [synth.blurred_noise(s, 2.0, seed=40 + i) for i, s in enumerate(shapes)]
    tabs = tb.build_critical_tables(tb.pack_images(imgs, align=1))
    rng = np.random.default_rng(4)
    dirs = rng.normal(size=(len(imgs), 9, 2))
    dirs[:, 0, 1] = 0.0                                         # a zero coordinate in every image
    rep0 = tb.exact_representation(tabs, 0, torch.from_numpy(dirs).cuda())
    rep1 = tb.exact_representation(tabs, 1, torch.from_numpy(dirs).cuda())
    t = np.linspace(-1.0, 1.0, 41)
    got_r = tb.radon_exact_eval(rep0, rep1, t).cpu().numpy()
    for b, img in enumerate(imgs):
        ref = O.critical_tables(img)
        for di in range(dirs.shape[1]):
            T, E = rep0.segment(b, di)
            Tw, Ew = O.ect_exact(ref, dirs[b, di])
            np.testing.assert_array_equal(T, Tw)
            np.testing.assert_array_equal(E, Ew)
            np.testing.assert_array_equal(got_r[b, di], O.radon_values(ref, dirs[b, di], t))


def test_exact_cap_too_small(tb):
    img = IMAGES["bern64"]
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    d = torch.from_numpy(_dirs(2)).cuda()
    with pytest.raises(tb.TopotError):
        tb.exact_representation(tabs, 0, d, cap=3)


def test_exact_full_size_2048(tb):
    """Tables of a 2048^2 GRF image (about 4e5 points per table, a hundred radix tiles per
    segment joined by look-back), two images sharing 5 directions (one axis-aligned,
    one with a zero coordinate): both representations bit-exact."""
    imgs = [synth.grf((2048, 2048), 16.0, seed=20), synth.grf((2048, 2048), 16.0, seed=21)]
    tabs = tb.build_critical_tables(tb.pack_images(imgs))
    dirs = np.concatenate([synth.random_2d_dirs(3, 22, 0.01, 1.0), np.array([[0.0, -1.0], [0.7, 0.0]])])
    d = torch.from_numpy(dirs).cuda()
    rep0 = tb.exact_representation(tabs, 0, d)
    rep1 = tb.exact_representation(tabs, 1, d)
    for b, img in enumerate(imgs):
        ref = O.critical_tables(img)
        for di, xi in enumerate(dirs):
            T, E = rep0.segment(b, di)
            Tw, Ew = O.ect_exact(ref, xi)
            np.testing.assert_array_equal(T, Tw)
            np.testing.assert_array_equal(E, Ew)
            T, E = rep1.segment(b, di)
            Tw, Ew = O.radon_exact(ref, xi)
            np.testing.assert_array_equal(T, Tw)
            np.testing.assert_array_equal(E, Ew)
