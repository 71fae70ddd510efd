"""Top-dimensional construction (Section 4.1: one top cell per pixel, lower cells carry the
minimum over the pixels containing them) on the GPU against the oracle: tables on the
pixel corners bit-exact, ECT / Radon bit-exact and hybrid transforms within 1e-6 on them."""
import numpy as np
import pytest

import oracle as O
from paper_2405_02256_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_02256_gb300 import binding
    binding.load()
    return binding


IMAGES = {
    "single_pixel": np.array([[9]], dtype=np.uint8),
    "row1x5": synth.uniform_u8((1, 5), seed=1),
    "example4x4": np.array([[1, 0, 0, 0], [0, 1, 1, 0], [1, 1, 1, 1], [1, 1, 0, 0]], dtype=np.uint8),
    "bern64": synth.bernoulli((64, 64), 0.5, seed=0),
    "grf150x211": synth.grf((150, 211), 6.0, seed=1),
    "wide3x5000": synth.uniform_u8((3, 5000), seed=3),
    "tall600x4": synth.uniform_u8((600, 4), seed=4),
    "i32_2d": np.random.default_rng(5).integers(-1000, 1000, size=(40, 55)).astype(np.int32),
    "cube1": np.array([[[3]]], dtype=np.uint8),
    "bern9x10x11": synth.bernoulli((9, 10, 11), 0.5, seed=6),
    "grf20x33x40": synth.grf((20, 33, 40), 4.0, seed=7),
    "i32_3d": np.random.default_rng(6).integers(-50, 50, size=(8, 9, 10)).astype(np.int32),
    # 8-bit images take a u8 corner image where 255 also stands for "no pixel"
    "all255_7x9": np.full((7, 9), 255, dtype=np.uint8),
    "border255_31x47": np.pad(synth.uniform_u8((29, 45), seed=8), 1, constant_values=255),
    "corners255_16x16": np.where(np.outer(np.arange(16) % 15 == 0, np.arange(16) % 15 == 0), 255,
                                 synth.uniform_u8((16, 16), seed=9)).astype(np.uint8),
    "bin0_255_6x7x8": (synth.bernoulli((6, 7, 8), 0.5, seed=10) * 255).astype(np.uint8),
    "all255_3x4x5": np.full((3, 4, 5), 255, dtype=np.uint8),
    "grf2x3x700": synth.grf((2, 3, 700), 3.0, seed=11),
}


def _check(tabs, b, ref):
    n = len(ref.shape)
    for o in range(1 << n):
        idx, val = tabs.table(b, o, 0)
        np.testing.assert_array_equal(idx, ref.lower_idx[o])
        np.testing.assert_array_equal(val, ref.lower_val[o])
        assert tabs.info(b, o)[2] == ref.chi
    for r in range(1 << (n - 1)):
        idx, val = tabs.table(b, r, 1)
        np.testing.assert_array_equal(idx, ref.delta_idx[r])
        np.testing.assert_array_equal(val, ref.delta_val[r])


@pytest.mark.parametrize("name", list(IMAGES))
def test_top_tables_and_transforms(tb, name):
    img = IMAGES[name]
    n = img.ndim
    tabs = tb.build_critical_tables(tb.pack_images([img]), construction="top")
    ref = O.critical_tables(img, "top")
    _check(tabs, 0, ref)
    if n == 2:
        dirs = np.concatenate([synth.circle_dirs(24), np.array([[0.0, 1.0], [-1.0, -0.0], [1.0, 1.0]])])
    else:
        dirs = np.concatenate([synth.fibonacci_dirs(24), np.array([[0.0, 0.0, 1.0], [1.0, -0.0, 0.0]])])
    R = synth.image_radius(n)
    d = torch.from_numpy(dirs).cuda()
    np.testing.assert_array_equal(tb.ect(tabs, d, -R, R, 65).cpu().numpy()[0], O.ect_grid(ref, dirs, -R, R, 65))
    np.testing.assert_array_equal(tb.radon(tabs, d, -R, R, 65).cpu().numpy()[0], O.radon_grid(ref, dirs, -R, R, 65))
    for kernel in ("laplace", "fourier", "bessel"):
        got = tb.hybrid_transform(tabs, kernel, d).cpu().numpy()[0]
        want, norm = O.hybrid_transform(ref, kernel, dirs)
        if kernel == "fourier":
            got = got[:, 0] + 1j * got[:, 1]
        assert np.all(np.abs(got - want) <= 1e-6 * np.maximum(norm, 1e-300)), kernel


def test_top_ragged_batch(tb):
    shapes = synth.ragged_shapes(11, 2, 80, seed=21)
    imgs = [synth.blurred_noise(s, 2.0, seed=60 + i) for i, s in enumerate(shapes)]
    tabs = tb.build_critical_tables(tb.pack_images(imgs, align=1), construction="top")
    for b, img in enumerate(imgs):
        _check(tabs, b, O.critical_tables(img, "top"))


def test_top_full_size_2048(tb):
    """A 2048^2 image (2049^2 corners, rows padded to 2064 bytes, runs of 4096 positions that
    cross rows): tables bit-exact."""
    img = synth.grf((2048, 2048), 16.0, seed=70)
    tabs = tb.build_critical_tables(tb.pack_images([img]), construction="top")
    _check(tabs, 0, O.critical_tables(img, "top"))
