"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Tables, ECT and Radon must be bit-exact; hybrid transforms and gradients must be
within 1e-6 of the oracle relative to sum |Delta kbar| (FP32C) or 1e-12 (FP64).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2405_02256_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HT_TOL = {"fp32c": 1e-6, "fp64": 1e-12}


@pytest.fixture(scope="module")
def tb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_02256_gb300 import binding
    binding.load()
    return binding


def _images():
    rng = np.random.default_rng(5)
    return {
        "example4x4": np.array([[1, 0, 0, 0], [0, 1, 1, 0], [1, 1, 1, 1], [1, 1, 0, 0]], dtype=np.uint8),
        "bern64": synth.bernoulli((64, 64), 0.5, seed=0),
        "grf150x211": synth.grf((150, 211), 6.0, seed=1),
        "grf96x256bin": synth.grf((96, 256), 8.0, seed=2, binary=True),
        "wide3x9000": synth.uniform_u8((3, 9000), seed=3),
        "tiny2x2": np.array([[3, 1], [2, 5]], dtype=np.uint8),
        "tall700x5": synth.uniform_u8((700, 5), seed=4),
        "const": np.full((33, 17), 7, dtype=np.uint8),
        "narrow1500x8": synth.uniform_u8((1500, 8), seed=13),
        "narrow1030x9": synth.grf((1030, 9), 3.0, seed=14),
        "grf20x4096": synth.grf((20, 4096), 6.0, seed=15),
        "wide2x4097": synth.uniform_u8((2, 4097), seed=16),
        "bern9x10x11": synth.bernoulli((9, 10, 11), 0.5, seed=6),
        "grf20x33x64": synth.grf((20, 33, 64), 4.0, seed=7),
        "cube2": np.full((2, 2, 2), 1, dtype=np.uint8),
        "wide3d_3x4x1100": synth.uniform_u8((3, 4, 1100), seed=17),     # row pieces, unaligned rows
        "wide3d_2x3x2048": synth.grf((2, 3, 2048), 3.0, seed=18),      # row pieces, aligned rows
        "grf40x40x48bin": synth.grf((40, 40, 48), 5.0, seed=8, binary=True),
        "i32_2d": rng.integers(-1000, 1000, size=(50, 70)).astype(np.int32),
        "i32_3d": rng.integers(-50, 50, size=(12, 13, 14)).astype(np.int32),
    }


IMAGES = _images()


def _check_tables(tabs, b, img):
    ref = O.critical_tables(img)
    n = img.ndim
    for o in range(1 << n):
        idx, val = tabs.table(b, o, 0)
        np.testing.assert_array_equal(idx, ref.lower_idx[o])
        np.testing.assert_array_equal(val, ref.lower_val[o])
        _, _, chi = tabs.info(b, o)
        assert chi == ref.chi
    for r in range(1 << (n - 1)):
        idx, val = tabs.table(b, r, 1)
        np.testing.assert_array_equal(idx, ref.delta_idx[r])
        np.testing.assert_array_equal(val, ref.delta_val[r])
    return ref


@pytest.mark.parametrize("name", list(IMAGES))
def test_tables_bit_exact(tb, name):
    img = IMAGES[name]
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    _check_tables(tabs, 0, img)


def test_tables_ragged_batch(tb):
    shapes = synth.ragged_shapes(37, 2, 90, seed=11)
    imgs = [synth.blurred_noise(s, 2.0, seed=100 + i) for i, s in enumerate(shapes)]
    imgs[3] = synth.bernoulli(imgs[3].shape, 0.5, seed=9)
    tabs = tb.build_critical_tables(tb.pack_images(imgs, align=1))   # unaligned starts too
    for b, img in enumerate(imgs):
        _check_tables(tabs, b, img)


def test_tables_unaligned_pixel_buffer(tb):
    # whole rows 16-byte aligned relative to the buffer, but the buffer itself starts one
    # byte past a 16-byte boundary: the staging falls back from bulk copies to plain loads
    imgs = [synth.grf((40, 64), 4.0, seed=90), synth.grf((6, 10, 32), 3.0, seed=91)]
    for img in imgs:
        b = tb.pack_images([img])
        px = torch.zeros(b.pixels.numel() + 1, dtype=torch.uint8, device="cuda")
        px[1:] = b.pixels
        tabs = tb.tables_create(b.shapes, b.offsets)
        tabs.build(px[1:])
        tabs.sync()
        _check_tables(tabs, 0, img)


def _dirs_2d():
    d = [synth.circle_dirs(32), synth.random_2d_dirs(40, 3, 0.01, 1.0),
         np.array([[0.0, 1.0], [1.0, 0.0], [-0.0, -1.0], [-1.0, -0.0], [0.0, 0.0], [1.0, 1.0], [1.0, -1.0]])]
    return np.concatenate(d)


def _dirs_3d():
    return np.concatenate([synth.fibonacci_dirs(48), synth.sphere_dirs(20, 4, 0.05, 2.0),
                           np.array([[0.0, 0.0, 1.0], [1.0, 0.0, -0.0], [0.5, -0.5, 0.0]])])


@pytest.mark.parametrize("name", ["example4x4", "bern64", "grf150x211", "wide3x9000", "tiny2x2", "const",
                                  "bern9x10x11", "grf20x33x64", "i32_2d", "i32_3d"])
@pytest.mark.parametrize("T", [64, 2, 301])
def test_ect_radon_bit_exact(tb, name, T):
    img = IMAGES[name]
    n = img.ndim
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    ref = O.critical_tables(img)
    dirs = _dirs_2d() if n == 2 else _dirs_3d()
    R = synth.image_radius(n)
    d = torch.from_numpy(dirs).cuda()
    got = tb.ect(tabs, d, -R, R, T).cpu().numpy()[0]
    np.testing.assert_array_equal(got, O.ect_grid(ref, dirs, -R, R, T))
    got = tb.radon(tabs, d, -R, R, T).cpu().numpy()[0]
    np.testing.assert_array_equal(got, O.radon_grid(ref, dirs, -R, R, T))


def test_ect_exact_ties(tb):
    """Lattice directions whose dot products hit thresholds in exact arithmetic."""
    img = synth.bernoulli((65, 65), 0.5, seed=12)
    ref = O.critical_tables(img)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    dirs = np.array([[1.0, 1.0], [1.0, -1.0], [-2.0, 2.0], [3.0, 0.0], [0.0, -0.5], [0.25, 0.75]])
    d = torch.from_numpy(dirs).cuda()
    for (a, b, T) in [(-1.0, 1.0, 129), (-2.0, 2.0, 257), (-0.5, 0.75, 81)]:
        np.testing.assert_array_equal(tb.ect(tabs, d, a, b, T).cpu().numpy()[0], O.ect_grid(ref, dirs, a, b, T))
        np.testing.assert_array_equal(tb.radon(tabs, d, a, b, T).cpu().numpy()[0],
                                      O.radon_grid(ref, dirs, a, b, T))


def test_ect_per_image_directions(tb):
    imgs = [synth.grf((40 + 3 * i, 50 - 2 * i), 4.0, seed=20 + i) for i in range(5)]
    tabs = tb.build_critical_tables(tb.pack_images(imgs))
    dirs = np.stack([synth.random_2d_dirs(24, 30 + i, 0.1, 2.0) for i in range(5)])
    d = torch.from_numpy(dirs).cuda()
    got_e = tb.ect(tabs, d, -0.8, 0.8, 33).cpu().numpy()
    got_r = tb.radon(tabs, d, -0.8, 0.8, 33).cpu().numpy()
    for b, img in enumerate(imgs):
        ref = O.critical_tables(img)
        np.testing.assert_array_equal(got_e[b], O.ect_grid(ref, dirs[b], -0.8, 0.8, 33))
        np.testing.assert_array_equal(got_r[b], O.radon_grid(ref, dirs[b], -0.8, 0.8, 33))


@pytest.mark.parametrize("td", [8, 16, 32, 64])
def test_ect_tile_shapes(tb, td):
    img = synth.grf((120, 130), 5.0, seed=40)
    ref = O.critical_tables(img)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    tabs.set_tuning(ect_dirs_per_warp=td, ect_chunk=1024)
    dirs = synth.random_2d_dirs(70, 41, 0.2, 1.5)
    d = torch.from_numpy(dirs).cuda()
    np.testing.assert_array_equal(tb.ect(tabs, d, -1, 1, 50).cpu().numpy()[0], O.ect_grid(ref, dirs, -1, 1, 50))
    np.testing.assert_array_equal(tb.radon(tabs, d, -1, 1, 50).cpu().numpy()[0],
                                  O.radon_grid(ref, dirs, -1, 1, 50))


def _ht_err(got, want, norm, kernel):
    if kernel == "fourier":
        got = got[..., 0] + 1j * got[..., 1]
    return np.max(np.abs(got - want) / np.maximum(norm, 1e-300))


@pytest.mark.parametrize("kernel", ["laplace", "fourier", "bessel", "sine"])
@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
@pytest.mark.parametrize("name", ["example4x4", "bern64", "grf150x211", "grf20x33x64", "i32_2d", "bern9x10x11"])
def test_hybrid_transform(tb, kernel, precision, name):
    img = IMAGES[name]
    n = img.ndim
    ref = O.critical_tables(img)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    dirs = _dirs_2d() if n == 2 else _dirs_3d()
    d = torch.from_numpy(dirs).cuda()
    got = tb.hybrid_transform(tabs, kernel, d, precision).cpu().numpy()[0]
    want, norm = O.hybrid_transform(ref, kernel, dirs)
    assert _ht_err(got, want, norm, kernel) <= HT_TOL[precision]


@pytest.mark.parametrize("dl,split", [(1, 1), (2, 1), (4, 1), (8, 1), (2, 2), (4, 2)])
def test_hybrid_transform_tiles(tb, dl, split):
    img = synth.grf((200, 180), 6.0, seed=50)
    ref = O.critical_tables(img)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    tabs.set_tuning(ht_dirs_per_lane=dl, ht_chunk=2048, ht_warp_split=split)
    dirs = synth.random_2d_dirs(1100, 51, 0.01, 1.0)
    d = torch.from_numpy(dirs).cuda()
    for kernel in ("laplace", "fourier", "bessel", "sine") if dl < 8 else ("laplace",):
        got = tb.hybrid_transform(tabs, kernel, d).cpu().numpy()[0]
        want, norm = O.hybrid_transform(ref, kernel, dirs)
        assert _ht_err(got, want, norm, kernel) <= 1e-6


def test_hybrid_transform_worked_example(tb, golden):
    img = np.array(golden["image"], dtype=np.uint8)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    d = torch.tensor([golden["ect"]["xi"]], dtype=torch.float64, device="cuda")
    v = tb.hybrid_transform(tabs, "laplace", d, "fp64").item()
    assert abs(v - (2 * math.exp(-2 / 3) - math.exp(2 / 3) - math.exp(4 / 3))) < 1e-12
    assert abs(v - golden["hybrid_transform"]["value_printed"]) < 5e-4


@pytest.mark.parametrize("kernel", ["laplace", "fourier", "bessel", "sine"])
@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
@pytest.mark.parametrize("per_image", [False, True])
def test_gradient(tb, kernel, precision, per_image):
    imgs = [synth.grf((60, 70), 4.0, seed=60), synth.grf((20, 25, 30), 3.0, seed=61)][:1]
    imgs = [imgs[0], synth.grf((55, 66), 3.0, seed=62)]
    tabs = tb.build_critical_tables(tb.pack_images(imgs))
    B = len(imgs)
    rng = np.random.default_rng(63)
    if per_image:
        dirs = np.stack([synth.random_2d_dirs(50, 64 + b, 0.1, 1.0) for b in range(B)])
    else:
        dirs = synth.random_2d_dirs(50, 64, 0.1, 1.0)
    D = 50
    nc = 2 if kernel == "fourier" else 1
    gout = rng.standard_normal((B, D, nc)) if nc == 2 else rng.standard_normal((B, D))
    d = torch.from_numpy(dirs).cuda()
    got = tb.hybrid_transform_grad(tabs, kernel, d, torch.from_numpy(gout).cuda(), precision).cpu().numpy()
    want = np.zeros_like(dirs)
    scale = np.zeros_like(dirs)
    for b, img in enumerate(imgs):
        ref = O.critical_tables(img)
        db = dirs[b] if per_image else dirs
        g, gn = O.hybrid_transform_grad(ref, kernel, db)
        if kernel == "fourier":
            contrib = gout[b, :, 0:1] * g.real + gout[b, :, 1:2] * g.imag
            sc = (np.abs(gout[b, :, 0:1]) + np.abs(gout[b, :, 1:2])) * gn
        else:
            contrib = gout[b][:, None] * g
            sc = np.abs(gout[b])[:, None] * gn
        if per_image:
            want[b] += contrib
            scale[b] += sc
        else:
            want += contrib
            scale += sc
    assert np.max(np.abs(got - want) / scale) <= 2 * HT_TOL[precision]


@pytest.mark.parametrize("dl", [1, 2, 4])
def test_gradient_tiles(tb, dl):
    # the adjoint at every number of directions per lane (Fourier stops at one pair)
    img = synth.grf((90, 80), 4.0, seed=68)
    ref = O.critical_tables(img)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    tabs.set_tuning(ht_dirs_per_lane=dl, ht_chunk=1024)
    dirs = synth.random_2d_dirs(600, 69, 0.05, 1.0)
    rng = np.random.default_rng(70)
    d = torch.from_numpy(dirs).cuda()
    for kernel in ("laplace", "fourier", "bessel", "sine"):
        nc = 2 if kernel == "fourier" else 1
        gout = rng.standard_normal((1, 600, 2)) if nc == 2 else rng.standard_normal((1, 600))
        got = tb.hybrid_transform_grad(tabs, kernel, d, torch.from_numpy(gout).cuda()).cpu().numpy()
        g, gn = O.hybrid_transform_grad(ref, kernel, dirs)
        if kernel == "fourier":
            want = gout[0, :, 0:1] * g.real + gout[0, :, 1:2] * g.imag
            sc = (np.abs(gout[0, :, 0:1]) + np.abs(gout[0, :, 1:2])) * gn
        else:
            want = gout[0][:, None] * g
            sc = np.abs(gout[0])[:, None] * gn
        assert np.max(np.abs(got - want) / sc) <= 2e-6, kernel


def test_autograd_function(tb):
    img = synth.grf((50, 40), 4.0, seed=70)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    dirs = torch.from_numpy(synth.random_2d_dirs(16, 71, 0.2, 1.0)).cuda().requires_grad_(True)
    target = torch.from_numpy(synth.perturb(dirs.detach().cpu().numpy(), 0.05, 72)).cuda()
    ht = tb.HybridTransform.apply(dirs, tabs, "laplace", "fp32c")
    with torch.no_grad():
        ht_t = tb.hybrid_transform(tabs, "laplace", target)
    loss = ((ht - ht_t) ** 2).sum()
    loss.backward()
    g_direct = tb.hybrid_transform_grad(tabs, "laplace", dirs.detach(), 2 * (ht - ht_t).detach())
    torch.testing.assert_close(dirs.grad, g_direct, rtol=1e-12, atol=1e-12)


def test_errors_are_reported(tb):
    img = synth.bernoulli((8, 8), 0.5, seed=1)
    batch = tb.pack_images([img])
    tabs = tb.build_critical_tables(batch)
    d = torch.zeros((3, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(tb.TopotError) as e:
        tb.ect(tabs, d, 1.0, -1.0, 10)
    assert e.value.status == 1
    with pytest.raises(tb.TopotError):
        tb.ect(tabs, d, -1.0, 1.0, 1)
    bad = tb.ImageBatch(batch.pixels, np.array([[1, 64]]), np.array([0]))
    with pytest.raises(tb.TopotError) as e:
        tb.build_critical_tables(bad)
    assert e.value.status == 1


def test_int32_range_check(tb):
    img = np.zeros((8, 8), dtype=np.int32)
    img[3, 3] = 1 << 27
    with pytest.raises(tb.TopotError) as e:
        tb.build_critical_tables(tb.pack_images([img]))
    assert e.value.status == 5


def test_rebuild_async_and_deterministic(tb):
    imgs = [synth.grf((128, 128), 5.0, seed=80), synth.grf((128, 128), 5.0, seed=81)]
    b0 = tb.pack_images([imgs[0]])
    b1 = tb.pack_images([imgs[1]])
    tabs = tb.tables_create(b0.shapes, b0.offsets)
    tabs.build(b1.pixels)
    tabs.sync()
    _check_tables(tabs, 0, imgs[1])
    tabs.build(b0.pixels)
    dirs = torch.from_numpy(synth.random_2d_dirs(64, 82, 0.01, 1.0)).cuda()
    h1 = tb.hybrid_transform(tabs, "fourier", dirs)
    h2 = tb.hybrid_transform(tabs, "fourier", dirs)
    assert torch.equal(h1, h2)
    tabs.sync()
    _check_tables(tabs, 0, imgs[0])


@pytest.mark.parametrize("kernel", ["laplace", "fourier", "bessel", "sine"])
def test_gradient_3d(tb, kernel):
    img = synth.grf((18, 21, 24), 3.0, seed=65)
    ref = O.critical_tables(img)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    dirs = synth.sphere_dirs(160, 66, 0.1, 1.0)
    rng = np.random.default_rng(67)
    nc = 2 if kernel == "fourier" else 1
    gout = rng.standard_normal((1, 160, 2)) if nc == 2 else rng.standard_normal((1, 160))
    got = tb.hybrid_transform_grad(tabs, kernel, torch.from_numpy(dirs).cuda(),
                                   torch.from_numpy(gout).cuda()).cpu().numpy()
    g, gn = O.hybrid_transform_grad(ref, kernel, dirs)
    if kernel == "fourier":
        want = gout[0, :, 0:1] * g.real + gout[0, :, 1:2] * g.imag
        sc = (np.abs(gout[0, :, 0:1]) + np.abs(gout[0, :, 1:2])) * gn
    else:
        want = gout[0][:, None] * g
        sc = np.abs(gout[0])[:, None] * gn
    assert np.max(np.abs(got - want) / sc) <= 2e-6
