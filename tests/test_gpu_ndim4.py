"""n = 4 through the same C ABI (the generic-n path) against the CPU oracle.

The method is stated for cubical complexes of any dimension (Section 2.1; 2^n sign
vectors, Section 3).  Tables must be bit-exact, ECT and Radon bit-exact, hybrid
transforms within 1e-6 of sum |Delta kbar| (FP32C) or 1e-12 (FP64), gradients within
2e-6 of sum |terms|, exact representations bit-exact.
"""
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
    "bern5x6x7x8": synth.bernoulli((5, 6, 7, 8), 0.5, seed=501),
    "grf9x10x11x12": synth.grf((9, 10, 11, 12), 3.0, seed=502),
    "grf4x5x6x70": synth.grf((4, 5, 6, 70), 2.5, seed=503),
    "const3x3x3x3": np.full((3, 3, 3, 3), 9, dtype=np.uint8),
    "tiny2x2x2x2": np.array(np.arange(16) * 13 % 7, dtype=np.uint8).reshape(2, 2, 2, 2),
    "i32_6x5x4x7": np.random.default_rng(504).integers(-20000, 20000, size=(6, 5, 4, 7)).astype(np.int32),
}


def dirs4(count, seed, lo, hi):
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((count, 4))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    d = g * rng.uniform(lo, hi, size=(count, 1))
    # every orthant, axis-aligned and zero coordinates (+0 and -0)
    extra = np.array([[1, 0, 0, 0], [0, -1, 0, 0], [0, 0, 0.5, -0.0], [-0.0, 0.3, -0.2, 0.1]], dtype=np.float64)
    return np.concatenate([d, extra])


def _check_tables(tabs, b, img):
    ref = O.critical_tables(img)
    for o in range(16):
        idx, val = tabs.table(b, o, 0)
        np.testing.assert_array_equal(idx, ref.lower_idx[o])
        np.testing.assert_array_equal(val, ref.lower_val[o])
        assert tabs.info(b, o)[2] == ref.chi
    for r in range(8):
        idx, val = tabs.table(b, r, 1)
        np.testing.assert_array_equal(idx, ref.delta_idx[r])
        np.testing.assert_array_equal(val, ref.delta_val[r])
    return ref


@pytest.mark.parametrize("name", list(IMAGES))
def test_tables_4d(tb, name):
    img = IMAGES[name]
    _check_tables(tb.build_critical_tables(tb.pack_images([img])), 0, img)


def test_tables_4d_batch(tb):
    imgs = [IMAGES["bern5x6x7x8"], IMAGES["tiny2x2x2x2"], IMAGES["grf9x10x11x12"]]
    tabs = tb.build_critical_tables(tb.pack_images(imgs, align=1))
    for b, img in enumerate(imgs):
        _check_tables(tabs, b, img)


@pytest.mark.parametrize("name", ["bern5x6x7x8", "grf9x10x11x12", "i32_6x5x4x7", "const3x3x3x3"])
@pytest.mark.parametrize("T", [2, 33])
def test_ect_radon_4d(tb, name, T):
    img = IMAGES[name]
    ref = O.critical_tables(img)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    dirs = dirs4(60, 505, 0.1, 2.0)
    d = torch.from_numpy(dirs).cuda()
    R = synth.image_radius(4)
    np.testing.assert_array_equal(tb.ect(tabs, d, -R, R, T).cpu().numpy()[0], O.ect_grid(ref, dirs, -R, R, T))
    np.testing.assert_array_equal(tb.radon(tabs, d, -R, R, T).cpu().numpy()[0], O.radon_grid(ref, dirs, -R, R, T))


def test_ect_4d_exact_ties(tb):
    """Directions and thresholds on the vertex lattice: dot products equal to thresholds."""
    img = IMAGES["grf9x10x11x12"]
    ref = O.critical_tables(img)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    dirs = np.array([[1.0, 1.0, 1.0, 1.0], [1.0, -1.0, 0.0, 2.0], [0.0, 0.0, -3.0, 0.0]])
    d = torch.from_numpy(dirs).cuda()
    for a, b, T in [(-2.0, 2.0, 33), (-1.5, 1.5, 19)]:
        np.testing.assert_array_equal(tb.ect(tabs, d, a, b, T).cpu().numpy()[0], O.ect_grid(ref, dirs, a, b, T))
        np.testing.assert_array_equal(tb.radon(tabs, d, a, b, T).cpu().numpy()[0], O.radon_grid(ref, dirs, a, b, T))


def _fwd_err(got, want, norm, kernel):
    if kernel == "fourier":
        got = got[..., 0] + 1j * got[..., 1]
    return np.max(np.abs(got - want) / np.maximum(norm, 1e-300))


@pytest.mark.parametrize("kernel", ["laplace", "fourier", "bessel", "sine"])
@pytest.mark.parametrize("name", ["bern5x6x7x8", "grf9x10x11x12", "i32_6x5x4x7"])
def test_hybrid_transform_4d(tb, kernel, name):
    img = IMAGES[name]
    ref = O.critical_tables(img)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    dirs = np.concatenate([dirs4(70, 506, 0.01, 1.0), dirs4(30, 507, 2.0, 12.0)])
    d = torch.from_numpy(dirs).cuda()
    want, norm = O.hybrid_transform(ref, kernel, dirs)
    for prec, tol in (("fp32c", 1e-6), ("fp64", 1e-12)):
        got = tb.hybrid_transform(tabs, kernel, d, prec).cpu().numpy()[0]
        assert _fwd_err(got, want, norm, kernel) <= tol, prec


@pytest.mark.parametrize("kernel", ["laplace", "fourier", "bessel", "sine"])
def test_gradient_4d(tb, kernel):
    imgs = [IMAGES["grf9x10x11x12"], IMAGES["bern5x6x7x8"]]
    tabs = tb.build_critical_tables(tb.pack_images(imgs))
    dirs = dirs4(50, 508, 0.1, 3.0)
    D = len(dirs)
    rng = np.random.default_rng(509)
    gout = rng.standard_normal((2, D, 2)) if kernel == "fourier" else rng.standard_normal((2, D))
    d = torch.from_numpy(dirs).cuda()
    want = np.zeros_like(dirs)
    scale = np.zeros_like(dirs)
    for b, img in enumerate(imgs):
        g, gn = O.hybrid_transform_grad(O.critical_tables(img), kernel, dirs)
        if kernel == "fourier":
            want += gout[b, :, 0:1] * g.real + gout[b, :, 1:2] * g.imag
            scale += (np.abs(gout[b, :, 0:1]) + np.abs(gout[b, :, 1:2])) * gn
        else:
            want += gout[b][:, None] * g
            scale += np.abs(gout[b])[:, None] * gn
    for prec, tol in (("fp32c", 2e-6), ("fp64", 1e-11)):
        got = tb.hybrid_transform_grad(tabs, kernel, d, torch.from_numpy(gout).cuda(), prec).cpu().numpy()
        assert np.max(np.abs(got - want) / scale) <= tol, prec


def test_table_kernel_4d(tb):
    img = IMAGES["grf9x10x11x12"]
    ref = O.critical_tables(img)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    s = np.linspace(-1.5, 1.5, 257)
    vals = np.tanh(2.0 * s)
    kt = tb.KernelTable(vals, -1.5, 1.5)
    dirs = dirs4(40, 510, 0.1, 2.0)
    d = torch.from_numpy(dirs).cuda()
    want, norm = O.hybrid_transform(ref, O.table_kernel(vals, -1.5, 1.5), dirs)
    for prec, tol in (("fp32c", 1e-6), ("fp64", 1e-12)):
        got = tb.hybrid_transform(tabs, kt, d, prec).cpu().numpy()[0]
        assert np.max(np.abs(got - want) / norm) <= tol
    kt.free()


def test_exact_representation_4d(tb):
    img = IMAGES["grf9x10x11x12"]
    ref = O.critical_tables(img)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    dirs = dirs4(12, 511, 0.2, 2.0)
    d = torch.from_numpy(dirs).cuda()
    rep = tb.exact_representation(tabs, 0, d)
    rep1 = tb.exact_representation(tabs, 1, d)
    for i, xi in enumerate(dirs):
        T, E = rep.segment(0, i)
        Tw, Ew = O.ect_exact(ref, xi)
        np.testing.assert_array_equal(T, Tw)
        np.testing.assert_array_equal(E, Ew)
        T1, E1 = rep1.segment(0, i)
        Tw1, Ew1 = O.radon_exact(ref, xi)
        np.testing.assert_array_equal(T1, Tw1)
        np.testing.assert_array_equal(E1, Ew1)


def test_4d_errors(tb):
    img = IMAGES["bern5x6x7x8"]
    with pytest.raises(tb.TopotError) as e:
        tb.build_critical_tables(tb.pack_images([img]), construction="top")
    assert e.value.status == 2
    big = np.zeros((3, 3, 3, 3), dtype=np.int32)
    big[1, 1, 1, 1] = 1 << 25     # n = 4 keeps int32 values below 2^25
    with pytest.raises(tb.TopotError) as e:
        tb.build_critical_tables(tb.pack_images([big]))
    assert e.value.status == 5
