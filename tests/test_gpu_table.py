"""Tabulated kernels (kbar given by samples) through the C ABI against the CPU oracle.

The oracle's reading (oracle.table_kernel): piecewise-linear kbar between the samples,
constant outside [s_min, s_max], kappa the segment slope.  Forward within 1e-6 of
sum |Delta kbar| in FP32C for smooth tables (the FP32 table position carries an error
of about 1e-7 (s_max - s_min), so the bound needs |kappa| (s_max - s_min) ~ |kbar|),
1e-12 in FP64 for any table.
"""
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


def _smooth(K, a, b):
    s = a + (b - a) / (K - 1) * np.arange(K)
    return np.sin(2.0 * s) + 0.3 * s * s


def _images():
    return {
        "bern64": synth.bernoulli((64, 64), 0.5, seed=0),
        "grf150x211": synth.grf((150, 211), 6.0, seed=1),
        "grf20x33x64": synth.grf((20, 33, 64), 4.0, seed=7),
        "i32_2d": np.random.default_rng(5).integers(-1000, 1000, size=(50, 70)).astype(np.int32),
    }


IMAGES = _images()


def _dirs(n, count, seed):
    if n == 2:
        return np.concatenate([synth.random_2d_dirs(count, seed, 0.05, 1.5),
                               np.array([[0.0, 1.0], [1.0, -0.0], [1.0, 1.0], [-0.5, 0.25]])])
    return np.concatenate([synth.sphere_dirs(count, seed, 0.05, 1.5), np.array([[0.0, 0.0, 1.0], [0.5, -0.5, 0.0]])])


def _err(got, want, norm):
    return np.max(np.abs(got - want) / np.maximum(norm, 1e-300))


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
@pytest.mark.parametrize("K", [2, 33, 4096, 16384])
@pytest.mark.parametrize("name", list(IMAGES))
def test_table_forward(tb, name, K, precision):
    img = IMAGES[name]
    n = img.ndim
    ref = O.critical_tables(img)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    dirs = _dirs(n, 150, 70 + K)
    # the table covers only part of the dot products: both constant ends are used
    M = 0.5 * 1.5 * n
    a, b = -0.8 * M, 0.9 * M
    y = _smooth(K, a, b)
    kt = tb.KernelTable(y, a, b)
    got = tb.hybrid_transform(tabs, kt, torch.from_numpy(dirs).cuda(), precision).cpu().numpy()[0]
    want, norm = O.hybrid_transform(ref, O.table_kernel(y, a, b), dirs)
    assert _err(got, want, norm) <= HT_TOL[precision]
    kt.free()


@pytest.mark.parametrize("dl", [1, 2, 4])
def test_table_forward_tiles_and_rough_samples(tb, dl):
    img = synth.grf((200, 180), 6.0, seed=50)
    ref = O.critical_tables(img)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    tabs.set_tuning(ht_dirs_per_lane=dl, ht_chunk=2048)
    dirs = synth.random_2d_dirs(700, 51, 0.01, 1.0)
    d = torch.from_numpy(dirs).cuda()
    a, b = -0.6, 0.7
    y = _smooth(257, a, b)
    kt = tb.KernelTable(y, a, b)
    got = tb.hybrid_transform(tabs, kt, d).cpu().numpy()[0]
    want, norm = O.hybrid_transform(ref, O.table_kernel(y, a, b), dirs)
    assert _err(got, want, norm) <= 1e-6
    # random samples: FP64 exact to rounding; FP32C within the position error
    # |du| <= 16 K 2^-24 (|u| < 2 K, a few roundings) times the largest sample step, summed over |Delta|
    yr = np.random.default_rng(52).normal(size=50)
    kr = tb.KernelTable(yr, a, b)
    want, norm = O.hybrid_transform(ref, O.table_kernel(yr, a, b), dirs)
    got = tb.hybrid_transform(tabs, kr, d, "fp64").cpu().numpy()[0]
    assert _err(got, want, norm) <= 1e-12
    got = tb.hybrid_transform(tabs, kr, d).cpu().numpy()[0]
    l1 = np.array([np.sum(np.abs(O.oracle._ht_terms(ref, xi)[2])) for xi in dirs], dtype=np.float64)
    bound = 16 * 50 * 2.0 ** -24 * np.max(np.abs(np.diff(yr))) * l1 + 1e-6 * norm
    assert np.all(np.abs(got - want) <= bound)
    kt.free()
    kr.free()


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
@pytest.mark.parametrize("n", [2, 3])
def test_table_gradient(tb, precision, n):
    imgs = [synth.grf((60, 70), 4.0, seed=60), synth.grf((55, 66), 3.0, seed=62)] if n == 2 else \
        [synth.grf((20, 25, 30), 3.0, seed=61)]
    tabs = tb.build_critical_tables(tb.pack_images(imgs))
    B = len(imgs)
    D = 60
    dirs = synth.random_2d_dirs(D, 64, 0.1, 1.0) if n == 2 else synth.sphere_dirs(D, 65, 0.1, 1.0)
    a, b = -0.55 * n, 0.6 * n
    y = _smooth(257, a, b)
    kt = tb.KernelTable(y, a, b)
    gout = np.random.default_rng(63).standard_normal((B, D))
    got = tb.hybrid_transform_grad(tabs, kt, torch.from_numpy(dirs).cuda(), torch.from_numpy(gout).cuda(),
                                   precision).cpu().numpy()
    want = np.zeros_like(dirs)
    scale = np.zeros_like(dirs)
    for bi, img in enumerate(imgs):
        g, gn = O.hybrid_transform_grad(O.critical_tables(img), O.table_kernel(y, a, b), dirs)
        want += gout[bi][:, None] * g
        scale += np.abs(gout[bi])[:, None] * gn
    # FP32C: a dot product within the position error of a knot may take the neighbouring
    # slope; for samples of a smooth kbar the two slopes differ by about h max|kbar''|
    tol = 1e-10 if precision == "fp64" else 2e-5
    assert np.max(np.abs(got - want) / np.maximum(scale, 1e-300)) <= tol
    kt.free()


def test_table_autograd_and_errors(tb):
    img = synth.grf((40, 50), 3.0, seed=66)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    kt = tb.KernelTable(_smooth(65, -1.0, 1.0), -1.0, 1.0)
    d = torch.from_numpy(synth.random_2d_dirs(20, 67, 0.1, 1.0)).cuda().requires_grad_(True)
    out = tb.HybridTransform.apply(d, tabs, kt, "fp64")
    out.sum().backward()
    g = tb.hybrid_transform_grad(tabs, kt, d.detach(), torch.ones(1, 20, dtype=torch.float64, device="cuda"), "fp64")
    assert torch.equal(d.grad, g)
    # the TABLE kernel id is not accepted without its table
    L = tb.load()
    o = torch.empty(1, 20, dtype=torch.float64, device="cuda")
    st = L.hybrid_transform(tabs.handle, tb.TABLE, 0, tb._ptr(d.detach()), 20, 0, tb._ptr(o), tb._stream(None))
    assert st == 1 and b"TABLE" in L.topot_last_error()
    with pytest.raises(tb.TopotError):
        tb.KernelTable(np.zeros(16385), 0.0, 1.0)
    kt.free()
