"""Slabs of a volume (Section 5.3: parallelisation over vertex subsets) through the C ABI.

A slab handle's tables are the volume's tables restricted to the slab's planes (the
lower-star values depend on the 3^n neighbourhood in the whole volume), so they are
checked bit for bit against the oracle's tables of the whole volume filtered by plane.
The slabs' ECT and Radon parts, added by slab_sum, equal the volume's bit for bit; the
hybrid transforms and gradients are within the parity tolerance of the oracle.
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


@pytest.fixture(scope="module")
def sl(tb):
    from paper_2405_02256_gb300 import slabs
    return slabs


VOLUMES = {
    "bern9x10x11": synth.bernoulli((9, 10, 11), 0.5, seed=401),
    "grf20x33x64": synth.grf((20, 33, 64), 4.0, seed=402),
    "grf40x40x48bin": synth.grf((40, 40, 48), 5.0, seed=403, binary=True),
    "wide3x4x1100": synth.uniform_u8((3, 4, 1100), seed=404),
    "i32_12x13x14": np.random.default_rng(405).integers(-50, 50, size=(12, 13, 14)).astype(np.int32),
}


def restrict(ref, z0, z1):
    """The oracle's tables of the whole volume restricted to planes [z0, z1)."""
    m0, m1 = ref.m[0], ref.m[1]
    lo, hi = z0 * m0 * m1, z1 * m0 * m1
    out = O.CriticalTables(shape=ref.shape)
    for idx, val in zip(ref.lower_idx, ref.lower_val):
        k = (idx >= lo) & (idx < hi)
        out.lower_idx.append(idx[k])
        out.lower_val.append(val[k])
    for idx, val in zip(ref.delta_idx, ref.delta_val):
        k = (idx >= lo) & (idx < hi)
        out.delta_idx.append(idx[k])
        out.delta_val.append(val[k])
    out.chi = int(out.lower_val[0].sum())
    return out


def partitions(depth):
    cuts = {1: [(0, depth)], 2: [(0, depth // 2), (depth // 2, depth)]}
    if depth >= 3:
        cuts[3] = [(0, 1), (1, depth - 1), (depth - 1, depth)]   # one-plane slabs at both ends
    return list(cuts.values())


@pytest.mark.parametrize("name", list(VOLUMES))
def test_slab_tables_bit_exact(tb, sl, name):
    vol = VOLUMES[name]
    ref = O.critical_tables(vol)
    for ranges in partitions(vol.shape[0]):
        tabs = sl.build_slab_tables(vol, ranges)
        for b, (z0, z1) in enumerate(ranges):
            want = restrict(ref, z0, z1)
            for o in range(8):
                idx, val = tabs.table(b, o, 0)
                np.testing.assert_array_equal(idx, want.lower_idx[o])
                np.testing.assert_array_equal(val, want.lower_val[o])
                assert tabs.info(b, o)[2] == want.chi
            for r in range(4):
                idx, val = tabs.table(b, r, 1)
                np.testing.assert_array_equal(idx, want.delta_idx[r])
                np.testing.assert_array_equal(val, want.delta_val[r])


@pytest.mark.parametrize("name", list(VOLUMES))
def test_slab_transforms_sum_to_volume(tb, sl, name):
    vol = VOLUMES[name]
    ref = O.critical_tables(vol)
    dirs = np.concatenate([synth.fibonacci_dirs(40), synth.sphere_dirs(24, 406, 0.05, 2.0),
                           np.array([[0.0, 0.0, 1.0], [1.0, -0.0, 0.0]])])
    d = torch.from_numpy(dirs).cuda()
    R = synth.image_radius(3)
    ect_w = O.ect_grid(ref, dirs, -R, R, 33)
    rad_w = O.radon_grid(ref, dirs, -R, R, 33)
    for ranges in partitions(vol.shape[0])[1:]:
        tabs = sl.build_slab_tables(vol, ranges)
        got = tb.slab_sum(tb.ect(tabs, d, -R, R, 33)).cpu().numpy()
        np.testing.assert_array_equal(got, ect_w)
        got = tb.slab_sum(tb.radon(tabs, d, -R, R, 33)).cpu().numpy()
        np.testing.assert_array_equal(got, rad_w)
        for kernel in ("laplace", "fourier", "bessel", "sine"):
            want, norm = O.hybrid_transform(ref, kernel, dirs)
            for prec, tol in (("fp32c", 1e-6), ("fp64", 1e-12)):
                got = tb.slab_sum(tb.hybrid_transform(tabs, kernel, d, prec)).cpu().numpy()
                if kernel == "fourier":
                    got = got[..., 0] + 1j * got[..., 1]
                assert np.max(np.abs(got - want) / norm) <= tol, (kernel, prec)
        # the gradient: with shared directions the slabs (images) are summed by the call
        gout = torch.ones((len(ranges), len(dirs)), dtype=torch.float64, device="cuda")
        got = tb.hybrid_transform_grad(tabs, "laplace", d, gout).cpu().numpy()
        g, gn = O.hybrid_transform_grad(ref, "laplace", dirs)
        assert np.max(np.abs(got - g) / gn) <= 2e-6


def test_slab_errors(tb):
    shapes = np.array([[8, 8, 8]])
    with pytest.raises(tb.TopotError):
        tb.tables_create_slab(shapes, [0], [[3, 3]])          # empty slab
    with pytest.raises(tb.TopotError):
        tb.tables_create_slab(shapes, [0], [[0, 9]])          # beyond the volume
    with pytest.raises(tb.TopotError):
        tb.tables_create_slab(np.array([[8, 8]]), [0], [[0, 4]])   # 2-D
    parts = torch.full((3, 5), 2 ** 30, dtype=torch.int32, device="cuda")
    with pytest.raises(tb.TopotError) as e:
        tb.slab_sum(parts)
    assert e.value.status == 5


def test_slabs_256_cube(tb, sl):
    """The 256^3 binary GRF volume of the volume workload in 4 slabs;
    ECT and Radon at 2048 Fibonacci directions x 256 thresholds bit-exact against the
    whole volume, Fourier at 8192 directions within 2e-6 of the whole volume's FP32C
    result relative to sum |Delta kbar| (the oracle's, on 96 sampled directions, within 1e-6)."""
    vol = synth.grf((256, 256, 256), 8.0, seed=410, binary=True)
    whole = tb.build_critical_tables(tb.pack_images([vol]))
    tabs = sl.build_slab_tables(vol, sl.slab_bounds(256, 4))
    dirs_e = torch.from_numpy(synth.fibonacci_dirs(2048)).cuda()
    R = synth.image_radius(3)
    for f in (tb.ect, tb.radon):
        want = f(whole, dirs_e, -R, R, 256)[0]
        got = tb.slab_sum(f(tabs, dirs_e, -R, R, 256))
        assert torch.equal(got, want)
    dirs_h_np = synth.scale_norms(synth.fibonacci_dirs(8192), 411, 0.05, 2.0)
    dirs_h = torch.from_numpy(dirs_h_np).cuda()
    got = tb.slab_sum(tb.hybrid_transform(tabs, "fourier", dirs_h)).cpu().numpy()
    whole_h = tb.hybrid_transform(whole, "fourier", dirs_h)[0].cpu().numpy()
    ref = O.critical_tables(vol)
    sample = np.random.default_rng(412).choice(8192, 96, replace=False)
    want, norm = O.hybrid_transform(ref, "fourier", dirs_h_np[sample])
    g = got[sample, 0] + 1j * got[sample, 1]
    w = whole_h[sample, 0] + 1j * whole_h[sample, 1]
    assert np.max(np.abs(g - want) / norm) <= 1e-6
    assert np.max(np.abs(g - w) / norm) <= 2e-6
