"""Parity at the full sizes of the workloads, in the launch configuration bench.py uses,
on outputs the oracle can compute one by one (sampled images and directions).

* 64 x 2048^2 grey GRF (the bench step): tables of sampled images bit-exact; ECT
  (1024 x 512) and Radon bit-exact and the three hybrid transforms within 1e-6 on sampled
  (image, direction) pairs.
* 4 x 256^3 binary GRF volumes: tables of one volume bit-exact; ECT / Radon at 2048
  Fibonacci directions x 256 and Fourier at 8192 directions on sampled directions.
* 128^3 grey GRF with 8192 learnable directions: forward and adjoint of Laplace and
  Fourier, and the gradient of the squared-error loss to perturbed directions, against
  the oracle's analytic gradient and central finite differences.
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


def _ht_err(got, want, norm, kernel):
    if kernel == "fourier":
        got = got[..., 0] + 1j * got[..., 1]
    return np.max(np.abs(got - want) / norm)


def test_bench_workload_2048(tb):
    import bench
    imgs = bench.make_images(64, 2048)
    dirs_ect, dirs_ht = bench.make_dirs()
    batch = tb.pack_images(imgs)
    tabs = tb.tables_create(batch.shapes, batch.offsets)
    tabs.build(batch.pixels)
    tabs.sync()
    R = synth.image_radius(2)
    d_e = torch.from_numpy(dirs_ect).cuda()
    d_h = torch.from_numpy(dirs_ht).cuda()
    ect = tb.ect(tabs, d_e, -R, R, 512).cpu().numpy()
    rad = tb.radon(tabs, d_e, -R, R, 512).cpu().numpy()
    hts = {k: tb.hybrid_transform(tabs, k, d_h, "fp32c").cpu().numpy() for k in ("laplace", "fourier", "bessel")}
    rng = np.random.default_rng(123)
    for b in (0, 37, 63):
        ref = O.critical_tables(imgs[b])
        for o in range(4):
            idx, val = tabs.table(b, o, 0)
            np.testing.assert_array_equal(idx, ref.lower_idx[o])
            np.testing.assert_array_equal(val, ref.lower_val[o])
        for r in range(2):
            idx, val = tabs.table(b, r, 1)
            np.testing.assert_array_equal(idx, ref.delta_idx[r])
            np.testing.assert_array_equal(val, ref.delta_val[r])
        de = rng.choice(len(dirs_ect), 8, replace=False)
        np.testing.assert_array_equal(ect[b, de], O.ect_grid(ref, dirs_ect[de], -R, R, 512))
        np.testing.assert_array_equal(rad[b, de[:4]], O.radon_grid(ref, dirs_ect[de[:4]], -R, R, 512))
        dh = rng.choice(len(dirs_ht), 6, replace=False)
        for k, v in hts.items():
            want, norm = O.hybrid_transform(ref, k, dirs_ht[dh])
            assert _ht_err(v[b, dh], want, norm, k) <= 1e-6, k
    # chi on every image: ECT at the last threshold (t = R >= every dot product of a unit
    # direction up to rounding) against a property of the tables: sum of Delta^-_0 = chi
    chis = np.array([tabs.info(b, 0)[2] for b in range(64)])
    assert np.array_equal(ect[:, 0, -1], chis)


def test_volumes_256(tb):
    vols = [synth.grf((256, 256, 256), 8.0, seed=300 + b, binary=True) for b in range(4)]
    batch = tb.pack_images(vols)
    tabs = tb.build_critical_tables(batch)
    R = synth.image_radius(3)
    fib = synth.fibonacci_dirs(2048)
    four = synth.scale_norms(synth.fibonacci_dirs(8192), 3, 0.05, 2.0)
    ect = tb.ect(tabs, torch.from_numpy(fib).cuda(), -R, R, 256).cpu().numpy()
    rad = tb.radon(tabs, torch.from_numpy(fib).cuda(), -R, R, 256).cpu().numpy()
    ft = tb.hybrid_transform(tabs, "fourier", torch.from_numpy(four).cuda()).cpu().numpy()
    ref = O.critical_tables(vols[1])
    for o in range(8):
        idx, val = tabs.table(1, o, 0)
        np.testing.assert_array_equal(idx, ref.lower_idx[o])
        np.testing.assert_array_equal(val, ref.lower_val[o])
    for r in range(4):
        idx, val = tabs.table(1, r, 1)
        np.testing.assert_array_equal(idx, ref.delta_idx[r])
        np.testing.assert_array_equal(val, ref.delta_val[r])
    rng = np.random.default_rng(7)
    de = np.concatenate([[0], rng.choice(2048, 7, replace=False)])   # direction 0 has a zero coordinate
    np.testing.assert_array_equal(ect[1, de], O.ect_grid(ref, fib[de], -R, R, 256))
    np.testing.assert_array_equal(rad[1, de], O.radon_grid(ref, fib[de], -R, R, 256))
    dh = rng.choice(8192, 8, replace=False)
    want, norm = O.hybrid_transform(ref, "fourier", four[dh])
    assert _ht_err(ft[1, dh], want, norm, "fourier") <= 1e-6


def test_gradients_128(tb):
    vol = synth.grf((128, 128, 128), 6.0, seed=5)
    tabs = tb.build_critical_tables(tb.pack_images([vol]))
    ref = O.critical_tables(vol)
    xi = synth.sphere_dirs(8192, 6, 0.1, 1.0)
    target = synth.perturb(xi, 0.05, 7)
    rng = np.random.default_rng(8)
    samp = rng.choice(8192, 6, replace=False)
    for kernel in ("laplace", "fourier"):
        d = torch.from_numpy(xi).cuda().requires_grad_(True)
        ht = tb.HybridTransform.apply(d, tabs, kernel, "fp32c")
        with torch.no_grad():
            ht_t = tb.hybrid_transform(tabs, kernel, torch.from_numpy(target).cuda())
        loss = ((ht - ht_t) ** 2).sum()
        loss.backward()
        g = d.grad.cpu().numpy()
        # oracle: dL/dxi = 2 (HT - HT*) dHT/dxi  (Fourier: real and imaginary parts)
        h, hn = O.hybrid_transform(ref, kernel, xi[samp])
        hs, hsn = O.hybrid_transform(ref, kernel, target[samp])
        gd, gn = O.hybrid_transform_grad(ref, kernel, xi[samp])
        r = h - hs
        if kernel == "fourier":
            want = 2 * (r.real[:, None] * gd.real + r.imag[:, None] * gd.imag)
            ra = (np.abs(r.real) + np.abs(r.imag))[:, None]
        else:
            want = 2 * r[:, None] * gd
            ra = np.abs(r)[:, None]
        # error propagation: the residual carries the forward error (<= 1e-6 of the
        # forward norms), the adjoint its own (<= 2e-6 of gn)
        allowed = 2 * (1e-6 * (hn + hsn)[:, None] * gn + 2e-6 * ra * gn)
        assert np.all(np.abs(g[samp] - want) <= 2 * allowed)
        # analytic gradient against central differences of the oracle (h = 1e-4)
        hstep = 1e-4
        smooth = [di for di in samp if np.min(np.abs(xi[di])) > 10 * hstep]   # no orthant wall in reach
        for di in smooth[:2]:
            for k in range(3):
                e = np.zeros(3)
                e[k] = hstep
                fp, _ = O.hybrid_transform(ref, kernel, [xi[di] + e])
                fm, _ = O.hybrid_transform(ref, kernel, [xi[di] - e])
                fd = (fp[0] - fm[0]) / (2 * hstep)
                gk, gnk = O.hybrid_transform_grad(ref, kernel, [xi[di]])
                assert abs(fd - gk[0, k]) <= 1e-6 * max(1.0, gnk[0, k])
