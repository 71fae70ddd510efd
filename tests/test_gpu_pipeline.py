"""Ragged batches in one persistent launch per operation, replayed as a CUDA graph, and
the autotuner (GPU).  Results are compared with eager calls and with the CPU oracle."""
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


def _ragged(count, seed, lo=28, hi=160):
    shapes = synth.ragged_shapes(count, lo, hi, seed=seed)
    return [synth.blurred_noise(s, 2.0, seed=seed * 1000 + i) for i, s in enumerate(shapes)]


def _pipeline(tb, imgs, ect_dirs, ht_dirs, T=64, ktab=None):
    batch = tb.pack_images(imgs)
    R = synth.image_radius(2)
    hybrid = [("laplace", ht_dirs, "fp32c"), ("fourier", ht_dirs, "fp32c")]
    if ktab is not None:
        hybrid.append((ktab, ht_dirs, "fp32c"))
    pipe = tb.Pipeline(batch.shapes, batch.offsets, batch.pixels.numel(),
                       ect=(ect_dirs, -R, R, T), radon=(ect_dirs, -R, R, T), hybrid=hybrid)
    return pipe, batch


def test_graph_replay_matches_eager_and_follows_new_pixels(tb):
    imgs_a = _ragged(60, 1)
    imgs_b = [synth.blurred_noise(im.shape, 2.0, seed=7000 + i) for i, im in enumerate(imgs_a)]
    ect_dirs = torch.from_numpy(synth.circle_dirs(64)).cuda()
    ht_dirs = torch.from_numpy(synth.circle_dirs(256)).cuda()
    knots = np.linspace(-0.8, 0.8, 129)
    ktab = tb.KernelTable(np.exp(-4.0 * knots * knots), -0.8, 0.8)   # a tabulated kernel in the graph too
    pipe, batch_a = _pipeline(tb, imgs_a, ect_dirs, ht_dirs, ktab=ktab)
    batch_b = tb.pack_images(imgs_b)
    pipe.pixels.copy_(batch_a.pixels)
    pipe.capture()
    R = synth.image_radius(2)
    for batch in (batch_a, batch_b, batch_a):
        pipe.run(batch.pixels)
        torch.cuda.synchronize()
        eager = tb.build_critical_tables(batch)
        assert torch.equal(pipe.ect_out, tb.ect(eager, ect_dirs, -R, R, 64))
        assert torch.equal(pipe.radon_out, tb.radon(eager, ect_dirs, -R, R, 64))
        assert torch.equal(pipe.hybrid_out[0], tb.hybrid_transform(eager, "laplace", ht_dirs))
        assert torch.equal(pipe.hybrid_out[1], tb.hybrid_transform(eager, "fourier", ht_dirs))
        assert torch.equal(pipe.hybrid_out[2], tb.hybrid_transform(eager, ktab, ht_dirs))


def test_ragged_batch_against_oracle(tb):
    """Ragged grey-level images (sides log-uniform in [28, 160]), ECT 64 x 64 and Laplace
    at 256 unit directions for every image, through the captured graph."""
    imgs = _ragged(90, 2)
    ect_np = synth.circle_dirs(64)
    ht_np = synth.random_2d_dirs(256, 3, 1.0, 1.0 + 1e-12)
    pipe, batch = _pipeline(tb, imgs, torch.from_numpy(ect_np).cuda(), torch.from_numpy(ht_np).cuda())
    pipe.pixels.copy_(batch.pixels)
    pipe.capture().run()
    torch.cuda.synchronize()
    R = synth.image_radius(2)
    ect = pipe.ect_out.cpu().numpy()
    rad = pipe.radon_out.cpu().numpy()
    lap = pipe.hybrid_out[0].cpu().numpy()
    for b, img in enumerate(imgs):
        ref = O.critical_tables(img)
        np.testing.assert_array_equal(ect[b], O.ect_grid(ref, ect_np, -R, R, 64))
        np.testing.assert_array_equal(rad[b], O.radon_grid(ref, ect_np, -R, R, 64))
        want, norm = O.hybrid_transform(ref, "laplace", ht_np)
        assert np.max(np.abs(lap[b] - want) / norm) <= 1e-6


def test_autotuner_picks_a_valid_tuning(tb, tmp_path, monkeypatch):
    from paper_2405_02256_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "cache.json"))
    img = synth.grf((300, 280), 6.0, seed=4)
    ref = O.critical_tables(img)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    dirs_np = synth.random_2d_dirs(512, 5, 0.05, 1.0)
    dirs = torch.from_numpy(dirs_np).cuda()
    best = autotune.tune(tabs, "hybrid", dirs, kernel="fourier",
                         space=[dict(ht_dirs_per_lane=d, ht_chunk=c, ht_ctas_per_sm=0) for d in (2, 4) for c in (0, 4096)])
    assert best["tuning"]["ht_dirs_per_lane"] in (2, 4) and tabs.tuning["ht_dirs_per_lane"] in (2, 4)
    got = tb.hybrid_transform(tabs, "fourier", dirs).cpu().numpy()[0]
    want, norm = O.hybrid_transform(ref, "fourier", dirs_np)
    assert np.max(np.abs(got[:, 0] + 1j * got[:, 1] - want) / norm) <= 1e-6
    best = autotune.tune(tabs, "ect", dirs, T=40, t_min=-0.7, t_max=0.7,
                         space=[dict(ect_dirs_per_warp=d, ect_chunk=0, ect_ctas_per_sm=0) for d in (16, 32)])
    np.testing.assert_array_equal(tb.ect(tabs, dirs, -0.7, 0.7, 40).cpu().numpy()[0],
                                  O.ect_grid(ref, dirs_np, -0.7, 0.7, 40))
    again = autotune.tune(tabs, "ect", dirs, T=40, t_min=-0.7, t_max=0.7)   # from the cache
    assert again["tuning"] == best["tuning"]
