"""The 10,000-image ragged batch at full size, in the launch configuration bench.py times:
10,000 ragged grey images (sides 28-512) in one CUDA graph with tuned tiles, ECT at 64
directions x 64 thresholds and Laplace at 256 directions (FP32C).  Sampled images --
the largest, the smallest and random ones -- are checked against the oracle: tables and
ECT bit-exact, Laplace within 1e-6 of sum |Delta kbar|."""
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


def test_ragged_10000_in_bench_configuration(tb):
    import bench
    imgs, ect_h, ht_h = bench.ragged_workload()
    batch = tb.pack_images(imgs)
    pipe = bench.ragged_pipeline(tb, batch, ect_h, ht_h, "cuda")
    pipe.run()                       # a replay of the captured graph
    torch.cuda.synchronize()
    pipe.tables.sync()
    sizes = np.array([im.size for im in imgs])
    rng = np.random.default_rng(600)
    sample = sorted({int(np.argmax(sizes)), int(np.argmin(sizes)), *rng.choice(len(imgs), 14, replace=False).tolist()})
    ect_all = pipe.ect_out.cpu().numpy()
    ht_all = pipe.hybrid_out[0].cpu().numpy()
    R = synth.image_radius(2)
    for b in sample:
        ref = O.critical_tables(imgs[b])
        for o in range(4):
            idx, val = pipe.tables.table(b, o, 0)
            np.testing.assert_array_equal(idx, ref.lower_idx[o])
            np.testing.assert_array_equal(val, ref.lower_val[o])
        np.testing.assert_array_equal(ect_all[b], O.ect_grid(ref, ect_h, -R, R, 64))
        want, norm = O.hybrid_transform(ref, "laplace", ht_h)
        assert np.max(np.abs(ht_all[b] - want) / norm) <= 1e-6, b
    assert set(pipe.tuned) == {"ect", "laplace"}
