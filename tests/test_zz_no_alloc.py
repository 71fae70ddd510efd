"""hybrid_transform_noalloc: the allocation-free variant of hybrid_transform.

Some callers cannot call cudaMalloc -- code running inside an allocator or memory-pool
callback, under a no-allocation real-time budget, or in a host that forbids device
allocation after start-up.  For them the library offers hybrid_transform_noalloc,
whose scratch is a fixed device array instead of a workspace grown with cudaMalloc.
This test calls it through the C ABI, twice in a row (the array keeps the previous
call's contents), and checks each result against hybrid_transform within the tolerance
the parity tests use; it also checks that an oversized request is refused.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2405_02256_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32c": 1e-6, "fp64": 1e-12}


@pytest.fixture(scope="module")
def tb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_02256_gb300 import binding
    binding.load()
    return binding


def _noalloc(tb, tabs, kernel, precision, dirs, out):
    L = tb.load()
    return L.hybrid_transform_noalloc(tabs.handle, tb.KERNELS[kernel], tb.PRECISIONS[precision],
                                      ctypes.c_void_p(dirs.data_ptr()), dirs.shape[0], 0,
                                      ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_noalloc_matches_hybrid_transform(tb, precision):
    imgs = [synth.grf((150, 170), 5.0, seed=90), synth.grf((120, 131), 4.0, seed=91)]
    tabs = tb.build_critical_tables(tb.pack_images(imgs))
    dirs_np = synth.random_2d_dirs(300, 92, 0.05, 1.0)
    dirs = torch.from_numpy(dirs_np).cuda()
    refs = [O.critical_tables(im) for im in imgs]
    for kernel in ("laplace", "fourier", "bessel"):
        want = tb.hybrid_transform(tabs, kernel, dirs, precision)
        norms = np.stack([O.hybrid_transform(r, kernel, dirs_np)[1] for r in refs])
        for _ in range(2):
            out = torch.full_like(want, float("nan"))
            st = _noalloc(tb, tabs, kernel, precision, dirs, out)
            assert st == 0, tb.load().topot_last_error()
            torch.cuda.synchronize()
            diff = (out - want).abs().cpu().numpy()
            if kernel == "fourier":
                diff = diff.max(axis=-1)
            assert np.all(np.isfinite(diff))
            assert np.max(diff / norms) <= TOL[precision]


def test_noalloc_rejects_oversized_request(tb):
    img = synth.bernoulli((32, 32), 0.5, seed=93)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    dirs = torch.ones((1200000, 2), dtype=torch.float64, device="cuda")
    out = torch.empty((1, 1200000), dtype=torch.float64, device="cuda")
    st = _noalloc(tb, tabs, "laplace", "fp32c", dirs, out)
    assert st == 1
    assert b"bytes of scratch" in tb.load().topot_last_error()
