"""hybrid_transform_noalloc: the allocation-free variant of hybrid_transform.

Some callers cannot call cudaMalloc -- code running inside an allocator or memory-pool
callback, under a no-allocation real-time budget, or in a host that forbids device
allocation after start-up.  For them the library offers hybrid_transform_noalloc,
whose scratch is a fixed device array instead of a workspace grown with cudaMalloc.
This test calls it through the C ABI, twice in a row (the array keeps the previous
call's contents), for every kernel, shared and per-image directions, and checks each
result against hybrid_transform within the tolerance the parity tests use.  It checks
that a call on a fresh handle reserves no device memory, and that an oversized request
is refused.
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


def _noalloc(tb, tabs, kernel, precision, dirs, out, per_image=0):
    L = tb.load()
    D = dirs.shape[-2] if dirs.dim() == 3 else dirs.shape[0]
    return L.hybrid_transform_noalloc(tabs.handle, tb.KERNELS[kernel], tb.PRECISIONS[precision],
                                      ctypes.c_void_p(dirs.data_ptr()), D, per_image,
                                      ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _check(tb, tabs, kernel, precision, dirs, norms, per_image):
    want = tb.hybrid_transform(tabs, kernel, dirs, precision)
    for _ in range(2):
        out = torch.full_like(want, float("nan"))
        st = _noalloc(tb, tabs, kernel, precision, dirs, out, per_image)
        assert st == 0, tb.load().topot_last_error()
        torch.cuda.synchronize()
        diff = (out - want).abs().cpu().numpy()
        if kernel == "fourier":
            diff = diff.max(axis=-1)
        assert np.all(np.isfinite(diff))
        assert np.max(diff / norms) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_noalloc_matches_hybrid_transform(tb, precision):
    imgs = [synth.grf((150, 170), 5.0, seed=90), synth.grf((120, 131), 4.0, seed=91)]
    tabs = tb.build_critical_tables(tb.pack_images(imgs))
    dirs_np = synth.random_2d_dirs(300, 92, 0.05, 1.0)
    dirs = torch.from_numpy(dirs_np).cuda()
    refs = [O.critical_tables(im) for im in imgs]
    for kernel in ("laplace", "fourier", "bessel", "sine"):
        norms = np.stack([O.hybrid_transform(r, kernel, dirs_np)[1] for r in refs])
        _check(tb, tabs, kernel, precision, dirs, norms, 0)


def test_noalloc_per_image_directions(tb):
    imgs = [synth.grf((90, 100), 4.0, seed=94), synth.grf((70, 81), 3.0, seed=95)]
    tabs = tb.build_critical_tables(tb.pack_images(imgs))
    dirs_np = np.stack([synth.random_2d_dirs(140, 96 + b, 0.05, 2.5) for b in range(2)])
    dirs = torch.from_numpy(dirs_np).cuda()
    refs = [O.critical_tables(im) for im in imgs]
    for kernel in ("laplace", "fourier", "bessel", "sine"):
        norms = np.stack([O.hybrid_transform(refs[b], kernel, dirs_np[b])[1] for b in range(2)])
        _check(tb, tabs, kernel, "fp32c", dirs, norms, 1)


def test_noalloc_reserves_no_device_memory(tb):
    """After start-up, a call on a fresh handle (whose workspace hybrid_transform would
    have to allocate) reserves no device memory: free memory does not drop."""
    img = synth.grf((200, 210), 5.0, seed=97)
    batch = tb.pack_images([img])
    dirs = torch.from_numpy(synth.random_2d_dirs(2000, 98, 0.05, 1.0)).cuda()
    outs = {k: torch.empty((1, 2000, 2) if k == "fourier" else (1, 2000), dtype=torch.float64, device="cuda")
            for k in ("laplace", "fourier", "bessel", "sine")}
    warm = tb.build_critical_tables(batch)
    for k, o in outs.items():   # start-up: the array's address and every kernel's code
        assert _noalloc(tb, warm, k, "fp32c", dirs, o) == 0, tb.load().topot_last_error()
    fresh = tb.build_critical_tables(batch)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k, o in outs.items():
        assert _noalloc(tb, fresh, k, "fp32c", dirs, o) == 0, tb.load().topot_last_error()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    # a workspace would take at least 1 MiB (cudaMalloc granularity 2 MiB)
    assert free0 - free1 < (1 << 20), (free0, free1)


def test_noalloc_rejects_oversized_request(tb):
    img = synth.bernoulli((32, 32), 0.5, seed=93)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    dirs = torch.ones((1200000, 2), dtype=torch.float64, device="cuda")
    out = torch.empty((1, 1200000), dtype=torch.float64, device="cuda")
    st = _noalloc(tb, tabs, "laplace", "fp32c", dirs, out)
    assert st == 1
    assert b"bytes of scratch" in tb.load().topot_last_error()
