"""The C-ABI library builds, loads and exports every symbol include/topot.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "topot.h")) as f:
        text = f.read()
    return re.findall(r"^TOPOT_API\s+[\w\s\*]+?\b(\w+)\s*\(", text, flags=re.M)


@pytest.fixture(scope="module")
def lib_path():
    from paper_2405_02256_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = set(_declared())
    for required in ("build_critical_tables", "ect", "radon", "hybrid_transform", "hybrid_transform_grad",
                     "tables_info", "tables_copy_to_host", "free_tables", "topot_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_the_same_symbols(lib_path):
    from paper_2405_02256_gb300 import binding
    assert set(binding.API_SYMBOLS) == set(_declared())
    binding.load(lib_path)


def test_last_error_without_gpu(lib_path):
    """Host-side validation answers without touching a device."""
    from paper_2405_02256_gb300 import binding
    L = binding.load(lib_path)
    h = ctypes.c_void_p()
    shapes = (ctypes.c_int64 * 2)(4, 4)
    offs = (ctypes.c_int64 * 1)(0)
    # n = 5 is rejected before any CUDA call, and so are the top construction in 4-D and
    # slabs of anything but 3-D volumes
    st = L.tables_create(0, 5, shapes, offs, 1, 0, ctypes.byref(h))
    assert st == 1 and b"n must be 2, 3 or 4" in L.topot_last_error()
    st = L.tables_create(0, 4, shapes, offs, 1, 1, ctypes.byref(h))
    assert st == 2 and b"top-dimensional" in L.topot_last_error()
    zr = (ctypes.c_int64 * 2)(0, 2)
    st = L.tables_create_slab(0, 2, shapes, offs, zr, 1, ctypes.byref(h))
    assert st == 2 and b"slabs of 3-D volumes" in L.topot_last_error()
    assert L.slab_sum_f64(None, 1, 1, None, None) == 1
    st = L.tables_create(0, 2, shapes, offs, 1, 7, ctypes.byref(h))
    assert st == 1 and b"construction" in L.topot_last_error()


def test_kernel_table_validation_without_gpu(lib_path):
    """kernel_table_create rejects bad samples and ranges before any CUDA call."""
    from paper_2405_02256_gb300 import binding
    L = binding.load(lib_path)
    h = ctypes.c_void_p()
    y = (ctypes.c_double * 3)(1.0, 2.0, 3.0)
    assert L.kernel_table_create(y, 1, 0.0, 1.0, ctypes.byref(h)) == 1
    assert b"K" in L.topot_last_error()
    assert L.kernel_table_create(y, 3, 1.0, 1.0, ctypes.byref(h)) == 1
    assert L.kernel_table_create(y, 3, 0.0, float("inf"), ctypes.byref(h)) == 1
    bad = (ctypes.c_double * 3)(1.0, float("nan"), 3.0)
    assert L.kernel_table_create(bad, 3, 0.0, 1.0, ctypes.byref(h)) == 1
    assert b"non-finite" in L.topot_last_error()
    big = (ctypes.c_double * 3)(1.0, 3e37, 3.0)
    assert L.kernel_table_create(big, 3, 0.0, 1.0, ctypes.byref(h)) == 1
    assert b"1e37" in L.topot_last_error()
    assert L.hybrid_transform_table(None, None, 0, None, 1, 0, None, None) == 1
    L.kernel_table_free(None)
