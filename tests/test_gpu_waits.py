"""The bounded device-side waits give up and report TOPOT_ERR_TIMEOUT instead of hanging:
a spin on a flag that nothing sets and an mbarrier phase that never completes, each
limited to 50 ms; the context stays usable afterwards (an extraction right after is
bit-exact against the oracle)."""
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


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_reports_timeout(tb, which):
    L = tb.load()
    st = L.topot_selftest_wait(which, 50, tb._stream(None))
    assert st == 6, tb.STATUS.get(st, st)          # TIMEOUT
    assert b"timed out" in L.topot_last_error()
    img = synth.grf((70, 90), 4.0, seed=3)
    tabs = tb.build_critical_tables(tb.pack_images([img]))
    ref = O.critical_tables(img)
    for o in range(4):
        idx, val = tabs.table(0, o, 0)
        np.testing.assert_array_equal(idx, ref.lower_idx[o])
        np.testing.assert_array_equal(val, ref.lower_val[o])


def test_selftest_rejects_bad_arguments(tb):
    L = tb.load()
    assert L.topot_selftest_wait(2, 50, tb._stream(None)) == 1
    assert L.topot_selftest_wait(0, 0, tb._stream(None)) == 1
