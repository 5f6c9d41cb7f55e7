"""Failure detection without a GPU fault: a bounded wait on a barrier that nothing completes gives
up after its limit and reports MER_ERR_TIMEOUT through the host status; the context keeps
working afterwards."""
import ctypes as ct

import pytest

from .gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout():
    torch = need_gpu()
    from paper_2309_15676_gb300 import _lib
    L = _lib.load()
    waited = ct.c_double()
    st = L.mer_wait_selftest(0.02, ct.byref(waited))
    assert st == 4, st                            # MER_ERR_TIMEOUT
    assert 0.02 <= waited.value < 0.5, waited.value
    # the device is still usable
    x = torch.arange(1024, device="cuda", dtype=torch.float32)
    assert float(x.sum().item()) == 1023 * 1024 / 2
