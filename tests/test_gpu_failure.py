"""Device-side failure path without a GPU fault: a bounded wait on an
mbarrier phase that nothing completes runs out, the kernel records
SPINSUM_ERR_TIMEOUT and returns; the host reads it through
spinsum_check_status and the context stays usable."""
import ctypes

import numpy as np
import pytest

import workloads as wl
from tests.gpu_helpers import assert_bitexact, gpu_run

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    import torch
    import oracle
    import paper_1705_06661_gb300 as ss
    from paper_1705_06661_gb300 import _binding
    st = torch.cuda.current_stream().cuda_stream
    ss.spinsum_check_status(st)
    f = _binding.lib.ss_selftest_wait_timeout
    f.argtypes = [ctypes.c_longlong, ctypes.c_void_p]
    f.restype = ctypes.c_int
    assert f(1000, st) == 0
    with pytest.raises(ss.SpinsumError, match="TIMEOUT"):
        ss.spinsum_check_status(st)
    # the status word was cleared and the context still works
    ss.spinsum_check_status(st)
    A = wl.integers(7, (8, 8, 8, 5, 5, 5))
    assert_bitexact(gpu_run(A, 3, wl.table2(1)), oracle.spinsum(A, 3, wl.table2(1)), "after timeout")
