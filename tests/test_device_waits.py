"""Bounded device waits give up and report instead of hanging the GPU.

Every wait of the library's kernels on an mbarrier has a time limit; when it
runs out the kernel records a timeout, returns, and the host call reports
NEUROSIM_E_TIMEOUT.  neurosim_debug_expiring_wait runs that same wait on an
mbarrier that nothing arrives on (with a 1 ms limit), so the wait must run
out; with the arrival it must complete.  The GPU context stays usable
afterwards: a later library call still computes.
"""
import ctypes as C
import time

import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def test_wait_without_arrival_times_out_and_context_survives():
    from paper_2602_15018_gb300 import _lib, device_log
    L = _lib.lib()
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.neurosim_debug_expiring_wait(1, 1_000_000, st) == 0                  # arrival: completes
    t = time.perf_counter()
    rc = L.neurosim_debug_expiring_wait(0, 1_000_000, st)                         # no arrival: 1 ms limit
    dt = time.perf_counter() - t
    assert rc == 5, rc                                                              # NEUROSIM_E_TIMEOUT
    assert b"gave up" in L.neurosim_last_error()
    assert dt < 5.0
    assert L.neurosim_debug_expiring_wait(0, 10, st) == 1                          # limit out of range
    x = torch.tensor([1.0, 2.0, 0.5], device="cuda")
    y = device_log(x)
    torch.cuda.synchronize()
    assert abs(float(y[1]) - 0.6931472) < 1e-6
