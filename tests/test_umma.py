"""The tensor-core GEMM core (tcgen05, TMEM accumulators, BF16 operands in
shared memory) against a host GEMM, for every operand layout."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _gemm(mode, A, B, M, N, K):
    from paper_2602_15018_gb300 import _lib
    L = _lib.lib()
    a = A.to(torch.bfloat16).cuda().contiguous()
    b = B.to(torch.bfloat16).cuda().contiguous()
    c = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    rc = L.neurosim_debug_umma_gemm(mode, M, N, K, C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()),
                                    C.c_void_p(c.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(rc)
    return c.cpu()


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (304, 256, 200), (77, 48, 136), (96, 32, 192), (64, 16, 136)])
@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4, 5, 6])
def test_gemm_layouts(mode, M, N, K):
    g = torch.Generator().manual_seed(M * 1000 + N * 10 + K + mode)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).float()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).float()
    ref = (A.double() @ B.double().T).float()
    a_mn, b_mn = mode in (1, 3, 6), mode in (2, 3, 6)     # modes 4 and 5 (TMA) are K-major
    a_in = A.T.contiguous() if a_mn else A
    b_in = B.T.contiguous() if b_mn else B
    if (a_mn and M % 8) or (b_mn and N % 8):
        pytest.skip("MN-major operands need rows % 8 == 0")
    out = _gemm(mode, a_in, b_in, M, N, K)
    # products of BF16 values are exact in FP32; only the FP32 sum order differs
    tol = 1e-5 * K * (A.abs().max() * B.abs().max()).item()
    assert torch.isfinite(out).all()
    assert (out - ref).abs().max().item() <= tol
