"""The tensor-core GEMM core (tcgen05.mma, BF16 in, FP32 accumulate) against a
host GEMM of the same BF16-rounded operands (GPU).  It pins the shared-memory
descriptors, the instruction descriptor and the TMEM read-back layout that
the learned preconditioner's layer kernels use."""
import numpy as np
import pytest
import torch

import paper_0810_5365_gb300 as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,K,N", [(128, 16, 16), (256, 144, 16), (128, 80, 32),
                                   (384, 256, 256), (128, 48, 48)])
def test_tc_gemm_matches_host(M, K, N):
    g = torch.Generator().manual_seed(M * 7 + K * 3 + N)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(K, N, generator=g).to(torch.bfloat16)
    want = A.double() @ B.double()
    D = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    W.wd_tc_gemm_bf16(D, A.cuda(), B.cuda(), M, K, N)
    got = D.cpu().double()
    # FP32 accumulation of K exact BF16 x BF16 products
    scale = (A.double().abs() @ B.double().abs())
    assert torch.all(torch.isfinite(got))
    assert torch.max((got - want).abs() / scale).item() <= K * 2.0 ** -23


def test_tc_gemm_rejects_bad_shapes():
    a = torch.zeros(128 * 16, dtype=torch.bfloat16, device="cuda")
    d = torch.zeros(128 * 16, dtype=torch.float32, device="cuda")
    for M, K, N in [(64, 16, 16), (128, 8, 16), (128, 16, 8), (128, 272, 16)]:
        with pytest.raises(W.WdError) as e:
            W.wd_tc_gemm_bf16(d, a, a, M, K, N)
        assert e.value.status == W.WD_ERR_ARG


def test_bounded_wait_times_out_and_context_stays_usable():
    """The failure path of the bounded device waits, run on purpose: a wait on
    an mbarrier that nothing completes gives up after its polls, the call
    reports WD_ERR_TIMEOUT, and the next tensor-core launch is still exact."""
    assert W.wd_wait_selftest(1 << 14) == W.WD_ERR_TIMEOUT
    assert W.wd_wait_selftest(0) == W.WD_ERR_ARG
    test_tc_gemm_matches_host(128, 48, 48)
