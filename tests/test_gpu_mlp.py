"""Tensor-core (tcgen05) GEMM and surrogate-network kernels against plain
fp32 PyTorch references on the same bf16 inputs."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ssa():
    from paper_2605_00479_gb300 import build, ssa as mod
    build.build()
    mod.lib()
    return mod


@pytest.mark.parametrize("M,N,K", [(128, 16, 16), (300, 256, 256), (257, 128, 512), (1024, 256, 16), (64, 64, 32),
                                   (384, 16, 768)])
def test_gemm_matches_fp32_reference(ssa, M, N, K):
    """D = A B^T with bf16 operands and fp32 accumulation; the reference sums
    the same bf16 products in fp32 (differences come only from summation
    order: |err| <= K * 2^-23 * sum|a||b|)."""
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = torch.full((M, N), float("nan"), device="cuda")
    rc = ssa.lib().ssa_mlp_gemm_bf16(M, N, K, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                     ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    ref = A.double() @ B.double().T
    bound = K * 2.0 ** -23 * (A.double().abs() @ B.double().abs().T) + 1e-30
    err = (D.double() - ref).abs()
    assert torch.all(err <= bound), float((err / bound).max())
