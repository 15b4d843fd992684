"""The tcgen05 BF16 GEMM (C = A B^T, FP32 accumulation in tensor memory)
against a float64 product of the same bfloat16 values."""
import numpy as np
import pytest

from paper_2310_07854_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (256, 256, 256), (1024, 512, 1024),
                                   (384, 768, 192), (128, 256, 4096)])
def test_gemm_bf16_matches_float64(M, N, K):
    import torch
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = (torch.rand(M, K, generator=g) * 2 - 1).to(torch.bfloat16)
    Bm = (torch.rand(N, K, generator=g) * 2 - 1).to(torch.bfloat16)
    C = torch.full((M, N), float("nan"), device="cuda")
    B.vapr_gemm_bf16(A.cuda(), Bm.cuda(), C, M, N, K)
    torch.cuda.synchronize()
    a = A.to(torch.float64).numpy()
    b = Bm.to(torch.float64).numpy()
    want = a @ b.T
    bound = np.abs(a) @ np.abs(b).T  # sum of |a_ik b_jk|
    err = np.abs(C.cpu().numpy().astype(np.float64) - want)
    # float32 accumulation: error <= K * 2^-24 * sum|a b| (with margin 4)
    assert np.all(err <= 4 * K * 2.0 ** -24 * bound + 1e-30), err.max()
    assert B.vapr_device_error() == 0


def test_gemm_identity_and_structure():
    """A = I: C reproduces B exactly (each output sums one product)."""
    import torch
    M = N = K = 256
    A = torch.eye(M, K, dtype=torch.bfloat16)
    Bm = (torch.randn(N, K) * 3).to(torch.bfloat16)
    C = torch.empty((M, N), device="cuda")
    B.vapr_gemm_bf16(A.cuda(), Bm.cuda(), C, M, N, K)
    assert torch.equal(C.cpu(), Bm.float().T.contiguous())
