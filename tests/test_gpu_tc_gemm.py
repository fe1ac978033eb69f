"""The tcgen05 tensor-core GEMM against a float64 product of the same bf16
inputs (fp32 accumulation: only the summation order differs)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (256, 256, 1024), (1000, 128, 192), (384, 512, 256),
                                   (64, 256, 4096)])
def test_tc_gemm_matches_float64(M, N, K):
    import torch

    import paper_2404_06452_gb300 as pkg

    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    C = torch.full((M, N), float("nan"), device="cuda", dtype=torch.float32)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    pkg.paam_tc_gemm_bf16(A, B, C, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = A.double() @ B.double().T
    tol = 1e-5 * (A.double().abs() @ B.double().abs().T) + 1e-6
    assert torch.all((C.double() - ref).abs() <= tol), float((C.double() - ref).abs().max())
