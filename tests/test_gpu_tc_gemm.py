"""The tcgen05 tensor-core GEMM against a float64 product of the same bf16
inputs (fp32 accumulation: only the summation order differs)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


# The last three shapes take the persistent weight-stationary kernel (one
# column tile, K <= 256, at least 4 row tiles per SM), with a ragged last tile.
@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (256, 256, 1024), (1000, 128, 192), (384, 512, 256),
                                   (64, 256, 4096), (100000, 256, 256), (90001, 128, 64), (80000, 64, 192)])
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


def test_activation_matches_its_definition():
    """GELU (tanh form) and its derivative as the epilogues evaluate them, against
    float64: one ex2.approx and one rcp.approx keep them within ~1e-6 relative."""
    import torch

    import paper_2404_06452_gb300 as pkg
    from oracle import mlp

    z = np.concatenate([np.linspace(-12, 12, 200001), [0.0, -0.0, 1e-30, -1e-30, 40.0, -40.0, 300.0, -300.0]])
    z = z.astype(np.float32)
    zt = torch.from_numpy(z).cuda()
    g = torch.empty_like(zt)
    d = torch.empty_like(zt)
    pkg.paam_diag_gelu(zt, g, d)
    torch.cuda.synchronize()
    z64 = z.astype(np.float64)
    ref_g, ref_d = mlp.gelu(z64), mlp.gelu_grad(z64)
    got_g, got_d = g.cpu().numpy().astype(np.float64), d.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got_g - ref_g) <= 2e-6 * np.abs(ref_g) + 1e-30 + 1e-7 * np.abs(z64) * (np.abs(z64) < 20))
    assert np.all(np.abs(got_d - ref_d) <= 4e-6 * (np.abs(ref_d) + np.abs(z64 * ref_d)) + 1e-6)
