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


def test_activation_within_its_error_bound():
    """GELU and GELU' of the network's epilogues against float64 erf: the
    Abramowitz-Stegun 7.1.26 erf is within 1.5e-7, and fp32 evaluation adds a
    few ulps."""
    import torch
    from scipy.special import erf

    import paper_2404_06452_gb300 as pkg

    z = np.concatenate([np.linspace(-12, 12, 200001), [0.0, -0.0, 1e-30, -1e-30, 40.0, -40.0]]).astype(np.float32)
    zt = torch.from_numpy(z).cuda()
    g = torch.empty_like(zt)
    d = torch.empty_like(zt)
    pkg.paam_diag_gelu(zt, g, d)
    torch.cuda.synchronize()
    z64 = z.astype(np.float64)
    cdf = 0.5 * (1.0 + erf(z64 / np.sqrt(2.0)))
    ref_g = z64 * cdf
    ref_d = cdf + z64 * np.exp(-0.5 * z64 * z64) / np.sqrt(2.0 * np.pi)
    tol = 1e-7 * np.abs(z64) + 4e-7 + 1e-6 * np.abs(ref_g)
    assert np.all(np.abs(g.cpu().numpy() - ref_g) <= tol), np.max(np.abs(g.cpu().numpy() - ref_g) - tol)
    assert np.all(np.abs(d.cpu().numpy() - ref_d) <= 3e-7 * np.abs(z64) + 4e-7 + 1e-6 * np.abs(ref_d))
