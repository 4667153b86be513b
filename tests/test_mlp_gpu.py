"""Tensor-core (tcgen05 / TMEM / TMA) BF16 GEMM of the surrogate against a PyTorch FP32 reference."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ck():
    import torch
    from paper_1209_6038_gb300 import build, cloak
    build.build()
    cloak.load()
    torch.cuda.init()
    return cloak


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (128, 256, 256), (384, 96, 128), (1024, 256, 64),
                                   (256, 208, 1024), (128, 64, 4096)])
def test_gemm_matches_fp32_reference(ck, M, N, K):
    import torch
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    a = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    b = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    c = torch.full((M, N), float("nan"), device="cuda")
    ck.cloak_mlp_gemm(a, b, c)
    ref = a.float() @ b.float().t()
    # same BF16 inputs, FP32 accumulation: differences are summation-order rounding only
    tol = 1e-5 * K ** 0.5 * ref.abs().max().item() + 1e-4
    assert torch.isfinite(c).all()
    assert (c - ref).abs().max().item() <= tol


def test_gemm_rejects_bad_shapes(ck):
    import torch
    a = torch.zeros(100, 64, device="cuda", dtype=torch.bfloat16)
    b = torch.zeros(16, 64, device="cuda", dtype=torch.bfloat16)
    c = torch.zeros(100, 16, device="cuda")
    with pytest.raises(ck.CloakError):
        ck.cloak_mlp_gemm(a, b, c)
