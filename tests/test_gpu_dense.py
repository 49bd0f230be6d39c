"""Dense mixed-precision building blocks: the tcgen05 BF16 GEMM against a
plain FP32 product of the same BF16 inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2104_04609_gb300 import binding

    return binding


@pytest.mark.parametrize("N", [16, 48, 256])
def test_tcgen05_gemm_matches_fp32(B, N):
    g = torch.Generator(device="cpu").manual_seed(N)
    M, K = 384, 512          # 3 CTAs, 8 K slices: the 4-stage ring wraps twice
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    Bm = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.osrc_gemm_bf16(A, Bm, C, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = A.float() @ Bm.float().T
    assert torch.isfinite(C).all()
    rel = float((C - ref).abs().max() / ref.abs().max())
    assert rel < 1e-5, rel


def test_tcgen05_gemm_rejects_bad_shapes(B):
    A = torch.zeros(100, 64, dtype=torch.bfloat16, device="cuda")
    Bm = torch.zeros(16, 64, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(100, 16, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(B.OsrcError):
        B.osrc_gemm_bf16(A, Bm, C, err)
