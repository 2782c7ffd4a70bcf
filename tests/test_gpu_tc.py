"""The tcgen05 building block of the dense form (operands in the 32-, 64- and
128-byte swizzled K-major layouts) against torch.matmul on the same BF16
operands (FP32 accumulation; only the summation order differs)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_0342_gb300 import build
    build.build()
    from paper_1410_0342_gb300 import glrm
    return glrm


@pytest.mark.parametrize("M,N,K", [(128, 64, 16), (256, 128, 32), (384, 192, 64), (128, 64, 128),
                                   (256, 320, 64)])
def test_tc_gemm_matches_matmul(G, M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = torch.full((M, N), float("nan"), device="cuda")
    G.glrm_tc_gemm_bf16(A, B, D)
    ref = A.float() @ B.float().T
    torch.testing.assert_close(D, ref, rtol=1e-5, atol=1e-4)


@pytest.mark.parametrize("M,N,K", [(100, 64, 16), (128, 64, 48), (128, 64, 80), (128, 40, 32)])
def test_tc_gemm_rejects_bad_shapes(G, M, N, K):
    A = torch.zeros(M, K, device="cuda", dtype=torch.bfloat16)
    B = torch.zeros(N, K, device="cuda", dtype=torch.bfloat16)
    D = torch.zeros(M, N, device="cuda")
    with pytest.raises(G.GLRMError) as e:
        G.glrm_tc_gemm_bf16(A, B, D)
    assert e.value.code == G.GLRM_ERR_RANGE
