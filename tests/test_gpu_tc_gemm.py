"""The tcgen05 BF16 GEMM (mc_tc_gemm_bf16) against an FP64 product of the same BF16 inputs."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_04200_gb300 import build as b
    b.build()
    from paper_1901_04200_gb300 import _lib
    return _lib


@pytest.mark.parametrize("M,N,K,ks", [(128, 16, 64, 64), (128, 32, 64, 64), (128, 256, 64, 64),
                                      (256, 256, 256, 256), (128, 48, 320, 320), (4096, 256, 256, 256),
                                      (256, 256, 8192, 512), (256, 16, 8192, 1024)])
def test_tc_gemm_matches_fp64(L, M, N, K, ks):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn((M, K), device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn((N, K), device="cuda", generator=g).to(torch.bfloat16)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    D = L.tc_gemm_bf16(A, B, ks, err)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = torch.stack([A[:, s * ks:(s + 1) * ks].double() @ B[:, s * ks:(s + 1) * ks].double().T
                       for s in range(K // ks)])
    scale = ref.abs().max().item()
    assert (D.double() - ref).abs().max().item() <= 1e-5 * scale, (D.double() - ref).abs().max().item()


def test_tc_gemm_strided_operands(L):
    """Row strides larger than K (operands that are column windows of wider buffers)."""
    M, N, K = 256, 64, 128
    A = torch.randn((M, 3 * K), device="cuda").to(torch.bfloat16)
    B = torch.randn((N, 2 * K), device="cuda").to(torch.bfloat16)
    Aw, Bw = A[:, K:2 * K], B[:, :K]
    D = L.tc_gemm_bf16(Aw, Bw)
    ref = Aw.double() @ Bw.double().T
    assert (D[0].double() - ref).abs().max().item() <= 1e-5 * ref.abs().max().item()
