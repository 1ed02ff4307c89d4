"""The tcgen05 BF16 GEMM (rank-r correction of Eq. 14) against a plain FP32
product of the same BF16-rounded operands.  Tolerance: the products of two
BF16 numbers are exact in FP32, so the only difference is the FP32
summation order: |err| <= K * 2^-23 * sum|a||b| (checked with margin)."""
import numpy as np
import pytest

from paper_1912_06525_gb300 import katz

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def padded(rows, K, seed):
    ld = (K + 7) // 8 * 8
    g = torch.Generator().manual_seed(seed)
    X = torch.zeros((rows, ld), dtype=torch.bfloat16)
    X[:, :K] = torch.randn((rows, K), generator=g).to(torch.bfloat16)
    return X.cuda()


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (200, 72, 150), (128, 1024, 2000),
                                   (2000, 1024, 128), (1, 16, 8), (333, 257, 777)])
def test_tc_gemm_matches_fp32_reference(M, N, K):
    A = padded(M, K, 1)
    B = padded(N, K, 2)
    C = torch.randn((M, N), dtype=torch.float32, device="cuda")
    C0 = C.clone()
    katz.katz_gemm_bf16(A, B, C, K=K, alpha=0.5, beta=2.0)
    Ak = A[:, :K]
    Bk = B[:, :K]
    torch.cuda.synchronize()
    ref = 0.5 * (Ak.float() @ Bk.float().T) + 2.0 * C0
    bound = K * 2.0 ** -22 * (0.5 * (Ak.float().abs() @ Bk.float().abs().T)) + 1e-6 * C0.abs()
    assert torch.all((C - ref).abs() <= 4 * bound + 1e-30), float((C - ref).abs().max())


def test_tc_gemm_rejects_bad_strides():
    A = torch.zeros((16, 12), dtype=torch.bfloat16, device="cuda")
    C = torch.zeros((16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(katz.KatzError):
        katz.katz_gemm_bf16(A, A, C)


def fp32_matrix(rows, K, seed, ld=None):
    ld = ld or (K + 3) // 4 * 4
    g = torch.Generator().manual_seed(seed)
    X = torch.zeros((rows, ld), dtype=torch.float32)
    X[:, :K] = torch.randn((rows, K), generator=g) * torch.exp(torch.randn((rows, 1), generator=g))
    return X.cuda()


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (200, 72, 150), (1000, 1024, 2000),
                                   (4097, 264, 37), (1, 16, 4), (333, 257, 777)])
def test_tc_gemm_tf32x3_is_fp32_accurate(M, N, K):
    """Three TF32 products of the split operands against an FP64 product:
    the error stays within FP32 accumulation bounds, |err| <= (K + 8) 2^-23
    sum_k |a_ik||b_jk| (a single TF32 product would be ~2^-11)."""
    A = fp32_matrix(M, K, 1)
    B = fp32_matrix(N, K, 2)
    C = torch.randn((M, N), dtype=torch.float32, device="cuda")
    C0 = C.clone()
    katz.katz_gemm_tf32x3(A, B, C, K=K, alpha=0.75, beta=-1.5)
    torch.cuda.synchronize()
    Ad, Bd = A[:, :K].double(), B[:, :K].double()
    ref = 0.75 * (Ad @ Bd.T) - 1.5 * C0.double()
    bound = (K + 8) * 2.0 ** -23 * (0.75 * (Ad.abs() @ Bd.abs().T)) + 2.0 ** -22 * 1.5 * C0.double().abs()
    err = (C.double() - ref).abs()
    assert torch.all(err <= bound + 1e-30), float((err / (bound + 1e-30)).max())
