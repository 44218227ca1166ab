"""The warm-start network's tcgen05 GEMM (BF16 operands, FP32 accumulation in tensor memory)
against the plain definition C = A B^T evaluated in FP64 on the same BF16 values."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2309_08093_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2309_08093_gb300 import lib  # noqa: E402


@pytest.mark.parametrize("M,N,K,pad", [(128, 128, 64, 0), (200, 300, 192, 8), (256, 512, 1024, 0),
                                       (1, 7, 64, 0), (130, 129, 320, 16), (384, 256, 4096, 0),
                                       # enough 128 x 256 tiles for the wide-tile kernel (one per SM)
                                       (2048, 2560, 128, 0), (2000, 2600, 192, 8)])
def test_gemm_bf16_tn_matches_fp64(M, N, K, pad):
    g = torch.Generator(device="cuda")
    g.manual_seed(M * 7919 + N * 31 + K)
    lda = ldb = K + pad
    A = torch.randn(M, lda, generator=g, device="cuda").to(torch.bfloat16)
    B = torch.randn(N, ldb, generator=g, device="cuda").to(torch.bfloat16)
    ldc = N + 3
    C = torch.full((M, ldc), float("nan"), device="cuda")
    rc = lib.tt_mlp_gemm_bf16(A, B, C, M, N, K, lda, ldb, ldc)
    torch.cuda.synchronize()
    assert rc == lib.TT_OK
    a = A.float().cpu().numpy().astype(np.float64)[:, :K]
    b = B.float().cpu().numpy().astype(np.float64)[:, :K]
    ref = a @ b.T
    absum = np.abs(a) @ np.abs(b).T
    got = C.cpu().numpy().astype(np.float64)
    assert np.all(np.isnan(got[:, N:]))          # nothing written past column N
    got = got[:, :N]
    err = np.abs(got - ref)
    # FP32 accumulation of exact BF16 products: |error| <= K 2^-23 sum_k |a_k b_k| (a deterministic
    # bound with a factor 2 for the accumulator's rounding); typical errors are far smaller
    assert np.all(err <= K * 2.0 ** -23 * absum + 1e-30), float(np.max(err / (absum + 1e-30)))
    assert float(np.median(err / (absum + 1e-30))) <= 1e-6


def test_gemm_rejects_bad_shapes():
    A = torch.zeros(128, 64, device="cuda", dtype=torch.bfloat16)
    C = torch.zeros(128, 128, device="cuda")
    assert lib.tt_mlp_gemm_bf16(A, A, C, 128, 128, 60, 64, 64, 128) == lib.TT_EINVAL   # K % 64
    assert lib.tt_mlp_gemm_bf16(A, A, C, 128, 128, 64, 60, 64, 128) == lib.TT_EINVAL   # lda % 8
    assert lib.tt_mlp_gemm_bf16(A, A, C, 0, 128, 64, 64, 64, 128) == lib.TT_EINVAL     # M
