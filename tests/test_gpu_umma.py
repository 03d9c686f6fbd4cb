"""The tcgen05 tile (tt_umma_gemm_bf16) against a plain product: C = A B^T
for bfloat16 A [128][K], B [N][K].  Products of bfloat16 values are exact in
FP32, so the tensor-core result differs from the FP64 product only by FP32
accumulation rounding: relative 1e-5 of sum |a||b| per element."""
import numpy as np
import pytest
import torch

from paper_2504_16446_gb300 import tt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2504_16446_gb300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("N,K", [(32, 64), (16, 16), (128, 128), (256, 256), (48, 32)])
def test_tile_matches_plain_product(N, K):
    gen = torch.Generator(device="cuda")
    gen.manual_seed(N * 1000 + K)
    A = torch.randn((128, K), device="cuda", generator=gen).to(torch.bfloat16)
    B = torch.randn((N, K), device="cuda", generator=gen).to(torch.bfloat16)
    C = tt.umma_gemm_bf16(A, B).cpu().numpy().astype(np.float64)
    a, b = A.double().cpu().numpy(), B.double().cpu().numpy()
    ref = a @ b.T
    bound = np.abs(a) @ np.abs(b).T
    assert np.all(np.abs(C - ref) <= 1e-5 * bound + 1e-30)


def test_structured_operands_locate_rows_and_columns():
    """A = identity rows, B = a ramp: C[m][n] = B[n][m] picks out single
    elements, so a wrong row/column mapping cannot cancel out."""
    K, N = 128, 64
    A = torch.zeros((128, K), dtype=torch.bfloat16, device="cuda")
    A[torch.arange(128), torch.arange(128)] = 1.0
    Bf = (torch.arange(N * K, device="cuda", dtype=torch.float32) % 251).reshape(N, K)
    C = tt.umma_gemm_bf16(A, Bf.to(torch.bfloat16))
    torch.testing.assert_close(C, Bf.T.contiguous(), rtol=0, atol=0)
