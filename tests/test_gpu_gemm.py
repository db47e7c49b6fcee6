"""The tensor-core GEMM (tcgen05, BF16 x BF16 -> FP32) against a float64 product of the
same BF16 values.  Products of two BF16 numbers are exact in FP32; only the order of the
FP32 sums differs, so |D - D_ref| <= 1e-5 * K * max|a| max|b| holds with a wide margin."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (128, 256, 64), (200, 100, 50), (300, 256, 256),
                                   (1, 1, 1), (257, 129, 130), (1024, 128, 256)])
@pytest.mark.parametrize("layout", ["nt", "tn"])
def test_gemm_matches_float64(asx, M, N, K, layout):
    import torch
    from paper_2406_14933_gb300 import asx as A
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    a = torch.randn(M, K, generator=g).to(torch.bfloat16)
    b = torch.randn(N, K, generator=g).to(torch.bfloat16)
    ref = a.double() @ b.double().T
    if layout == "nt":            # A row-major M x K, B row-major N x K
        da, db = a.cuda(), b.cuda()
        sam, sak, sbn, sbk = K, 1, K, 1
    else:                         # both stored transposed (K x M and K x N), read with strides
        da, db = a.T.contiguous().cuda(), b.T.contiguous().cuda()
        sam, sak, sbn, sbk = 1, M, 1, N
    d = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    A.asx_gemm_bf16(M, N, K, da, sam, sak, db, sbn, sbk, d, N, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    err = (d.double().cpu() - ref).abs().max().item()
    scale = float(a.float().abs().max() * b.float().abs().max()) * K
    assert err <= 1e-5 * scale + 1e-6, (err, scale)
