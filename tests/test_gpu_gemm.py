"""The tensor-core GEMM (tcgen05, BF16 x BF16 -> FP32) against a float64 product of the
same BF16 values.  Products of two BF16 numbers are exact in FP32; only the order of the
FP32 sums differs, so |D - D_ref| <= 1e-5 * K * max|a| max|b| holds with a wide margin.

The layout letters say how the two factors of D = A R (R = B^T, K x N) are stored, as in
BLAS: A "n" is M x K row-major, "t" is its transpose; R "n" is K x N row-major, "t" is
its transpose (B as N x K).  Each operand is staged by TMA tiles when its layout allows
(16-byte aligned, one unit stride, the other a multiple of 8 elements) -- K-contiguous
tiles for A "n" and R "t", row-contiguous tiles otherwise -- and element by element
through its strides when not.  nt / tn / nn / tt with M, N, K multiples of 8 run the TMA
staging in all four combinations, with ragged last tiles and chunks and boxes wider than
the matrix; odd strides run the element-by-element staging, alone or beside a TMA
operand."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(M, N, K, layout, seed_extra=0):
    import torch
    from paper_2406_14933_gb300 import asx as A
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K + seed_extra)
    a = torch.randn(M, K, generator=g).to(torch.bfloat16)
    b = torch.randn(N, K, generator=g).to(torch.bfloat16)
    ref = a.double() @ b.double().T
    if layout[0] == "n":          # A row-major M x K
        da, sam, sak = a.cuda(), K, 1
    else:                         # A stored transposed (K x M)
        da, sam, sak = a.T.contiguous().cuda(), 1, M
    if layout[1] == "t":          # B row-major N x K (the product's B^T)
        db, sbn, sbk = b.cuda(), K, 1
    else:                         # B stored as K x N
        db, sbn, sbk = b.T.contiguous().cuda(), 1, N
    d = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    A.asx_gemm_bf16(M, N, K, da, sam, sak, db, sbn, sbk, d, N, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    err = (d.double().cpu() - ref).abs().max().item()
    scale = float(a.float().abs().max() * b.float().abs().max()) * K
    assert err <= 1e-5 * scale + 1e-6, (err, scale)


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (128, 256, 64), (200, 100, 50), (300, 256, 256),
                                   (1, 1, 1), (257, 129, 130), (1024, 128, 256)])
@pytest.mark.parametrize("layout", ["nt", "tn"])
def test_gemm_matches_float64(asx, M, N, K, layout):
    _run(M, N, K, layout)


@pytest.mark.parametrize("M,N,K", [(136, 264, 200), (200, 104, 72), (8, 8, 8), (256, 256, 256),
                                   (128, 64, 1024), (384, 128, 640)])
@pytest.mark.parametrize("layout", ["nt", "tn", "nn", "tt"])
def test_gemm_tma_staging(asx, M, N, K, layout):
    _run(M, N, K, layout, seed_extra=1)


@pytest.mark.parametrize("M,N,K,layout", [(200, 100, 64, "nn"),    # B's stride 100: element staging
                                          (130, 64, 96, "tt"),     # A's stride 130: element staging
                                          (64, 72, 36, "tn"),      # TMA, boxes past all edges
                                          (72, 64, 40, "nt")])     # A's stride 40: TMA; K ragged
def test_gemm_mixed_staging(asx, M, N, K, layout):
    _run(M, N, K, layout, seed_extra=2)
