"""Cross-checks of the tensor-core GEMMs against cuBLAS (torch) at the
benchmark's 8192^3 size: an independent implementation, beside the FP64
oracle that the parity tests use."""
import pytest
import torch

import paper_2606_15991_gb300 as tp
from oracle import gemm as ogemm

pytestmark = pytest.mark.gpu


def _operands():
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    a = torch.randn(8192, 8192, device="cuda", generator=g).to(torch.bfloat16)
    bt = torch.randn(8192, 8192, device="cuda", generator=g).to(torch.bfloat16)
    return a, bt


def _gemm_c(ctx):
    c = torch.empty(8192, 8192, device="cuda", dtype=torch.bfloat16)
    p = tp.tp_partition_create(ctx, c, (256, 256))
    tp.tp_partition_map(p, tp.MAP_STRIDED, ctx.sm_count // 2)
    return c, p


def test_bf16_8192_matches_cublas(ctx):
    """Both accumulate in FP32 and round once to bf16; accumulation order
    differences move a few elements by one bf16 step."""
    a, bt = _operands()
    c, p = _gemm_c(ctx)
    tp.tp_gemm(ctx, p, a, bt.t(), tp.gemm_config(bm=256, bn=256, group_m=8))
    ref = torch.matmul(a, bt.t())
    assert ogemm.rel_frobenius(c.float(), ref.float()) <= 2e-3
    tp.tp_partition_destroy(p)


def test_fp8_8192_matches_cublas_scaled_mm(ctx):
    """Same E4M3 codes and per-tensor scales: tp_gemm_fp8 against
    torch._scaled_mm (cuBLAS FP8)."""
    if not hasattr(torch, "_scaled_mm"):
        pytest.skip("torch._scaled_mm unavailable")
    a, bt = _operands()
    amax, scale = torch.zeros(2, device="cuda"), torch.zeros(2, device="cuda")
    qa = torch.empty(8192, 8192, device="cuda", dtype=torch.float8_e4m3fn)
    qb = torch.empty(8192, 8192, device="cuda", dtype=torch.float8_e4m3fn)
    for i, (src, q) in enumerate(((a, qa), (bt, qb))):
        pq = tp.tp_partition_create(ctx, q, (16, 8192))
        tp.tp_amax(ctx, src, amax[i:i + 1])
        tp.tp_quantize_fp8(ctx, pq, src, amax[i:i + 1], scale[i:i + 1])
        tp.tp_partition_destroy(pq)
    c, p = _gemm_c(ctx)
    tp.tp_gemm_fp8(ctx, p, qa, qb.t(), scale[0:1], scale[1:2], tp.gemm_config(bm=256, bn=256, group_m=8))
    inv = 1.0 / scale
    ref = torch._scaled_mm(qa, qb.t(), scale_a=inv[0:1].reshape(()).contiguous(),
                           scale_b=inv[1:2].reshape(()).contiguous(), out_dtype=torch.bfloat16)
    assert ogemm.rel_frobenius(c.float(), ref.float()) <= 2e-3
    tp.tp_partition_destroy(p)
