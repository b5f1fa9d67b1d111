"""GPU edge cases: empty outputs, odd lengths and unaligned views (the
scalar path), and sizes whose element indices pass 2^31 (64-bit indexing in
the map and GEMM kernels), checked against the FP64 oracle on samples."""
import numpy as np
import pytest
import torch

import paper_2606_15991_gb300 as tp
import synth
from oracle import gemm as ogemm
from oracle import lowp
from oracle import maps as omaps
from oracle import partition as opart

pytestmark = pytest.mark.gpu


def test_empty_map_and_gemm_are_no_ops(ctx):
    z = torch.empty(0, device="cuda")
    p = tp.tp_partition_create(ctx, z, (4,))
    assert tp.tp_partition_query(p)["num_tiles"] == 0
    tp.tp_map_axpy(ctx, p, 0.5, z, z.clone())
    tp.tp_partition_destroy(p)
    for m, n in ((0, 64), (128, 0)):
        a = torch.zeros(m, 64, device="cuda", dtype=torch.bfloat16)
        bt = torch.zeros(n, 64, device="cuda", dtype=torch.bfloat16)
        c = torch.zeros(m, n, device="cuda", dtype=torch.bfloat16)
        pc = tp.tp_partition_create(ctx, c, (128, 64))
        tp.tp_gemm(ctx, pc, a, bt.t(), tp.gemm_config(bm=128, bn=64))
        tp.tp_partition_destroy(pc)


@pytest.mark.parametrize("dt", ["f32", "bf16"])
@pytest.mark.parametrize("n,tile,offset", [(1, 4, 0), (4097, 4096, 0), (4099, 1000, 0), (10000, 4096, 1),
                                           (12345, 333, 3)])
def test_odd_lengths_and_unaligned_views(ctx, dt, n, tile, offset):
    """Lengths that are no multiple of the vector width, tiles that are no
    multiple of it, and views starting `offset` elements into their storage
    (not 16-byte aligned) take the scalar path; every element is written
    once and matches the oracle to one rounding."""
    torch_dt = torch.float32 if dt == "f32" else torch.bfloat16
    xs = synth.tensor(synth.normal(n + offset, 1), dt).cuda()
    ys = synth.tensor(synth.normal(n + offset, 2), dt).cuda()
    zs = torch.full((n + offset,), float("nan"), device="cuda", dtype=torch_dt)
    x, y, z = xs[offset:], ys[offset:], zs[offset:]
    p = tp.tp_partition_create(ctx, z, (tile,))
    counts = torch.zeros(n, dtype=torch.int32, device="cuda")
    owner = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    tp.tp_map_axpy(ctx, p, 0.5, x, y, tp.make_exec(write_counts=counts, write_owner=owner))
    tp.tp_partition_destroy(p)
    ref = omaps.axpy(0.5, x.cpu(), y.cpu())
    if dt == "bf16":
        ref = lowp.round_bf16(ref)
        assert np.array_equal(z.cpu().double().numpy(), ref)   # fp32 fma of bf16 values, one bf16 rounding
    else:
        assert np.all(np.abs(z.cpu().double().numpy() - ref) <= 2.0 ** -24 * np.abs(ref) + 1e-37)
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    assert np.array_equal(owner.cpu().numpy(), opart.owner_map((n,), (tile,)))
    if offset:
        assert torch.isnan(zs[:offset]).all()                   # nothing before the view was touched


def test_map_past_two_to_the_31_elements(ctx):
    """2^31 + 12345 bf16 elements (4 GiB per tensor): tiles and element
    indices past 2^31 must not wrap. Sampled around the boundary and at the
    end, against the oracle."""
    n = (1 << 31) + 12345
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    x = torch.randn(n, device="cuda", generator=g, dtype=torch.float32).to(torch.bfloat16)
    y = torch.randn(n, device="cuda", generator=g, dtype=torch.float32).to(torch.bfloat16)
    z = torch.empty_like(x)
    p = tp.tp_partition_create(ctx, z, (4096,))
    tp.tp_map_axpy(ctx, p, 0.5, x, y)
    tp.tp_partition_destroy(p)
    idx = torch.cat([torch.arange(0, 64), torch.arange((1 << 31) - 4096, (1 << 31) + 4096), torch.arange(n - 4200, n)])
    idx = idx.cuda()
    ref = lowp.round_bf16(omaps.axpy(0.5, x[idx].cpu(), y[idx].cpu()))
    assert np.array_equal(z[idx].cpu().double().numpy(), ref)
    del x, y, z
    torch.cuda.empty_cache()


@pytest.mark.parametrize("bm", [128, 256])
def test_gemm_output_past_two_to_the_31_elements(ctx, bm):
    """C of 65664 x 32768 bf16 (2.15e9 elements, 4.3 GB) with K = 64: row
    offsets row * N pass 2^31. Sampled tiles in the last rows, integer
    inputs (exact), against the oracle."""
    m, n, k = 65664, 32768, 64
    a = synth.to_bf16(synth.integers(m * k, 3, -4, 4)).reshape(m, k).cuda()
    bt = synth.to_bf16(synth.integers(n * k, 4, -4, 4)).reshape(n, k).cuda()
    c = torch.empty(m, n, device="cuda", dtype=torch.bfloat16)
    p = tp.tp_partition_create(ctx, c, (bm, 256))
    tp.tp_partition_map(p, tp.MAP_STRIDED, ctx.sm_count // (2 if bm == 256 else 1))
    tp.tp_gemm(ctx, p, a, bt.t(), tp.gemm_config(bm=bm, bn=256, group_m=8))
    tp.tp_partition_destroy(p)
    for r0, c0 in ((m - 128, n - 256), (65536, 0), (32768, 16384), (0, 0)):
        rs, cs = slice(r0, r0 + 128), slice(c0, c0 + 256)
        exact = ogemm.gemm(a[rs].cpu(), bt[cs].cpu().t())
        assert np.array_equal(c[rs, cs].cpu().double().numpy(), lowp.round_bf16(exact)), (r0, c0)
    del a, bt, c
    torch.cuda.empty_cache()
