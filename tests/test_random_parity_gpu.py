"""Seeded randomized parity sweeps: tensor-core GEMMs over random shapes
(ragged in every dimension), tile shapes, map kinds and program counts, and
element-wise maps over random lengths, tiles, dtypes and map kinds; each
result against the FP64 oracle, each owner map against the oracle's
schedule."""
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


def _draws(count, seed):
    u = synth.uniform(count * 8, seed, 0.0, 1.0, dtype=np.float64).reshape(count, 8)
    return u


@pytest.mark.parametrize("case", range(24))
def test_random_gemm(ctx, case):
    u = _draws(24, 101)[case]
    m = 1 + int(u[0] * 700)
    n = 8 * (1 + int(u[1] * 90))                 # C rows stay 16-byte aligned
    k = 8 * (1 + int(u[2] * 80))                 # K rows are a multiple of 16 bytes
    bm = 128 if u[3] < 0.5 else 256
    bn = (32, 64, 128, 192, 256)[int(u[4] * 5)] if bm == 128 else (64, 128, 192, 256)[int(u[4] * 4)]
    kind = tp.MAP_IDENTITY if u[5] < 0.25 else tp.MAP_STRIDED
    a = synth.to_bf16(synth.integers(m * k, 200 + case, -4, 4)).reshape(m, k).cuda()
    bt = synth.to_bf16(synth.integers(n * k, 300 + case, -4, 4)).reshape(n, k).cuda()
    c = torch.full((m, n), float("nan"), device="cuda", dtype=torch.bfloat16)
    p = tp.tp_partition_create(ctx, c, (bm, bn))
    tiles = tp.tp_partition_query(p)["num_tiles"]
    P = tiles
    if kind == tp.MAP_STRIDED:
        P = max(1, min(tiles, 1 + int(u[6] * min(tiles, ctx.sm_count // (2 if bm == 256 else 1)))))
        tp.tp_partition_map(p, kind, P)
    G = (1, 2, 8)[int(u[7] * 3)]
    counts = torch.zeros(m * n, dtype=torch.int32, device="cuda")
    owner = torch.full((m * n,), -1, dtype=torch.int32, device="cuda")
    tp.tp_gemm(ctx, p, a, bt.t(), tp.gemm_config(bm=bm, bn=bn, group_m=G),
               tp.make_exec(write_counts=counts, write_owner=owner))
    tp.tp_partition_destroy(p)
    exact = ogemm.gemm(a.cpu(), bt.cpu().t())
    assert np.array_equal(c.cpu().double().numpy(), lowp.round_bf16(exact)), (m, n, k, bm, bn, kind, P, G)
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    if kind == tp.MAP_IDENTITY:
        ref_owner = opart.gemm_owner_map(m, n, bm, bn)
    else:
        ref_owner = opart.gemm_owner_map_cut(m, n, bm, bn, P, G)
    assert np.array_equal(owner.cpu().numpy(), ref_owner), (m, n, k, bm, bn, kind, P, G)


@pytest.mark.parametrize("case", range(24))
def test_random_map(ctx, case):
    u = _draws(24, 202)[case]
    n = 1 + int(u[0] ** 2 * 300000)
    dt = "f32" if u[1] < 0.5 else "bf16"
    tile = (1, 7, 64, 1000, 4096, 8192)[int(u[2] * 6)]
    kinds = (tp.MAP_IDENTITY, tp.MAP_STRIDED, tp.MAP_QUEUE)
    kind = kinds[int(u[3] * 3)]
    op = ("axpy", "gelu_mul", "scale", "add_accum")[int(u[4] * 4)]
    x = synth.tensor(synth.normal(n, 400 + case), dt).cuda()
    y = synth.tensor(synth.normal(n, 500 + case), dt).cuda()
    c0 = synth.tensor(synth.normal(n, 600 + case), dt).cuda()
    out = c0.clone() if op == "add_accum" else torch.full_like(x, float("nan"))
    p = tp.tp_partition_create(ctx, out, (tile,))
    tiles = tp.tp_partition_query(p)["num_tiles"]
    P = tiles
    if kind != tp.MAP_IDENTITY:
        P = max(1, min(tiles, 1 + int(u[5] * 600)))
        tp.tp_partition_map(p, kind, P)
    counts = torch.zeros(n, dtype=torch.int32, device="cuda")
    owner = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    ex = tp.make_exec(write_counts=counts, write_owner=owner)
    {"axpy": lambda: tp.tp_map_axpy(ctx, p, 0.5, x, y, ex),
     "gelu_mul": lambda: tp.tp_map_gelu_mul(ctx, p, x, y, ex),
     "scale": lambda: tp.tp_map_scale(ctx, p, x, y, ex),
     "add_accum": lambda: tp.tp_map_add_accum(ctx, p, x, y, ex)}[op]()
    tp.tp_partition_destroy(p)
    ref = {"axpy": lambda: omaps.axpy(0.5, x.cpu(), y.cpu()), "gelu_mul": lambda: omaps.gelu_mul(x.cpu(), y.cpu()),
           "scale": lambda: omaps.scale(x.cpu(), y.cpu()),
           "add_accum": lambda: omaps.add_accum(c0.cpu(), x.cpu(), y.cpu())}[op]().reshape(-1)
    got = out.cpu().double().numpy().reshape(-1)
    r = np.abs(ref)
    if op == "add_accum":
        bound = 2 * 2.0 ** -24 * (np.abs(c0.cpu().double().numpy()) + np.abs(x.cpu().double().numpy())
                                  + np.abs(y.cpu().double().numpy()))
    elif op == "gelu_mul":
        bound = 2e-5 * r
    else:
        bound = 2.0 ** -24 * r
    if dt == "bf16":
        bound = bound + (2.0 ** -8 + 2.0 ** -24) * r
    assert np.all(np.abs(got - ref) <= bound + 1e-37), (n, dt, tile, kind, op)
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    if kind != tp.MAP_QUEUE:                       # the queue decides owners at run time
        kname = {tp.MAP_IDENTITY: "identity", tp.MAP_STRIDED: "strided"}[kind]
        assert np.array_equal(owner.cpu().numpy(), opart.owner_map((n,), (tile,), P, kname))
    else:
        assert owner.min().item() >= 0 and owner.max().item() < P


@pytest.mark.parametrize("case", range(8))
def test_random_grouped(ctx, case):
    """Random groups (1..24 problems, M in [1, 900], N in [1, 700], K a
    multiple of 8 up to 512, both orientations, single CTAs or pairs):
    integer inputs, every C_i bit-exact against the oracle and every element
    of every C_i written exactly once."""
    from oracle import grouped as ogrouped

    u = synth.uniform(8 * 64, 700, 0.0, 1.0, dtype=np.float64).reshape(8, 64)[case]
    count = 1 + int(u[0] * 24)
    pair = u[1] < 0.5
    probs, shapes = [], []
    for i in range(count):
        m = 1 + int(u[2 + 3 * (i % 20)] ** 2 * 900)
        n = 1 + int(u[3 + 3 * (i % 20)] * 700)
        k = 8 * (1 + int(u[4 + 3 * (i % 20)] * 64))
        a = synth.to_bf16(synth.integers(m * k, 800 + 10 * case + i, -4, 4)).reshape(m, k).cuda()
        bt = synth.to_bf16(synth.integers(n * k, 900 + 10 * case + i, -4, 4)).reshape(n, k).cuda()
        probs.append((a, bt.t(), torch.full((m, n), float("nan"), device="cuda", dtype=torch.bfloat16)))
        shapes.append((m, n, k))
    plan = tp.tp_grouped_plan_create(ctx, probs, cta_pair=pair)
    total, swapped = tp.tp_grouped_plan_info(plan)
    assert swapped == [m <= 256 for m, _, _ in shapes]
    n_el = sum(m * n for m, n, _ in shapes)
    counts = torch.zeros(n_el, dtype=torch.int32, device="cuda")
    owner = torch.full((n_el,), -1, dtype=torch.int32, device="cuda")
    tp.tp_grouped_gemm(ctx, plan, 0, tp.make_exec(write_counts=counts, write_owner=owner))
    tp.tp_grouped_plan_destroy(plan)
    for (a, b, c), shape in zip(probs, shapes):
        exact = ogemm.gemm(a.cpu(), b.cpu())
        assert np.array_equal(c.cpu().double().numpy(), lowp.round_bf16(exact)), shape
    assert opart.check_counts(counts.cpu().numpy())["ok"]
