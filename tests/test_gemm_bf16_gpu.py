"""GPU parity of the BF16 tcgen05 GEMM (TMA -> shared-memory ring -> tcgen05.mma
-> TMEM -> bf16 epilogue) against the FP64 oracle, and its tile coverage, for
64-row tiles (tcgen05 M = 64), 128-row tiles and 256-row tiles on CTA pairs."""
import numpy as np
import pytest
import torch

import paper_2606_15991_gb300 as tp
import synth
from oracle import gemm as ogemm
from oracle import lowp
from oracle import partition as opart

pytestmark = pytest.mark.gpu


def _bf16(n, seed, kind="normal", lo=-4, hi=4):
    if kind == "normal":
        return synth.to_bf16(synth.normal(n, seed))
    return synth.to_bf16(synth.integers(n, seed, lo, hi))


def _operands(m, n, k, seed=0, kind="normal"):
    a = _bf16(m * k, seed, kind).reshape(m, k).cuda()
    bt = _bf16(n * k, seed + 1, kind).reshape(n, k).cuda()      # B stored N x K (K-major)
    return a, bt


def _gemm(ctx, a, bt, bn=128, kind=tp.MAP_STRIDED, P=None, group_m=1, stages=0, count=False, bm=128,
          checked=False, split_k=0, cut_limit=0, out=None, bk=0):
    m, n = a.shape[0], bt.shape[0]
    c = torch.full((m, n), float("nan"), device="cuda", dtype=torch.bfloat16) if out is None else out
    p = tp.tp_partition_create(ctx, c, (bm, bn))
    if kind != tp.MAP_IDENTITY:
        tiles = tp.tp_partition_query(p)["num_tiles"]
        default = ctx.sm_count // 2 if bm == 256 else ctx.sm_count
        tp.tp_partition_map(p, kind, tiles if split_k > 1 and P is None else min(P or default, tiles))
    counts = owner = None
    if count:
        counts = torch.zeros(m * n, dtype=torch.int32, device="cuda")
        owner = torch.full((m * n,), -1, dtype=torch.int32, device="cuda")
    tp.tp_gemm(ctx, p, a, bt.t(), tp.gemm_config(bm=bm, bn=bn, group_m=group_m, stages=stages, split_k=split_k,
                                                 cut_limit=cut_limit, bk=bk),
               tp.make_exec(write_counts=counts, write_owner=owner, checked=checked))
    info = tp.tp_partition_query(p)
    tp.tp_partition_destroy(p)
    return c, counts, owner, info


@pytest.mark.parametrize("bm,bn", [(64, 32), (64, 64), (64, 96), (64, 128), (64, 192), (64, 256),
                                   (128, 32), (128, 64), (128, 96), (128, 128), (128, 160), (128, 192), (128, 256),
                                   (256, 64), (256, 128), (256, 192), (256, 256)])
def test_random_within_tolerance(ctx, bm, bn):
    m, n, k = 384, 512, 640
    a, bt = _operands(m, n, k, seed=bn)
    c, _, _, _ = _gemm(ctx, a, bt, bn=bn, bm=bm)
    ref = ogemm.gemm(a.cpu(), bt.cpu().t())
    err = ogemm.rel_frobenius(c.cpu(), ref)
    assert err <= 1e-2
    assert err <= 5e-3          # expected ~2e-3: bf16 output rounding dominates


@pytest.mark.parametrize("bm", [64, 128, 256])
@pytest.mark.parametrize("kind", [tp.MAP_IDENTITY, tp.MAP_STRIDED])
def test_integer_inputs_bit_exact(ctx, kind, bm):
    """Integer entries in [-4, 4]: every partial sum is exact in FP32, so C must
    equal the round-to-nearest-even bf16 of the exact integer product."""
    m, n, k = 256, 384, 512
    a, bt = _operands(m, n, k, seed=3, kind="int")
    c, _, _, _ = _gemm(ctx, a, bt, bn=128, kind=kind, P=5, bm=bm)
    exact = ogemm.gemm(a.cpu(), bt.cpu().t())
    assert np.array_equal(c.cpu().double().numpy(), lowp.round_bf16(exact))


def test_identity_and_permutation_bit_exact(ctx):
    k = 256
    bt = _bf16(192 * k, 5).reshape(192, k).cuda()             # B^T: 192 x 256
    eye = torch.eye(k, dtype=torch.bfloat16, device="cuda")
    c, _, _, _ = _gemm(ctx, eye, bt, bn=64)                    # I . B = B
    assert torch.equal(c, bt.t())
    perm = torch.tensor([(53 * i + 7) % k for i in range(k)])
    P = torch.zeros(k, k, dtype=torch.bfloat16)
    P[torch.arange(k), perm] = 1.0
    c, _, _, _ = _gemm(ctx, P.cuda(), bt, bn=64)
    assert torch.equal(c, bt.t()[perm.cuda()])


@pytest.mark.parametrize("bm", [64, 128, 256])
@pytest.mark.parametrize("m,n,k", [(1, 32, 8), (129, 65, 72), (300, 200, 136), (130, 1000, 8), (7, 8, 4104)])
def test_ragged_shapes(ctx, m, n, k, bm):
    a, bt = _operands(m, n, k, seed=m + n)
    c, counts, owner, info = _gemm(ctx, a, bt, bn=64, count=True, P=3, bm=bm)
    ref = ogemm.gemm(a.cpu(), bt.cpu().t())
    assert ogemm.rel_frobenius(c.cpu(), ref) <= 1e-2
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    assert np.array_equal(owner.cpu().numpy(), opart.gemm_owner_map_cut(m, n, bm, 64, info["num_programs"], 1))


@pytest.mark.parametrize("bm", [64, 128, 256])
@pytest.mark.parametrize("P,group_m,stages", [(7, 2, 0), (148, 8, 3), (1, 1, 2), (64, 4, 6)])
def test_mapped_partition_coverage(ctx, P, group_m, stages, bm):
    m, n, k = 1024, 1280, 256
    a, bt = _operands(m, n, k, seed=P)
    c, counts, owner, info = _gemm(ctx, a, bt, bn=128, P=P, group_m=group_m, stages=stages, count=True, bm=bm)
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    assert np.array_equal(owner.cpu().numpy(),
                          opart.gemm_owner_map_cut(m, n, bm, 128, info["num_programs"], group_m))
    assert ogemm.rel_frobenius(c.cpu(), ogemm.gemm(a.cpu(), bt.cpu().t())) <= 1e-2
    # without cutting the last round, the owners are exactly the strided map's
    c1, counts1, owner1, info1 = _gemm(ctx, a, bt, bn=128, P=P, group_m=group_m, stages=stages, count=True, bm=bm,
                                       cut_limit=1)
    assert np.array_equal(owner1.cpu().numpy(),
                          opart.gemm_owner_map(m, n, bm, 128, info1["num_programs"], "strided", group_m))
    assert torch.equal(c1, c)


@pytest.mark.parametrize("bm", [64, 128, 256])
def test_plain_partition_one_program_per_tile(ctx, bm):
    m, n, k = 512, 768, 128
    a, bt = _operands(m, n, k, seed=9)
    c, counts, owner, info = _gemm(ctx, a, bt, bn=256, kind=tp.MAP_IDENTITY, count=True, bm=bm)
    assert info["num_programs"] == info["num_tiles"] == (512 // bm) * 3
    assert np.array_equal(owner.cpu().numpy(), opart.gemm_owner_map(m, n, bm, 256))
    assert ogemm.rel_frobenius(c.cpu(), ogemm.gemm(a.cpu(), bt.cpu().t())) <= 1e-2


def test_layout_and_alignment_errors(ctx):
    a = torch.zeros(256, 100, dtype=torch.bfloat16, device="cuda")    # K*2 = 200 bytes: not 16-aligned
    bt = torch.zeros(128, 100, dtype=torch.bfloat16, device="cuda")
    c = torch.zeros(256, 128, dtype=torch.bfloat16, device="cuda")
    p = tp.tp_partition_create(ctx, c, (128, 128))
    with pytest.raises(tp.TPError) as e:
        tp.tp_gemm(ctx, p, a, bt.t())
    assert e.value.status == tp._lib.ERR_ALIGN
    a2 = torch.zeros(256, 128, dtype=torch.bfloat16, device="cuda")
    b_rowmajor = torch.zeros(128, 128, dtype=torch.bfloat16, device="cuda")   # K x N, N contiguous
    with pytest.raises(tp.TPError) as e:
        tp.tp_gemm(ctx, p, a2, b_rowmajor)
    assert e.value.status == tp._lib.ERR_UNSUPPORTED
    tp.tp_partition_destroy(p)
    p = tp.tp_partition_create(ctx, c, (96, 128))             # tiles have 64, 128 or 256 rows
    with pytest.raises(tp.TPError) as e:
        tp.tp_gemm(ctx, p, a2, b_rowmajor.t())
    assert e.value.status == tp._lib.ERR_UNSUPPORTED
    tp.tp_partition_destroy(p)


def test_8192_cubed_sampled_tiles(ctx):
    """The 8192^3 configuration with N(0,1) bf16 inputs, launched as the
    benchmark launches it (76 persistent CTA pairs, 256 x 256 tiles, stages
    of 2 K blocks, raster bands of 8); error over 64 sampled 128 x 128
    output tiles against FP64."""
    M = N = K = 8192
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    a = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    bt = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    c, _, _, _ = _gemm(ctx, a, bt, bn=256, bm=256, group_m=8, bk=128)
    tiles = synth.sample_tiles(64, 64, 64, seed=0)
    rows = sorted({tm for tm, _ in tiles})
    cols = sorted({tn for _, tn in tiles})
    a_h = {tm: a[tm * 128:(tm + 1) * 128].cpu() for tm in rows}
    b_h = {tn: bt[tn * 128:(tn + 1) * 128].cpu() for tn in cols}
    got, ref = [], []
    for tm, tn in tiles:
        ref.append(ogemm.gemm(a_h[tm], b_h[tn].t()))
        got.append(c[tm * 128:(tm + 1) * 128, tn * 128:(tn + 1) * 128].cpu().double().numpy())
    err = ogemm.rel_frobenius(np.stack(got), np.stack(ref))
    assert err <= 1e-2
    del a, bt, c
    torch.cuda.empty_cache()


@pytest.mark.parametrize("bm", [64, 128, 256])
@pytest.mark.parametrize("kind,P,group_m", [(tp.MAP_IDENTITY, None, 1), (tp.MAP_STRIDED, 7, 1),
                                            (tp.MAP_STRIDED, None, 8)])
@pytest.mark.parametrize("m,n,k", [(384, 512, 640), (300, 200, 136), (1, 96, 64)])
def test_checked_launch_matches_release(ctx, bm, kind, P, group_m, m, n, k):
    """TP_EXEC_CHECKED (every tile validated against the map and claimed
    before its store) stores exactly what the release launch stores, each
    element once, and raises no race on a correct map."""
    a, bt = _operands(m, n, k, seed=m + n)
    rel, _, _, _ = _gemm(ctx, a, bt, bn=64, bm=bm, kind=kind, P=P, group_m=group_m)
    chk, counts, _, _ = _gemm(ctx, a, bt, bn=64, bm=bm, kind=kind, P=P, group_m=group_m, checked=True, count=True)
    assert torch.equal(rel, chk)
    assert opart.check_counts(counts.cpu().numpy())["ok"]


def test_checked_launch_in_a_graph(ctx):
    """The claim bitmap is cleared by a node of the graph, so every replay of
    a captured checked GEMM re-checks from scratch (no stale claims)."""
    a, bt = _operands(512, 512, 256, seed=11)
    c = torch.zeros(512, 512, device="cuda", dtype=torch.bfloat16)
    p = tp.tp_partition_create(ctx, c, (256, 128))
    tp.tp_partition_map(p, tp.MAP_STRIDED, 5)
    s = torch.cuda.Stream()
    g = tp.tp_graph_begin(ctx, s)
    tp.tp_gemm(ctx, p, a, bt.t(), tp.gemm_config(bm=256, bn=128), tp.make_exec(tp.CAPTURE, s, checked=True))
    tp.tp_graph_end(g)
    for _ in range(3):
        tp.tp_graph_replay(g, tp.make_exec(stream=s))
    ref = ogemm.gemm(a.cpu(), bt.cpu().t())
    assert ogemm.rel_frobenius(c.cpu(), ref) <= 1e-2
    tp.tp_graph_destroy(g)
    tp.tp_partition_destroy(p)


def test_checked_flag_rejected_where_unsupported(ctx):
    a = torch.ones(64, 64, device="cuda")
    c = torch.zeros(64, 64, device="cuda")
    p = tp.tp_partition_create(ctx, c, (64, 64))
    with pytest.raises(tp.TPError) as e:                      # the FP32 SIMT GEMM
        tp.tp_gemm(ctx, p, a, a, None, tp.make_exec(checked=True))
    assert e.value.status == tp._lib.ERR_UNSUPPORTED
    tp.tp_partition_destroy(p)


@pytest.mark.parametrize("bm", [64, 128, 256])
@pytest.mark.parametrize("limit", [0, 2, 3, 8])
def test_last_round_cut_along_n(ctx, bm, limit):
    """The tiles of the last, partial round cut along N into narrow tiles run
    by otherwise idle programs: every element is stored once, by the program
    the oracle's schedule names, and C is bit-identical to the uncut run
    (integer inputs: the exact product rounded once)."""
    m, n, k = 1024, 640, 512            # 128-row tiles: 8 x 5 = 40 tiles of 128 columns; 64-row: 80; 256-row: 20
    P = 9 if bm == 256 else 13          # 40 mod 13 = 1, 80 mod 13 = 2 and 20 mod 9 = 2 tiles in the last round
    bn = 128
    T = (m // bm) * (n // bn)
    D, S = opart.gemm_cut_schedule(T, P, bn, 64 if bm == 256 else 32, limit or 4)
    assert S >= 2
    a, bt = _operands(m, n, k, seed=3, kind="int")
    c, counts, owner, info = _gemm(ctx, a, bt, bn=bn, P=P, bm=bm, count=True, cut_limit=limit)
    assert np.array_equal(c.cpu().double().numpy(), lowp.round_bf16(ogemm.gemm(a.cpu(), bt.cpu().t())))
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    assert np.array_equal(owner.cpu().numpy(), opart.gemm_owner_map_cut(m, n, bm, bn, P, 1, limit or 4))
    a, bt = _operands(m, n, k, seed=4)
    c1, _, _, _ = _gemm(ctx, a, bt, bn=bn, P=P, bm=bm, cut_limit=limit)
    c0, _, _, _ = _gemm(ctx, a, bt, bn=bn, P=P, bm=bm, cut_limit=1)
    assert torch.equal(c1, c0)
    assert ogemm.rel_frobenius(c1.cpu(), ogemm.gemm(a.cpu(), bt.cpu().t())) <= 5e-3


def test_cut_limit_validation(ctx):
    a, bt = _operands(256, 256, 128)
    with pytest.raises(tp.TPError) as e:
        _gemm(ctx, a, bt, bn=64, P=3, cut_limit=9)
    assert e.value.status == tp._lib.ERR_INVALID


# ------------------------------------------------------------------ split-K
@pytest.mark.parametrize("S,bn", [(2, 64), (2, 256), (4, 128), (4, 256), (8, 256)])
@pytest.mark.parametrize("m,n,k", [(384, 512, 640), (300, 200, 1000), (1, 256, 4104), (129, 96, 520)])
def test_split_k_parity(ctx, S, bn, m, n, k):
    """split_k = S: each tile's K blocks are cut into S contiguous slices run
    by the CTAs of one cluster and summed in slice order. Integer inputs are
    exact in FP32 whatever the order, so C equals the exactly rounded product;
    N(0,1) inputs stay within the BF16 gate; two runs are bit-identical."""
    if (k + 63) // 64 < S:
        pytest.skip("fewer K blocks than slices")
    a, bt = _operands(m, n, k, seed=S + bn, kind="int")
    c, counts, owner, info = _gemm(ctx, a, bt, bn=bn, kind=tp.MAP_IDENTITY, split_k=S, count=True)
    assert np.array_equal(c.cpu().double().numpy(), lowp.round_bf16(ogemm.gemm(a.cpu(), bt.cpu().t())))
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    assert np.array_equal(owner.cpu().numpy(), opart.gemm_owner_map(m, n, 128, bn))
    a, bt = _operands(m, n, k, seed=S + bn + 1)
    c1, _, _, _ = _gemm(ctx, a, bt, bn=bn, kind=tp.MAP_IDENTITY, split_k=S)
    c2, _, _, _ = _gemm(ctx, a, bt, bn=bn, kind=tp.MAP_IDENTITY, split_k=S)
    assert torch.equal(c1, c2)
    assert ogemm.rel_frobenius(c1.cpu(), ogemm.gemm(a.cpu(), bt.cpu().t())) <= 5e-3


@pytest.mark.parametrize("S", [2, 4])
def test_split_k_strided_and_checked(ctx, S):
    """A strided map with one tile per program (P = tiles, band raster) and the
    checked launch give the same C as the identity map, each element stored
    once by the program the map names."""
    m, n, k = 512, 768, 384
    a, bt = _operands(m, n, k, seed=31 + S)
    ref, _, _, _ = _gemm(ctx, a, bt, bn=256, kind=tp.MAP_IDENTITY, split_k=S)
    c, counts, owner, info = _gemm(ctx, a, bt, bn=256, kind=tp.MAP_STRIDED, group_m=2, split_k=S, count=True)
    assert torch.equal(c, ref)
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    assert np.array_equal(owner.cpu().numpy(),
                          opart.gemm_owner_map(m, n, 128, 256, info["num_programs"], "strided", 2))
    chk, counts, _, _ = _gemm(ctx, a, bt, bn=256, kind=tp.MAP_STRIDED, group_m=2, split_k=S, checked=True,
                              count=True)
    assert torch.equal(chk, ref)
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    rel, _, _, _ = _gemm(ctx, a, bt, bn=256, kind=tp.MAP_STRIDED, group_m=2, split_k=S, checked=True)
    assert torch.equal(rel, ref)


def test_split_k_in_a_graph(ctx):
    a, bt = _operands(256, 512, 2048, seed=41)
    c = torch.zeros(256, 512, device="cuda", dtype=torch.bfloat16)
    p = tp.tp_partition_create(ctx, c, (128, 256))
    s = torch.cuda.Stream()
    g = tp.tp_graph_begin(ctx, s)
    tp.tp_gemm(ctx, p, a, bt.t(), tp.gemm_config(bm=128, bn=256, split_k=8), tp.make_exec(tp.CAPTURE, s))
    tp.tp_graph_end(g)
    for _ in range(3):
        tp.tp_graph_replay(g, tp.make_exec(stream=s))
    ref, _, _, _ = _gemm(ctx, a, bt, bn=256, kind=tp.MAP_IDENTITY, split_k=8)
    assert torch.equal(c, ref)
    assert ogemm.rel_frobenius(c.cpu(), ogemm.gemm(a.cpu(), bt.cpu().t())) <= 5e-3
    tp.tp_graph_destroy(g)
    tp.tp_partition_destroy(p)


@pytest.mark.parametrize("kw,status", [(dict(bm=256, bn=256, split_k=2), "ERR_UNSUPPORTED"),
                                       (dict(bn=256, split_k=3), "ERR_INVALID"),
                                       (dict(bn=256, split_k=16), "ERR_INVALID"),
                                       (dict(bn=64, split_k=4), "ERR_UNSUPPORTED"),      # 64 / 4 < 32 columns
                                       (dict(bn=256, split_k=8, k=448), "ERR_UNSUPPORTED"),  # 7 K blocks
                                       (dict(bn=128, split_k=2, P=3), "ERR_UNSUPPORTED")])   # tiles > programs
def test_split_k_validation(ctx, kw, status):
    kw = dict(kw)
    k = kw.pop("k", 512)
    a, bt = _operands(512, 512, k)
    with pytest.raises(tp.TPError) as e:
        _gemm(ctx, a, bt, **kw)
    assert e.value.status == getattr(tp._lib, status)


def test_split_k_resident_programs(ctx):
    one = tp.tp_gemm_resident_programs(ctx, tp.gemm_config(bm=128, bn=256))
    for S in (2, 4, 8):
        n = tp.tp_gemm_resident_programs(ctx, tp.gemm_config(bm=128, bn=256, split_k=S))
        assert 0 < n * S <= one


# ------------------------------------------------------- TMA-store epilogue
@pytest.mark.parametrize("bm", [64, 128, 256])
@pytest.mark.parametrize("m,n,k", [(129, 72, 200), (300, 200, 136), (1, 32, 8), (130, 1000, 8), (65, 65, 72)])
def test_epilogue_stays_inside_c(ctx, bm, m, n, k):
    """C is a view inside a guarded allocation: the epilogue (TMA stores
    clipped at C's bounds when rows are 16-byte aligned, plain stores
    otherwise) writes every element of C and nothing around it."""
    a, bt = _operands(m, n, k, seed=m * 7 + n)
    guard = 4096
    buf = torch.full((guard + m * n + guard,), 3.0, device="cuda", dtype=torch.bfloat16)
    c = buf[guard:guard + m * n].view(m, n)
    c.fill_(float("nan"))
    _gemm(ctx, a, bt, bn=64, bm=bm, P=3, out=c)
    assert torch.all(buf[:guard] == 3.0) and torch.all(buf[guard + m * n:] == 3.0)
    assert ogemm.rel_frobenius(c.cpu(), ogemm.gemm(a.cpu(), bt.cpu().t())) <= 1e-2


def test_plain_and_staged_epilogues_agree(ctx):
    """256 x 256 tiles on CTA pairs: a 7-stage ring leaves no room for the
    staging area (plain stores), the default 6-stage ring stages C for TMA
    stores; both round the same FP32 sums, so C is bit-identical."""
    a, bt = _operands(1024, 768, 1024, seed=51)
    c6, _, _, _ = _gemm(ctx, a, bt, bn=256, bm=256, P=5)
    c7, _, _, _ = _gemm(ctx, a, bt, bn=256, bm=256, P=5, stages=7)
    assert torch.equal(c6, c7)


@pytest.mark.parametrize("bm,P", [(64, 0), (64, 9), (128, 0), (128, 7), (256, 0), (256, 5)])
def test_unchecked_raw_pointer_gemm_matches_partitioned(ctx, bm, P):
    """tp_gemm_unchecked runs the same schedule on a raw C pointer: C is
    bit-identical to tp_gemm on the equivalent partition (plain for
    num_programs = 0, strided otherwise), and matches the oracle."""
    m, n, k = 640, 768, 320
    a, bt = _operands(m, n, k, seed=21)
    kind = tp.MAP_IDENTITY if P == 0 else tp.MAP_STRIDED
    ref, _, _, _ = _gemm(ctx, a, bt, bn=128, kind=kind, P=P or None, bm=bm)
    c = torch.full((m, n), float("nan"), device="cuda", dtype=torch.bfloat16)
    s = torch.cuda.Stream()
    tp.tp_gemm_unchecked(ctx, c, a, bt.t(), tp.gemm_config(bm=bm, bn=128, num_programs=P), s)
    s.synchronize()
    assert torch.equal(c, ref)
    assert ogemm.rel_frobenius(c.cpu(), ogemm.gemm(a.cpu(), bt.cpu().t())) <= 1e-2
    with pytest.raises(tp.TPError) as e:
        tp.tp_gemm_unchecked(ctx, c, a, bt.t(), tp.gemm_config(bm=96, bn=128), s)
    assert e.value.status == tp._lib.ERR_INVALID


def test_resident_programs(ctx):
    """The resident-program query: CTA pairs for 256-row tiles, CTAs for
    64- and 128-row tiles, never more than the SMs allow."""
    pairs = tp.tp_gemm_resident_programs(ctx, tp.gemm_config(bm=256, bn=256))
    ctas = tp.tp_gemm_resident_programs(ctx, tp.gemm_config(bm=128, bn=256))
    ctas64 = tp.tp_gemm_resident_programs(ctx, tp.gemm_config(bm=64, bn=64))
    print(f"resident: {ctas} CTAs, {pairs} CTA pairs, {ctas64} CTAs of 64 x 64 tiles")
    assert 0 < pairs <= ctx.sm_count // 2 and 0 < ctas <= ctx.sm_count and 0 < ctas64 <= ctx.sm_count
    with pytest.raises(tp.TPError) as e:
        tp.tp_gemm_resident_programs(ctx, tp.gemm_config(bm=96, bn=256))
    assert e.value.status == tp._lib.ERR_UNSUPPORTED
    # swap-AB tiles run on CTA pairs
    for w in (32, 64, 128):
        sw = tp.tp_gemm_resident_programs(ctx, tp.gemm_config(bm=w, bn=128, bk=256, swap_ab=1))
        assert 0 < sw <= ctx.sm_count // 2, (w, sw)
    with pytest.raises(tp.TPError) as e:
        tp.tp_gemm_resident_programs(ctx, tp.gemm_config(bm=64, bn=64, swap_ab=1))
    assert e.value.status == tp._lib.ERR_UNSUPPORTED


@pytest.mark.parametrize("bn", [96, 160, 224])
def test_epilogue_mixed_block_widths_bit_exact(ctx, bn):
    """Tile widths that are odd multiples of 32 columns store 32 x 64 blocks
    and one 32 x 32 block per 32-row slice; integer inputs make C exact, so
    every element is checked, including ragged edges."""
    m, n, k = 300, 3 * bn + 40, 256
    a, bt = _operands(m, n, k, seed=bn, kind="int")
    c, _, _, _ = _gemm(ctx, a, bt, bn=bn, P=5)
    assert np.array_equal(c.cpu().double().numpy(), lowp.round_bf16(ogemm.gemm(a.cpu(), bt.cpu().t())))


@pytest.mark.parametrize("m", [1, 16, 64, 65, 100])
def test_64_row_tiles_equal_128_row_tiles(ctx, m):
    """A 64-row tile (tcgen05 M = 64: D row r in TMEM lane 32(r/16) + r%16)
    accumulates each C element over K in the same order as a 128-row tile,
    so C is bit-identical, and both equal the exact integer product rounded
    once when every partial sum is exact."""
    n, k = 640, 1032
    a, bt = _operands(m, n, k, seed=m)
    c64, counts, owner, info = _gemm(ctx, a, bt, bn=128, bm=64, P=7, count=True)
    c128, _, _, _ = _gemm(ctx, a, bt, bn=128, bm=128, P=7)
    assert torch.equal(c64, c128)
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    assert np.array_equal(owner.cpu().numpy(), opart.gemm_owner_map_cut(m, n, 64, 128, info["num_programs"], 1))
    ai, bi = _operands(m, n, k, seed=m + 1, kind="int")
    c, _, _, _ = _gemm(ctx, ai, bi, bn=64, bm=64, P=5)
    assert np.array_equal(c.cpu().double().numpy(), lowp.round_bf16(ogemm.gemm(ai.cpu(), bi.cpu().t())))


@pytest.mark.parametrize("bm,bn", [(64, 64), (128, 128), (128, 256), (256, 256)])
@pytest.mark.parametrize("bk", [128, 256])
@pytest.mark.parametrize("m,n,k", [(300, 520, 1024), (129, 200, 448), (64, 256, 192), (257, 96, 4160)])
def test_multi_block_stages_bit_identical(ctx, bm, bn, bk, m, n, k):
    """Stages of 2 or 4 K blocks (each operand one 3-D TMA box per stage;
    K-block counts that do not fill the last stage leave zero-filled blocks
    that are not multiplied) issue the same MMAs in the same K order as one
    block per stage: C is bit-identical, every element stored once, and the
    integer product exact."""
    if bm == 256 and bn % 64:
        pytest.skip("256-row tiles take multiples of 64 columns")
    a, bt = _operands(m, n, k, seed=k + bm)
    ref, _, _, _ = _gemm(ctx, a, bt, bn=bn, bm=bm, P=7)
    c = torch.full((m, n), float("nan"), device="cuda", dtype=torch.bfloat16)
    p = tp.tp_partition_create(ctx, c, (bm, bn))
    tp.tp_partition_map(p, tp.MAP_STRIDED, min(7, tp.tp_partition_query(p)["num_tiles"]))
    counts = torch.zeros(m * n, dtype=torch.int32, device="cuda")
    owner = torch.full((m * n,), -1, dtype=torch.int32, device="cuda")
    tp.tp_gemm(ctx, p, a, bt.t(), tp.gemm_config(bm=bm, bn=bn, bk=bk), tp.make_exec(write_counts=counts,
                                                                                    write_owner=owner))
    tp.tp_partition_destroy(p)
    assert torch.equal(c, ref)
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    ai, bi = _operands(m, n, k, seed=k + bm + 1, kind="int")
    c2 = torch.empty(m, n, device="cuda", dtype=torch.bfloat16)
    p = tp.tp_partition_create(ctx, c2, (bm, bn))
    tp.tp_partition_map(p, tp.MAP_STRIDED, min(5, tp.tp_partition_query(p)["num_tiles"]))
    tp.tp_gemm(ctx, p, ai, bi.t(), tp.gemm_config(bm=bm, bn=bn, bk=bk))
    tp.tp_partition_destroy(p)
    assert np.array_equal(c2.cpu().double().numpy(), lowp.round_bf16(ogemm.gemm(ai.cpu(), bi.cpu().t())))


def test_multi_block_stages_fallback_and_validation(ctx):
    """K not a multiple of the 64-element K block runs one block per stage
    (same C); bk values other than 1, 2 or 4 K blocks are refused."""
    m, n, k = 200, 256, 520
    a, bt = _operands(m, n, k, seed=77)
    ref, _, _, _ = _gemm(ctx, a, bt, bn=128, bm=128, P=3)
    c, _, _, _ = _gemm(ctx, a, bt, bn=128, bm=128, P=3, bk=256)
    assert torch.equal(c, ref)
    for bad in (96, 192, 512):
        with pytest.raises(tp.TPError) as e:
            _gemm(ctx, a, bt, bn=128, bm=128, P=3, bk=bad)
        assert e.value.status == tp._lib.ERR_INVALID


def _swap_gemm(ctx, a, bt, w, P, bk=0, count=False, checked=False):
    """C = A B on swap-AB tiles (cfg.swap_ab): the partition's tiles are W
    rows x 128 columns of C, each computed as C^T = B^T A^T by a CTA pair."""
    m, n = a.shape[0], bt.shape[0]
    c = torch.full((m, n), float("nan"), device="cuda", dtype=torch.bfloat16)
    p = tp.tp_partition_create(ctx, c, (w, 128))
    tp.tp_partition_map(p, tp.MAP_STRIDED, min(P, tp.tp_partition_query(p)["num_tiles"]))
    counts = owner = None
    if count:
        counts = torch.zeros(m * n, dtype=torch.int32, device="cuda")
        owner = torch.full((m * n,), -1, dtype=torch.int32, device="cuda")
    tp.tp_gemm(ctx, p, a, bt.t(), tp.gemm_config(bm=w, bn=128, bk=bk, swap_ab=1),
               tp.make_exec(write_counts=counts, write_owner=owner, checked=checked))
    info = tp.tp_partition_query(p)
    tp.tp_partition_destroy(p)
    return c, counts, owner, info


@pytest.mark.parametrize("w", [32, 64, 128])
@pytest.mark.parametrize("bk", [64, 256])
@pytest.mark.parametrize("m,n,k", [(64, 1024, 1024), (37, 520, 2048), (128, 384, 1088), (1, 300, 192),
                                   (100, 1160, 640)])
def test_swap_ab_tiles(ctx, w, bk, m, n, k):
    """Swap-AB tiles: the MMA's 128 rows are C columns (64 rows of B^T per
    CTA of the pair) and its W columns are C rows (W/2 rows of A per CTA); the
    epilogue writes each TMEM lane's values down a column of C. Integer inputs
    give the exact product rounded once; random inputs are within the BF16
    gate of the FP64 oracle and equal a normal tile's C; every element is
    stored once, by the program the strided map gives its tile."""
    a, bt = _operands(m, n, k, seed=w + k, kind="int")
    c, counts, owner, info = _swap_gemm(ctx, a, bt, w, P=5, bk=bk, count=True)
    assert np.array_equal(c.cpu().double().numpy(), lowp.round_bf16(ogemm.gemm(a.cpu(), bt.cpu().t())))
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    assert np.array_equal(owner.cpu().numpy(),
                          opart.gemm_owner_map_cut(m, n, w, 128, info["num_programs"], 1, limit=1))
    a, bt = _operands(m, n, k, seed=w + k + 1)
    c, _, _, _ = _swap_gemm(ctx, a, bt, w, P=7, bk=bk)
    assert ogemm.rel_frobenius(c.cpu(), ogemm.gemm(a.cpu(), bt.cpu().t())) <= 5e-3
    # each C element is accumulated over K in the same order as on a normal
    # tile, so C is bit-identical to it (swap-AB is in the autotuner's
    # single-pass class)
    ref, _, _, _ = _gemm(ctx, a, bt, bn=64, bm=64, P=7)
    assert torch.equal(c, ref)


def test_swap_ab_checked_raw_and_validation(ctx):
    """The checked launch claims swap-AB tiles like any other (same C); the
    raw-pointer entry runs the same schedule; swap_ab with FP8, with tiles
    other than W x 128, or with split_k is refused."""
    m, n, k = 64, 1000, 512
    a, bt = _operands(m, n, k, seed=41)
    ref, _, _, _ = _swap_gemm(ctx, a, bt, 64, P=3, bk=128)
    c, _, _, _ = _swap_gemm(ctx, a, bt, 64, P=3, bk=128, checked=True)
    assert torch.equal(c, ref)
    for w in (64, 32):
        raw = torch.full((m, n), float("nan"), device="cuda", dtype=torch.bfloat16)
        tp.tp_gemm_unchecked(ctx, raw, a, bt.t(), tp.gemm_config(bm=w, bn=128, bk=128, swap_ab=1, num_programs=3))
        torch.cuda.synchronize()
        assert torch.equal(raw, ref), w
    for tile, kw in (((64, 64), {}), ((48, 128), {}), ((64, 128), {"split_k": 2})):
        cc = torch.empty(m, n, device="cuda", dtype=torch.bfloat16)
        p = tp.tp_partition_create(ctx, cc, tile)
        tp.tp_partition_map(p, tp.MAP_STRIDED, 2)
        with pytest.raises(tp.TPError) as e:
            tp.tp_gemm(ctx, p, a, bt.t(), tp.gemm_config(bm=tile[0], bn=tile[1], swap_ab=1, **kw))
        assert e.value.status == tp._lib.ERR_UNSUPPORTED
        tp.tp_partition_destroy(p)
    # swap_ab values other than 0 and 1 are reserved
    cc = torch.empty(m, n, device="cuda", dtype=torch.bfloat16)
    p = tp.tp_partition_create(ctx, cc, (64, 128))
    with pytest.raises(tp.TPError) as e:
        tp.tp_gemm(ctx, p, a, bt.t(), tp.gemm_config(bm=64, bn=128, swap_ab=2))
    assert e.value.status == tp._lib.ERR_INVALID
    tp.tp_partition_destroy(p)
