"""GPU parity of the grouped persistent BF16 GEMM (one launch, device tile
queue, swap-AB for small M and for the partial last band of larger M on CTA
pairs) against the FP64 oracle, and queue coverage (every element of every
C_i written exactly once)."""
import numpy as np
import pytest
import torch

import paper_2606_15991_gb300 as tp
import synth
from oracle import gemm as ogemm
from oracle import grouped as ogrouped
from oracle import lowp
from oracle import partition as opart

pytestmark = pytest.mark.gpu

# (257, ...), (300, ...) and (448, ...) have a partial last 256-row band of
# at most 192 rows, which CTA pairs run as a swap-AB tail; (449, ...) and
# (1000, ...) have longer partial bands, run as normal tiles
SMALL = [(1, 300, 64), (17, 128, 136), (256, 520, 72), (257, 384, 128), (300, 1000, 200), (64, 96, 4104),
         (33, 2048, 512), (1000, 256, 64), (448, 600, 96), (449, 520, 64)]


def _problems(shapes, kind="normal", seed=0):
    probs = []
    for i, (m, n, k) in enumerate(shapes):
        if kind == "normal":
            a = synth.to_bf16(synth.normal(m * k, seed + 3 * i)).reshape(m, k)
            bt = synth.to_bf16(synth.normal(n * k, seed + 3 * i + 1)).reshape(n, k)
        else:
            a = synth.to_bf16(synth.integers(m * k, seed + 3 * i, -4, 4)).reshape(m, k)
            bt = synth.to_bf16(synth.integers(n * k, seed + 3 * i + 1, -4, 4)).reshape(n, k)
        c = torch.full((m, n), float("nan"), dtype=torch.bfloat16, device="cuda")
        probs.append((a.cuda(), bt.cuda().t(), c))
    return probs


def _run(ctx, probs, count=False, programs=0, pair=True):
    plan = tp.tp_grouped_plan_create(ctx, probs, cta_pair=pair)
    total, swapped = tp.tp_grouped_plan_info(plan)
    counts = owner = None
    if count:
        n = sum(c.numel() for _, _, c in probs)
        counts = torch.zeros(n, dtype=torch.int32, device="cuda")
        owner = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    tp.tp_grouped_gemm(ctx, plan, programs, tp.make_exec(write_counts=counts, write_owner=owner))
    tp.tp_grouped_plan_destroy(plan)
    return total, swapped, counts, owner


@pytest.mark.parametrize("pair", [True, False])
def test_small_group_parity_and_coverage(ctx, pair):
    probs = _problems(SMALL)
    total, swapped, counts, owner = _run(ctx, probs, count=True, pair=pair)
    assert swapped == [m <= 256 for m, _, _ in SMALL]
    rows = 256 if pair else 128
    cfg = [(rows, ((m + 31) // 32) * 32, True) if m <= 256 else (rows, 256, False) for m, _, _ in SMALL]
    assert total == sum(ogrouped.problem_tiles(m, n, *c)[0] for (m, n, _), c in zip(SMALL, cfg))
    for (a, b, c), shape in zip(probs, SMALL):
        assert ogemm.rel_frobenius(c.cpu(), ogemm.gemm(a.cpu(), b.cpu())) <= 1e-2, shape
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    assert owner.min().item() >= 0 and owner.max().item() < ctx.sm_count


@pytest.mark.parametrize("pair", [True, False])
@pytest.mark.parametrize("programs", [0, 1, 7])
def test_integer_group_bit_exact(ctx, programs, pair):
    probs = _problems(SMALL[:6], kind="int", seed=5)
    _run(ctx, probs, programs=programs, pair=pair)
    for a, b, c in probs:
        exact = ogemm.gemm(a.cpu(), b.cpu())
        assert np.array_equal(c.cpu().double().numpy(), lowp.round_bf16(exact))


@pytest.mark.parametrize("pair", [True, False])
def test_swap_problems_with_few_rows_bit_exact(ctx, pair):
    """Swap problems of at most 64 rows take 3 K blocks per ring stage on CTA
    pairs: K of 1, 3, 5, 8 and 10 blocks (the last stage full, holding 1 or
    2 blocks, or a single stage), integer inputs, C equal to the rounded
    exact product; the same problems on single CTAs too."""
    shapes = [(1, 256, 64), (64, 384, 192), (17, 300, 320), (33, 2048, 512), (40, 520, 640)]
    probs = _problems(shapes, kind="int", seed=9)
    _, swapped, counts, _ = _run(ctx, probs, count=True, pair=pair)
    assert all(swapped)
    for a, b, c in probs:
        exact = ogemm.gemm(a.cpu(), b.cpu())
        assert np.array_equal(c.cpu().double().numpy(), lowp.round_bf16(exact))
    assert opart.check_counts(counts.cpu().numpy())["ok"]


@pytest.mark.parametrize("pair", [True, False])
def test_swap_threshold_and_single_problem(ctx, pair):
    probs = _problems([(200, 640, 256)])
    plan = tp.tp_grouped_plan_create(ctx, probs, swap_max_m=0, cta_pair=pair)   # force the normal orientation
    assert tp.tp_grouped_plan_info(plan)[1] == [False]
    tp.tp_grouped_gemm(ctx, plan)
    tp.tp_grouped_plan_destroy(plan)
    a, b, c = probs[0]
    assert ogemm.rel_frobenius(c.cpu(), ogemm.gemm(a.cpu(), b.cpu())) <= 1e-2


def test_plan_rejections(ctx):
    a = torch.zeros(8, 100, dtype=torch.bfloat16, device="cuda")   # K*2 = 200 bytes
    b = torch.zeros(16, 100, dtype=torch.bfloat16, device="cuda").t()
    c = torch.zeros(8, 16, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(tp.TPError) as e:
        tp.tp_grouped_plan_create(ctx, [(a, b, c)])
    assert e.value.status == tp._lib.ERR_ALIGN
    with pytest.raises(tp.TPError) as e:
        tp.tp_grouped_plan_create(ctx, [(a[:, :96], b[:96, :], torch.zeros(8, 15, dtype=torch.bfloat16,
                                                                             device="cuda"))])
    assert e.value.status == tp._lib.ERR_SHAPE


def test_async_busy_and_graph_replay(ctx):
    probs = _problems(SMALL[:4], seed=9)
    plan = tp.tp_grouped_plan_create(ctx, probs)
    s, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    ev = tp.tp_event_create(ctx)
    with torch.cuda.stream(s):
        torch.cuda._sleep(100_000_000)
    tp.tp_grouped_gemm(ctx, plan, 0, tp.make_exec(mode=tp.ASYNC, stream=s, event=ev))
    with pytest.raises(tp.TPError) as e:      # the group's outputs are held by the in-flight launch
        tp.tp_grouped_gemm(ctx, plan, 0, tp.make_exec(stream=s2))
    assert e.value.status == tp._lib.ERR_BUSY
    with pytest.raises(tp.TPError) as e:
        tp.tp_grouped_plan_destroy(plan)
    assert e.value.status == tp._lib.ERR_BUSY
    tp.tp_event_wait(ev)
    eager = [c.clone() for _, _, c in probs]
    for _, _, c in probs:
        c.zero_()
    g = tp.tp_graph_begin(ctx, s)
    tp.tp_grouped_gemm(ctx, plan, 0, tp.make_exec(mode=tp.CAPTURE, stream=s))
    tp.tp_graph_end(g)
    for _ in range(3):
        tp.tp_graph_replay(g, tp.make_exec(stream=s))
    for (_, _, c), e0 in zip(probs, eager):
        assert torch.equal(c, e0)
    tp.tp_graph_destroy(g)
    tp.tp_event_destroy(ev)
    tp.tp_grouped_plan_destroy(plan)


@pytest.mark.parametrize("pair", [True, False])
def test_full_group_sampled(ctx, pair):
    """The 64-problem group (M log-uniform on [1, 4096], four (K, N) pairs,
    seed 0), launched as the benchmark launches it; per problem, error over up
    to two sampled 128 x 128 blocks of C against FP64."""
    shapes = synth.grouped_problems(64, seed=0)
    g = torch.Generator(device="cuda")
    probs = []
    for i, (m, n, k) in enumerate(shapes):
        g.manual_seed(1000 + i)
        a = torch.randn(m, k, device="cuda", generator=g).to(torch.bfloat16)
        bt = torch.randn(n, k, device="cuda", generator=g).to(torch.bfloat16)
        probs.append((a, bt.t(), torch.full((m, n), float("nan"), dtype=torch.bfloat16, device="cuda")))
    _run(ctx, probs, pair=pair)
    got, ref = [], []
    for i, ((m, n, k), (a, b, c)) in enumerate(zip(shapes, probs)):
        gm, gn = -(-m // 128), -(-n // 128)
        for tm, tn in synth.sample_tiles(gm, gn, 2, seed=i):
            rs, cs = slice(tm * 128, min(m, (tm + 1) * 128)), slice(tn * 128, min(n, (tn + 1) * 128))
            r = ogemm.gemm(a[rs].cpu(), b[:, cs].cpu())
            ref.append(r.reshape(-1))
            got.append(c[rs, cs].cpu().double().numpy().reshape(-1))
        assert not torch.isnan(c).any(), i
    assert ogemm.rel_frobenius(np.concatenate(got), np.concatenate(ref)) <= 1e-2
    del probs
    torch.cuda.empty_cache()
