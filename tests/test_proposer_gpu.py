"""GPU tests of the autotuner and the learned tile proposer: the MLP's
forward, gradients and Adam steps against the FP64 oracle, the autotuner's
table and cache, the single-pass class (configs that give bit-identical C,
the only ones a proposal may pick), proposals equal to the exhaustive pick
bit for bit on held-out shapes, and a small end-to-end train/evaluate run
measured against the best fixed config, the untrained network and
exhaustive tuning time."""
import os

import numpy as np
import pytest
import torch

import paper_2606_15991_gb300 as tp
import synth
from oracle import gemm as ogemm
from oracle import mlp as omlp
from paper_2606_15991_gb300 import proposer

pytestmark = pytest.mark.gpu

F, H, C = 5, 64, 32


def _split(flat):
    o, out = 0, {}
    for k, shape in (("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (C, H)), ("b3", (C,))):
        n = int(np.prod(shape))
        out[k] = np.asarray(flat[o:o + n], np.float64).reshape(shape)
        o += n
    return out


def _flat(p):
    return np.concatenate([p[k].reshape(-1) for k in omlp.PARAMS])


def _batch(B=96, seed=0):
    X = synth.uniform(B * F, seed, 0, 14, dtype=np.float64).reshape(B, F).astype(np.float32)
    T = synth.uniform(B * C, seed + 1, 0, 1, dtype=np.float64).reshape(B, C).astype(np.float32)
    V = (synth.uniform(B * C, seed + 2, 0, 1, dtype=np.float64) > 0.2).astype(np.float32).reshape(B, C)
    return X, T, V


def test_mlp_forward_grad_adam_match_oracle(ctx):
    p0 = proposer.init_params(F, H, C, seed=3)
    X, T, V = _batch()
    m = tp.tp_mlp_create(ctx, F, H, C, 96, p0)
    Xd, Td, Vd = (torch.from_numpy(a).cuda() for a in (X, T, V))
    Y = torch.empty(96, C, device="cuda")
    tp.tp_mlp_forward(m, Xd, Y)
    P = _split(p0)
    Yref, cache = omlp.forward(P, X.astype(np.float64))
    assert np.max(np.abs(Y.cpu().numpy() - Yref)) <= 1e-5 * max(1.0, np.abs(Yref).max())
    loss = torch.zeros(1, device="cuda")
    G = torch.empty(len(p0), device="cuda")
    tp.tp_mlp_loss_grad(m, Xd, Td, Vd, loss, G)
    assert abs(loss.item() - omlp.loss(Yref, T, V)) <= 1e-5 * omlp.loss(Yref, T, V)
    gref = _flat(omlp.backward(P, cache, Yref, T, V))
    assert np.linalg.norm(G.cpu().numpy() - gref) <= 1e-4 * np.linalg.norm(gref)
    # three Adam steps against the oracle's trajectory
    mom = {k: np.zeros_like(v) for k, v in P.items()}
    vel = {k: np.zeros_like(v) for k, v in P.items()}
    for t in range(1, 4):
        tp.tp_mlp_train_step(m, Xd, Td, Vd, 1e-3, loss)
        Yr, cr = omlp.forward(P, X.astype(np.float64))
        P, mom, vel = omlp.adam_step(P, omlp.backward(P, cr, Yr, T, V), mom, vel, t, 1e-3)
    got = tp.tp_mlp_get_params(m)
    assert np.max(np.abs(got - _flat(P))) <= 1e-5
    tp.tp_mlp_destroy(m)


def test_mlp_learns_separable_toy_on_gpu(ctx):
    S = 512
    X = synth.uniform(S * F, 40, 0, 1, dtype=np.float64).reshape(S, F).astype(np.float32)
    cls = X[:, :3].argmax(axis=1)
    T = np.zeros((S, C), np.float32)
    T[np.arange(S), cls] = 1.0
    V = np.ones_like(T)
    mlp, hist = proposer.train(ctx, X, T, V, epochs=150, batch=128, lr=1e-2, seed=5)
    assert hist[-1] < 0.2 * hist[0]
    acc = (proposer.scores(mlp, X).argmax(axis=1) == cls).mean()
    assert acc > 0.95
    tp.tp_mlp_destroy(mlp)


def test_features_targets_and_save_load(ctx, tmp_path):
    assert tp.tp_mlp_features(1024, 3, 16384, "fp8") == pytest.approx(list(omlp.features(1024, 3, 16384, 1)))
    # a config that did not run (0 TFLOP/s) is trained towards score 0
    tg, mk = tp.tp_mlp_targets([2.0, 0.0, 4.0, 1.0])
    assert tg == [0.5, 0.0, 1.0, 0.25] and mk == [1.0, 1.0, 1.0, 1.0]
    tg, mk = tp.tp_mlp_targets([0.0, 0.0])
    assert tg == [0.0, 0.0] and mk == [0.0, 0.0]
    p0 = proposer.init_params(F, H, C, seed=9)
    m = tp.tp_mlp_create(ctx, F, H, C, 8, p0)
    path = os.path.join(tmp_path, "mlp.txt")
    tp.tp_mlp_save(m, path)
    tp.tp_mlp_set_params(m, np.zeros_like(p0))
    tp.tp_mlp_load(m, path)
    assert np.array_equal(tp.tp_mlp_get_params(m), p0)
    tp.tp_mlp_destroy(m)


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_autotune_table_cache_and_numerics(ctx, dtype, tmp_path):
    space = tp.tp_autotune_space(dtype)
    assert len(space) == 72 and all(cfg.split_k <= 1 and not cfg.swap_ab for cfg in space)
    M, N, K = 700, 900, 1024
    best, table, best_tf = tp.tp_autotune(ctx, M, N, K, dtype)
    assert len(table) == len(space) and all(t > 0 for t in table)
    assert best_tf == max(table) or best_tf >= 0.99 * max(table)
    assert best.split_k <= 1
    assert tp.tp_autotune_lookup(ctx, M, N, K, dtype).bn == best.bn
    assert tp.tp_autotune_lookup(ctx, M, N, K, dtype, split_k=True) is None     # that search has not run
    # the split-K opt-in times the same 72 configs plus the split ones
    best_s, table_s, _ = tp.tp_autotune(ctx, M, N, K, dtype, split_k=True)
    assert len(table_s) == 77 and all(t > 0 for t in table_s[:72])
    assert tp.tp_autotune_lookup(ctx, M, N, K, dtype, split_k=True) is not None
    t = tp.tp_autotune_time(ctx, M, N, K, dtype, best, repeats=3)
    assert 0.5 * best_tf < t < 2.0 * best_tf
    path = os.path.join(tmp_path, "cache.txt")
    tp.tp_autotune_save(ctx, path)
    tp.tp_autotune_load(ctx, path)
    assert tp.tp_autotune_lookup(ctx, M, N, K, dtype).bn == best.bn
    # every single-pass config computes the same C (each element is summed
    # over K in the same order by one program), so tuning or proposing among
    # them never changes numerics; split-K configs sum K slices in a fixed
    # order of their own (deterministic, within the BF16 gate)
    if dtype == "bf16":
        a = synth.to_bf16(synth.normal(M * K, 1)).reshape(M, K).cuda()
        bt = synth.to_bf16(synth.normal(N * K, 2)).reshape(N, K).cuda()
        ref = None
        for cfg in tp.tp_autotune_space(dtype, split_k=True, swap_ab=True):
            c = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
            p = tp.tp_partition_create(ctx, c, (cfg.bm, cfg.bn))
            tiles = tp.tp_partition_query(p)["num_tiles"]
            pair = cfg.bm == 256 or cfg.swap_ab
            tp.tp_partition_map(p, tp.MAP_STRIDED, min(tiles, ctx.sm_count // (2 if pair else 1)))
            tp.tp_gemm(ctx, p, a, bt.t(), cfg)
            tp.tp_partition_destroy(p)
            if cfg.split_k > 1:
                assert ogemm.rel_frobenius(c.cpu(), ogemm.gemm(a.cpu(), bt.cpu().t())) <= 5e-3
            elif ref is None:
                ref = c
            else:
                assert torch.equal(c, ref)


@pytest.fixture(scope="module")
def trained(ctx):
    """A proposer trained on 512 exhaustively tuned shapes (both dtypes,
    dimensions log-uniform on [1, 16384], the benchmark's range), with its
    training tables."""
    shapes = proposer.sample_shapes(512, seed=1)
    X, T, V, TF = proposer.collect(ctx, shapes)
    mlp, hist = proposer.train(ctx, X, T, V, epochs=400, batch=64, lr=3e-3)
    yield mlp, hist, T, V
    tp.tp_mlp_destroy(mlp)


def test_small_end_to_end_gain(ctx, trained):
    """Evaluate the trained proposer on 200 held-out shapes of the same range.
    It must reach the stated median regret (<= 5% of the exhaustive best) and
    lose less than the same network untrained. Against the best fixed config
    (the method without it: the config with the best mean relative speed over
    the training shapes) it must lose less in mean and in p90 regret, with the
    proposal, the exhaustive pick and the default re-timed (median of 3
    timings) so that one noisy sample decides nothing; the single-pass
    configs differ most on large shapes, where the fixed config loses most.
    It must also choose a config far faster than exhaustive tuning."""
    import time

    mlp, hist, T, V = trained
    assert hist[-1] < 0.5 * hist[0]
    test_shapes = proposer.sample_shapes(200, seed=2)
    t0 = time.perf_counter()
    Xt, Tt, Vt, TFt = proposer.collect(ctx, test_shapes)
    t_exhaustive = (time.perf_counter() - t0) / len(test_shapes)
    dflt = proposer.default_config(T, V)
    r = proposer.evaluate(mlp, Xt, TFt, dflt)
    assert r["median_regret"] <= 0.05
    prop = proposer.propose_indices(ctx, mlp, test_shapes)
    rt = proposer.retimed_regret(ctx, test_shapes, TFt, prop, dflt, repeats=3)
    print("proposer vs fixed default (re-timed):", rt)
    assert rt["median_regret"] <= 0.05
    assert rt["mean_regret"] < rt["mean_regret_default"], rt
    assert rt["p90_regret"] < rt["p90_regret_default"], rt
    NC = len(tp.tp_autotune_space("bf16"))
    untrained = tp.tp_mlp_create(ctx, F, H, NC, 256, proposer.init_params(F, H, NC, seed=0))
    r0 = proposer.evaluate(untrained, Xt, TFt, 0)
    assert r["mean_regret"] < r0["mean_regret"]
    t0 = time.perf_counter()
    for m, n, k, dt in test_shapes:
        cfg, score, fb = tp.tp_propose(ctx, mlp, m, n, k, dt, min_score=-1e9)
        assert not fb and cfg.split_k <= 1
    t_propose = (time.perf_counter() - t0) / len(test_shapes)
    assert t_propose * 20 < t_exhaustive
    cfg, score, fb = tp.tp_propose(ctx, mlp, 20000, 64, 64, "bf16")      # outside the trained range
    assert fb and cfg.bm in (128, 256) and cfg.split_k <= 1
    tp.tp_mlp_destroy(untrained)


def test_proposals_equal_exhaustive_pick_bit_for_bit(ctx, trained):
    """On 40 held-out BF16 shapes, C computed with the config tp_propose
    returns equals, bit for bit, C computed with the exhaustive autotuner's
    pick for the same shape and inputs: the proposal never changes numerics,
    whether or not it picks the same config."""
    mlp = trained[0]
    shapes = [(m, n, k) for m, n, k, _ in proposer.sample_shapes(80, seed=7, hi=4096)][:40]
    differ = 0
    for i, (m, n, k) in enumerate(shapes):
        prop, _, fb = tp.tp_propose(ctx, mlp, m, n, k, "bf16", min_score=-1e9)
        assert not fb and prop.split_k <= 1
        exh, _, _ = tp.tp_autotune(ctx, m, n, k, "bf16")
        differ += (prop.bm, prop.bn, prop.bk, prop.group_m, prop.swap_ab) != (exh.bm, exh.bn, exh.bk, exh.group_m,
                                                                             exh.swap_ab)
        a = synth.to_bf16(synth.normal(m * k, 100 + i)).reshape(m, k).cuda()
        bt = synth.to_bf16(synth.normal(n * k, 200 + i)).reshape(n, k).cuda()
        outs = []
        for cfg in (prop, exh):
            c = torch.full((m, n), float("nan"), dtype=torch.bfloat16, device="cuda")
            p = tp.tp_partition_create(ctx, c, (cfg.bm, cfg.bn))
            tiles = tp.tp_partition_query(p)["num_tiles"]
            pair = cfg.bm == 256 or cfg.swap_ab
            tp.tp_partition_map(p, tp.MAP_STRIDED, min(tiles, ctx.sm_count // (2 if pair else 1)))
            tp.tp_gemm(ctx, p, a, bt.t(), cfg)
            tp.tp_partition_destroy(p)
            outs.append(c)
        assert torch.equal(outs[0], outs[1]), (m, n, k)
        assert not torch.isnan(outs[0]).any()
    assert differ > 0      # the check covered proposals that differ from the exhaustive pick


def test_split_k_is_opt_in_only(ctx):
    """An MLP biased towards the last outputs cannot reach a split-K config
    (the proposer's outputs are the single-pass class), the fallback searches
    the single-pass class, and only the explicit split-K search can return a
    split config, on a shape where split programs pay off."""
    space = tp.tp_autotune_space("bf16")
    NC = len(space)
    params = proposer.init_params(F, H, NC, seed=3)
    params[-NC:] = 100.0 + np.arange(NC)
    m = tp.tp_mlp_create(ctx, F, H, NC, 8, params)
    cfg, _, fb = tp.tp_propose(ctx, m, 128, 256, 4096, "bf16", min_score=-1e9)
    assert not fb and cfg.split_k <= 1
    cfg, _, fb = tp.tp_propose(ctx, m, 128, 256, 4096, "bf16", min_score=1e9)   # forced fallback
    assert fb and cfg.split_k <= 1
    best, table, _ = tp.tp_autotune(ctx, 128, 256, 4096, "bf16", split_k=True)
    assert len(table) == 77 and max(table[72:]) > 0
    tp.tp_mlp_destroy(m)
    # an MLP whose output count is the split-inclusive space is refused
    bad = tp.tp_mlp_create(ctx, F, H, 77, 8, proposer.init_params(F, H, 77, seed=3))
    with pytest.raises(tp.TPError):
        tp.tp_propose(ctx, bad, 128, 256, 4096, "bf16", min_score=-1e9)
    tp.tp_mlp_destroy(bad)


def test_autotune_cache_reads_older_files(ctx, tmp_path):
    """v1 and v2 cache lines (no flags column) came from searches that
    included split-K: a single-pass winner loads under both searches, a
    split winner only under the split-K search; v3 lines lack bk (0); v4
    lines lack swap_ab (0); v5 saves write the flags, bk and swap_ab."""
    path = os.path.join(tmp_path, "v1.txt")
    with open(path, "w") as f:
        f.write("tp-autotune-cache v1\n")
        f.write("1111 2222 3344 1 256 128 3 8 76 1234.500\n")
    tp.tp_autotune_load(ctx, path)
    cfg = tp.tp_autotune_lookup(ctx, 1111, 2222, 3344, "bf16")
    assert (cfg.bm, cfg.bn, cfg.bk, cfg.stages, cfg.group_m, cfg.num_programs, cfg.split_k) == (256, 128, 0, 3, 8, 76, 0)
    assert tp.tp_autotune_lookup(ctx, 1111, 2222, 3344, "bf16", split_k=True).bn == 128
    path2 = os.path.join(tmp_path, "v2.txt")
    with open(path2, "w") as f:
        f.write("tp-autotune-cache v2\n")
        f.write("128 256 4096 1 128 256 0 1 0 4 300.0\n")
    tp.tp_autotune_load(ctx, path2)
    assert tp.tp_autotune_lookup(ctx, 128, 256, 4096, "bf16", split_k=True).split_k == 4
    path3 = os.path.join(tmp_path, "v3.txt")
    with open(path3, "w") as f:
        f.write("tp-autotune-cache v3\n")
        f.write("333 444 512 1 0 64 128 0 1 0 0 99.0\n")
    tp.tp_autotune_load(ctx, path3)
    assert (tp.tp_autotune_lookup(ctx, 333, 444, 512, "bf16").bm, tp.tp_autotune_lookup(ctx, 333, 444, 512).bk) == (64, 0)
    tp.tp_autotune(ctx, 640, 384, 512, "bf16")
    best = tp.tp_autotune_lookup(ctx, 640, 384, 512, "bf16")
    out = os.path.join(tmp_path, "v4.txt")
    tp.tp_autotune_save(ctx, out)
    lines = open(out).read().splitlines()
    assert lines[0] == "tp-autotune-cache v5"
    assert any(line.split()[:12] == ["1111", "2222", "3344", "1", "0", "256", "128", "0", "3", "8", "76", "0"]
               for line in lines[1:])
    assert not any(line.split()[:5] == ["128", "256", "4096", "1", "0"] and line.split()[11] == "4"
                   for line in lines[1:])
    assert any(line.split()[:8] == ["640", "384", "512", "1", "0", str(best.bm), str(best.bn), str(best.bk)]
               for line in lines[1:])
    tp.tp_autotune_load(ctx, out)
    assert tp.tp_autotune_lookup(ctx, 640, 384, 512, "bf16").bk == best.bk
    path4 = os.path.join(tmp_path, "v4.txt")
    with open(path4, "w") as f:
        f.write("tp-autotune-cache v4\n")
        f.write("64 8192 8192 1 0 64 64 256 0 1 0 0 290.0\n")
    tp.tp_autotune_load(ctx, path4)
    cfg = tp.tp_autotune_lookup(ctx, 64, 8192, 8192, "bf16")
    assert (cfg.bm, cfg.bn, cfg.bk, cfg.swap_ab) == (64, 64, 256, 0)
    swap = [c for c in tp.tp_autotune_space("bf16", swap_ab=True) if c.swap_ab][2]
    path5 = os.path.join(tmp_path, "v5.txt")
    with open(path5, "w") as f:
        f.write("tp-autotune-cache v5\n")
        f.write(f"32 4096 2048 1 2 {swap.bm} {swap.bn} {swap.bk} 0 1 0 0 1 150.0\n")
        f.write(f"32 4096 4096 1 0 {swap.bm} {swap.bn} {swap.bk} 0 1 0 0 1 150.0\n")   # not from such a search
    tp.tp_autotune_load(ctx, path5)
    cfg = tp.tp_autotune_lookup(ctx, 32, 4096, 2048, "bf16", swap_ab=True)
    assert (cfg.bm, cfg.bn, cfg.bk, cfg.swap_ab) == (swap.bm, swap.bn, swap.bk, 1)
    assert tp.tp_autotune_lookup(ctx, 32, 4096, 4096, "bf16") is None


def test_swap_ab_search_is_opt_in(ctx):
    """TP_TUNE_SWAP_AB adds the swap-AB configs to the search: on a BF16
    problem of 64 rows the W = 64 and W = 128 ones are timed (W = 32 tiles
    would need two tile rows and are skipped), none on FP8; the winner is
    cached under that flag, and it computes C bit for bit like the default
    search's winner (both in the single-pass class)."""
    M, N, K = 64, 2048, 1024
    space = tp.tp_autotune_space("bf16", swap_ab=True)
    best, table, _ = tp.tp_autotune(ctx, M, N, K, "bf16", swap_ab=True)
    assert len(table) == len(space) == 78
    assert all((t > 0) == (not c.swap_ab or c.bm >= M) for t, c in zip(table, space))
    assert tp.tp_autotune_lookup(ctx, M, N, K, "bf16", swap_ab=True) is not None
    _, t8, _ = tp.tp_autotune(ctx, M, N, K, "fp8", swap_ab=True)
    assert all(t == 0 for t in t8[72:]) and all(t > 0 for t in t8[:72])
    dflt, _, _ = tp.tp_autotune(ctx, M, N, K, "bf16")
    a = synth.to_bf16(synth.normal(M * K, 11)).reshape(M, K).cuda()
    bt = synth.to_bf16(synth.normal(N * K, 12)).reshape(N, K).cuda()
    outs = []
    for cfg in (best, dflt, space[74]):          # space[74]: W = 64, 2 K blocks per stage
        c = torch.full((M, N), float("nan"), dtype=torch.bfloat16, device="cuda")
        p = tp.tp_partition_create(ctx, c, (cfg.bm, cfg.bn))
        tiles = tp.tp_partition_query(p)["num_tiles"]
        pair = cfg.bm == 256 or cfg.swap_ab
        tp.tp_partition_map(p, tp.MAP_STRIDED, min(tiles, ctx.sm_count // (2 if pair else 1)))
        tp.tp_gemm(ctx, p, a, bt.t(), cfg)
        tp.tp_partition_destroy(p)
        outs.append(c)
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[1], outs[2])
