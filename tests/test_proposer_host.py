"""Host-side arithmetic of the tile-proposer experiment (no GPU): the regret
summary and the fixed default config, on hand-made tables."""
import numpy as np

from paper_2606_15991_gb300 import proposer


def test_regret_stats_hand_worked():
    # 4 shapes x 3 configs (TFLOP/s); the proposals pick configs 0, 2, 1, 1
    TF = np.array([[100.0, 50.0, 80.0],
                   [10.0, 20.0, 40.0],
                   [30.0, 30.0, 60.0],
                   [5.0, 4.0, 1.0]])
    r = proposer.regret_stats(TF, [0, 2, 1, 1], default_index=2)
    reg = np.array([0.0, 0.0, 0.5, 0.2])              # 1 - chosen / best, shape by shape
    reg_def = np.array([0.2, 0.0, 0.0, 0.8])
    assert np.isclose(r["median_regret"], np.median(reg)) and np.isclose(r["mean_regret"], 0.175)
    assert np.isclose(r["p90_regret"], np.percentile(reg, 90))
    assert np.isclose(r["mean_regret_default"], 0.25) and np.isclose(r["median_regret_default"], 0.1)
    assert r["exact_pick_rate"] == 0.5 and r["shapes"] == 4 and r["fallback_rate"] == 0.0
    # shapes whose top score is below min_score fall back to the exhaustive pick (regret 0)
    r = proposer.regret_stats(TF, [0, 2, 1, 1], 2, top_score=[0.9, 0.9, 0.1, 0.1], min_score=0.5)
    assert r["fallback_rate"] == 0.5 and r["median_regret_with_fallback"] == 0.0
    assert np.isclose(r["mean_regret"], 0.175)       # the proposal's own regret is unchanged


def test_default_config_is_best_on_average():
    # relative speeds (targets) of 3 configs on 3 training shapes; the masked
    # entry (a config that did not run) counts as 0
    T = np.array([[1.0, 0.9, 0.2], [0.5, 1.0, 1.0], [1.0, 0.8, 0.0]], np.float32)
    V = np.array([[1, 1, 1], [1, 1, 1], [1, 1, 0]], np.float32)
    assert proposer.default_config(T, V) == 1       # column sums 2.5, 2.7, 1.2


def test_tuned_config_programs():
    """A launch config from an autotuned one: persistent programs up to the
    SM count in CTAs, or in CTA pairs for 256-row and swap-AB tiles, one
    program per tile for split-K; swap_ab and the K per stage carry over."""
    from types import SimpleNamespace

    from paper_2606_15991_gb300 import experiments, gemm_config

    ctx = SimpleNamespace(sm_count=152)
    cases = [(gemm_config(bm=128, bn=256, bk=128), 1000, 152),
             (gemm_config(bm=256, bn=256, group_m=8), 1000, 76),
             (gemm_config(bm=64, bn=128, bk=256, swap_ab=1), 1000, 76),
             (gemm_config(bm=64, bn=128, swap_ab=1), 40, 40),
             (gemm_config(bm=128, bn=128, split_k=4), 24, 24),
             (gemm_config(bm=128, bn=64, num_programs=7), 100, 7)]
    for best, tiles, progs in cases:
        cfg = experiments.tuned_config(ctx, best, tiles)
        assert cfg.num_programs == progs, (best.bm, best.swap_ab, best.split_k)
        assert (cfg.bm, cfg.bn, cfg.bk, cfg.swap_ab, cfg.split_k) == (best.bm, best.bn, best.bk, best.swap_ab,
                                                                     best.split_k)
