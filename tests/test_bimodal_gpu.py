"""The bimodal GEMM queue (Appendix B): the drain strategies run to
completion on a small queue, and the grouped launch of the full 2000-unit
queue (80% 512^3, 20% 2048^3, distinct outputs, shared operands) matches the
FP64 oracle on sampled tiles of sampled units."""
import numpy as np
import pytest
import torch

import paper_2606_15991_gb300 as tp
import synth
from oracle import gemm as ogemm
from paper_2606_15991_gb300 import experiments

pytestmark = pytest.mark.gpu


def test_kinds_are_twenty_percent_large_interleaved():
    k = experiments.bimodal_kinds(2000)
    assert sum(k) == 400 and k[:10] == [0, 0, 0, 0, 1, 0, 0, 0, 0, 1]


def test_drain_strategies_small_queue(ctx):
    r = experiments.bimodal_queue(ctx, n_units=40, streams=(1, 3), small=256, large=512, reps=1)
    assert r["serial"]["wu_per_ms"] > 0 and r["grouped"]["wu_per_ms"] > 0
    for name in ("threaded", "async"):
        assert set(r[name]) == {1, 3} and all(v["wu_per_ms"] > 0 for v in r[name].values())


def test_full_queue_grouped_sampled(ctx):
    kinds = experiments.bimodal_kinds(2000)
    sizes = (512, 2048)
    A = [synth.to_bf16(synth.normal(n * n, 10 + i)).reshape(n, n).cuda() for i, n in enumerate(sizes)]
    BT = [synth.to_bf16(synth.normal(n * n, 20 + i)).reshape(n, n).cuda() for i, n in enumerate(sizes)]
    outs = [torch.full((sizes[k], sizes[k]), float("nan"), device="cuda", dtype=torch.bfloat16) for k in kinds]
    plan = tp.tp_grouped_plan_create(ctx, [(A[k], BT[k].t(), c) for k, c in zip(kinds, outs)])
    tp.tp_grouped_gemm(ctx, plan)
    tp.tp_grouped_plan_destroy(plan)
    units = sorted(set(int(u) for u in synth.integers(24, 5, 0, 1999)) | {0, 4, 1999})
    got, ref = [], []
    for u in units:
        n = sizes[kinds[u]]
        c = outs[u]
        assert not torch.isnan(c).any(), u
        for tm, tn in synth.sample_tiles(n // 128, n // 128, 1, seed=u):
            rs, cs = slice(tm * 128, (tm + 1) * 128), slice(tn * 128, (tn + 1) * 128)
            ref.append(ogemm.gemm(A[kinds[u]][rs].cpu(), BT[kinds[u]][cs].cpu().t()).reshape(-1))
            got.append(c[rs, cs].cpu().double().numpy().reshape(-1))
    assert ogemm.rel_frobenius(np.concatenate(got), np.concatenate(ref)) <= 1e-2
    del outs
    torch.cuda.empty_cache()


def test_fresh_thread_first_call(ctx):
    """A thread that has made no CUDA call yet can launch through the
    library (the context's device is made current at the entry point), and a
    caller's different current device would be restored afterwards."""
    import threading

    a = synth.to_bf16(synth.normal(256 * 64, 3)).reshape(256, 64).cuda()
    bt = synth.to_bf16(synth.normal(128 * 64, 4)).reshape(128, 64).cuda()
    c = torch.empty(256, 128, device="cuda", dtype=torch.bfloat16)
    err = []

    def body():
        try:
            p = tp.tp_partition_create(ctx, c, (128, 128))
            tp.tp_gemm(ctx, p, a, bt.t(), tp.gemm_config(bm=128, bn=128))
            tp.tp_partition_destroy(p)
        except BaseException as e:
            err.append(e)

    t = threading.Thread(target=body)
    t.start()
    t.join()
    assert not err, err
    assert ogemm.rel_frobenius(c.cpu(), ogemm.gemm(a.cpu(), bt.cpu().t())) <= 1e-2
