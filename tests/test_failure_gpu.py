"""Failure detection without a GPU fault: a device wait on a barrier that
nothing signals gives up after its limit, the host reads TP_ERR_TIMEOUT in
every execution mode, and the context keeps working afterwards."""
import time

import pytest
import torch

import paper_2606_15991_gb300 as tp
import synth
from oracle import gemm as ogemm

pytestmark = pytest.mark.gpu

LIMIT = 50_000_000     # 50 ms


def test_sync_timeout_then_recovery(ctx):
    tp.tp_diag_bounded_wait(ctx, LIMIT, True)                      # signalled: completes
    t0 = time.perf_counter()
    with pytest.raises(tp.TPError) as e:
        tp.tp_diag_bounded_wait(ctx, LIMIT, False)
    assert e.value.status == tp._lib.ERR_TIMEOUT
    assert time.perf_counter() - t0 >= 0.045                      # the wait ran to its limit
    tp.tp_diag_bounded_wait(ctx, LIMIT, True)                      # error word was cleared
    # real work still runs correctly on the same context
    a = synth.to_bf16(synth.normal(256 * 128, 1)).reshape(256, 128).cuda()
    bt = synth.to_bf16(synth.normal(256 * 128, 2)).reshape(256, 128).cuda()
    c = torch.empty(256, 256, device="cuda", dtype=torch.bfloat16)
    p = tp.tp_partition_create(ctx, c, (128, 128))
    tp.tp_gemm(ctx, p, a, bt.t(), tp.gemm_config(bm=128, bn=128))
    tp.tp_partition_destroy(p)
    assert ogemm.rel_frobenius(c.cpu(), ogemm.gemm(a.cpu(), bt.cpu().t())) <= 1e-2


def test_async_and_graph_report_the_timeout(ctx):
    s = torch.cuda.Stream()
    ev = tp.tp_event_create(ctx)
    tp.tp_diag_bounded_wait(ctx, LIMIT, False, tp.make_exec(tp.ASYNC, s, ev))
    with pytest.raises(tp.TPError) as e:
        tp.tp_event_wait(ev)
    assert e.value.status == tp._lib.ERR_TIMEOUT
    tp.tp_diag_bounded_wait(ctx, LIMIT, True, tp.make_exec(tp.ASYNC, s, ev))
    tp.tp_event_wait(ev)
    g = tp.tp_graph_begin(ctx, s)
    tp.tp_diag_bounded_wait(ctx, LIMIT, False, tp.make_exec(tp.CAPTURE, s))
    tp.tp_graph_end(g)
    for _ in range(2):                                             # every replay times out again
        with pytest.raises(tp.TPError) as e:
            tp.tp_graph_replay(g, tp.make_exec(stream=s))
        assert e.value.status == tp._lib.ERR_TIMEOUT
    tp.tp_graph_destroy(g)
    tp.tp_event_destroy(ev)


def test_limit_validation(ctx):
    for bad in (0, 999, 2_000_000_001):
        with pytest.raises(tp.TPError) as e:
            tp.tp_diag_bounded_wait(ctx, bad, True)
        assert e.value.status == tp._lib.ERR_INVALID


@pytest.mark.parametrize("mode", ["sync", "async", "split"])
def test_gemm_injected_timeout_drains_and_reports(ctx, mode):
    """TP_EXEC_INJECT_TIMEOUT leaves each program's first K block unloaded:
    the tensor-core GEMM's MMA issuer runs out its (50 ms) bounded wait, the
    kernel drains its copies and MMAs, frees TMEM and returns; the host reads
    TP_ERR_TIMEOUT (SYNC on return, ASYNC from the event) and the context,
    the partition and the next GEMM all work afterwards."""
    a = synth.to_bf16(synth.normal(384 * 512, 5)).reshape(384, 512).cuda()
    bt = synth.to_bf16(synth.normal(256 * 512, 6)).reshape(256, 512).cuda()
    c = torch.zeros(384, 256, device="cuda", dtype=torch.bfloat16)
    p = tp.tp_partition_create(ctx, c, (128, 128))
    if mode == "split":
        cfg = tp.gemm_config(bm=128, bn=128, split_k=2)
    else:
        tp.tp_partition_map(p, tp.MAP_STRIDED, 4)
        cfg = tp.gemm_config(bm=128, bn=128)
    s = torch.cuda.Stream()
    t0 = time.perf_counter()
    with pytest.raises(tp.TPError) as e:
        if mode == "async":
            ev = tp.tp_event_create(ctx)
            tp.tp_gemm(ctx, p, a, bt.t(), cfg, tp.make_exec(tp.ASYNC, s, ev, inject_timeout=True))
            try:
                tp.tp_event_wait(ev)
            finally:
                tp.tp_event_destroy(ev)
        else:
            tp.tp_gemm(ctx, p, a, bt.t(), cfg, tp.make_exec(stream=s, inject_timeout=True))
    assert e.value.status == tp._lib.ERR_TIMEOUT
    assert time.perf_counter() - t0 >= 0.045                      # the wait ran to its limit
    assert not tp.tp_partition_query(p)["busy"]
    tp.tp_gemm(ctx, p, a, bt.t(), cfg, tp.make_exec(stream=s))
    assert ogemm.rel_frobenius(c.cpu(), ogemm.gemm(a.cpu(), bt.cpu().t())) <= 1e-2
    tp.tp_partition_destroy(p)


def test_injected_timeout_is_refused_where_not_implemented(ctx):
    a = torch.zeros(256, 128, device="cuda", dtype=torch.bfloat16)
    bt = torch.zeros(256, 128, device="cuda", dtype=torch.bfloat16)
    c = torch.zeros(256, 256, device="cuda", dtype=torch.bfloat16)
    p = tp.tp_partition_create(ctx, c, (256, 128))                 # CTA-pair tiles
    with pytest.raises(tp.TPError) as e:
        tp.tp_gemm(ctx, p, a, bt.t(), tp.gemm_config(bm=256, bn=128), tp.make_exec(inject_timeout=True))
    assert e.value.status == tp._lib.ERR_UNSUPPORTED
    tp.tp_partition_destroy(p)
    x = torch.zeros(4096, device="cuda")
    z = torch.zeros(4096, device="cuda")
    pz = tp.tp_partition_create(ctx, z, (4096,))
    with pytest.raises(tp.TPError) as e:
        tp.tp_map_axpy(ctx, pz, 1.0, x, x, tp.make_exec(inject_timeout=True))
    assert e.value.status == tp._lib.ERR_UNSUPPORTED
    tp.tp_partition_destroy(pz)
