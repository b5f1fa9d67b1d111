"""GPU tests of the four execution modes of §3.2 / §5.2 on a chain of N
dependent y = x * g launches over one 2048-element BF16 tile: every mode
leaves x * g^N rounded to BF16 after each op (the oracle's composition, bit
for bit: the product of two BF16 values is exact in FP32), and no partition
stays held once the chain has completed."""
import numpy as np
import pytest
import torch

import paper_2606_15991_gb300 as tp
import synth
from oracle import lowp
from oracle import maps as omaps
from paper_2606_15991_gb300 import experiments

pytestmark = pytest.mark.gpu


def _oracle_chain(x, g, N):
    y = np.asarray(x, np.float64)
    for _ in range(N):
        y = lowp.round_bf16(omaps.scale(y, g))
    return y


@pytest.fixture
def chain(ctx):
    x = synth.to_bf16(synth.normal(2048, 3)).cuda()
    g = synth.to_bf16(1.0 + 0.05 * synth.normal(2048, 4)).cuda()
    s = torch.cuda.Stream()
    ch = experiments.ExecChain(ctx, x, g, s)
    yield ch, x.cpu().double().numpy(), g.cpu().double().numpy()
    ch.close()


@pytest.mark.parametrize("mode", ["sync", "chained", "async", "graph"])
@pytest.mark.parametrize("N", [1, 2, 7, 64, 333])
def test_chain_result_every_mode(chain, mode, N):
    ch, x, g = chain
    ch.reset()
    if mode == "graph":
        gr = ch.capture(N)
        assert np.array_equal(ch.output(0).cpu().double().numpy(), x)   # capture ran nothing
        ch.replay(gr)
        tp.tp_graph_destroy(gr)
    else:
        {"sync": ch.run_sync, "chained": ch.run_chained, "async": ch.run_async}[mode](N)
    got = ch.output(N).cpu().double().numpy()
    assert np.array_equal(got, _oracle_chain(x, g, N))
    for p in ch.parts:
        assert not tp.tp_partition_query(p)["busy"]


def test_graph_replays_repeat_the_chain(chain):
    ch, x, g = chain
    ch.reset()
    gr = ch.capture(4)                 # even N: the chain reads and ends in buffer 0
    for r in range(1, 4):
        ch.replay(gr)
        assert np.array_equal(ch.output(0).cpu().double().numpy(), _oracle_chain(x, g, 4 * r))
    tp.tp_graph_destroy(gr)


def test_scaling_driver_small(ctx):
    r = experiments.exec_mode_scaling(ctx, Ns=(1, 10), reps=3, warmup=1)
    for m in ("sync", "chained", "async", "graph", "graph_device"):
        for N in (1, 10):
            v = r["us_per_op"][m][N]
            assert 0 < v["min"] <= v["p75"]
    assert r["binding_us"] > 0


def test_event_reuse_across_streams_waits_for_the_first(ctx):
    """An event that still tracks unfinished work on one stream cannot be
    re-recorded by work on another stream (that would release the first
    work's holds early); once the first work is done it can."""
    x = torch.ones(4096, device="cuda")
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    p1, p2 = tp.tp_partition_create(ctx, y1, (1024,)), tp.tp_partition_create(ctx, y2, (1024,))
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    ev = tp.tp_event_create(ctx)
    with torch.cuda.stream(s1):
        torch.cuda._sleep(50_000_000)
    tp.tp_map_scale(ctx, p1, x, x, tp.make_exec(tp.ASYNC, s1, ev))
    with pytest.raises(tp.TPError) as e:
        tp.tp_map_scale(ctx, p2, x, x, tp.make_exec(tp.ASYNC, s2, ev))
    assert e.value.status == tp._lib.ERR_BUSY
    assert tp.tp_partition_query(p1)["busy"] and not tp.tp_partition_query(p2)["busy"]
    s1.synchronize()
    tp.tp_map_scale(ctx, p2, x, x, tp.make_exec(tp.ASYNC, s2, ev))   # first work finished: released, re-recorded
    assert not tp.tp_partition_query(p1)["busy"]
    tp.tp_event_wait(ev)
    assert not tp.tp_partition_query(p2)["busy"]
    assert torch.equal(y1, x) and torch.equal(y2, x)
    tp.tp_event_destroy(ev)
    tp.tp_partition_destroy(p1)
    tp.tp_partition_destroy(p2)
