"""The multi-process path of bench.py on CPU: two or four gloo ranks (one process
per GPU on a GPU node) agree on the slowest rank's step time, read their
rank from the launcher's environment, and the whole-job value is the
world size times one rank's bytes over that time (weak scaling, no data
exchange between ranks)."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    import torch
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    got_ws, got_rank, got_local = bench._dist()
    ms = bench._barrier_max(10.0 + 5.0 * rank, ws, torch.device("cpu"))
    value = bench.weak_scaling_value(got_ws, 3.0e9, ms)
    all_ok = bench._all_ranks_ok(True, ws, torch.device("cpu"))
    one_failed = bench._all_ranks_ok(rank == 0, ws, torch.device("cpu"))   # ranks past 0 report a failure
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got_ws, got_rank, got_local, ms, value, all_ok, one_failed))


@pytest.mark.timeout(150)
@pytest.mark.parametrize("world", [2, 4])
def test_gloo_ranks_take_the_max_step_time(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    slowest = 10.0 + 5.0 * (world - 1)
    for rank, ws, r, local, ms, value, all_ok, one_failed in out:
        assert all_ok and not one_failed                   # every rank sees the same verdict
        assert (ws, r, local) == (world, rank, rank)
        assert ms == slowest                                # the slowest rank's time, on every rank
        assert value == pytest.approx(world * 3.0e9 / (slowest * 1e-3) / 1e12)


def test_single_process_defaults(monkeypatch):
    import bench

    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench._dist() == (1, 0, 0)
    assert bench._barrier_max(7.0, 1, None) == 7.0
    assert bench.weak_scaling_value(1, 1e12, 1000.0) == pytest.approx(1.0)
    assert bench._all_ranks_ok(True, 1, None) and not bench._all_ranks_ok(False, 1, None)
