"""Measurement drivers for the secondary experiments of §5 (built on the
library's C ABI; every kernel that runs is the library's).

exec_mode_scaling (§5.2, "Execution Mode Overhead"): a pipeline of N
dependent y = x * g launches over one 2048-element tile, run four ways:
  sync      N calls in TP_SYNC mode: each synchronizes its stream (the
            individual `sync_on` calls);
  chained   N TP_ASYNC calls queued on one stream, then one blocking
            tp_event_wait (the `then` chain run with one `sync`);
  async     the same chain, then the host polls tp_event_query, yielding its
            thread between polls (the host is free while the GPU runs, as
            with `.await`);
  graph     the N launches captured once (TP_CAPTURE) and replayed with one
            tp_graph_replay per pipeline.
Host wall time per pipeline / N = microseconds per op; min and p75 over
repetitions, as in the paper's figure. The calls go through ctypes with
argument structs built once, so the per-call cost of the binding itself (the
`binding_us` figure, an empty ABI call) is part of every host-side number.
"""
from __future__ import annotations

import ctypes
import os
import time

import numpy as np
import torch

from . import (ASYNC, CAPTURE, SYNC, _lib, make_exec, tensor_desc, tp_event_create, tp_event_destroy,
               tp_graph_begin, tp_graph_destroy, tp_graph_end, tp_partition_create, tp_partition_destroy)


def _check(st: int, what: str) -> None:
    if st != _lib.OK:
        raise _lib.TPError(st, _lib.lib().tp_last_error_detail().decode(), what)


class ExecChain:
    """Two ping-pong buffers of `n` elements; op i computes
    buf[(i + 1) % 2] = buf[i % 2] * g, so every op depends on the previous one
    and the output after N ops is x * g^N (rounded per op in the buffer dtype)."""

    def __init__(self, ctx, x, g, stream):
        self.ctx, self.stream = ctx, stream
        self.g = g
        self.bufs = [x.clone(), torch.empty_like(x)]
        self.parts = [tp_partition_create(ctx, b, (x.numel(),)) for b in self.bufs]
        self.ev = tp_event_create(ctx)
        self.dx = [tensor_desc(b) for b in self.bufs]
        self.dg = tensor_desc(g)
        self.ex = {SYNC: make_exec(SYNC, stream), ASYNC: make_exec(ASYNC, stream, self.ev),
                   CAPTURE: make_exec(CAPTURE, stream)}
        L = _lib.lib()
        self._f = L.tp_map_scale
        self._args = {m: [(ctx.handle, self.parts[(i + 1) % 2].handle, ctypes.byref(self.dx[i]),
                           ctypes.byref(self.dg), ctypes.byref(self.ex[m])) for i in range(2)]
                      for m in (SYNC, ASYNC, CAPTURE)}
        self._wait = L.tp_event_wait
        self._query = L.tp_event_query
        self._replay = L.tp_graph_replay
        self._done = ctypes.c_int32()
        self.x0 = x

    def reset(self) -> None:
        self.bufs[0].copy_(self.x0)
        torch.cuda.synchronize()

    def output(self, N: int):
        return self.bufs[N % 2]

    def _launch(self, mode: int, N: int) -> None:
        f, a = self._f, self._args[mode]
        for i in range(N):
            st = f(*a[i & 1])
            if st:
                _check(st, "tp_map_scale")

    def run_sync(self, N: int) -> None:
        self._launch(SYNC, N)

    def run_chained(self, N: int) -> None:
        self._launch(ASYNC, N)
        _check(self._wait(self.ev.handle), "tp_event_wait")

    def run_async(self, N: int) -> None:
        self._launch(ASYNC, N)
        q, h, d = self._query, self.ev.handle, ctypes.byref(self._done)
        while True:
            _check(q(h, d), "tp_event_query")
            if self._done.value:
                return
            os.sched_yield()

    def capture(self, N: int):
        g = tp_graph_begin(self.ctx, self.stream)
        self._launch(CAPTURE, N)
        tp_graph_end(g)
        return g

    def replay(self, graph) -> None:
        _check(self._replay(graph.handle, ctypes.byref(self.ex[SYNC])), "tp_graph_replay")

    def close(self) -> None:
        tp_event_destroy(self.ev)
        for p in self.parts:
            tp_partition_destroy(p)


def binding_floor_us(reps: int = 20000) -> float:
    """Host cost of one ctypes call into the library (tp_version)."""
    L = _lib.lib()
    a, b = ctypes.c_int32(), ctypes.c_int32()
    ra, rb = ctypes.byref(a), ctypes.byref(b)
    f = L.tp_version
    t0 = time.perf_counter_ns()
    for _ in range(reps):
        f(ra, rb)
    return (time.perf_counter_ns() - t0) / reps / 1e3


def exec_mode_scaling(ctx, Ns=(1, 2, 5, 10, 20, 50, 100, 200, 500, 1000), reps: int = 30, warmup: int = 3,
                      n: int = 2048, dtype=torch.bfloat16, seed: int = 0) -> dict:
    dev = torch.device("cuda", torch.cuda.current_device())
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    x = torch.randn(n, device=dev, generator=gen).to(dtype)
    g = (1.0 + 0.01 * torch.randn(n, device=dev, generator=gen)).to(dtype)
    s = torch.cuda.Stream(device=dev)
    ch = ExecChain(ctx, x, g, s)
    out = {"n": n, "dtype": str(dtype).replace("torch.", ""), "reps": reps, "Ns": list(Ns),
           "binding_us": binding_floor_us()}
    modes = {"sync": ch.run_sync, "chained": ch.run_chained, "async": ch.run_async}
    res = {m: {} for m in ("sync", "chained", "async", "graph", "graph_device")}
    for N in Ns:
        graph = ch.capture(N)
        runners = dict(modes)
        runners["graph"] = lambda _N, gr=graph: ch.replay(gr)
        for name, fn in runners.items():
            for _ in range(warmup):
                fn(N)
            ts = []
            for _ in range(reps):
                t0 = time.perf_counter_ns()
                fn(N)
                ts.append((time.perf_counter_ns() - t0) / 1e3 / N)
            res[name][N] = {"min": float(np.min(ts)), "p75": float(np.percentile(ts, 75))}
        # device-side time of the replayed pipeline (CUDA events on its stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        dts = []
        for _ in range(max(3, reps // 3)):
            with torch.cuda.stream(s):
                e0.record(s)
                _check(_lib.lib().tp_graph_replay(graph.handle, ctypes.byref(ch.ex[ASYNC])), "tp_graph_replay")
                e1.record(s)
            _check(ch._wait(ch.ev.handle), "tp_event_wait")
            e1.synchronize()
            dts.append(e0.elapsed_time(e1) * 1e3 / N)
        res["graph_device"][N] = {"min": float(np.min(dts)), "p75": float(np.percentile(dts, 75))}
        tp_graph_destroy(graph)
    ch.close()
    out["us_per_op"] = res
    return out


def graph_time_ms(ctx, stream, record, reps: int, replays: int = 3) -> float:
    """Device time (ms) of one recorded op: `record(ex)` is captured `reps`
    times into one graph (ex = a TP_CAPTURE exec on `stream`), the graph is
    replayed once to warm up, then `replays` times, each bracketed by CUDA
    events on `stream`; returns the fastest replay / reps."""
    g = tp_graph_begin(ctx, stream)
    cap = make_exec(CAPTURE, stream)
    for _ in range(reps):
        record(cap)
    tp_graph_end(g)
    ex = make_exec(SYNC, stream)
    _check(_lib.lib().tp_graph_replay(g.handle, ctypes.byref(ex)), "tp_graph_replay")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = None
    for _ in range(replays):
        e0.record(stream)
        _check(_lib.lib().tp_graph_replay(g.handle, ctypes.byref(ex)), "tp_graph_replay")
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) / reps
        best = t if best is None else min(best, t)
    tp_graph_destroy(g)
    return best


def tuned_config(ctx, best, tiles: int):
    """A launch config from an autotuned one: persistent programs (CTAs, CTA
    pairs for 256-row and swap-AB tiles) up to the SM count, or one split
    program per tile for a split-K config."""
    from . import gemm_config
    if best.split_k > 1:
        progs = tiles
    else:
        pair = best.bm == 256 or best.swap_ab
        progs = min(best.num_programs or (ctx.sm_count // (2 if pair else 1)), tiles)
    return gemm_config(bm=best.bm, bn=best.bn, bk=best.bk, stages=best.stages, group_m=best.group_m,
                       num_programs=progs, swap_ab=best.swap_ab, split_k=best.split_k)


class _Captured:
    """`reps` back-to-back calls captured once into a graph (the library's
    for `record(ex)`, torch's for a plain callable); time() replays it once,
    bracketed by CUDA events on `stream`, and returns ms per call."""

    def __init__(self, ctx, stream, reps: int, record=None, torch_fn=None):
        self.stream, self.reps = stream, reps
        self.e0, self.e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if record is not None:
            self.g = tp_graph_begin(ctx, stream)
            cap = make_exec(CAPTURE, stream)
            for _ in range(reps):
                record(cap)
            tp_graph_end(self.g)
            self.ex = make_exec(SYNC, stream)
            self.torch_graph = None
        else:
            with torch.cuda.stream(stream):
                torch_fn()
            torch.cuda.synchronize()
            self.torch_graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.torch_graph, stream=stream):
                for _ in range(reps):
                    torch_fn()
            self.g = None
        self.time()                                    # warm-up replay

    def time(self) -> float:
        if self.g is not None:
            self.e0.record(self.stream)
            _check(_lib.lib().tp_graph_replay(self.g.handle, ctypes.byref(self.ex)), "tp_graph_replay")
            self.e1.record(self.stream)
        else:
            with torch.cuda.stream(self.stream):
                self.e0.record(self.stream)
                self.torch_graph.replay()
                self.e1.record(self.stream)
        self.e1.synchronize()
        return self.e0.elapsed_time(self.e1) / self.reps

    def close(self) -> None:
        if self.g is not None:
            tp_graph_destroy(self.g)
        self.torch_graph = None


def _interleaved(variants: dict, rounds: int) -> tuple:
    """Median and lowest ms per call of each captured variant over `rounds`
    rounds (at least two per variant), each round replaying every variant
    once in turn, the starting variant rotating from round to round, so that
    clock and power drift (and the burst after an idle gap) fall on all
    variants alike."""
    names = list(variants)
    ts = {k: [] for k in names}
    for r in range(max(rounds, 2 * len(names))):
        for k in names[r % len(names):] + names[:r % len(names)]:
            ts[k].append(variants[k].time())
    med = {k: float(np.median(v)) for k, v in ts.items()}
    return med, {k: min(v) for k, v in ts.items()}


def _torch_graph_time_ms(fn, stream, reps: int, replays: int = 3) -> float:
    with torch.cuda.stream(stream):
        fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        for _ in range(reps):
            fn()
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = None
    for _ in range(replays):
        with torch.cuda.stream(stream):
            e0.record(stream)
            g.replay()
            e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) / reps
        best = t if best is None else min(best, t)
    del g
    return best


def _host_enqueue_us(fn, calls: int = 200) -> float:
    t0 = time.perf_counter_ns()
    for _ in range(calls):
        fn()
    t = (time.perf_counter_ns() - t0) / calls / 1e3
    torch.cuda.synchronize()
    return t


def gemm_size_sweep(ctx, sizes=(1024, 2048, 4096, 8192, 16384, 32768), target_ms: float = 25.0,
                    with_cublas: bool = True, rounds: int = 3, log=None) -> list:
    """§5.1's safety-overhead GEMM sweep, M = N = K over `sizes`, BF16 in,
    FP32 accumulate, BF16 out, tile config tuned once per size by the
    exhaustive autotuner and shared by every variant:
      safe        tp_gemm on a strided mapped partition (the safe API);
      checked     the same with TP_EXEC_CHECKED (every tile validated
                  against the map and claimed on the device before its store);
      unchecked   tp_gemm_unchecked: the same schedule on a raw C pointer;
      plain       tp_gemm on a plain partition (one program per tile);
      cublas      torch.matmul (cuBLAS) into a preallocated C, for context.
    Device time per GEMM from CUDA graphs of back-to-back launches (operands
    stay L2/HBM-resident between launches, as in a loop of GEMMs), the median
    (`ms`, and the TFLOP/s from it) and the lowest (`ms_min`) of at least ten
    interleaved rounds over the variants. safe and unchecked launch the same
    kernel with the same arguments, so their gap is the spread of the
    measurement. Host
    enqueue cost per call (safe vs unchecked, ctypes arguments built once) is
    reported for the smallest size."""
    from . import (tp_autotune, tp_gemm, tp_gemm_unchecked, tp_partition_map, tp_partition_query, gemm_config,
                   MAP_STRIDED)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    gen = torch.Generator(device=dev)
    out = []
    for n in sizes:
        gen.manual_seed(n)
        a = torch.randn(n, n, device=dev, generator=gen).to(torch.bfloat16)
        bt = torch.randn(n, n, device=dev, generator=gen).to(torch.bfloat16)
        c = torch.empty(n, n, device=dev, dtype=torch.bfloat16)
        flops = 2.0 * n ** 3
        t0 = time.perf_counter()
        best, table, best_tf = tp_autotune(ctx, n, n, n, "bf16")
        t_tune = time.perf_counter() - t0
        reps = int(min(200, max(1, np.ceil(target_ms / (flops / (best_tf * 1e12) * 1e3)))))
        tiles = -(-n // best.bm) * -(-n // best.bn)
        cfg = tuned_config(ctx, best, tiles)
        progs = cfg.num_programs
        p = tp_partition_create(ctx, c, (best.bm, best.bn))
        tp_partition_map(p, MAP_STRIDED, progs)
        pp = tp_partition_create(ctx, c, (best.bm, best.bn))
        bT = bt.t()
        chk = make_exec(CAPTURE, stream, checked=True)
        ucfg = tuned_config(ctx, best, tiles)
        pcfg = gemm_config(bm=best.bm, bn=best.bn, bk=best.bk, stages=best.stages, split_k=best.split_k)
        variants = {
            "safe": _Captured(ctx, stream, reps, record=lambda ex: tp_gemm(ctx, p, a, bT, cfg, ex)),
            "checked": _Captured(ctx, stream, reps, record=lambda ex: tp_gemm(ctx, p, a, bT, cfg, chk)),
            "unchecked": _Captured(ctx, stream, reps,
                                   record=lambda ex: tp_gemm_unchecked(ctx, c, a, bT, ucfg, stream)),
            "plain": _Captured(ctx, stream, reps, record=lambda ex: tp_gemm(ctx, pp, a, bT, pcfg, ex)),
        }
        if with_cublas:
            c2 = torch.empty_like(c)
            variants["cublas"] = _Captured(ctx, stream, reps, torch_fn=lambda: torch.matmul(a, bT, out=c2))
        ms, ms_min = _interleaved(variants, rounds)
        for v in variants.values():
            v.close()
        if with_cublas:
            del c2
        row = {"n": n, "tile": [best.bm, best.bn], "bk": best.bk, "stages": best.stages, "group_m": best.group_m,
               "split_k": best.split_k,
               "programs": progs, "tiles": tiles, "reps": reps, "tune_s": t_tune,
               "ms": ms, "ms_min": ms_min, "tflops": {k: flops / (v * 1e-3) / 1e12 for k, v in ms.items()}}
        row["checked_overhead"] = ms["checked"] / ms["safe"] - 1.0
        row["unchecked_vs_safe"] = ms["safe"] / ms["unchecked"]
        if with_cublas:
            row["safe_vs_cublas"] = ms["cublas"] / ms["safe"]
        if n == sizes[0]:
            row["host_enqueue_us"] = _enqueue_costs(ctx, p, c, a, bT, cfg, ucfg, stream)
        out.append(row)
        if log:
            log(f"n={n}: " + ", ".join(f"{k} {v:.0f} TF" for k, v in row["tflops"].items()))
        tp_partition_destroy(p)
        tp_partition_destroy(pp)
        del a, bt, c, bT
        torch.cuda.empty_cache()
    return out


def _enqueue_costs(ctx, p, c, a, bT, cfg, ucfg, stream) -> dict:
    """Host time per call to enqueue one GEMM: the safe entry (partition,
    alias and busy checks, ASYNC completion event) vs the raw entry."""
    L = _lib.lib()
    ev = tp_event_create(ctx)
    da, db = tensor_desc(a), tensor_desc(bT)
    ex = make_exec(ASYNC, stream, ev)
    sargs = (ctx.handle, p.handle, ctypes.byref(da), ctypes.byref(db), ctypes.byref(cfg), ctypes.byref(ex))
    uargs = (ctx.handle, ctypes.c_void_p(c.data_ptr()), ctypes.byref(da), ctypes.byref(db), ctypes.byref(ucfg),
             ctypes.c_void_p(stream.cuda_stream))
    fs, fu = L.tp_gemm, L.tp_gemm_unchecked

    def safe():
        _check(fs(*sargs), "tp_gemm")

    def raw():
        _check(fu(*uargs), "tp_gemm_unchecked")

    for fn in (safe, raw):
        _host_enqueue_us(fn, 20)
    res = {"safe": _host_enqueue_us(safe), "unchecked": _host_enqueue_us(raw)}
    _check(L.tp_event_wait(ev.handle), "tp_event_wait")
    tp_event_destroy(ev)
    return res


class _Worker:
    """One stream with its own outputs (one C per work-unit size) and ctypes
    arguments built once for SYNC and ASYNC launches of tp_gemm."""

    def __init__(self, ctx, stream, A, BT, cfgs):
        from . import tp_partition_map, MAP_STRIDED
        self.stream = stream
        self.ev = tp_event_create(ctx)
        self.c = [torch.empty(a.shape[0], b.shape[0], device=a.device, dtype=torch.bfloat16) for a, b in zip(A, BT)]
        self.p = []
        for c, cfg in zip(self.c, cfgs):
            p = tp_partition_create(ctx, c, (cfg.bm, cfg.bn))
            tp_partition_map(p, MAP_STRIDED, cfg.num_programs)
            self.p.append(p)
        self.da = [tensor_desc(a) for a in A]
        self.db = [tensor_desc(b.t()) for b in BT]
        self.cfgs = cfgs
        self.ex = {SYNC: make_exec(SYNC, stream), ASYNC: make_exec(ASYNC, stream, self.ev)}
        self.args = {m: [(ctx.handle, self.p[k].handle, ctypes.byref(self.da[k]), ctypes.byref(self.db[k]),
                          ctypes.byref(cfgs[k]), ctypes.byref(self.ex[m])) for k in range(len(A))]
                     for m in (SYNC, ASYNC)}
        L = _lib.lib()
        self._f, self._q = L.tp_gemm, L.tp_event_query
        self._done = ctypes.c_int32()
        self.active = False

    def run_sync(self, k: int) -> None:
        _check(self._f(*self.args[SYNC][k]), "tp_gemm")

    def launch_async(self, k: int) -> None:
        _check(self._f(*self.args[ASYNC][k]), "tp_gemm")
        self.active = True

    def poll(self) -> bool:
        _check(self._q(self.ev.handle, ctypes.byref(self._done)), "tp_event_query")
        if self._done.value:
            self.active = False
        return not self.active

    def close(self) -> None:
        tp_event_destroy(self.ev)
        for p in self.p:
            tp_partition_destroy(p)


def bimodal_kinds(n_units: int = 2000) -> list:
    """Work unit i is Large when i % 5 == 4: 20% Large interleaved with 80%
    Small, in a fixed order."""
    return [1 if i % 5 == 4 else 0 for i in range(n_units)]


def bimodal_queue(ctx, n_units: int = 2000, streams=(1, 2, 4, 8, 16, 32), small: int = 512, large: int = 2048,
                  reps: int = 3, log=None) -> dict:
    """The bimodal work-distribution experiment (Appendix B): a queue of
    `n_units` BF16 GEMMs, 80% Small (small^3) interleaved with 20% Large
    (large^3), drained as
      serial      one host thread, one stream, a SYNC tp_gemm per unit;
      threaded    S host threads, one stream each, SYNC per unit, units
                  taken from a shared counter;
      async       one host thread driving S streams: each stream has one
                  ASYNC unit in flight, the host polls tp_event_query and
                  issues the next unit on whichever stream finished;
      grouped     every unit as one problem of a single grouped persistent
                  launch (distinct outputs; plan built outside the timing).
    Work units per millisecond (WU/ms) of host wall time, best of `reps`."""
    import itertools
    import threading

    from . import (tp_autotune, tp_grouped_gemm, tp_grouped_plan_create, tp_grouped_plan_destroy, gemm_config)

    dev = torch.device("cuda", torch.cuda.current_device())
    gen = torch.Generator(device=dev)
    sizes = (small, large)
    A, BT = [], []
    for n in sizes:
        gen.manual_seed(n)
        A.append(torch.randn(n, n, device=dev, generator=gen).to(torch.bfloat16))
        BT.append(torch.randn(n, n, device=dev, generator=gen).to(torch.bfloat16))
    cfgs = []
    for n in sizes:
        best, _, _ = tp_autotune(ctx, n, n, n, "bf16")
        cfgs.append(tuned_config(ctx, best, -(-n // best.bm) * -(-n // best.bn)))
    kinds = bimodal_kinds(n_units)
    flops = sum(2.0 * sizes[k] ** 3 for k in kinds)
    S_max = max(streams)
    pool = [torch.cuda.Stream(device=dev) for _ in range(S_max)]
    workers = [_Worker(ctx, s, A, BT, cfgs) for s in pool]

    def timed(fn) -> float:
        fn()                                   # warm-up pass
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            t0 = time.perf_counter_ns()
            fn()
            t = (time.perf_counter_ns() - t0) / 1e6
            best = t if best is None else min(best, t)
        return best

    def serial():
        w = workers[0]
        for k in kinds:
            w.run_sync(k)

    def threaded(S):
        ctr = itertools.count()
        errors = []

        def body(w):
            try:
                while True:
                    i = next(ctr)
                    if i >= n_units:
                        return
                    w.run_sync(kinds[i])
            except BaseException as e:          # re-raised on the driving thread
                errors.append(e)

        ts = [threading.Thread(target=body, args=(workers[j],)) for j in range(S)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        if errors:
            raise errors[0]

    def async_(S):
        ws = workers[:S]
        nxt = 0
        while True:
            busy = False
            for w in ws:
                if w.active and not w.poll():
                    busy = True
                    continue
                if nxt < n_units:
                    w.launch_async(kinds[nxt])
                    nxt += 1
                    busy = True
            if not busy:
                return

    res = {"units": n_units, "small": small, "large": large, "large_fraction": sum(kinds) / n_units,
           "gflop": flops / 1e9, "configs": [{"bm": c.bm, "bn": c.bn, "stages": c.stages, "group_m": c.group_m,
                                              "programs": c.num_programs} for c in cfgs]}
    ms = timed(serial)
    res["serial"] = {"ms": ms, "wu_per_ms": n_units / ms}
    if log:
        log(f"serial: {n_units / ms:.1f} WU/ms")
    for name, fn in (("threaded", threaded), ("async", async_)):
        res[name] = {}
        for S in streams:
            ms = timed(lambda: fn(S))
            res[name][S] = {"ms": ms, "wu_per_ms": n_units / ms}
            if log:
                log(f"{name} S={S}: {n_units / ms:.1f} WU/ms")
    for w in workers:
        w.close()
    # grouped: one launch over all units, each with its own output
    outs = [torch.empty(sizes[k], sizes[k], device=dev, dtype=torch.bfloat16) for k in kinds]
    probs = [(A[k], BT[k].t(), c) for k, c in zip(kinds, outs)]
    t0 = time.perf_counter()
    plan = tp_grouped_plan_create(ctx, probs)
    t_plan = (time.perf_counter() - t0) * 1e3
    s0 = pool[0]
    ex = make_exec(SYNC, s0)
    ms = timed(lambda: tp_grouped_gemm(ctx, plan, 0, ex))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s0)
    tp_grouped_gemm(ctx, plan, 0, ex)
    e1.record(s0)
    e1.synchronize()
    dev_ms = e0.elapsed_time(e1)
    res["grouped"] = {"ms": ms, "wu_per_ms": n_units / ms, "device_ms": dev_ms, "plan_ms": t_plan,
                      "tflops": flops / (dev_ms * 1e-3) / 1e12}
    if log:
        log(f"grouped: {n_units / ms:.1f} WU/ms ({flops / (dev_ms * 1e-3) / 1e12:.0f} TFLOP/s device)")
    tp_grouped_plan_destroy(plan)
    del outs, probs
    torch.cuda.empty_cache()
    return res
