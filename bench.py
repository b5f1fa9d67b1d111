"""Benchmark of the partitioned tile-program hot path on GB300.

Default workload (one "step"): the four element-wise maps over 2^28 elements
with the output partitioned into 4096-element tiles, each run once:
z = 0.5 x + y and y = gelu_tanh(x) * w, in fp32 and in bf16 (fp32 math).
`value` is HBM throughput in TB/s: algorithmic bytes of the step (2 reads + 1
write per element per map, as the paper counts its element-wise add) divided
by the device time of the step. Inputs are 0.5-1 GiB per tensor, far larger
than the 129 MB L2, so no flush is needed between steps.

Secondary rows (the other hot-path configurations) are measured after the
timed region and reported under "rows".

--impl reference times the FP64 CPU oracle on the host cores instead.
Multi-GPU (torchrun): every rank runs the same per-GPU workload on its own
GPU (weak scaling, no collective on the data path); the step time is the max
over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ELEMS = 1 << 28
TILE = 4096
ALPHA = 0.5
MAPS = [("axpy", "f32"), ("gelu_mul", "f32"), ("axpy", "bf16"), ("gelu_mul", "bf16")]
ESIZE = {"f32": 4, "bf16": 2}
NOMINAL = {"hbm_gbs": 8000.0, "bf16_tflops": 2250.0, "fp8_tflops": 4500.0}   # GB300 dense, per GPU
METRIC = "GEMM TFLOP/s & map TB/s vs GB300 roofline; grouped vs plain speedup at stated error"
WORKLOAD = "element-wise maps over 2^28 elements, fp32 and bf16: z=0.5*x+y and y=gelu_tanh(x)*w, 4096-element tiles"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained"), "src": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "src": "fallback"}


def _traffic(kernel: str, src_file: str):
    """dram bytes per launch for `kernel` from profiles/dram_traffic.txt, only
    if the kernel's source file is unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    src = os.path.join(ROOT, "paper_2606_15991_gb300", "csrc", src_file)
    if not os.path.exists(path) or not os.path.exists(src):
        return None
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    for line in open(path):
        f = line.split()
        if len(f) >= 3 and not line.startswith("#") and f[0] == kernel and f[2] == digest:
            return float(f[1])
    return None


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait(timeout=5)
        sm = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 8 for i in range(4) if r[4 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier_max(value: float, ws: int, backend_dev):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=backend_dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(ws: int, bytes_per_rank_step: float, max_ms_per_step: float) -> float:
    """Whole-job TB/s: every rank moves the same bytes per step; the job's
    step time is the slowest rank's."""
    return ws * bytes_per_rank_step / (max_ms_per_step * 1e-3) / 1e12


def _all_ranks_ok(ok: bool, ws: int, backend_dev) -> bool:
    """True on every rank when `ok` holds on every rank (a MIN all-reduce)."""
    if ws == 1:
        return ok
    import torch
    import torch.distributed as dist

    t = torch.tensor([1 if ok else 0], dtype=torch.int32, device=backend_dev)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    return bool(t.item())


def _map_bytes(dt: str) -> int:
    return 3 * ESIZE[dt] * N_ELEMS


# --------------------------------------------------------------------- CPU oracle leg
def cpu_oracle_sample(seconds: float = 12.0):
    """Times the FP64 oracle maps (as they stand) on a 2^22-element sample of
    the same four maps, repeated until `seconds` elapse; returns TB/s over the
    same algorithmic byte count the GPU is charged."""
    import numpy as np

    import synth
    from oracle import maps as omaps

    n = 1 << 22
    data = {}
    for _, dt in MAPS:
        if dt not in data:
            x = synth.tensor(synth.normal(n, 1), dt).double().numpy()
            y = synth.tensor(synth.normal(n, 2), dt).double().numpy()
            data[dt] = (x, y)
    reps = 0
    bytes_done = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        for op, dt in MAPS:
            x, y = data[dt]
            z = omaps.axpy(ALPHA, x, y) if op == "axpy" else omaps.gelu_mul(x, y)
            z.astype(np.float32)
            bytes_done += 3 * ESIZE[dt] * n
        reps += 1
    el = time.perf_counter() - t0
    return {"value": bytes_done / el / 1e12, "unit": "TB/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} passes of the 4 maps over 2^22 of the 2^28 elements (numpy float64, 1 thread), "
                      f"{el:.1f} s"}


def cpu_oracle_gemm_rows(seconds: float = 4.0) -> dict:
    """The FP64 GEMM oracle (as it stands: a float64 matmul over the exact
    input values) on the host: the full 512^3 FP32 configuration, and 128x128
    output tiles of the 8192^3 configuration (K = 8192) timed and
    extrapolated to the 4096 tiles of the full product."""
    import numpy as np

    import synth
    from oracle import gemm as ogemm

    out = {}
    a = synth.uniform(512 * 512, 0).reshape(512, 512)
    b = synth.uniform(512 * 512, 1).reshape(512, 512)
    reps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds / 2:
        ogemm.gemm(a, b)
        reps += 1
    el = (time.perf_counter() - t0) / reps
    out["gemm_f32_512"] = {"tflops": 2 * 512 ** 3 / el / 1e12, "ms": el * 1e3, "kind": "oracle", "sample": "full"}
    K = 8192
    at = synth.normal(128 * K, 2).reshape(128, K)
    bt = synth.normal(128 * K, 3).reshape(K, 128)
    reps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds / 2:
        ogemm.gemm(at, bt)
        reps += 1
    el = (time.perf_counter() - t0) / reps
    out["gemm_bf16_8192"] = {"tflops": 2 * 128 * 128 * K / el / 1e12, "ms_extrapolated": el * 4096 * 1e3,
                             "kind": "oracle", "sample": f"{reps} 128x128 output tiles with K = 8192, "
                                                          "extrapolated to the 4096 tiles of 8192^3"}
    # the 64-problem group: one output tile (128 x 128, or M x 128 for M <
    # 128) per problem with that problem's full K, extrapolated to every
    # tile of every problem
    probs = synth.grouped_problems(64, seed=0)
    t_total, flops, tiles_timed, t0_all = 0.0, 0.0, 0, time.perf_counter()
    for i, (m, n, k) in enumerate(probs):
        tm = min(m, 128)
        at = synth.normal(tm * k, 10 + 2 * i).reshape(tm, k)
        bt = synth.normal(k * 128, 11 + 2 * i).reshape(k, 128)
        t0 = time.perf_counter()
        ogemm.gemm(at, bt)
        el = time.perf_counter() - t0
        tiles_timed += 1
        t_total += el * (-(-m // 128)) * (-(-n // 128))
        flops += 2.0 * m * n * k
    out["grouped_64"] = {"tflops": flops / t_total / 1e12, "ms_extrapolated": t_total * 1e3, "kind": "oracle",
                         "sample": f"{tiles_timed} output tiles (one per problem, full K), extrapolated to every "
                                   f"tile of the 64 problems; {time.perf_counter() - t0_all:.1f} s"}
    out["threads"] = "numpy's BLAS threads (all host cores unless limited)"
    return out


def _oracle_worker_init(n: int, seed: int):
    """Pool worker: its own 2^22-element sample of the four maps' inputs (the
    bf16 values rounded by the oracle's bf16 definition)."""
    import numpy as np

    import synth
    from oracle import lowp

    global _ORACLE_DATA
    x = synth.normal(n, 1 + 2 * seed).astype(np.float32).astype(np.float64)
    y = synth.normal(n, 2 + 2 * seed).astype(np.float32).astype(np.float64)
    _ORACLE_DATA = {"f32": (x, y), "bf16": (lowp.round_bf16(x), lowp.round_bf16(y))}


def _oracle_worker_run(seconds: float):
    import numpy as np

    from oracle import maps as omaps

    n = len(_ORACLE_DATA["f32"][0])
    done, reps = 0, 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        for op, dt in MAPS:
            x, y = _ORACLE_DATA[dt]
            z = omaps.axpy(ALPHA, x, y) if op == "axpy" else omaps.gelu_mul(x, y)
            z.astype(np.float32)
            done += 3 * ESIZE[dt] * n
        reps += 1
    return done, time.perf_counter() - t0, reps


class OraclePool:
    """The FP64 oracle maps (as they stand) run by one spawned process per
    host core, each on its own 2^22-element sample; run(seconds) returns the
    aggregate TB/s over the algorithmic bytes the GPU is charged."""

    def __init__(self, n: int = 1 << 22):
        import multiprocessing as mp

        self.cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        self.n = n
        ctx = mp.get_context("spawn")   # the parent holds a CUDA context: never fork it
        self.pool = ctx.Pool(self.cores, initializer=_oracle_worker_init_indexed, initargs=(n, ctx.Value("i", 0)))

    def run(self, seconds: float) -> dict:
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker_run, [seconds] * self.cores, chunksize=1)
        wall = time.perf_counter() - t0
        done = sum(r[0] for r in res)
        reps = sum(r[2] for r in res)
        return {"value": done / wall / 1e12, "unit": "TB/s", "cores": self.cores, "kind": "oracle",
                "sample": f"{self.cores} processes, each {reps // self.cores}+ passes of the 4 maps over its own "
                          f"2^22 of the 2^28 elements (numpy float64), {wall:.1f} s wall"}

    def close(self):
        self.pool.close()
        self.pool.join()


def _oracle_worker_init_indexed(n: int, counter):
    with counter.get_lock():
        i = counter.value
        counter.value += 1
    _oracle_worker_init(n, i)


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    pool = OraclePool()
    steps = []
    for _ in range(args.warmup):
        pool.run(1.0)
    for _ in range(args.steps):
        steps.append(pool.run(max(1.0, 30.0 / max(1, args.steps))))
    pool.close()
    vals = [s["value"] for s in steps]
    v = statistics.median(vals)
    base = steps[0]
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "TB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "bounded CPU sample per step"},
        "cpu_baseline": {"value": v, "unit": "TB/s", "cores": base["cores"], "kind": "oracle",
                         "sample": base["sample"]},
        "e2e": {"value": v, "unit": "TB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# --------------------------------------------------------------------- GPU leg
def run_ours(args):
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_2606_15991_gb300 import build as _build

    _build.build()
    import paper_2606_15991_gb300 as tp

    ctx = tp.tp_ctx_create(dev.index)
    stream = torch.cuda.Stream(device=dev)
    gen = torch.Generator(device=dev)
    inputs = {}
    for dt in ("f32", "bf16"):
        tdt = torch.float32 if dt == "f32" else torch.bfloat16
        gen.manual_seed(1)
        x = torch.randn(N_ELEMS, device=dev, generator=gen).to(tdt)
        gen.manual_seed(2)
        y = torch.randn(N_ELEMS, device=dev, generator=gen).to(tdt)
        inputs[dt] = (x, y)
    tens = {}   # one output tensor + partition per map: a partition in flight is held exclusively
    for op, dt in MAPS:
        x, y = inputs[dt]
        z = torch.empty_like(x)
        tens[(op, dt)] = (x, y, z, tp.tp_partition_create(ctx, z, (TILE,)))
    torch.cuda.synchronize()
    ex = tp.make_exec(stream=stream)
    ex.mode = tp.ASYNC   # launches are chained on the stream; the event wait ends the step
    ev = tp.tp_event_create(ctx)
    ex.event = ev.handle.value

    def launch(op, dt):
        x, y, z, p = tens[(op, dt)]
        if op == "axpy":
            tp.tp_map_axpy(ctx, p, ALPHA, x, y, ex)
        else:
            tp.tp_map_gelu_mul(ctx, p, x, y, ex)

    def step():
        for op, dt in MAPS:
            launch(op, dt)
        tp.tp_event_wait(ev)   # releases the partitions (host-side protocol)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    # per-launch events on the launching stream (for the roofline)
    evs = {k: [] for k in MAPS}
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    # The timed steps are chained on one stream (§3.2's asynchronous
    # pipeline: same-stream launches may rewrite a partition still held by
    # the previous step); the event wait after the last step releases them.
    t_start.record(stream)
    for _ in range(args.steps):
        for op, dt in MAPS:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            launch(op, dt)
            e1.record(stream)
            evs[(op, dt)].append((e0, e1))
    t_end.record(stream)
    tp.tp_event_wait(ev)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    el_ms = t_start.elapsed_time(t_end)
    el_ms = _barrier_max(el_ms, ws, dev)
    ms_step = el_ms / args.steps
    step_bytes = sum(_map_bytes(dt) for _, dt in MAPS)
    value = weak_scaling_value(ws, step_bytes, ms_step)

    per_kernel = {}
    for k, lst in evs.items():
        d = [a.elapsed_time(b) for a, b in lst]
        per_kernel[k] = sum(d) / len(d)
    peaks = _peaks()
    dom = max(per_kernel, key=per_kernel.get)
    dom_bytes = _map_bytes(dom[1])
    achieved = dom_bytes / (per_kernel[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": f"map_vec_kernel<{dom[0]},{dom[1]}>", "achieved": achieved,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "peak_src": peaks["src"], "frac_of_nominal": achieved / NOMINAL["hbm_gbs"],
                "traffic": _traffic(f"{dom[0]}_{dom[1]}", "map_kernels.cu"),
                "algorithmic_bytes_per_launch": dom_bytes,
                "per_map_gbs": {f"{o}_{d}": _map_bytes(d) / (t * 1e-3) / 1e9 for (o, d), t in per_kernel.items()}}

    # ---------------- end-to-end through the C ABI with pinned host buffers
    e2e = None
    if not args.skip_e2e:
        e2e = _e2e_leg(tp, ctx, ex, ev, inputs, tens, step_bytes, ws, dev, args)

    rows = {}
    if not args.skip_rows and rank == 0:
        rows = secondary_rows(tp, ctx, dev, stream, peaks, args)

    cpu = None
    if rank == 0 and ws == 1 and not args.skip_cpu:
        pool = OraclePool()
        pool.run(1.0)
        cpu = pool.run(args.cpu_seconds)
        pool.close()
        single = cpu_oracle_sample(seconds=args.cpu_seconds / 2)
        cpu["single_thread"] = {"value": single["value"], "unit": "TB/s", "sample": single["sample"]}
        cpu["rows"] = cpu_oracle_gemm_rows()
        cpu["host"] = {"nproc": os.cpu_count(), "affinity_cpus": len(os.sched_getaffinity(0))
                       if hasattr(os, "sched_getaffinity") else None}

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "TB/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "elements": N_ELEMS, "tile": TILE, "alpha": ALPHA,
                       "storage_dtypes": ["f32", "bf16"], "arithmetic": "f32 (bf16 inputs widened, results rounded)",
                       "maps": [f"{o}_{d}" for o, d in MAPS], "l2": "inputs larger than L2 (no flush)",
                       "parallelism": f"replicas x{ws}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": len(MAPS) * args.steps, "clocks": clocks, "rows": rows,
        }))
    if ws > 1:
        torch.distributed.destroy_process_group()


E2E_CHUNKS = 16   # pipeline chunks of the end-to-end step (2^24 elements each)


def _e2e_leg(tp, ctx, ex, ev, inputs, tens, step_bytes, ws, dev, args):
    """The maps step end to end through the C ABI, inputs and outputs in
    pinned host memory. Every step copies its inputs (x and y of both dtypes)
    to the device, runs the four maps and copies their results back, in
    E2E_CHUNKS chunks pipelined over three streams (copies in, maps, copies
    out), so both directions of the host link stay busy while the kernels
    run; each input crosses the link once per step, as it would for a user
    running the four maps on host data. (The maps reading and writing host
    memory directly, each map fetching its own inputs over the link, ran at
    0.30 TB/s on GB300, bound by the ~210 GB/s host-to-device direction.)"""
    import torch

    # every rank must hold its pinned buffers before any rank times (the
    # ranks meet in a collective afterwards), so they agree first
    err = None
    try:
        host_in = {dt: (x.cpu().pin_memory(), y.cpu().pin_memory()) for dt, (x, y) in inputs.items()}
        host_out = {(op, dt): torch.empty(N_ELEMS, dtype=inputs[dt][0].dtype).pin_memory() for op, dt in MAPS}
    except (RuntimeError, MemoryError) as e:
        err = f"{type(e).__name__}: {str(e)[:200]}"
    if _all_ranks_ok(err is None, ws, dev) is False:
        return {"value": None, "unit": "TB/s", "unavailable": err or "pinned host buffers unavailable on another rank"}
    L = N_ELEMS // E2E_CHUNKS
    chunks = [slice(c * L, (c + 1) * L) for c in range(E2E_CHUNKS)]
    parts = {(op, dt, c): tp.tp_partition_create(ctx, tens[(op, dt)][2][sl], (TILE,))
             for op, dt in MAPS for c, sl in enumerate(chunks)}
    s_in, s_map, s_out = (torch.cuda.Stream(device=dev) for _ in range(3))
    ev_map = tp.tp_event_create(ctx)
    ex_map = tp.make_exec(stream=s_map)
    ex_map.mode = tp.ASYNC
    ex_map.event = ev_map.handle.value
    e2e_steps = max(2, min(args.steps, 5))

    def e2e_step():
        for c, sl in enumerate(chunks):
            with torch.cuda.stream(s_in):
                for dt, (hx, hy) in host_in.items():
                    dx, dy = inputs[dt]
                    dx[sl].copy_(hx[sl], non_blocking=True)
                    dy[sl].copy_(hy[sl], non_blocking=True)
            landed = torch.cuda.Event()
            landed.record(s_in)
            s_map.wait_event(landed)
            for op, dt in MAPS:
                dx, dy = inputs[dt]
                if op == "axpy":
                    tp.tp_map_axpy(ctx, parts[(op, dt, c)], ALPHA, dx[sl], dy[sl], ex_map)
                else:
                    tp.tp_map_gelu_mul(ctx, parts[(op, dt, c)], dx[sl], dy[sl], ex_map)
            mapped = torch.cuda.Event()
            mapped.record(s_map)
            s_out.wait_event(mapped)
            with torch.cuda.stream(s_out):
                for op, dt in MAPS:
                    host_out[(op, dt)][sl].copy_(tens[(op, dt)][2][sl], non_blocking=True)
        tp.tp_event_wait(ev_map)
        s_out.synchronize()

    e2e_step()
    torch.cuda.synchronize()
    each = []
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
        each.append(time.perf_counter())
    t1 = time.perf_counter()
    each = [round((b - a) * 1e3, 2) for a, b in zip([t0] + each[:-1], each)]
    e2e_ms = _barrier_max((t1 - t0) * 1e3 / e2e_steps, ws, dev)
    # the results read back on the host: a strided sample of every output is
    # compared with a device-resident run of the same maps on the same inputs
    for op, dt in MAPS:
        x, y, z, p = tens[(op, dt)]
        if op == "axpy":
            tp.tp_map_axpy(ctx, p, ALPHA, x, y)
        else:
            tp.tp_map_gelu_mul(ctx, p, x, y)
        assert torch.equal(host_out[(op, dt)][::4097], z[::4097].cpu()), (op, dt)
    h2d = sum(2 * ESIZE[dt] * N_ELEMS for dt in host_in)
    d2h = sum(ESIZE[dt] * N_ELEMS for _, dt in MAPS)
    e2e = {"value": weak_scaling_value(ws, step_bytes, e2e_ms), "unit": "TB/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "ms_each_step": each, "steps": e2e_steps,
           "transfer": f"pinned host inputs copied in and results copied out every step, in {E2E_CHUNKS} chunks "
                       "pipelined with the maps over three streams (each input crosses the link once per step)"}
    for p in parts.values():
        tp.tp_partition_destroy(p)
    tp.tp_event_destroy(ev_map)
    return e2e


def _graph_time(tp, ctx, stream, record, reps: int, replays: int = 3) -> float:
    """Device time (ms) of one recorded op (`record(ex)` captured `reps`
    times into one graph and replayed; the fastest replay / reps)."""
    from paper_2606_15991_gb300 import experiments

    return experiments.graph_time_ms(ctx, stream, record, reps, replays)


def secondary_rows(tp, ctx, dev, stream, peaks, args):
    """Other hot-path configurations. Each op is captured back to back into
    a CUDA graph and replayed; per-op time = replay time / ops (CUDA events)."""
    import torch

    import synth

    rows = {}
    # FP32 FFMA GEMM 512^3, 64x64 tiles (64 programs)
    a = torch.from_numpy(synth.uniform(512 * 512, seed=0)).reshape(512, 512).to(dev)
    b = torch.from_numpy(synth.uniform(512 * 512, seed=1)).reshape(512, 512).to(dev)
    c = torch.empty(512, 512, device=dev)
    p = tp.tp_partition_create(ctx, c, (64, 64))
    f32cfg = tp.gemm_config(bk=32, split_k=2)
    ms = _graph_time(tp, ctx, stream, lambda ex: tp.tp_gemm(ctx, p, a, b, f32cfg, ex), reps=50)
    rows["gemm_f32_512"] = {"tflops": 2 * 512 ** 3 / (ms * 1e-3) / 1e12, "ms": ms, "programs": 64,
                            "split_k": 2, "bk": 32,
                            "note": "64 tile programs, each a cluster of 2 CTAs splitting K (128 of 152 SMs), "
                                    "operands fed by TMA into a ring of 32-wide K chunks"}
    tp.tp_partition_destroy(p)
    del a, b, c

    # BF16 and FP8 tcgen05 GEMM 8192^3, 256x256 tiles on CTA pairs
    M = N = K = 8192
    flops = 2 * M * N * K
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    a = torch.randn(M, K, device=dev, generator=g).to(torch.bfloat16)
    bt = torch.randn(N, K, device=dev, generator=g).to(torch.bfloat16)   # B stored N x K (K-major)
    c = torch.empty(M, N, device=dev, dtype=torch.bfloat16)
    # 256 x 256 tiles on CTA pairs, stages of 2 K blocks, raster bands of 8
    cfg = tp.gemm_config(bm=256, bn=256, group_m=8, bk=128)
    p = tp.tp_partition_create(ctx, c, (256, 256))
    tp.tp_partition_map(p, tp.MAP_STRIDED, min(ctx.sm_count // 2, tp.tp_partition_query(p)["num_tiles"]))
    ms = _graph_time(tp, ctx, stream, lambda ex: tp.tp_gemm(ctx, p, a, bt.t(), cfg, ex), reps=10)
    ms_cublas = _torch_graph_time(stream, lambda: torch.matmul(a, bt.t(), out=c), reps=10)
    tf = flops / (ms * 1e-3) / 1e12
    rows["gemm_bf16_8192"] = {
        "tflops": tf, "ms": ms, "tile": [256, 256], "programs": ctx.sm_count // 2, "bk": 128, "group_m": 8,
        "cublas_tflops_same_run": flops / (ms_cublas * 1e-3) / 1e12, "vs_cublas_same_run": ms_cublas / ms,
        "roofline": {"bound": "tensor", "achieved": tf, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                     "frac_of_nominal": tf / NOMINAL["bf16_tflops"],
                     "frac": tf / peaks["bf16_tflops"], "peak_src": peaks["src"] + " bf16 burst"}}

    # FP8: amax + quantize (HBM passes, reported separately) and the GEMM
    amax = torch.zeros(2, device=dev)
    scale = torch.zeros(2, device=dev)
    qa = torch.empty(M, K, device=dev, dtype=torch.float8_e4m3fn)
    qbt = torch.empty(N, K, device=dev, dtype=torch.float8_e4m3fn)
    pqa = tp.tp_partition_create(ctx, qa, (16, K))
    pqb = tp.tp_partition_create(ctx, qbt, (16, K))

    def quant(ex):
        tp.tp_amax(ctx, a, amax[0:1], ex)
        tp.tp_amax(ctx, bt, amax[1:2], ex)
        tp.tp_quantize_fp8(ctx, pqa, a, amax[0:1], scale[0:1], ex)
        tp.tp_quantize_fp8(ctx, pqb, bt, amax[1:2], scale[1:2], ex)

    qms = _graph_time(tp, ctx, stream, quant, reps=5)
    qbytes = 2 * (2 * M * K * 2 + M * K)   # per operand: amax read + quantize read (bf16) + write (fp8)
    # stages of 2 K blocks of 128 codes, raster bands of 16
    cfg8 = tp.gemm_config(bm=256, bn=256, group_m=16, bk=256)
    ms8 = _graph_time(tp, ctx, stream,
                      lambda ex: tp.tp_gemm_fp8(ctx, p, qa, qbt.t(), scale[0:1], scale[1:2], cfg8, ex), reps=10)
    inv = (1.0 / scale).contiguous()
    sa, sb = inv[0:1].reshape(()).contiguous(), inv[1:2].reshape(()).contiguous()
    ms8_cublas = _torch_graph_time(stream, lambda: torch._scaled_mm(qa, qbt.t(), scale_a=sa, scale_b=sb,
                                                                    out_dtype=torch.bfloat16), reps=10)
    tf8 = flops / (ms8 * 1e-3) / 1e12
    peak8 = 2 * peaks["bf16_tflops"]
    rows["gemm_fp8_8192"] = {
        "tflops": tf8, "ms": ms8, "tile": [256, 256], "bk": 256, "group_m": 16,
        "cublas_tflops_same_run": flops / (ms8_cublas * 1e-3) / 1e12, "vs_cublas_same_run": ms8_cublas / ms8,
        "quantize_ms": qms, "quantize_gbs": qbytes / (qms * 1e-3) / 1e9,
        "tflops_incl_quantize": flops / ((ms8 + qms) * 1e-3) / 1e12,
        "roofline": {"bound": "tensor", "achieved": tf8, "peak": peak8, "unit": "TFLOP/s", "frac": tf8 / peak8,
                     "frac_of_nominal": tf8 / NOMINAL["fp8_tflops"],
                     "peak_src": peaks["src"] + " bf16 burst x 2 (nominal fp8:bf16 dense ratio)"}}
    for h in (p, pqa, pqb):
        tp.tp_partition_destroy(h)
    del a, bt, c, qa, qbt
    torch.cuda.empty_cache()
    rows["small_gemm"] = small_gemm_row(tp, ctx, dev, stream)
    rows["grouped_64"] = grouped_row(tp, ctx, dev, stream, peaks)
    rows["decode_64"] = decode_row(tp, ctx, dev, stream, peaks)
    if not args.skip_proposer:
        rows["proposer"] = proposer_row(tp, ctx, args.train_shapes, args.test_shapes, args.epochs)
    if not args.skip_experiments:
        rows["experiments"] = experiment_rows(tp, ctx, peaks)
    return rows


def experiment_rows(tp, ctx, peaks) -> dict:
    """The paper's three measurement studies in short form, each run here in
    full: the BF16 GEMM size sweep with safe / checked / unchecked / plain
    launches and cuBLAS (§5.1), microseconds per op of the four execution
    modes (§5.2), and the bimodal GEMM queue (Appendix B). About 45 s."""
    from paper_2606_15991_gb300 import experiments

    sweep = experiments.gemm_size_sweep(ctx, (1024, 2048, 4096, 8192, 16384, 32768))
    modes = experiments.exec_mode_scaling(ctx, reps=30)
    bim = experiments.bimodal_queue(ctx, reps=3)
    us = modes["us_per_op"]
    plateau = max(list(bim["threaded"].values()) + list(bim["async"].values()), key=lambda r: r["wu_per_ms"])
    return {
        "gemm_sweep": [{"n": r["n"], "tile": r["tile"], "bk": r["bk"],
                        "tflops": {k: round(v, 1) for k, v in r["tflops"].items()},
                        "checked_overhead": r["checked_overhead"], "unchecked_vs_safe": r["unchecked_vs_safe"],
                        "safe_vs_cublas": r.get("safe_vs_cublas"),
                        "frac_of_measured_bf16_safe": r["tflops"]["safe"] / peaks["bf16_tflops"]} for r in sweep],
        "exec_modes_us_per_op": {m: {str(n): us[m][n]["min"] for n in (1, 10, 100, 1000) if n in us[m]}
                                 for m in us},
        "exec_modes_note": "minimum us per op of an N-launch chain (2048-element bf16 tile), host wall time",
        "bimodal_wu_per_ms": {"serial": bim["serial"]["wu_per_ms"], "best_threads_or_streams": plateau["wu_per_ms"],
                              "grouped": bim["grouped"]["wu_per_ms"]},
        "paper_reference_numbers": {"rtx5090_us_per_op_at_1000": {"sync": 7.3, "chained": 3.4, "async": 3.4,
                                                                  "graph": 0.8},
                                    "b200_bimodal_wu_per_ms": {"serial": 37, "plateau_S8": 77}},
    }


def _torch_graph_time(stream, fn, reps: int, replays: int = 3) -> float:
    """Device time (ms) of one torch call (cuBLAS): `reps` calls captured
    into one CUDA graph and replayed; the fastest replay / reps."""
    from paper_2606_15991_gb300 import experiments

    cap = experiments._Captured(None, stream, reps, torch_fn=fn)
    ms = min(cap.time() for _ in range(replays))
    cap.close()
    return ms


def small_gemm_row(tp, ctx, dev, stream):
    """Small and skinny BF16 GEMMs on each shape's autotuned config (the
    single-pass class, whose configs all compute C bit-identically), on the
    split-K opt-in's pick and, for M <= 128, on the swap-AB opt-in's pick
    (same class), against cuBLAS (torch.matmul) in the same run; for
    M <= 256 also swap-AB through the grouped kernel (one-problem group)."""
    import torch

    from paper_2606_15991_gb300 import experiments

    out = {}
    for m, n, k in ((1024, 1024, 1024), (2048, 2048, 2048), (64, 8192, 8192), (64, 16384, 4096)):
        g = torch.Generator(device=dev)
        g.manual_seed(m + n + k)
        a = torch.randn(m, k, device=dev, generator=g).to(torch.bfloat16)
        bt = torch.randn(n, k, device=dev, generator=g).to(torch.bfloat16)
        c = torch.empty(m, n, device=dev, dtype=torch.bfloat16)
        fl = 2.0 * m * n * k
        reps = 50
        row = {}
        searches = [("single_pass", False, False), ("split_k_opt_in", True, False)]
        if m <= 128:
            searches.append(("swap_ab_opt_in", False, True))
        for name, split, swap in searches:
            best, _, _ = tp.tp_autotune(ctx, m, n, k, "bf16", split_k=split, swap_ab=swap)
            p = tp.tp_partition_create(ctx, c, (best.bm, best.bn))
            cfg = experiments.tuned_config(ctx, best, tp.tp_partition_query(p)["num_tiles"])
            tp.tp_partition_map(p, tp.MAP_STRIDED, cfg.num_programs)
            ms = _graph_time(tp, ctx, stream, lambda ex: tp.tp_gemm(ctx, p, a, bt.t(), cfg, ex), reps=reps)
            tp.tp_partition_destroy(p)
            row[name] = {"us": ms * 1e3, "tflops": fl / (ms * 1e-3) / 1e12,
                         "config": {f: getattr(best, f) for f in ("bm", "bn", "bk", "group_m", "split_k", "swap_ab")}}
        if m <= 256:
            # the same product computed swap-AB (C^T = B^T A^T: 128 or 256 N rows
            # per MMA, N = M) by the grouped kernel as a one-problem group
            for pair in (True, False):
                plan = tp.tp_grouped_plan_create(ctx, [(a, bt.t(), c)], -1, pair)
                ms = _graph_time(tp, ctx, stream, lambda ex: tp.tp_grouped_gemm(ctx, plan, 0, ex), reps=reps)
                tp.tp_grouped_plan_destroy(plan)
                row["swap_ab_pairs" if pair else "swap_ab_single_ctas"] = {"us": ms * 1e3,
                                                                          "tflops": fl / (ms * 1e-3) / 1e12}
        ms_cb = _torch_graph_time(stream, lambda: torch.matmul(a, bt.t(), out=c), reps=reps)
        row["cublas_us"] = ms_cb * 1e3
        for name, _, _ in searches:
            row[name]["vs_cublas"] = ms_cb / (row[name]["us"] * 1e-3)
        row["b_stream_gbs_single_pass"] = 2.0 * n * k / (row["single_pass"]["us"] * 1e-6) / 1e9
        out[f"{m}x{n}x{k}"] = row
    return out


def decode_row(tp, ctx, dev, stream, peaks):
    """Batch-1 decode-shaped chain, 64 layers (d 5120, QKV 10240, gate/up
    2 x 25600, down 25600 -> 5120), bf16 N(0, 0.02) weights: fused kernels
    replayed as one CUDA graph against one synced call per step."""
    import torch

    d, nq, ni, L = 5120, 10240, 25600, 64
    g = torch.Generator(device=dev)
    layers = []
    for i in range(L):
        g.manual_seed(100 + i)
        layers.append(tuple((torch.randn(r, k, device=dev, generator=g) * 0.02).to(torch.bfloat16)
                            for r, k in ((nq, d), (2 * ni, d), (d, ni))))
    wbytes = sum(w.numel() * 2 for lay in layers for w in lay)
    g.manual_seed(11)
    h0 = torch.randn(d, device=dev, generator=g)
    h = h0.clone()
    ch = tp.DecodeChain(ctx, h, layers)
    gr = tp.tp_graph_begin(ctx, stream)
    ch.record_fused(tp.make_exec(mode=tp.CAPTURE, stream=stream))
    tp.tp_graph_end(gr)
    launches_graph = tp.tp_graph_kernel_count(gr)
    ex = tp.make_exec(stream=stream)
    tp.tp_graph_replay(gr, ex)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(5):
        e0.record(stream)
        tp.tp_graph_replay(gr, ex)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms_graph = min(ts)
    tp.tp_graph_destroy(gr)

    def wall(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            t = (time.perf_counter() - t0) * 1e3
            best = t if best is None else min(best, t)
        return best

    sync_ex = tp.make_exec(stream=stream)
    ms_plain = wall(lambda: ch.record_unfused(sync_ex))
    ms_fused_sync = wall(lambda: ch.record_fused(sync_ex))
    ch.close()
    roof = wbytes / (peaks["hbm_gbs"] * 1e9) * 1e3
    del layers
    torch.cuda.empty_cache()
    return {"ms_graph_fused": ms_graph, "ms_plain_sync_unfused": ms_plain, "ms_sync_fused": ms_fused_sync,
            "speedup_vs_plain": ms_plain / ms_graph, "speedup_vs_sync_fused": ms_fused_sync / ms_graph,
            "speedup_bound_vs_plain": ms_plain / roof, "weight_gb": wbytes / 1e9,
            "weight_gbs_graph": wbytes / (ms_graph * 1e-3) / 1e9, "roofline_ms": roof,
            "frac_of_roofline": roof / ms_graph, "launches_graph": launches_graph, "launches_plain": 6 * L,
            "note": "plain = 6 kernels per layer, each launched and synchronised on its own (per-call sync); "
                    "speedup_bound_vs_plain = plain time / HBM roofline time, the largest speed-up any "
                    "implementation streaming the weights once could reach against it"}


def grouped_rooflines_ms(shapes, peaks) -> tuple:
    """Roofline times (ms) of a group of BF16 GEMMs (M, N, K), each problem
    2MNK flops and 2(MK + KN + MN) bytes. The grouped launch can overlap
    HBM-bound and tensor-bound tiles, so its bound is max(total flops /
    tensor peak, total bytes / HBM peak): at the burst bf16 peak, and at the
    sustained one (the burst one when none is measured). The sum of the
    problems' own bounds (no overlap) is returned third."""
    flops = sum(2.0 * m * n * k for m, n, k in shapes)
    bytes_ = sum(2.0 * (m * k + k * n + m * n) for m, n, k in shapes)
    hbm = peaks["hbm_gbs"] * 1e9
    t_overlap = max(flops / (peaks["bf16_tflops"] * 1e12), bytes_ / hbm) * 1e3
    sust = peaks.get("bf16_tflops_sustained") or peaks["bf16_tflops"]
    t_overlap_sust = max(flops / (sust * 1e12), bytes_ / hbm) * 1e3
    t_sum = sum(max(2.0 * m * n * k / (peaks["bf16_tflops"] * 1e12), 2.0 * (m * k + k * n + m * n) / hbm)
                for m, n, k in shapes) * 1e3
    return t_overlap, t_overlap_sust, t_sum


def grouped_row(tp, ctx, dev, stream, peaks):
    """64 BF16 GEMMs (M log-uniform on [1, 4096], four (K, N) pairs, seed 0):
    one persistent grouped launch against 64 plain per-call launches."""
    import torch

    import synth

    shapes = synth.grouped_problems(64, seed=0)
    g = torch.Generator(device=dev)
    probs = []
    for i, (m, n, k) in enumerate(shapes):
        g.manual_seed(1000 + i)
        a = torch.randn(m, k, device=dev, generator=g).to(torch.bfloat16)
        bt = torch.randn(n, k, device=dev, generator=g).to(torch.bfloat16)
        probs.append((a, bt.t(), torch.empty(m, n, dtype=torch.bfloat16, device=dev)))
    flops = sum(2.0 * m * n * k for m, n, k in shapes)
    bytes_ = sum(2.0 * (m * k + k * n + m * n) for m, n, k in shapes)
    plan = tp.tp_grouped_plan_create(ctx, probs)
    total_tiles, swapped = tp.tp_grouped_plan_info(plan)
    ms_grouped = _graph_time(tp, ctx, stream, lambda ex: tp.tp_grouped_gemm(ctx, plan, 0, ex), reps=3)
    # plain per-call: one tp_gemm per problem (1-CTA tiles for M <= 128, CTA pairs above)
    parts = []
    for a, b, c in probs:
        bm = 128 if a.shape[0] <= 128 else 256
        p = tp.tp_partition_create(ctx, c, (bm, 256))
        tiles = tp.tp_partition_query(p)["num_tiles"]
        tp.tp_partition_map(p, tp.MAP_STRIDED, min(tiles, ctx.sm_count * 128 // bm))
        parts.append((p, tp.gemm_config(bm=bm, bn=256, group_m=8)))
    sync_ex = tp.make_exec(stream=stream)

    def plain_sync():
        for (a, b, c), (p, cfg) in zip(probs, parts):
            tp.tp_gemm(ctx, p, a, b, cfg, sync_ex)

    ev = tp.tp_event_create(ctx)
    async_ex = tp.make_exec(mode=tp.ASYNC, stream=stream, event=ev)

    def plain_chained():
        for (a, b, c), (p, cfg) in zip(probs, parts):
            tp.tp_gemm(ctx, p, a, b, cfg, async_ex)
        tp.tp_event_wait(ev)

    # plain per-call on each problem's autotuned config (single-pass class)
    from paper_2606_15991_gb300 import experiments

    tuned = []
    for (a, b, c), (m, n, k) in zip(probs, shapes):
        best, _, _ = tp.tp_autotune(ctx, m, n, k, "bf16")
        p = tp.tp_partition_create(ctx, c, (best.bm, best.bn))
        tiles = tp.tp_partition_query(p)["num_tiles"]
        cfg = experiments.tuned_config(ctx, best, tiles)
        tp.tp_partition_map(p, tp.MAP_STRIDED, cfg.num_programs)
        tuned.append((p, cfg))

    def tuned_sync():
        for (a, b, c), (p, cfg) in zip(probs, tuned):
            tp.tp_gemm(ctx, p, a, b, cfg, sync_ex)

    res = {}
    for name, fn in (("plain_sync", plain_sync), ("plain_chained", plain_chained), ("tuned_sync", tuned_sync)):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
        res[name] = min(ts)
    for p, _ in parts + tuned:
        tp.tp_partition_destroy(p)
    tp.tp_event_destroy(ev)
    tp.tp_grouped_plan_destroy(plan)
    t_overlap, t_overlap_sust, t_sum = grouped_rooflines_ms(shapes, peaks)
    del probs
    torch.cuda.empty_cache()
    return {"ms_grouped": ms_grouped, "ms_plain_sync": res["plain_sync"], "ms_plain_chained": res["plain_chained"],
            "ms_tuned_sync": res["tuned_sync"],
            "speedup_vs_plain_sync": res["plain_sync"] / ms_grouped,
            "speedup_vs_plain_chained": res["plain_chained"] / ms_grouped,
            "speedup_vs_tuned_sync": res["tuned_sync"] / ms_grouped,
            "tflops_grouped": flops / (ms_grouped * 1e-3) / 1e12, "gflop": flops / 1e9, "gbytes": bytes_ / 1e9,
            "tiles": total_tiles, "swapped_problems": int(sum(swapped)),
            "roofline_ms": t_overlap, "frac_of_roofline": t_overlap / ms_grouped,
            "roofline_peaks": f"{peaks['src']}: bf16 burst {peaks['bf16_tflops']} TFLOP/s, HBM {peaks['hbm_gbs']} GB/s",
            "roofline_ms_sustained": t_overlap_sust, "frac_of_roofline_sustained": t_overlap_sust / ms_grouped,
            "roofline_ms_per_problem_sum": t_sum, "frac_of_per_problem_sum": t_sum / ms_grouped,
            "note": "roofline = max(sum flops / bf16 peak, sum bytes / HBM peak) over the group (the launch overlaps "
                    "HBM-bound swap-AB tiles with tensor-bound tiles); _sustained uses the sustained bf16 peak; "
                    "per_problem_sum = sum over problems of max(flops / bf16 peak, bytes / HBM peak); "
                    "plain = one tp_gemm per problem on (128|256) x 256 tiles, group_m 8; tuned = one tp_gemm per "
                    "problem on its autotuned config; _sync = each call synchronised"}


def proposer_row(tp, ctx, train_n: int, test_n: int, epochs: int, log=None) -> dict:
    """The learned-proposer experiment: exhaustive tables of `train_n` shapes
    (BF16 and FP8, x 72 single-pass configs: ~20k autotuner measurements at
    278 shapes) for training on the GPU, `test_n` held-out shapes tuned
    exhaustively as the reference, proposals made by tp_propose. Regret is
    reported twice: against the exhaustive search's one timing per config, and with the
    proposal, the exhaustive pick and the fixed default re-timed (median of 3
    independent timings each) so that the reference is not the maximum of
    noisy samples."""
    import numpy as np

    from paper_2606_15991_gb300 import proposer

    train_shapes = proposer.sample_shapes(train_n, seed=1)
    test_shapes = proposer.sample_shapes(test_n, seed=2)
    t0 = time.perf_counter()
    X, T, V, TF = proposer.collect(ctx, train_shapes, log=log)
    t_collect = time.perf_counter() - t0
    t0 = time.perf_counter()
    mlp, hist = proposer.train(ctx, X, T, V, epochs=epochs, batch=64, lr=3e-3, log=log)
    t_train = time.perf_counter() - t0
    t0 = time.perf_counter()
    Xt, Tt, Vt, TFt = proposer.collect(ctx, test_shapes, log=log)
    t_exh = (time.perf_counter() - t0) / len(test_shapes)
    dflt = proposer.default_config(T, V)
    t0 = time.perf_counter()
    prop = proposer.propose_indices(ctx, mlp, test_shapes)
    t_prop = (time.perf_counter() - t0) / len(test_shapes)
    r = proposer.evaluate(mlp, Xt, TFt, dflt, prop=prop)
    t0 = time.perf_counter()
    rt = proposer.retimed_regret(ctx, test_shapes, TFt, prop, dflt, repeats=3)
    t_retime = time.perf_counter() - t0
    big = np.array([m * n * k >= 2 ** 33 for m, n, k, _ in test_shapes])
    reg = 1 - TFt[np.arange(len(TFt)), prop] / TFt.max(1)
    reg_d = 1 - TFt[:, dflt] / TFt.max(1)
    space = tp.tp_autotune_space("bf16")
    tp.tp_mlp_destroy(mlp)
    return {
        "space": "single-pass configs (bit-identical C; split-K excluded)", "configs": int(T.shape[1]),
        "train_shapes": len(train_shapes), "train_measurements": int(V.sum()), "test_shapes": len(test_shapes),
        "exhaustive_single_timing": r, "retimed_median_of_3": rt,
        "default_config": {n: getattr(space[dflt], n) for n in ("bm", "bn", "bk", "stages", "group_m", "split_k")},
        "large_shapes": int(big.sum()),
        "large_mean_regret": float(reg[big].mean()) if big.any() else None,
        "large_mean_regret_default": float(reg_d[big].mean()) if big.any() else None,
        "ms_exhaustive_per_shape": t_exh * 1e3, "ms_propose_per_shape": t_prop * 1e3,
        "tuning_time_saved_x": t_exh / t_prop, "loss_first_last": [hist[0], hist[-1]],
        "s_collect_train": t_collect, "s_train": t_train, "s_retime": t_retime}


def run_proposer(args):
    """The learned-proposer experiment alone; prints one JSON line."""
    from paper_2606_15991_gb300 import build as _build

    _build.build()
    import paper_2606_15991_gb300 as tp

    ctx = tp.tp_ctx_create(0)
    log = (lambda m: print(m, file=sys.stderr, flush=True))
    print(json.dumps({"case": "learned tile proposer",
                      **proposer_row(tp, ctx, args.train_shapes, args.test_shapes, args.epochs, log)}))


def run_exec_modes(args):
    """§5.2 execution-mode scaling: microseconds per op of an N-launch chain of
    y = x * g over a 2048-element BF16 tile, N = 1..1000, in the sync, chained,
    async and graph modes (host wall time; graph_device = CUDA-event time of
    the replayed graph). Prints one JSON line."""
    import torch

    from paper_2606_15991_gb300 import build as _build

    _build.build()
    import paper_2606_15991_gb300 as tp
    from paper_2606_15991_gb300 import experiments

    ctx = tp.tp_ctx_create(0)
    r = experiments.exec_mode_scaling(ctx, reps=args.reps)
    r["case"] = "execution-mode scaling"
    r["paper_rtx5090_us_per_op_at_1000"] = {"sync": 7.3, "chained": 3.4, "async": 3.4, "graph": 0.8}
    print(json.dumps(r))


def run_gemm_sweep(args):
    """§5.1 safety-overhead sweep: BF16 GEMM M = N = K = 1024..32768, safe
    (mapped partition) vs device-checked vs unchecked raw pointer vs plain
    partition, cuBLAS for context. Prints one JSON line."""
    import torch

    from paper_2606_15991_gb300 import build as _build

    _build.build()
    import paper_2606_15991_gb300 as tp
    from paper_2606_15991_gb300 import experiments

    ctx = tp.tp_ctx_create(0)
    peaks = _peaks()
    sizes = tuple(int(x) for x in args.sizes.split(","))
    log = (lambda m: print(m, file=sys.stderr, flush=True))
    rows = experiments.gemm_size_sweep(ctx, sizes, log=log)
    for r in rows:
        r["frac_of_measured_bf16"] = {k: v / peaks["bf16_tflops"] for k, v in r["tflops"].items()}
    print(json.dumps({"case": "gemm size sweep", "dtype": "bf16", "peak_bf16_tflops": peaks["bf16_tflops"],
                      "peak_src": peaks["src"], "rows": rows,
                      "paper_b200_8192": {"rust_pflops": 2.07, "vs_cublas": 0.964}}))


def run_bimodal(args):
    """Appendix B's bimodal work distribution: 2000 BF16 GEMMs (80% 512^3
    interleaved with 20% 2048^3) drained serially, by S threads, by one host
    thread over S streams, and as one grouped persistent launch; WU/ms (one
    work unit = one GEMM). Prints one JSON line."""
    import torch

    from paper_2606_15991_gb300 import build as _build

    _build.build()
    import paper_2606_15991_gb300 as tp
    from paper_2606_15991_gb300 import experiments

    ctx = tp.tp_ctx_create(0)
    log = (lambda m: print(m, file=sys.stderr, flush=True))
    r = experiments.bimodal_queue(ctx, reps=args.reps if args.reps != 30 else 3, log=log)
    r["case"] = "bimodal GEMM queue"
    r["paper_b200_wu_per_ms"] = {"serial": 37, "plateau_S8": 77}
    print(json.dumps(r))


def run_kernel(args):
    """One kernel on a (small) case, warm-up plus a few launches: the target of
    ncu captures. Prints a one-line JSON summary."""
    import torch

    from paper_2606_15991_gb300 import build as _build

    _build.build()
    import paper_2606_15991_gb300 as tp
    import synth

    ctx = tp.tp_ctx_create(0)
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev)
    g.manual_seed(1)
    k, n = args.kernel, args.size
    out = {"case": "kernel", "kernel": k}
    if k.startswith("map"):
        dt = torch.float32 if k.endswith("f32") else torch.bfloat16
        x = torch.randn(args.elements, device=dev, generator=g).to(dt)
        y = torch.randn(args.elements, device=dev, generator=g).to(dt)
        z = torch.empty_like(x)
        p = tp.tp_partition_create(ctx, z, (TILE,))
        fn = (lambda: tp.tp_map_axpy(ctx, p, ALPHA, x, y)) if "axpy" in k else (lambda: tp.tp_map_gelu_mul(ctx, p, x, y))
        out["elements"] = args.elements
    elif k in ("gemm_bf16", "gemm_fp8"):
        a = torch.randn(n, n, device=dev, generator=g).to(torch.bfloat16)
        bt = torch.randn(n, n, device=dev, generator=g).to(torch.bfloat16)
        c = torch.empty(n, n, device=dev, dtype=torch.bfloat16)
        p = tp.tp_partition_create(ctx, c, (256, 256))
        tp.tp_partition_map(p, tp.MAP_STRIDED, min(ctx.sm_count // 2, tp.tp_partition_query(p)["num_tiles"]))
        # the benchmark rows' configs: stages of 2 K blocks; raster bands of 8 (bf16) / 16 (fp8)
        cfg = tp.gemm_config(bm=256, bn=256, group_m=8 if k == "gemm_bf16" else 16, bk=128 if k == "gemm_bf16" else 256)
        if k == "gemm_bf16":
            fn = lambda: tp.tp_gemm(ctx, p, a, bt.t(), cfg)
        else:
            amax, scale = torch.zeros(2, device=dev), torch.zeros(2, device=dev)
            qa = torch.empty(n, n, device=dev, dtype=torch.float8_e4m3fn)
            qb = torch.empty(n, n, device=dev, dtype=torch.float8_e4m3fn)
            for src, q, i in ((a, qa, 0), (bt, qb, 1)):
                pq = tp.tp_partition_create(ctx, q, (16, n))
                tp.tp_amax(ctx, src, amax[i:i + 1])
                tp.tp_quantize_fp8(ctx, pq, src, amax[i:i + 1], scale[i:i + 1])
                tp.tp_partition_destroy(pq)
            fn = lambda: tp.tp_gemm_fp8(ctx, p, qa, qb.t(), scale[0:1], scale[1:2], cfg)
        out["size"] = n
    elif k == "gemm_f32":
        # the 512^3 FP32 configuration as the benchmark row runs it: 64 tile
        # programs, each a cluster of 2 CTAs splitting K
        a = torch.from_numpy(synth.uniform(512 * 512, seed=0)).reshape(512, 512).to(dev)
        b = torch.from_numpy(synth.uniform(512 * 512, seed=1)).reshape(512, 512).to(dev)
        c = torch.empty(512, 512, device=dev)
        p = tp.tp_partition_create(ctx, c, (64, 64))
        cfg = tp.gemm_config(bk=32, split_k=2)
        fn = lambda: tp.tp_gemm(ctx, p, a, b, cfg)
        out["size"] = 512
    elif k == "gemm_bf16_split":
        # few tiles, long K: M = 128, N = 256 * (size / 1024), K = 4096 as
        # split-K programs of 4 CTAs on 128 x 128 tiles
        nn = 256 * max(1, n // 1024)
        a = torch.randn(128, 4096, device=dev, generator=g).to(torch.bfloat16)
        bt = torch.randn(nn, 4096, device=dev, generator=g).to(torch.bfloat16)
        c = torch.empty(128, nn, device=dev, dtype=torch.bfloat16)
        p = tp.tp_partition_create(ctx, c, (128, 128))
        cfg = tp.gemm_config(bm=128, bn=128, split_k=4)
        fn = lambda: tp.tp_gemm(ctx, p, a, bt.t(), cfg)
        out["shape"] = [128, nn, 4096]
    elif k == "grouped":
        shapes = synth.grouped_problems(64, seed=0)[:args.group]
        probs = []
        for i, (m, nn, kk) in enumerate(shapes):
            g.manual_seed(1000 + i)
            probs.append((torch.randn(m, kk, device=dev, generator=g).to(torch.bfloat16),
                          torch.randn(nn, kk, device=dev, generator=g).to(torch.bfloat16).t(),
                          torch.empty(m, nn, device=dev, dtype=torch.bfloat16)))
        plan = tp.tp_grouped_plan_create(ctx, probs)
        fn = lambda: tp.tp_grouped_gemm(ctx, plan)
        out["problems"] = len(shapes)
    elif k == "decode":
        d, nq, ni = 5120, 10240, 25600
        lay = [tuple((torch.randn(r, c_, device=dev, generator=g) * 0.02).to(torch.bfloat16)
                     for r, c_ in ((nq, d), (2 * ni, d), (d, ni)))]
        h = torch.randn(d, device=dev, generator=g)
        ch = tp.DecodeChain(ctx, h, lay)
        fn = lambda: ch.record_fused()
    else:
        raise SystemExit(f"unknown kernel {k}")
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    out["ms_per_call_incl_sync"] = e0.elapsed_time(e1) / max(1, args.steps)
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-rows", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-proposer", action="store_true")
    ap.add_argument("--skip-experiments", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--case", default="maps", choices=["maps", "proposer", "kernel", "exec_modes", "gemm_sweep", "bimodal"],
                    help="maps: the benchmark step (default); proposer: the learned-proposer experiment; "
                         "kernel: one kernel on a small case (profiling target); "
                         "exec_modes: execution-mode scaling; gemm_sweep: GEMM size sweep; "
                         "bimodal: bimodal GEMM queue")
    ap.add_argument("--kernel", default="map_axpy_f32",
                    help="map_axpy_f32|map_axpy_bf16|map_gelu_f32|map_gelu_bf16|gemm_f32|gemm_bf16|gemm_bf16_split|"
                         "gemm_fp8|grouped|decode")
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--elements", type=int, default=1 << 26)
    ap.add_argument("--group", type=int, default=8)
    ap.add_argument("--train-shapes", type=int, default=278)
    ap.add_argument("--test-shapes", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=600)
    ap.add_argument("--reps", type=int, default=30)
    ap.add_argument("--sizes", default="1024,2048,4096,8192,16384,32768")
    args = ap.parse_args()
    if args.case == "proposer":
        run_proposer(args)
    elif args.case == "kernel":
        run_kernel(args)
    elif args.case == "exec_modes":
        run_exec_modes(args)
    elif args.case == "gemm_sweep":
        run_gemm_sweep(args)
    elif args.case == "bimodal":
        run_bimodal(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
