"""Partitioned tile-program kernels for GB300 (sm_103a) behind a C ABI.

Python binding of libtp.so with the same names as the C entry points
(include/tp.h). It marshals torch tensors into tp_tensor views and passes
torch's CUDA stream; all computation runs in the library's CUDA kernels.
There is no fallback: if libtp.so is missing or no GPU is present, the calls
raise.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import (ASYNC, CAPTURE, MAP_IDENTITY, MAP_QUEUE, MAP_STRIDED, SYNC, TPError, call,
                   tp_exec, tp_gemm_config, tp_partition_info, tp_tensor)

__all__ = [
    "TPError", "SYNC", "ASYNC", "CAPTURE", "MAP_IDENTITY", "MAP_STRIDED", "MAP_QUEUE",
    "tensor_desc", "make_exec", "gemm_config", "TUNE_SPLIT_K", "TUNE_SWAP_AB",
    "tp_version", "tp_ctx_create", "tp_ctx_destroy", "tp_ctx_info", "tp_tensor_init", "tp_tensor_view",
    "tp_partition_create", "tp_partition_map", "tp_partition_query", "tp_partition_destroy",
    "tp_event_create", "tp_event_query", "tp_event_wait", "tp_event_destroy",
    "tp_graph_begin", "tp_graph_end", "tp_graph_replay", "tp_graph_kernel_count", "tp_graph_destroy",
    "tp_map_axpy", "tp_map_gelu_mul", "tp_map_scale", "tp_map_add_accum", "tp_gemm",
    "tp_amax", "tp_quantize_fp8", "tp_gemm_fp8",
    "tp_grouped_plan_create", "tp_grouped_plan_info", "tp_grouped_plan_destroy", "tp_grouped_gemm",
    "tp_rmsnorm", "tp_gemv", "tp_silu_mul", "tp_residual_add", "tp_decode_norm_qkv_gu",
    "tp_decode_down_residual", "DecodeChain", "tp_permute_heads", "tp_permute_heads_unchecked",
    "tp_gemm_unchecked", "tp_diag_bounded_wait", "tp_gemm_resident_programs",
    "tp_autotune_space", "tp_autotune", "tp_autotune_time", "tp_autotune_lookup", "tp_autotune_save", "tp_autotune_load",
    "tp_mlp_create", "tp_mlp_destroy", "tp_mlp_num_params", "tp_mlp_get_params", "tp_mlp_set_params",
    "tp_mlp_forward", "tp_mlp_loss_grad", "tp_mlp_train_step", "tp_mlp_save", "tp_mlp_load",
    "tp_mlp_features", "tp_mlp_targets", "tp_propose",
]

_DTYPES = {
    torch.float32: _lib.F32,
    torch.bfloat16: _lib.BF16,
    torch.float8_e4m3fn: _lib.F8E4M3,
    torch.float64: _lib.F64,
    torch.int32: _lib.I32,
    torch.uint8: _lib.U8,
}
if hasattr(torch, "uint32"):
    _DTYPES[torch.uint32] = _lib.U32


def _i64(vals):
    arr = (ctypes.c_int64 * max(1, len(vals)))(*[int(v) for v in vals])
    return arr


def tensor_desc(t) -> tp_tensor:
    """tp_tensor view of a torch tensor (or a tp_tensor passed through)."""
    if isinstance(t, tp_tensor):
        return t
    if t.dtype not in _DTYPES:
        raise TypeError(f"unsupported dtype {t.dtype}")
    d = tp_tensor()
    call("tp_tensor_init", ctypes.byref(d), ctypes.c_void_p(t.data_ptr()), _DTYPES[t.dtype], t.dim(),
         _i64(t.shape), _i64(t.stride()))
    return d


def tp_tensor_init(t) -> tp_tensor:
    return tensor_desc(t)


def tp_tensor_view(base: tp_tensor, offset: int, shape, strides=None) -> tp_tensor:
    out = tp_tensor()
    call("tp_tensor_view", ctypes.byref(base), int(offset), len(shape), _i64(shape),
         _i64(strides) if strides is not None else None, ctypes.byref(out))
    return out


def tp_version():
    a, b = ctypes.c_int32(), ctypes.c_int32()
    call("tp_version", ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


class Context:
    def __init__(self, handle: int):
        self.handle = ctypes.c_void_p(handle)
        sm, ma, mi = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        call("tp_ctx_info", self.handle, ctypes.byref(sm), ctypes.byref(ma), ctypes.byref(mi))
        self.sm_count, self.cc = sm.value, (ma.value, mi.value)

    @property
    def _as_parameter_(self):
        return self.handle


def tp_ctx_create(device: int = 0) -> Context:
    h = ctypes.c_void_p()
    call("tp_ctx_create", int(device), ctypes.byref(h))
    return Context(h.value)


def tp_ctx_destroy(ctx: Context) -> None:
    if ctx.handle:
        call("tp_ctx_destroy", ctx.handle)
        ctx.handle = ctypes.c_void_p()


def tp_ctx_info(ctx: Context):
    return ctx.sm_count, ctx.cc


class Partition:
    """Handle of a partitioned mutable output; keeps the tensor alive."""

    def __init__(self, handle, tensor, ctx):
        self.handle = ctypes.c_void_p(handle)
        self.tensor = tensor
        self.ctx = ctx

    @property
    def _as_parameter_(self):
        return self.handle


def tp_partition_create(ctx, out, tile) -> Partition:
    d = tensor_desc(out)
    h = ctypes.c_void_p()
    call("tp_partition_create", ctx.handle if ctx is not None else None, ctypes.byref(d), _i64(tile),
         ctypes.byref(h))
    return Partition(h.value, out, ctx)


def tp_partition_map(p: Partition, kind: int, num_programs: int = 0) -> None:
    call("tp_partition_map", p.handle, int(kind), int(num_programs))


def tp_partition_query(p: Partition) -> dict:
    info = tp_partition_info()
    call("tp_partition_query", p.handle, ctypes.byref(info))
    r = info.rank
    return {"rank": r, "map_kind": info.map_kind, "shape": tuple(info.shape[:r]), "tile": tuple(info.tile[:r]),
            "grid": tuple(info.grid[:r]), "num_tiles": info.num_tiles, "num_programs": info.num_programs,
            "busy": bool(info.busy)}


def tp_partition_destroy(p: Partition) -> None:
    if p.handle:
        call("tp_partition_destroy", p.handle)
        p.handle = ctypes.c_void_p()


class Event:
    def __init__(self, handle):
        self.handle = ctypes.c_void_p(handle)


def tp_event_create(ctx) -> Event:
    h = ctypes.c_void_p()
    call("tp_event_create", ctx.handle, ctypes.byref(h))
    return Event(h.value)


def tp_event_query(ev: Event) -> bool:
    d = ctypes.c_int32()
    call("tp_event_query", ev.handle, ctypes.byref(d))
    return bool(d.value)


def tp_event_wait(ev: Event) -> None:
    call("tp_event_wait", ev.handle)


def tp_event_destroy(ev: Event) -> None:
    if ev.handle:
        call("tp_event_destroy", ev.handle)
        ev.handle = ctypes.c_void_p()


def _stream_handle(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Graph:
    def __init__(self, handle, stream):
        self.handle = ctypes.c_void_p(handle)
        self.stream = stream


def tp_graph_begin(ctx, stream) -> Graph:
    h = ctypes.c_void_p()
    call("tp_graph_begin", ctx.handle, ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(h))
    return Graph(h.value, stream)


def tp_graph_end(g: Graph) -> None:
    call("tp_graph_end", g.handle)


def tp_graph_replay(g: Graph, ex: tp_exec | None = None) -> None:
    call("tp_graph_replay", g.handle, ctypes.byref(ex if ex is not None else make_exec(stream=g.stream)))


def tp_graph_kernel_count(g: Graph) -> int:
    n = ctypes.c_int64()
    call("tp_graph_kernel_count", g.handle, ctypes.byref(n))
    return n.value


def tp_graph_destroy(g: Graph) -> None:
    if g.handle:
        call("tp_graph_destroy", g.handle)
        g.handle = ctypes.c_void_p()


def make_exec(mode: int = SYNC, stream=None, event: Event | None = None, write_counts=None,
              write_owner=None, checked: bool = False, inject_timeout: bool = False,
              static_weights: bool = False) -> tp_exec:
    """tp_exec for `mode` on `stream` (torch.cuda.Stream, raw handle, or None =
    torch's current stream). write_counts / write_owner: optional uint32 /
    int32 device tensors with one entry per output element. checked: the
    device-checked launch (TP_EXEC_CHECKED). inject_timeout: the tensor-core
    GEMM's failure-path test hook (TP_EXEC_INJECT_TIMEOUT). static_weights:
    the decode products may start reading their weights before the work
    queued ahead of them on the stream finishes (TP_EXEC_STATIC_WEIGHTS)."""
    ex = tp_exec()
    ex.mode = mode
    ex.flags = ((_lib.EXEC_CHECKED if checked else 0) | (_lib.EXEC_INJECT_TIMEOUT if inject_timeout else 0) |
                (_lib.EXEC_STATIC_WEIGHTS if static_weights else 0))
    ex.stream = _stream_handle(stream)
    ex.event = event.handle.value if event is not None else None
    ex.write_counts = write_counts.data_ptr() if write_counts is not None else None
    ex.write_owner = write_owner.data_ptr() if write_owner is not None else None
    return ex


def gemm_config(bm=0, bn=0, bk=0, stages=0, group_m=0, num_programs=0, swap_ab=0, split_k=0, cut_limit=0):
    return tp_gemm_config(bm, bn, bk, stages, group_m, num_programs, swap_ab, split_k, cut_limit)


def _ex(ex):
    return ctypes.byref(ex if ex is not None else make_exec())


def tp_map_axpy(ctx, z: Partition, alpha: float, x, y, ex: tp_exec | None = None) -> None:
    """z = alpha * x + y (element-wise; z is a partition)."""
    dx, dy = tensor_desc(x), tensor_desc(y)
    call("tp_map_axpy", ctx.handle, z.handle, float(alpha), ctypes.byref(dx), ctypes.byref(dy), _ex(ex))


def tp_map_gelu_mul(ctx, y: Partition, x, w, ex: tp_exec | None = None) -> None:
    """y = gelu_tanh(x) * w (element-wise)."""
    dx, dw = tensor_desc(x), tensor_desc(w)
    call("tp_map_gelu_mul", ctx.handle, y.handle, ctypes.byref(dx), ctypes.byref(dw), _ex(ex))


def tp_map_scale(ctx, y: Partition, x, g, ex: tp_exec | None = None) -> None:
    """y = x * g (element-wise)."""
    dx, dg = tensor_desc(x), tensor_desc(g)
    call("tp_map_scale", ctx.handle, y.handle, ctypes.byref(dx), ctypes.byref(dg), _ex(ex))


def tp_map_add_accum(ctx, c: Partition, a, b, ex: tp_exec | None = None) -> None:
    """c <- c + a + b (element-wise read-modify-write of the partition)."""
    da, db = tensor_desc(a), tensor_desc(b)
    call("tp_map_add_accum", ctx.handle, c.handle, ctypes.byref(da), ctypes.byref(db), _ex(ex))


def tp_gemm(ctx, c: Partition, a, b, cfg: tp_gemm_config | None = None, ex: tp_exec | None = None) -> None:
    """C = A . B into the partition c (see include/tp.h for layouts)."""
    da, db = tensor_desc(a), tensor_desc(b)
    call("tp_gemm", ctx.handle, c.handle, ctypes.byref(da), ctypes.byref(db),
         ctypes.byref(cfg) if cfg is not None else None, _ex(ex))


def tp_gemm_resident_programs(ctx, cfg: tp_gemm_config) -> int:
    """Programs (CTA pairs for 256-row tiles, else CTAs) resident at once."""
    n = ctypes.c_int32()
    call("tp_gemm_resident_programs", ctx.handle, ctypes.byref(cfg), ctypes.byref(n))
    return n.value


def tp_gemm_unchecked(ctx, c, a, b, cfg: tp_gemm_config, stream=None) -> None:
    """C = A . B into the raw contiguous BF16 tensor c (no partition; the
    unchecked baseline). cfg.num_programs = 0 launches one program per tile."""
    da, db = tensor_desc(a), tensor_desc(b)
    call("tp_gemm_unchecked", ctx.handle, c.data_ptr(), ctypes.byref(da), ctypes.byref(db), ctypes.byref(cfg),
         _stream_handle(stream))


def tp_diag_bounded_wait(ctx, limit_ns: int, arrive: bool, ex: tp_exec | None = None) -> None:
    """One bounded mbarrier wait on the GPU; never signalled (arrive=False),
    it gives up after limit_ns and the call raises TPError(TP_ERR_TIMEOUT)."""
    call("tp_diag_bounded_wait", ctx.handle, int(limit_ns), int(bool(arrive)), _ex(ex))


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr())


def tp_amax(ctx, x, amax, ex: tp_exec | None = None) -> None:
    """amax[0] = max |x| (amax: a float32 device tensor with one element)."""
    dx = tensor_desc(x)
    call("tp_amax", ctx.handle, ctypes.byref(dx), _dptr(amax), _ex(ex))


def tp_quantize_fp8(ctx, q: Partition, x, amax, scale, ex: tp_exec | None = None) -> None:
    """q = E4M3(satfinite(RN(x * 448 / amax))); scale[0] receives 448 / amax."""
    dx = tensor_desc(x)
    call("tp_quantize_fp8", ctx.handle, q.handle, ctypes.byref(dx), _dptr(amax), _dptr(scale), _ex(ex))


def tp_gemm_fp8(ctx, c: Partition, qa, qb, scale_a, scale_b, cfg: tp_gemm_config | None = None,
                ex: tp_exec | None = None) -> None:
    """C (bf16) = (qA . qB) / (scale_a * scale_b) from E4M3 operands."""
    da, db = tensor_desc(qa), tensor_desc(qb)
    call("tp_gemm_fp8", ctx.handle, c.handle, ctypes.byref(da), ctypes.byref(db), _dptr(scale_a),
         _dptr(scale_b), ctypes.byref(cfg) if cfg is not None else None, _ex(ex))


class GroupedPlan:
    """Handle of a planned group; keeps the problem tensors alive."""

    def __init__(self, handle, tensors, n):
        self.handle = ctypes.c_void_p(handle)
        self.tensors = tensors
        self.n = n


def tp_grouped_plan_create(ctx, problems, swap_max_m: int = -1, cta_pair: bool = True) -> GroupedPlan:
    """problems: [(A [M,K], B [K,N] K-major view, C [M,N])] of bf16 CUDA tensors."""
    arr = (_lib.tp_gemm_problem * len(problems))()
    keep = []
    for i, (a, b, c) in enumerate(problems):
        arr[i].a, arr[i].b, arr[i].c = tensor_desc(a), tensor_desc(b), tensor_desc(c)
        keep += [a, b, c]
    h = ctypes.c_void_p()
    call("tp_grouped_plan_create", ctx.handle, arr, len(problems), int(swap_max_m), int(bool(cta_pair)),
         ctypes.byref(h))
    return GroupedPlan(h.value, keep, len(problems))


def tp_grouped_plan_info(plan: GroupedPlan):
    total = ctypes.c_int64()
    sw = (ctypes.c_int32 * plan.n)()
    call("tp_grouped_plan_info", plan.handle, ctypes.byref(total), sw)
    return total.value, [bool(v) for v in sw]


def tp_grouped_plan_destroy(plan: GroupedPlan) -> None:
    if plan.handle:
        call("tp_grouped_plan_destroy", plan.handle)
        plan.handle = ctypes.c_void_p()


def tp_grouped_gemm(ctx, plan: GroupedPlan, num_programs: int = 0, ex: tp_exec | None = None) -> None:
    """All problems of the plan in one persistent launch over a device tile queue."""
    call("tp_grouped_gemm", ctx.handle, plan.handle, int(num_programs), _ex(ex))


def _opt(t):
    return ctypes.byref(tensor_desc(t)) if t is not None else None


def tp_rmsnorm(ctx, n_out: Partition, h, gamma=None, eps: float = 1e-6, ex: tp_exec | None = None) -> None:
    call("tp_rmsnorm", ctx.handle, n_out.handle, ctypes.byref(tensor_desc(h)), _opt(gamma), float(eps), _ex(ex))


def tp_gemv(ctx, y: Partition, w, x, ex: tp_exec | None = None) -> None:
    call("tp_gemv", ctx.handle, y.handle, ctypes.byref(tensor_desc(w)), ctypes.byref(tensor_desc(x)), _ex(ex))


def tp_silu_mul(ctx, a_out: Partition, gu, ex: tp_exec | None = None) -> None:
    call("tp_silu_mul", ctx.handle, a_out.handle, ctypes.byref(tensor_desc(gu)), _ex(ex))


def tp_residual_add(ctx, h: Partition, d, ex: tp_exec | None = None) -> None:
    call("tp_residual_add", ctx.handle, h.handle, ctypes.byref(tensor_desc(d)), _ex(ex))


def tp_decode_norm_qkv_gu(ctx, qkv: Partition, a_out: Partition, h, gamma, w_qkv, w_gu, eps: float = 1e-6,
                          ex: tp_exec | None = None) -> None:
    call("tp_decode_norm_qkv_gu", ctx.handle, qkv.handle, a_out.handle, ctypes.byref(tensor_desc(h)),
         _opt(gamma), ctypes.byref(tensor_desc(w_qkv)), ctypes.byref(tensor_desc(w_gu)), float(eps), _ex(ex))


def tp_decode_down_residual(ctx, h: Partition, w_down, a_in, ex: tp_exec | None = None) -> None:
    call("tp_decode_down_residual", ctx.handle, h.handle, ctypes.byref(tensor_desc(w_down)),
         ctypes.byref(tensor_desc(a_in)), _ex(ex))


def tp_permute_heads(ctx, dst: Partition, src, H: int, ex: tp_exec | None = None) -> None:
    """Partitioned head permutation (§3.5): dst tile (b, m, h) = src tile
    (b, h, m); dst is a partition of the (B*H, M, D) output with (1, BM, D) tiles."""
    call("tp_permute_heads", ctx.handle, dst.handle, ctypes.byref(tensor_desc(src)), int(H), _ex(ex))


def tp_permute_heads_unchecked(ctx, dst, src, BM: int, swap_bug: bool, ex: tp_exec | None = None) -> None:
    """Raw-pointer head permutation with Listing 5's grid; swap_bug stores at
    the swapped (racing) index. dst, src: contiguous F32 (B, H, M, D) tensors."""
    B, H, M, D = src.shape
    call("tp_permute_heads_unchecked", ctx.handle, dst.data_ptr(), src.data_ptr(), B, H, M, D, int(BM),
         int(bool(swap_bug)), _ex(ex))


class DecodeChain:
    """Buffers and partitions for a decode-shaped chain of layers
    [(W_qkv, W_gu, W_down), ...] acting on the residual stream h (fp32 [d])."""

    def __init__(self, ctx, h, layers, gamma=None, eps: float = 1e-6):
        self.ctx, self.h, self.layers, self.gamma, self.eps = ctx, h, layers, gamma, eps
        d = h.shape[0]
        nq = layers[0][0].shape[0]
        ni = layers[0][1].shape[0] // 2
        dev = h.device
        self.n = torch.empty(d, device=dev)
        self.qkv = torch.empty(nq, device=dev)
        self.gu = torch.empty(2 * ni, device=dev)
        self.a = torch.empty(ni, device=dev)
        self.dd = torch.empty(d, device=dev)
        self.p = {k: tp_partition_create(ctx, t, (t.shape[0],)) for k, t in
                  (("h", h), ("n", self.n), ("qkv", self.qkv), ("gu", self.gu), ("a", self.a), ("dd", self.dd))}

    def record_fused(self, ex: tp_exec | None = None) -> None:
        """Two launches per layer (three with the down projection's K slices):
        norm+QKV+gate/up+SiLU*mul, down+residual. The chain's weights stay
        fixed while it runs, so the launches carry TP_EXEC_STATIC_WEIGHTS."""
        ex = tp_exec.from_buffer_copy(ex) if ex is not None else make_exec()
        ex.flags |= _lib.EXEC_STATIC_WEIGHTS
        for w_qkv, w_gu, w_down in self.layers:
            tp_decode_norm_qkv_gu(self.ctx, self.p["qkv"], self.p["a"], self.h, self.gamma, w_qkv, w_gu,
                                  self.eps, ex)
            tp_decode_down_residual(self.ctx, self.p["h"], w_down, self.a, ex)

    def record_unfused(self, ex: tp_exec | None = None) -> None:
        """Six launches per layer, one per step of the chain."""
        for w_qkv, w_gu, w_down in self.layers:
            tp_rmsnorm(self.ctx, self.p["n"], self.h, self.gamma, self.eps, ex)
            tp_gemv(self.ctx, self.p["qkv"], w_qkv, self.n, ex)
            tp_gemv(self.ctx, self.p["gu"], w_gu, self.n, ex)
            tp_silu_mul(self.ctx, self.p["a"], self.gu, ex)
            tp_gemv(self.ctx, self.p["dd"], w_down, self.a, ex)
            tp_residual_add(self.ctx, self.p["h"], self.dd, ex)

    def close(self) -> None:
        for p in self.p.values():
            tp_partition_destroy(p)


_DT_CODE = {"bf16": _lib.BF16, "fp8": _lib.F8E4M3}


def _cfg_dict(c: tp_gemm_config) -> dict:
    return {n: getattr(c, n) for n, _ in tp_gemm_config._fields_}


TUNE_SPLIT_K = 1
TUNE_SWAP_AB = 2


def _tune_flags(split_k: bool, swap_ab: bool) -> int:
    return (TUNE_SPLIT_K if split_k else 0) | (TUNE_SWAP_AB if swap_ab else 0)


def tp_autotune_space(dtype: str = "bf16", split_k: bool = False, swap_ab: bool = False) -> list:
    """The autotuner's config space: the single-pass configs (index i =
    proposer output i), then, with swap_ab, the swap-AB configs, then, with
    split_k, the split-K configs."""
    fl = _tune_flags(split_k, swap_ab)
    n = ctypes.c_int32()
    call("tp_autotune_space", _DT_CODE[dtype], fl, None, 0, ctypes.byref(n))
    arr = (tp_gemm_config * n.value)()
    call("tp_autotune_space", _DT_CODE[dtype], fl, arr, n.value, ctypes.byref(n))
    return [arr[i] for i in range(n.value)]


def tp_autotune(ctx, M: int, N: int, K: int, dtype: str = "bf16", reps: int = 0, split_k: bool = False,
                swap_ab: bool = False):
    """Exhaustive search: returns (best config, [TFLOP/s per config], best TFLOP/s)."""
    cnt = len(tp_autotune_space(dtype, split_k, swap_ab))
    best = tp_gemm_config()
    table = (ctypes.c_float * cnt)()
    bt = ctypes.c_float()
    call("tp_autotune", ctx.handle, int(M), int(N), int(K), _DT_CODE[dtype], int(reps),
         _tune_flags(split_k, swap_ab), ctypes.byref(best), table, ctypes.byref(bt))
    return best, list(table), bt.value


def tp_autotune_time(ctx, M: int, N: int, K: int, dtype: str, cfg: tp_gemm_config, reps: int = 0,
                     repeats: int = 3) -> float:
    """Median TFLOP/s of `repeats` independent timings of one config."""
    out = ctypes.c_float()
    call("tp_autotune_time", ctx.handle, int(M), int(N), int(K), _DT_CODE[dtype], ctypes.byref(cfg), int(reps),
         int(repeats), ctypes.byref(out))
    return out.value


def tp_autotune_lookup(ctx, M: int, N: int, K: int, dtype: str = "bf16", split_k: bool = False,
                       swap_ab: bool = False):
    out = tp_gemm_config()
    found = ctypes.c_int32()
    call("tp_autotune_lookup", ctx.handle, int(M), int(N), int(K), _DT_CODE[dtype], _tune_flags(split_k, swap_ab),
         ctypes.byref(out), ctypes.byref(found))
    return out if found.value else None


def tp_autotune_save(ctx, path: str) -> None:
    call("tp_autotune_save", ctx.handle, path.encode())


def tp_autotune_load(ctx, path: str) -> None:
    call("tp_autotune_load", ctx.handle, path.encode())


class MLP:
    def __init__(self, handle, shape):
        self.handle = ctypes.c_void_p(handle)
        self.shape = shape


def tp_mlp_create(ctx, in_features: int, hidden: int, out: int, max_batch: int, init_params) -> MLP:
    """init_params: float32 numpy array of the flat parameter layout."""
    import numpy as np

    p = np.ascontiguousarray(init_params, dtype=np.float32)
    h = ctypes.c_void_p()
    call("tp_mlp_create", ctx.handle, in_features, hidden, out, max_batch, p.ctypes.data_as(ctypes.c_void_p),
         ctypes.byref(h))
    return MLP(h.value, (in_features, hidden, out))


def tp_mlp_destroy(m: MLP) -> None:
    if m.handle:
        call("tp_mlp_destroy", m.handle)
        m.handle = ctypes.c_void_p()


def tp_mlp_num_params(m: MLP) -> int:
    n = ctypes.c_int64()
    call("tp_mlp_num_params", m.handle, ctypes.byref(n))
    return n.value


def tp_mlp_get_params(m: MLP):
    import numpy as np

    out = np.empty(tp_mlp_num_params(m), dtype=np.float32)
    call("tp_mlp_get_params", m.handle, out.ctypes.data_as(ctypes.c_void_p))
    return out


def tp_mlp_set_params(m: MLP, params) -> None:
    import numpy as np

    p = np.ascontiguousarray(params, dtype=np.float32)
    call("tp_mlp_set_params", m.handle, p.ctypes.data_as(ctypes.c_void_p))


def tp_mlp_forward(m: MLP, X, Y, ex: tp_exec | None = None) -> None:
    """Y[batch, out] = MLP(X[batch, in]) (float32 CUDA tensors)."""
    call("tp_mlp_forward", m.handle, _dptr(X), X.shape[0], _dptr(Y), _ex(ex))


def tp_mlp_loss_grad(m: MLP, X, T, V, loss=None, grads=None, ex: tp_exec | None = None) -> None:
    call("tp_mlp_loss_grad", m.handle, _dptr(X), _dptr(T), _dptr(V), X.shape[0],
         _dptr(loss) if loss is not None else None, _dptr(grads) if grads is not None else None, _ex(ex))


def tp_mlp_train_step(m: MLP, X, T, V, lr: float, loss=None, ex: tp_exec | None = None) -> None:
    call("tp_mlp_train_step", m.handle, _dptr(X), _dptr(T), _dptr(V), X.shape[0], float(lr),
         _dptr(loss) if loss is not None else None, _ex(ex))


def tp_mlp_save(m: MLP, path: str) -> None:
    call("tp_mlp_save", m.handle, path.encode())


def tp_mlp_load(m: MLP, path: str) -> None:
    call("tp_mlp_load", m.handle, path.encode())


def tp_mlp_features(M: int, N: int, K: int, dtype: str = "bf16"):
    out = (ctypes.c_float * 5)()
    call("tp_mlp_features", int(M), int(N), int(K), _DT_CODE[dtype], out)
    return list(out)


def tp_mlp_targets(tflops):
    n = len(tflops)
    t = (ctypes.c_float * n)(*tflops)
    tgt, mask = (ctypes.c_float * n)(), (ctypes.c_float * n)()
    call("tp_mlp_targets", t, n, tgt, mask)
    return list(tgt), list(mask)


def tp_propose(ctx, m: MLP, M: int, N: int, K: int, dtype: str = "bf16", min_score: float = 0.0):
    """Returns (config, score, used_fallback)."""
    out = tp_gemm_config()
    score = ctypes.c_float()
    fb = ctypes.c_int32()
    call("tp_propose", ctx.handle, m.handle, int(M), int(N), int(K), _DT_CODE[dtype], float(min_score),
         ctypes.byref(out), ctypes.byref(score), ctypes.byref(fb))
    return out, score.value, bool(fb.value)
