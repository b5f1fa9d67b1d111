"""ctypes binding to libtp.so: structures and prototypes mirroring include/tp.h.

Argument marshalling only; every step of the computation runs in the library.
Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libtp.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "tp.h")

MAX_RANK = 8

# tp_status
OK, ERR_INVALID, ERR_RANK, ERR_ALIGN, ERR_ALIAS, ERR_BUSY, ERR_CAPTURE, ERR_UNSUPPORTED, ERR_CUDA, \
    ERR_TIMEOUT, ERR_SHAPE, ERR_RACE = range(12)
STATUS_NAMES = {0: "TP_OK", 1: "TP_ERR_INVALID", 2: "TP_ERR_RANK", 3: "TP_ERR_ALIGN", 4: "TP_ERR_ALIAS",
                5: "TP_ERR_BUSY", 6: "TP_ERR_CAPTURE", 7: "TP_ERR_UNSUPPORTED", 8: "TP_ERR_CUDA",
                9: "TP_ERR_TIMEOUT", 10: "TP_ERR_SHAPE", 11: "TP_ERR_RACE"}
# tp_exec.flags
EXEC_CHECKED = 1
EXEC_INJECT_TIMEOUT = 2
EXEC_STATIC_WEIGHTS = 4
# tp_dtype
F32, BF16, F8E4M3, F64, I32, U32, U8 = range(7)
# tp_map_kind
MAP_IDENTITY, MAP_STRIDED, MAP_QUEUE = range(3)
# tp_mode
SYNC, ASYNC, CAPTURE = range(3)


class tp_tensor(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("rank", ctypes.c_int32),
                ("shape", ctypes.c_int64 * MAX_RANK), ("strides", ctypes.c_int64 * MAX_RANK)]


class tp_exec(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("flags", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("event", ctypes.c_void_p), ("write_counts", ctypes.c_void_p),
                ("write_owner", ctypes.c_void_p)]


class tp_partition_info(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32), ("map_kind", ctypes.c_int32), ("shape", ctypes.c_int64 * 3),
                ("tile", ctypes.c_int64 * 3), ("grid", ctypes.c_int64 * 3), ("num_tiles", ctypes.c_int64),
                ("num_programs", ctypes.c_int64), ("busy", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class tp_gemm_config(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("bm", "bn", "bk", "stages", "group_m", "num_programs", "swap_ab", "split_k",
                 "cut_limit")]


class tp_gemm_problem(ctypes.Structure):
    _fields_ = [("a", tp_tensor), ("b", tp_tensor), ("c", tp_tensor)]


class TPError(RuntimeError):
    def __init__(self, status: int, detail: str, call: str):
        self.status = status
        self.detail = detail
        super().__init__(f"{call}: {STATUS_NAMES.get(status, status)}: {detail}")


_lib = None

_VP = ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_PI32 = ctypes.POINTER(ctypes.c_int32)
_PI64 = ctypes.POINTER(ctypes.c_int64)
_PT = ctypes.POINTER(tp_tensor)
_PE = ctypes.POINTER(tp_exec)

# name -> argtypes (all return tp_status unless listed in _RESTYPES)
_PROTOS = {
    "tp_error_string": [_I32],
    "tp_last_error_detail": [],
    "tp_version": [_PI32, _PI32],
    "tp_ctx_create": [_I32, _PP],
    "tp_ctx_destroy": [_VP],
    "tp_ctx_info": [_VP, _PI32, _PI32, _PI32],
    "tp_tensor_init": [_PT, _VP, _I32, _I32, _PI64, _PI64],
    "tp_tensor_view": [_PT, _I64, _I32, _PI64, _PI64, _PT],
    "tp_partition_create": [_VP, _PT, _PI64, _PP],
    "tp_partition_map": [_VP, _I32, _I64],
    "tp_partition_query": [_VP, ctypes.POINTER(tp_partition_info)],
    "tp_partition_destroy": [_VP],
    "tp_event_create": [_VP, _PP],
    "tp_event_query": [_VP, _PI32],
    "tp_event_wait": [_VP],
    "tp_event_destroy": [_VP],
    "tp_graph_begin": [_VP, _VP, _PP],
    "tp_graph_end": [_VP],
    "tp_graph_replay": [_VP, _PE],
    "tp_graph_kernel_count": [_VP, _PI64],
    "tp_graph_destroy": [_VP],
    "tp_map_axpy": [_VP, _VP, ctypes.c_float, _PT, _PT, _PE],
    "tp_map_gelu_mul": [_VP, _VP, _PT, _PT, _PE],
    "tp_map_scale": [_VP, _VP, _PT, _PT, _PE],
    "tp_map_add_accum": [_VP, _VP, _PT, _PT, _PE],
    "tp_gemm": [_VP, _VP, _PT, _PT, ctypes.POINTER(tp_gemm_config), _PE],
    "tp_amax": [_VP, _PT, _VP, _PE],
    "tp_quantize_fp8": [_VP, _VP, _PT, _VP, _VP, _PE],
    "tp_gemm_fp8": [_VP, _VP, _PT, _PT, _VP, _VP, ctypes.POINTER(tp_gemm_config), _PE],
    "tp_grouped_plan_create": [_VP, ctypes.POINTER(tp_gemm_problem), _I32, _I32, _I32, _PP],
    "tp_grouped_plan_info": [_VP, _PI64, _PI32],
    "tp_grouped_plan_destroy": [_VP],
    "tp_grouped_gemm": [_VP, _VP, _I32, _PE],
    "tp_rmsnorm": [_VP, _VP, _PT, _PT, ctypes.c_float, _PE],
    "tp_gemv": [_VP, _VP, _PT, _PT, _PE],
    "tp_silu_mul": [_VP, _VP, _PT, _PE],
    "tp_residual_add": [_VP, _VP, _PT, _PE],
    "tp_decode_norm_qkv_gu": [_VP, _VP, _VP, _PT, _PT, _PT, _PT, ctypes.c_float, _PE],
    "tp_decode_down_residual": [_VP, _VP, _PT, _PT, _PE],
    "tp_autotune_space": [_I32, _I32, ctypes.POINTER(tp_gemm_config), _I32, _PI32],
    "tp_autotune": [_VP, _I64, _I64, _I64, _I32, _I32, _I32, ctypes.POINTER(tp_gemm_config), _VP, _VP],
    "tp_autotune_time": [_VP, _I64, _I64, _I64, _I32, ctypes.POINTER(tp_gemm_config), _I32, _I32, _VP],
    "tp_autotune_lookup": [_VP, _I64, _I64, _I64, _I32, _I32, ctypes.POINTER(tp_gemm_config), _PI32],
    "tp_autotune_save": [_VP, ctypes.c_char_p],
    "tp_autotune_load": [_VP, ctypes.c_char_p],
    "tp_mlp_create": [_VP, _I32, _I32, _I32, _I32, _VP, _PP],
    "tp_mlp_destroy": [_VP],
    "tp_mlp_num_params": [_VP, _PI64],
    "tp_mlp_get_params": [_VP, _VP],
    "tp_mlp_set_params": [_VP, _VP],
    "tp_mlp_forward": [_VP, _VP, _I32, _VP, _PE],
    "tp_mlp_loss_grad": [_VP, _VP, _VP, _VP, _I32, _VP, _VP, _PE],
    "tp_mlp_train_step": [_VP, _VP, _VP, _VP, _I32, ctypes.c_float, _VP, _PE],
    "tp_mlp_save": [_VP, ctypes.c_char_p],
    "tp_mlp_load": [_VP, ctypes.c_char_p],
    "tp_mlp_features": [_I64, _I64, _I64, _I32, _VP],
    "tp_mlp_targets": [_VP, _I32, _VP, _VP],
    "tp_propose": [_VP, _VP, _I64, _I64, _I64, _I32, ctypes.c_float, ctypes.POINTER(tp_gemm_config), _VP, _PI32],
    "tp_map_axpy_queue_noalloc": [_VP, _VP, _VP, _I32, _I64, _I64, _I32, ctypes.c_float, _VP],
    "tp_diag_bounded_wait": [_VP, _I64, _I32, _PE],
    "tp_gemm_resident_programs": [_VP, ctypes.POINTER(tp_gemm_config), _PI32],
    "tp_gemm_unchecked": [_VP, _VP, _PT, _PT, ctypes.POINTER(tp_gemm_config), _VP],
    "tp_permute_heads": [_VP, _VP, _PT, _I64, _PE],
    "tp_permute_heads_unchecked": [_VP, _VP, _VP, _I64, _I64, _I64, _I64, _I64, _I32, _PE],
}
_RESTYPES = {"tp_error_string": ctypes.c_char_p, "tp_last_error_detail": ctypes.c_char_p}


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2606_15991_gb300.build.build() "
                               "(the CUDA library is required; there is no fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _PROTOS.items():
            if not hasattr(L, name):
                continue
            f = getattr(L, name)
            f.argtypes = args
            f.restype = _RESTYPES.get(name, ctypes.c_int32)
        _lib = L
    return _lib


def call(name: str, *args) -> None:
    """Call a tp_* entry point and raise TPError on a non-OK status."""
    L = lib()
    st = getattr(L, name)(*args)
    if st != OK:
        raise TPError(st, L.tp_last_error_detail().decode(), name)


def header_symbols() -> list[str]:
    """Every function name declared in include/tp.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:tp_status|const char\*)\s+(tp_\w+)\s*\(", text, re.M)))
