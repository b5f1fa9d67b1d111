"""Host-side tests of the C ABI: the library loads, exports every declared
symbol, and validates descriptors and partitions without touching a GPU."""
import ctypes

import numpy as np
import pytest

import paper_2606_15991_gb300 as tp
from oracle import partition as opart
from paper_2606_15991_gb300 import _lib


def _desc(shape, dtype=_lib.F32, ptr=0x10000, strides=None):
    d = _lib.tp_tensor()
    _lib.call("tp_tensor_init", ctypes.byref(d), ctypes.c_void_p(ptr), dtype, len(shape),
              tp._i64(shape), tp._i64(strides) if strides else None)
    return d


def _status(name, *args):
    return getattr(_lib.lib(), name)(*args)


def test_exports_every_declared_symbol(built_lib):
    syms = _lib.header_symbols()
    assert len(syms) >= 25
    missing = [s for s in syms if not hasattr(built_lib, s)]
    assert missing == []
    assert set(_lib._PROTOS) >= set(syms)


def test_error_strings_and_version(built_lib):
    for s in range(11):
        assert built_lib.tp_error_string(s)
    assert tp.tp_version() == (0, 2)


def test_tensor_init_validation(built_lib):
    d = _lib.tp_tensor()
    assert _status("tp_tensor_init", ctypes.byref(d), None, _lib.F32, 9, tp._i64([1] * 9), None) == _lib.ERR_RANK
    assert _status("tp_tensor_init", ctypes.byref(d), None, 99, 1, tp._i64([4]), None) == _lib.ERR_INVALID
    assert _status("tp_tensor_init", ctypes.byref(d), None, _lib.F32, 1, tp._i64([-1]), None) == _lib.ERR_INVALID
    d = _desc((3, 5))
    assert list(d.strides[:2]) == [5, 1]


def test_tensor_view_bounds(built_lib):
    base = _desc((100,), ptr=0x1000)
    v = tp.tp_tensor_view(base, 10, (20,))
    assert v.ptr == 0x1000 + 40 and v.shape[0] == 20
    with pytest.raises(tp.TPError) as e:
        tp.tp_tensor_view(base, 90, (20,))
    assert e.value.status == _lib.ERR_INVALID
    v2 = tp.tp_tensor_view(base, 0, (10, 10), (10, 1))
    assert v2.rank == 2


def _part(shape, tile, strides=None):
    d = _desc(shape, strides=strides)
    h = ctypes.c_void_p()
    st = _status("tp_partition_create", None, ctypes.byref(d), tp._i64(tile), ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("shape,tile", [((1024,), (128,)), ((10,), (4,)), ((5, 7, 3), (2, 3, 3)),
                                        ((2 ** 28,), (4096,)), ((512, 512), (64, 64)), ((0,), (4,))])
def test_partition_grid_matches_oracle(built_lib, shape, tile):
    st, h = _part(shape, tile)
    assert st == _lib.OK
    p = tp.Partition(h.value, None, None)
    q = tp.tp_partition_query(p)
    assert q["grid"] == opart.grid(shape, tile)
    assert q["num_tiles"] == opart.num_tiles(shape, tile)
    assert q["num_programs"] == q["num_tiles"] and q["map_kind"] == _lib.MAP_IDENTITY and not q["busy"]
    tp.tp_partition_destroy(p)


def test_partition_rejections(built_lib):
    assert _part((2, 2, 2, 2), (1, 1, 1, 1))[0] == _lib.ERR_RANK
    assert _part((8,), (0,))[0] == _lib.ERR_INVALID
    assert _part((4, 4), (2, 2), strides=(1, 4))[0] == _lib.ERR_UNSUPPORTED   # non-contiguous output


def test_mapped_partition_program_count(built_lib):
    st, h = _part((1000,), (64,))   # 16 tiles
    p = tp.Partition(h.value, None, None)
    for bad in (0, 17, -1):
        with pytest.raises(tp.TPError) as e:
            tp.tp_partition_map(p, _lib.MAP_STRIDED, bad)
        assert e.value.status == _lib.ERR_INVALID
    tp.tp_partition_map(p, _lib.MAP_STRIDED, 16)
    tp.tp_partition_map(p, _lib.MAP_QUEUE, 3)
    q = tp.tp_partition_query(p)
    assert q["num_programs"] == 3 and q["map_kind"] == _lib.MAP_QUEUE
    with pytest.raises(tp.TPError):
        tp.tp_partition_map(p, 7, 3)
    tp.tp_partition_map(p, _lib.MAP_IDENTITY)
    assert tp.tp_partition_query(p)["num_programs"] == 16
    tp.tp_partition_destroy(p)


def test_ops_reject_missing_context(built_lib):
    st, h = _part((64,), (64,))
    x = _desc((64,))
    ex = tp.make_exec(stream=0)
    assert _status("tp_map_axpy", None, h, ctypes.c_float(1.0), ctypes.byref(x), ctypes.byref(x),
                   ctypes.byref(ex)) == _lib.ERR_INVALID
    _status("tp_partition_destroy", h)
    n = ctypes.c_int64(-1)
    assert _status("tp_graph_kernel_count", None, ctypes.byref(n)) == _lib.ERR_INVALID
    assert n.value == -1


def test_ctx_create_without_gpu_fails_cleanly(built_lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = _status("tp_ctx_create", 0, ctypes.byref(h))
    assert st in (_lib.ERR_CUDA, _lib.ERR_INVALID) and not h.value
    assert built_lib.tp_last_error_detail()


def test_empty_outputs_with_any_strides_are_partitionable():
    # torch gives a (128, 0) tensor strides (1, 1): an empty view is contiguous
    import torch
    for shape in ((128, 0), (0, 64), (0,), (3, 0, 5)):
        t = torch.zeros(shape)
        p = tp.tp_partition_create(None, t, tuple(4 for _ in shape))
        assert tp.tp_partition_query(p)["num_tiles"] == 0
        tp.tp_partition_destroy(p)


def test_missing_library_fails_loudly(monkeypatch):
    # without the built CUDA library every call raises: there is no fallback path
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", "/nonexistent/libtp.so")
    with pytest.raises(RuntimeError, match="no fallback"):
        tp.tp_version()


def test_autotune_space_and_targets_on_the_host(built_lib):
    """The autotuner's space (host data): by default the 72 single-pass
    configs (rows 64, 128 or 256, columns 64..256, 1, 2 or 4 K blocks per
    stage, raster bands 1 or 8), which all compute C bit-identically; with
    the swap-AB opt-in followed by 6 swap-AB configs (W x 128 C tiles, W =
    32, 64 or 128, 2 or 4 K blocks per stage; the same class); with the
    split-K opt-in followed by the split-K configs, each with 128-row tiles
    and a column slice of at least 32 per K slice. BF16 and FP8 share the
    layout, with K blocks of 64 and 128 elements; undefined flag bits are
    refused. Training targets train a config that did not run towards 0."""
    whole = tp.tp_autotune_space("bf16")
    assert len(whole) == 72 and len(tp.tp_autotune_space("fp8")) == 72
    assert {(c.bm, c.bn, c.bk, c.group_m) for c in whole} == {
        (bm, bn, 64 * kb, g) for bm in (64, 128, 256) for bn in (64, 128, 192, 256) for kb in (1, 2, 4)
        for g in (1, 8)}
    assert all(c.swap_ab == 0 for c in whole)
    assert [c.bk for c in tp.tp_autotune_space("fp8")] == [2 * c.bk for c in whole]
    assert all(c.split_k == 0 and c.stages == 0 for c in whole)
    key = lambda c: (c.bm, c.bn, c.bk, c.stages, c.group_m, c.swap_ab)
    sw = tp.tp_autotune_space("bf16", swap_ab=True)
    assert [key(c) for c in sw[:72]] == [key(c) for c in whole]
    assert [(c.bm, c.bn, c.bk, c.group_m, c.swap_ab, c.split_k) for c in sw[72:]] == [
        (w, 128, 64 * kb, 1, 1, 0) for w in (32, 64, 128) for kb in (2, 4)]
    both = tp.tp_autotune_space("bf16", split_k=True, swap_ab=True)
    assert len(both) == 83 and [key(c) for c in both[:78]] == [key(c) for c in sw]
    full = tp.tp_autotune_space("bf16", split_k=True)
    assert len(full) == 77 and len(tp.tp_autotune_space("fp8", split_k=True)) == 77
    assert [key(c) for c in full[:72]] == [key(c) for c in whole]
    assert [key(c) for c in both[78:]] == [key(c) for c in full[72:]]
    split = full[72:]
    assert [(c.bn, c.split_k) for c in split] == [(128, 2), (128, 4), (256, 2), (256, 4), (256, 8)]
    assert all(c.bm == 128 and c.bn % (32 * c.split_k) == 0 for c in split)
    n = ctypes.c_int32()
    assert _lib.lib().tp_autotune_space(_lib.BF16, 4, None, 0, ctypes.byref(n)) == _lib.ERR_INVALID
    tg, mk = tp.tp_mlp_targets([3.0, 0.0, 1.5])
    assert tg == [1.0, 0.0, 0.5] and mk == [1.0, 1.0, 1.0]


def test_binding_constants_match_the_header():
    """Every enum constant the ctypes binding passes across the boundary
    (status codes, dtypes, map kinds, launch modes, exec and tuning flags)
    equals the value include/tp.h gives it."""
    import re

    header = open(_lib.HEADER).read()
    consts = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(TP_[A-Z0-9_]+)\s*=\s*(\d+)", header)}
    status = {name: code for code, name in _lib.STATUS_NAMES.items()}
    assert status == {k: v for k, v in consts.items() if k == "TP_OK" or k.startswith("TP_ERR_")}
    expect = {
        "TP_F32": _lib.F32, "TP_BF16": _lib.BF16, "TP_F8E4M3": _lib.F8E4M3, "TP_F64": _lib.F64,
        "TP_I32": _lib.I32, "TP_U32": _lib.U32, "TP_U8": _lib.U8,
        "TP_MAP_IDENTITY": _lib.MAP_IDENTITY, "TP_MAP_STRIDED": _lib.MAP_STRIDED, "TP_MAP_QUEUE": _lib.MAP_QUEUE,
        "TP_SYNC": _lib.SYNC, "TP_ASYNC": _lib.ASYNC, "TP_CAPTURE": _lib.CAPTURE,
        "TP_EXEC_CHECKED": _lib.EXEC_CHECKED, "TP_EXEC_INJECT_TIMEOUT": _lib.EXEC_INJECT_TIMEOUT,
        "TP_EXEC_STATIC_WEIGHTS": _lib.EXEC_STATIC_WEIGHTS,
        "TP_TUNE_SPLIT_K": tp.TUNE_SPLIT_K, "TP_TUNE_SWAP_AB": tp.TUNE_SWAP_AB,
    }
    for name, value in expect.items():
        assert consts[name] == value, name


def test_mlp_features_on_the_host(built_lib):
    """The proposer's input features (host code, no GPU): log2 M, log2 N,
    log2 K and a one-hot dtype, equal to the oracle's within fp32 rounding;
    a power of two gives its exponent exactly."""
    from oracle import mlp as omlp

    for (m, n, k), dt in (((1, 1, 16), "bf16"), ((1024, 3, 16384), "fp8"), ((777, 12345, 4100), "bf16")):
        got = tp.tp_mlp_features(m, n, k, dt)
        want = omlp.features(m, n, k, 0 if dt == "bf16" else 1)
        assert np.allclose(got, want, rtol=1e-6, atol=1e-6), (m, n, k, dt)
    assert tp.tp_mlp_features(4096, 8192, 16, "fp8") == [12.0, 13.0, 4.0, 0.0, 1.0]
