"""The allocation-free queue-mapped axpy (tp_map_axpy_queue_noalloc).

It serves callers that cannot call cudaMalloc (code running while another
component captures the stream into a CUDA graph, or inside a runtime whose
device memory belongs to its own arena allocator): it takes only the inputs
and the output and keeps its one piece of scratch, the tile-queue counter, in
a static device array. These tests call it through the C ABI and compare it
with tp_map_axpy on a queue-mapped partition, twice in a row (the second call
must find the shared counter cleared again). This file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2606_15991_gb300 as tp
import synth
from paper_2606_15991_gb300 import _lib

pytestmark = pytest.mark.gpu

DT = {"f32": (_lib.F32, torch.float32), "bf16": (_lib.BF16, torch.bfloat16)}


def _noalloc(z, x, y, dt, tile, programs, alpha, stream):
    return _lib.lib().tp_map_axpy_queue_noalloc(
        ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
        DT[dt][0], z.numel(), tile, programs, ctypes.c_float(alpha), ctypes.c_void_p(stream.cuda_stream))


def _reference(ctx, x, y, tile, programs, alpha, stream):
    z = torch.empty_like(x)
    p = tp.tp_partition_create(ctx, z, (tile,))
    tp.tp_partition_map(p, tp.MAP_QUEUE, programs)
    tp.tp_map_axpy(ctx, p, alpha, x, y, tp.make_exec(stream=stream))
    tp.tp_partition_destroy(p)
    return z


def _within_tolerance(got, ref, dt):
    # the tolerance the map parity tests use: one fp32 rounding, plus one bf16
    # rounding of the output for bf16
    g = got.double().cpu().numpy()
    r = ref.double().cpu().numpy()
    bound = 2.0 ** -24 * np.abs(r)
    if dt == "bf16":
        bound = bound + (2.0 ** -8 + 2.0 ** -24) * np.abs(r)
    return bool(np.all(np.abs(g - r) <= bound + 1e-37))


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_matches_queue_mapped_axpy_twice_in_a_row(ctx, dt):
    n, tile, programs = 4096 * 37 + 5, 4096, 7
    s = torch.cuda.Stream()
    for call, (seed, alpha) in enumerate([(11, 0.5), (21, -1.25)]):
        x = synth.tensor(synth.normal(n, seed), dt).cuda()
        y = synth.tensor(synth.normal(n, seed + 1), dt).cuda()
        z = torch.full_like(x, float("nan"))
        torch.cuda.synchronize()
        st = _noalloc(z, x, y, dt, tile, programs, alpha, s)
        assert st == _lib.OK, (call, _lib.lib().tp_last_error_detail())
        s.synchronize()
        ref = _reference(ctx, x, y, tile, programs, alpha, s)
        assert _within_tolerance(z, ref, dt), call
        assert not torch.isnan(z).any()


def test_unaligned_tile_and_one_program(ctx):
    n, tile = 1000, 7                       # tile not a multiple of the vector width
    s = torch.cuda.Stream()
    x = synth.tensor(synth.normal(n, 3), "f32").cuda()
    y = synth.tensor(synth.normal(n, 4), "f32").cuda()
    for _ in range(2):
        z = torch.empty_like(x)
        assert _noalloc(z, x, y, "f32", tile, 1, 0.5, s) == _lib.OK
        s.synchronize()
        assert _within_tolerance(z, _reference(ctx, x, y, tile, 1, 0.5, s), "f32")


def test_rejections_launch_nothing(ctx):
    L = _lib.lib()
    s = torch.cuda.Stream()
    x = torch.zeros(64, device="cuda")
    z = torch.zeros(64, device="cuda")
    # more tiles than the 32-bit scratch counter may hand out
    st = L.tp_map_axpy_queue_noalloc(ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                     ctypes.c_void_p(x.data_ptr()), _lib.F32, (1 << 31) + 1, 1, 1,
                                     ctypes.c_float(1.0), ctypes.c_void_p(s.cuda_stream))
    assert st == _lib.ERR_INVALID and b"2^31" in L.tp_last_error_detail()
    assert _noalloc(z, x, x, "f32", 16, 5, 1.0, s) == _lib.ERR_INVALID          # 5 programs, 4 tiles
    assert _noalloc(z, z, x, "f32", 16, 2, 1.0, s) == _lib.ERR_ALIAS
    assert L.tp_map_axpy_queue_noalloc(None, None, None, _lib.F32, 64, 16, 2, ctypes.c_float(1.0),
                                       None) == _lib.ERR_INVALID
    assert L.tp_map_axpy_queue_noalloc(None, None, None, _lib.F32, 0, 16, 2, ctypes.c_float(1.0),
                                       None) == _lib.OK                          # empty: nothing to do
