"""The allocation-free queue-mapped axpy (tp_map_axpy_queue_noalloc).

It serves callers that cannot call cudaMalloc: code inside a runtime or
plugin whose device memory belongs to the host application's arena
allocator, or code on a latency-critical path where an allocation, which can
synchronise the device, is not allowed. It takes only the inputs and the
output and keeps its one piece of scratch, the tile-queue counter, in a
static device array shared by every call.

These tests call it through the C ABI. Each result must equal tp_map_axpy on
a queue-mapped partition bit for bit (the same kernel arithmetic) and the
FP64 oracle element by element within the map tolerance (one fp32 rounding,
plus one bf16 rounding of the output for bf16), for fp32 and bf16, on aligned
and ragged sizes; on two calls in a row (the second must find the shared
counter cleared again) and on calls queued back to back on one stream with
no host synchronisation between them (each call's clear of the counter must
wait for the previous call's kernel). This file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2606_15991_gb300 as tp
import synth
from oracle import maps as omaps
from paper_2606_15991_gb300 import _lib

pytestmark = pytest.mark.gpu

DT = {"f32": (_lib.F32, torch.float32), "bf16": (_lib.BF16, torch.bfloat16)}


def _noalloc(z, x, y, dt, tile, programs, alpha, stream):
    return _lib.lib().tp_map_axpy_queue_noalloc(
        ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
        DT[dt][0], z.numel(), tile, programs, ctypes.c_float(alpha), ctypes.c_void_p(stream.cuda_stream))


def _reference(ctx, x, y, tile, programs, alpha, stream):
    """The same map through the context-owning entry point (tp_map_axpy on a
    TP_MAP_QUEUE partition)."""
    z = torch.empty_like(x)
    p = tp.tp_partition_create(ctx, z, (tile,))
    tp.tp_partition_map(p, tp.MAP_QUEUE, programs)
    tp.tp_map_axpy(ctx, p, alpha, x, y, tp.make_exec(stream=stream))
    tp.tp_partition_destroy(p)
    return z


def _within_oracle_tolerance(got, x, y, alpha, dt):
    """Element-wise check against the FP64 oracle: one fp32 rounding, plus
    one bf16 rounding of the output for bf16."""
    ref = omaps.axpy(alpha, x.cpu(), y.cpu())
    g = got.double().cpu().numpy()
    bound = 2.0 ** -24 * np.abs(ref)
    if dt == "bf16":
        bound = bound + (2.0 ** -8 + 2.0 ** -24) * np.abs(ref)
    return bool(np.all(np.abs(g - ref) <= bound + 1e-37))


def _inputs(n, dt, seed):
    x = synth.tensor(synth.normal(n, seed), dt).cuda()
    y = synth.tensor(synth.normal(n, seed + 1), dt).cuda()
    return x, y


@pytest.mark.parametrize("n", [4096 * 37, 4096 * 37 + 5])
@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_two_calls_in_a_row_equal_axpy_and_oracle(ctx, dt, n):
    tile, programs = 4096, 7
    s = torch.cuda.Stream()
    for call, (seed, alpha) in enumerate([(11, 0.5), (21, -1.25)]):
        x, y = _inputs(n, dt, seed)
        z = torch.full_like(x, float("nan"))
        torch.cuda.synchronize()
        st = _noalloc(z, x, y, dt, tile, programs, alpha, s)
        assert st == _lib.OK, (call, _lib.lib().tp_last_error_detail())
        s.synchronize()
        assert not torch.isnan(z).any(), call
        assert torch.equal(z, _reference(ctx, x, y, tile, programs, alpha, s)), call
        assert _within_oracle_tolerance(z, x, y, alpha, dt), call


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_calls_queued_back_to_back_on_one_stream(ctx, dt):
    n, tile, programs = (1 << 24) + 3 * 4096 + 7, 4096, 148
    s = torch.cuda.Stream()
    x, y = _inputs(n, dt, 31)
    alphas = [0.5, -2.0, 0.125]
    zs = [torch.full_like(x, float("nan")) for _ in alphas]
    torch.cuda.synchronize()
    for z, alpha in zip(zs, alphas):
        assert _noalloc(z, x, y, dt, tile, programs, alpha, s) == _lib.OK
    s.synchronize()
    for z, alpha in zip(zs, alphas):
        assert not torch.isnan(z).any(), alpha
        assert torch.equal(z, _reference(ctx, x, y, tile, programs, alpha, s)), alpha
        assert _within_oracle_tolerance(z, x, y, alpha, dt), alpha


def test_unaligned_tile_and_one_program(ctx):
    n, tile = 1000, 7                       # tile not a multiple of the vector width
    s = torch.cuda.Stream()
    x, y = _inputs(n, "f32", 3)
    for _ in range(2):
        z = torch.full_like(x, float("nan"))
        assert _noalloc(z, x, y, "f32", tile, 1, 0.5, s) == _lib.OK
        s.synchronize()
        assert torch.equal(z, _reference(ctx, x, y, tile, 1, 0.5, s))
        assert _within_oracle_tolerance(z, x, y, 0.5, "f32")


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
    s.synchronize()
    assert torch.equal(z, torch.zeros_like(z))
