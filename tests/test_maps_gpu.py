"""GPU parity of the element-wise map kernels against the FP64 oracle, write-count
coverage against the oracle's partition enumeration, and the launch protocol
(SYNC / ASYNC / CAPTURE, busy and alias rules) through the C ABI."""
import numpy as np
import pytest
import torch

import paper_2606_15991_gb300 as tp
import synth
from oracle import gemm as ogemm
from oracle import maps as omaps
from oracle import partition as opart

pytestmark = pytest.mark.gpu

TORCH_DT = {"f32": torch.float32, "bf16": torch.bfloat16}
FN = {"axpy": tp.tp_map_axpy, "gelu_mul": tp.tp_map_gelu_mul, "scale": tp.tp_map_scale,
      "add_accum": tp.tp_map_add_accum}
ALPHA = 0.5


def _inputs(n, dt, seed=1, shape=None):
    shape = shape or (n,)
    x = synth.tensor(synth.normal(n, seed), dt).reshape(shape).cuda()
    y = synth.tensor(synth.normal(n, seed + 1), dt).reshape(shape).cuda()
    c = synth.tensor(synth.normal(n, seed + 2), dt).reshape(shape).cuda()
    return x, y, c


def _ref(op, x, y, c0):
    if op == "axpy":
        r = omaps.axpy(ALPHA, x, y)
    elif op == "gelu_mul":
        r = omaps.gelu_mul(x, y)
    elif op == "scale":
        r = omaps.scale(x, y)
    else:
        r = omaps.add_accum(c0, x, y)
    return r.reshape(-1)


def _bound(op, dt, ref, x, y, c0):
    """Per-element error bound derived from the kernel's arithmetic (fp32
    operations, then one rounding to the output type)."""
    u32, u16 = 2.0 ** -24, 2.0 ** -8
    ref = np.abs(ref).reshape(-1)
    if op in ("axpy", "scale"):
        b = u32 * ref                                # one fp32 rounding (fma / mul)
    elif op == "add_accum":
        b = 2 * u32 * (np.abs(_f(c0)) + np.abs(_f(x)) + np.abs(_f(y)))
    else:
        b = 2e-5 * ref                               # base-2 exponential + fast division, see kernel
    if dt == "bf16":
        b = b + (u16 + u32) * ref
    return b + 1e-37


def _f(t):
    return t.double().cpu().numpy().reshape(-1)


def _run(ctx, op, dt, n, tile, kind=tp.MAP_IDENTITY, P=0, count=False, shape=None, seed=1):
    x, y, c = _inputs(n, dt, seed, shape)
    c0 = c.clone()
    out = c if op == "add_accum" else torch.empty_like(x)
    part = tp.tp_partition_create(ctx, out, tile)
    if kind != tp.MAP_IDENTITY:
        tp.tp_partition_map(part, kind, P)
    counts = owner = None
    if count:
        counts = torch.zeros(n, dtype=torch.int32, device="cuda")
        owner = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    ex = tp.make_exec(write_counts=counts, write_owner=owner)
    if op == "axpy":
        tp.tp_map_axpy(ctx, part, ALPHA, x, y, ex)
    else:
        FN[op](ctx, part, x, y, ex)
    tp.tp_partition_destroy(part)
    return x, y, c0, out, counts, owner


@pytest.mark.parametrize("dt", ["f32", "bf16"])
@pytest.mark.parametrize("op", ["axpy", "gelu_mul", "scale", "add_accum"])
@pytest.mark.parametrize("n,tile", [(4096 * 9 + 77, 4096), (1, 4096), (8, 8), (4096 * 3, 4096), (10007, 100)])
def test_map_parity(ctx, op, dt, n, tile):
    x, y, c0, out, _, _ = _run(ctx, op, dt, n, (tile,))
    ref = _ref(op, x, y, c0)
    got = _f(out)
    assert np.all(np.abs(got - ref) <= _bound(op, dt, ref, x, y, c0))
    gate = 1e-5 if dt == "f32" else 1e-2
    assert ogemm.rel_frobenius(got, ref) <= gate


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_map_closed_forms_bit_exact(ctx, dt):
    n = 4096 * 5 + 3
    x, y, _ = _inputs(n, dt)
    z = torch.empty_like(x)
    p = tp.tp_partition_create(ctx, z, (4096,))
    tp.tp_map_axpy(ctx, p, 0.0, x, y)          # x * 0 + b = b
    assert torch.equal(z, y)
    tp.tp_map_axpy(ctx, p, 1.0, x, torch.zeros_like(y))
    assert torch.equal(z, x)
    tp.tp_map_gelu_mul(ctx, p, x, torch.zeros_like(y))
    assert torch.count_nonzero(z).item() == 0
    tp.tp_map_gelu_mul(ctx, p, torch.zeros_like(x), y)
    assert torch.count_nonzero(z).item() == 0
    tp.tp_partition_destroy(p)


@pytest.mark.parametrize("kind,P", [(tp.MAP_IDENTITY, 0), (tp.MAP_STRIDED, 3), (tp.MAP_STRIDED, 1),
                                    (tp.MAP_STRIDED, 7)])
@pytest.mark.parametrize("dt,n,tile", [("f32", 4096 * 7 + 5, 4096), ("bf16", 3001, 256), ("f32", 999, 10)])
def test_write_counts_match_oracle_map(ctx, kind, P, dt, n, tile):
    x, y, c0, out, counts, owner = _run(ctx, "axpy", dt, n, (tile,), kind, P, count=True)
    kname = "identity" if kind == tp.MAP_IDENTITY else "strided"
    expect = opart.owner_map((n,), (tile,), P or None, kname)
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    assert np.array_equal(owner.cpu().numpy(), expect)


def test_write_counts_queue_map(ctx):
    n, tile, P = 4096 * 13 + 1, 4096, 5
    x, y, c0, out, counts, owner = _run(ctx, "gelu_mul", "f32", n, (tile,), tp.MAP_QUEUE, P, count=True)
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    o = owner.cpu().numpy()
    assert o.min() >= 0 and o.max() < P
    for t in range(opart.num_tiles((n,), (tile,))):   # one owner per tile
        assert len(set(o[t * tile:(t + 1) * tile].tolist())) == 1
    ref = _ref("gelu_mul", x, y, c0)
    assert np.all(np.abs(_f(out) - ref) <= _bound("gelu_mul", "f32", ref, x, y, c0))


@pytest.mark.parametrize("shape,tile", [((37, 53), (8, 16)), ((5, 6, 7), (2, 4, 3)), ((64, 64), (64, 64))])
def test_rank2_rank3_partitions(ctx, shape, tile):
    n = int(np.prod(shape))
    x, y, c0, out, counts, owner = _run(ctx, "axpy", "f32", n, tile, count=True, shape=shape)
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    assert np.array_equal(owner.cpu().numpy(), opart.owner_map(shape, tile))
    ref = _ref("axpy", x, y, c0)
    assert np.all(np.abs(_f(out) - ref) <= _bound("axpy", "f32", ref, x, y, c0))


def test_misaligned_views_use_scalar_path(ctx):
    n = 4096 * 2 + 9
    xb, yb, _ = _inputs(n + 1, "bf16")
    zb = torch.empty_like(xb)
    x, y, z = xb[1:], yb[1:], zb[1:]          # 2-byte offset: not 16-byte aligned
    p = tp.tp_partition_create(ctx, z, (4096,))
    tp.tp_map_axpy(ctx, p, ALPHA, x, y)
    ref = omaps.axpy(ALPHA, x, y)
    assert np.all(np.abs(_f(z) - ref) <= _bound("axpy", "bf16", ref, x, y, None))
    tp.tp_partition_destroy(p)


def test_empty_output(ctx):
    z = torch.empty(0, device="cuda")
    p = tp.tp_partition_create(ctx, z, (4096,))
    tp.tp_map_axpy(ctx, p, ALPHA, z.clone(), z.clone())
    tp.tp_partition_destroy(p)


def test_shape_dtype_and_alias_errors(ctx):
    buf = torch.zeros(8192, device="cuda")
    z = buf[:4096]
    p = tp.tp_partition_create(ctx, z, (1024,))
    with pytest.raises(tp.TPError) as e:
        tp.tp_map_axpy(ctx, p, 1.0, buf[2048:6144], torch.zeros(4096, device="cuda"))
    assert e.value.status == tp._lib.ERR_ALIAS
    with pytest.raises(tp.TPError) as e:
        tp.tp_map_axpy(ctx, p, 1.0, torch.zeros(4095, device="cuda"), torch.zeros(4096, device="cuda"))
    assert e.value.status == tp._lib.ERR_SHAPE
    with pytest.raises(tp.TPError) as e:
        tp.tp_map_axpy(ctx, p, 1.0, torch.zeros(4096, device="cuda", dtype=torch.bfloat16),
                       torch.zeros(4096, device="cuda"))
    assert e.value.status == tp._lib.ERR_SHAPE
    with pytest.raises(tp.TPError) as e:     # capture mode without an open graph
        tp.tp_map_axpy(ctx, p, 1.0, buf[4096:], buf[4096:], tp.make_exec(mode=tp.CAPTURE))
    assert e.value.status == tp._lib.ERR_CAPTURE
    tp.tp_partition_destroy(p)


def test_async_busy_protocol(ctx):
    n = 1 << 22
    x, y, _ = _inputs(n, "f32")
    z = torch.empty_like(x)
    s, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    p = tp.tp_partition_create(ctx, z, (4096,))
    ev = tp.tp_event_create(ctx)
    with torch.cuda.stream(s):
        torch.cuda._sleep(200_000_000)       # keep the stream busy (bounded spin)
        tp.tp_map_axpy(ctx, p, ALPHA, x, y, tp.make_exec(mode=tp.ASYNC, stream=s, event=ev))
    assert tp.tp_partition_query(p)["busy"]
    assert not tp.tp_event_query(ev)
    with pytest.raises(tp.TPError) as e:      # second writer on another stream while in flight
        tp.tp_map_axpy(ctx, p, ALPHA, x, y, tp.make_exec(stream=s2))
    assert e.value.status == tp._lib.ERR_BUSY
    z2 = torch.empty_like(x)
    p2 = tp.tp_partition_create(ctx, z2, (4096,))
    with pytest.raises(tp.TPError) as e:      # reader of the in-flight output on another stream
        tp.tp_map_axpy(ctx, p2, ALPHA, z, y, tp.make_exec(stream=s2))
    assert e.value.status == tp._lib.ERR_BUSY
    with pytest.raises(tp.TPError) as e:
        tp.tp_partition_destroy(p)
    assert e.value.status == tp._lib.ERR_BUSY
    with pytest.raises(tp.TPError) as e:
        tp.tp_partition_map(p, tp.MAP_STRIDED, 2)
    assert e.value.status == tp._lib.ERR_BUSY
    with pytest.raises(tp.TPError) as e:
        tp.tp_event_destroy(ev)
    assert e.value.status == tp._lib.ERR_BUSY
    # chained on the same stream (`then`): reads the in-flight output in stream order
    tp.tp_map_axpy(ctx, p2, ALPHA, z, y, tp.make_exec(mode=tp.ASYNC, stream=s, event=ev))
    tp.tp_event_wait(ev)
    assert not tp.tp_partition_query(p)["busy"] and not tp.tp_partition_query(p2)["busy"]
    assert tp.tp_event_query(ev)
    ref = omaps.axpy(ALPHA, x, y)
    assert np.all(np.abs(_f(z) - ref) <= _bound("axpy", "f32", ref, x, y, None))
    ref2 = omaps.axpy(ALPHA, ref, y)   # the chained result, composed in the oracle
    assert np.all(np.abs(_f(z2) - ref2) <= 2.0 ** -24 * (np.abs(ref2) + ALPHA * np.abs(ref)) + 1e-37)
    tp.tp_map_axpy(ctx, p2, ALPHA, z, y, tp.make_exec(stream=s2))   # now allowed from any stream
    for h in (p, p2):
        tp.tp_partition_destroy(h)
    tp.tp_event_destroy(ev)


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_graph_replay_bit_equal_to_eager(ctx, dt):
    n = 4096 * 33 + 17
    x, w, _ = _inputs(n, dt, seed=7)
    t = torch.empty_like(x)
    z = torch.empty_like(x)
    pt = tp.tp_partition_create(ctx, t, (4096,))
    pz = tp.tp_partition_create(ctx, z, (4096,))
    tp.tp_map_gelu_mul(ctx, pt, x, w)
    tp.tp_map_axpy(ctx, pz, ALPHA, t, x)
    eager_t, eager_z = t.clone(), z.clone()
    t.zero_()
    z.zero_()
    s = torch.cuda.Stream()
    g = tp.tp_graph_begin(ctx, s)
    cap = tp.make_exec(mode=tp.CAPTURE, stream=s)
    tp.tp_map_gelu_mul(ctx, pt, x, w, cap)
    tp.tp_map_axpy(ctx, pz, ALPHA, t, x, cap)     # reads the first node's output
    tp.tp_graph_end(g)
    assert torch.count_nonzero(z).item() == 0     # recorded, not executed
    for _ in range(50):
        tp.tp_graph_replay(g, tp.make_exec(stream=s))
    assert torch.equal(t, eager_t) and torch.equal(z, eager_z)
    ev = tp.tp_event_create(ctx)
    tp.tp_graph_replay(g, tp.make_exec(mode=tp.ASYNC, stream=s, event=ev))
    tp.tp_event_wait(ev)
    assert torch.equal(z, eager_z)
    tp.tp_graph_destroy(g)
    tp.tp_event_destroy(ev)
    for p in (pt, pz):
        tp.tp_partition_destroy(p)


@pytest.mark.parametrize("dt", ["f32", "bf16"])
@pytest.mark.parametrize("op", ["axpy", "gelu_mul"])
def test_full_size_sampled(ctx, op, dt):
    """2^28 elements, 4096-element tiles (the benchmarked launch): outputs at
    65536 sampled indices against the oracle evaluated at those indices."""
    n = 1 << 28
    x = torch.randn(n, device="cuda", generator=torch.Generator("cuda").manual_seed(1)).to(TORCH_DT[dt])
    y = torch.randn(n, device="cuda", generator=torch.Generator("cuda").manual_seed(2)).to(TORCH_DT[dt])
    z = torch.empty_like(x)
    p = tp.tp_partition_create(ctx, z, (4096,))
    FN[op](ctx, p, *((ALPHA, x, y) if op == "axpy" else (x, y)))
    idx = torch.from_numpy((synth.uniform(65536, seed=5, lo=0, hi=1, dtype=np.float64) * n).astype(np.int64))
    idx = torch.cat([idx, torch.tensor([0, n - 1])]).cuda()
    xs, ys = x[idx].cpu(), y[idx].cpu()
    ref = _ref(op, xs, ys, None)
    got = _f(z[idx])
    assert np.all(np.abs(got - ref) <= _bound(op, dt, ref, xs, ys, None))
    tp.tp_partition_destroy(p)
    del x, y, z
    torch.cuda.empty_cache()


def test_full_size_write_counts(ctx):
    n, tile = 1 << 28, 4096
    x = torch.zeros(n, device="cuda", dtype=torch.bfloat16)
    z = torch.empty_like(x)
    counts = torch.zeros(n, dtype=torch.int32, device="cuda")
    owner = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    p = tp.tp_partition_create(ctx, z, (tile,))
    tp.tp_map_axpy(ctx, p, ALPHA, x, x.clone(), tp.make_exec(write_counts=counts, write_owner=owner))
    assert bool((counts == 1).all())
    o = owner.view(-1, tile)
    assert bool((o == o[:, :1]).all())                               # one program per tile
    assert torch.unique(o[:, 0]).numel() == n // tile                # no program owns two tiles
    tp.tp_partition_destroy(p)
    del x, z, counts, owner
    torch.cuda.empty_cache()


@pytest.mark.parametrize("kind,P", [(tp.MAP_IDENTITY, 0), (tp.MAP_STRIDED, 5), (tp.MAP_QUEUE, 7)])
@pytest.mark.parametrize("shape,tile", [((40000,), (4096,)), ((37, 300), (8, 64)), ((5, 6, 7), (2, 3, 4))])
def test_checked_launch_matches_release(ctx, kind, P, shape, tile):
    """TP_EXEC_CHECKED on the maps: every tile is validated against the map
    and claimed before it is stored; on a correct map the result equals the
    release launch bit for bit, each element is written once, and repeated
    checked launches (the bitmap clears itself) keep succeeding."""
    n = int(np.prod(shape))
    x = synth.tensor(synth.normal(n, 11), "f32").reshape(shape).cuda()
    y = synth.tensor(synth.normal(n, 12), "f32").reshape(shape).cuda()
    rel, chk = torch.empty_like(x), torch.empty_like(x)
    outs = []
    for out in (rel, chk):
        p = tp.tp_partition_create(ctx, out, tile)
        if kind != tp.MAP_IDENTITY:
            tp.tp_partition_map(p, kind, P)
        outs.append(p)
    tp.tp_map_gelu_mul(ctx, outs[0], x, y)
    counts = torch.zeros(n, dtype=torch.int32, device="cuda")
    owner = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    for _ in range(3):
        counts.zero_()
        tp.tp_map_gelu_mul(ctx, outs[1], x, y, tp.make_exec(write_counts=counts, write_owner=owner, checked=True))
        assert torch.equal(rel, chk)
        assert opart.check_counts(counts.cpu().numpy())["ok"]
    for p in outs:
        tp.tp_partition_destroy(p)


def test_trace_log_lines():
    """TP_LOG: one stderr line per operation, including refused ones; nothing
    is printed without it."""
    import os
    import subprocess
    import sys

    code = ("import torch, paper_2606_15991_gb300 as tp\n"
            "ctx = tp.tp_ctx_create(0)\n"
            "x = torch.ones(8192, device='cuda'); z = torch.empty_like(x)\n"
            "p = tp.tp_partition_create(ctx, z, (4096,))\n"
            "tp.tp_map_axpy(ctx, p, 2.0, x, x)\n"
            "try:\n    tp.tp_map_axpy(ctx, p, 2.0, z, x)\nexcept tp.TPError:\n    pass\n"
            "torch.cuda.synchronize()\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, TP_LOG="1", PYTHONPATH=root)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stderr.splitlines() if l.startswith("[tp] ")]
    assert any(l.startswith("[tp] tp_map_axpy done mode=SYNC") and "tiles=2 programs=2" in l and "status=ok" in l
               for l in lines), lines
    assert any("tp_map_axpy refused" in l and "input aliases output" in l for l in lines), lines
    env.pop("TP_LOG")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "[tp] " not in r.stderr
