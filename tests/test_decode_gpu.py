"""GPU parity of the decode-shaped chain (RMSNorm -> QKV GEMV -> gate/up GEMV
-> SiLU*mul -> down GEMV -> residual) against the FP64 oracle, fused and
unfused, plus the 64-layer chain at the full dimensions against the oracle
and its graph replay against the eager run."""
import numpy as np
import pytest
import torch

import paper_2606_15991_gb300 as tp
import synth
from oracle import decode as odecode
from oracle import gemm as ogemm
from oracle import partition as opart

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _w(rows, k, seed):
    return synth.to_bf16(synth.normal(rows * k, seed, std=0.02)).reshape(rows, k).cuda()


def _layers(d, nq, ni, n, seed=0):
    return [(_w(nq, d, seed + 3 * i), _w(2 * ni, d, seed + 3 * i + 1), _w(d, ni, seed + 3 * i + 2))
            for i in range(n)]


def _vec(n, seed, std=1.0):
    return torch.from_numpy(synth.normal(n, seed, std=std)).cuda()


def _f(t):
    return t.double().cpu().numpy()


def _gemv_bound(w, x):
    """Summation bound of the kernel: chains of about k/64 + 12 fp32 adds."""
    k = w.shape[1]
    return (k / 64 + 12) * U32 * (np.abs(_f(w)) @ np.abs(_f(x))) + 1e-30


@pytest.mark.parametrize("rows,k", [(10240, 5120), (5120, 25600), (1, 8), (77, 1000), (300, 4104)])
def test_gemv_within_summation_bound(ctx, rows, k):
    w = _w(rows, k, rows + k)
    x = _vec(k, 5)
    y = torch.full((rows,), float("nan"), device="cuda")
    p = tp.tp_partition_create(ctx, y, (rows,))
    counts = torch.zeros(rows, dtype=torch.int32, device="cuda")
    owner = torch.full((rows,), -1, dtype=torch.int32, device="cuda")
    tp.tp_gemv(ctx, p, w, x, tp.make_exec(write_counts=counts, write_owner=owner))
    ref = _f(w) @ _f(x)
    assert np.all(np.abs(_f(y) - ref) <= _gemv_bound(w, x))
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    tp.tp_partition_destroy(p)


@pytest.mark.parametrize("d", [1, 100, 5120])
def test_rmsnorm_silu_residual(ctx, d):
    h = _vec(d, 1, std=3.0)
    gamma = _vec(d, 2)
    n = torch.empty(d, device="cuda")
    p = tp.tp_partition_create(ctx, n, (d,))
    tp.tp_rmsnorm(ctx, p, h, gamma, 1e-6)
    ref = odecode.rmsnorm(h.cpu(), gamma.cpu(), 1e-6)
    assert np.all(np.abs(_f(n) - ref) <= (d / 256 + 8) * U32 * np.abs(ref) + 1e-30)
    tp.tp_rmsnorm(ctx, p, h, None, 1e-6)
    assert np.allclose(_f(n), odecode.rmsnorm(h.cpu(), None, 1e-6), rtol=(d / 256 + 8) * U32, atol=0)
    tp.tp_partition_destroy(p)
    gu = _vec(2 * d, 3, std=4.0)
    a = torch.empty(d, device="cuda")
    p = tp.tp_partition_create(ctx, a, (d,))
    tp.tp_silu_mul(ctx, p, gu)
    g = gu.cpu().double().numpy()
    ref = odecode.silu(g[:d]) * g[d:]
    assert np.all(np.abs(_f(a) - ref) <= 1e-5 * np.abs(ref) + 1e-30)
    tp.tp_partition_destroy(p)
    hh = h.clone()
    p = tp.tp_partition_create(ctx, hh, (d,))
    dd = _vec(d, 4)
    tp.tp_residual_add(ctx, p, dd)
    assert np.all(np.abs(_f(hh) - (_f(h) + _f(dd))) <= U32 * np.abs(_f(h) + _f(dd)))
    tp.tp_partition_destroy(p)


@pytest.mark.parametrize("fused", [True, False])
def test_small_chain_against_oracle(ctx, fused):
    d, nq, ni, L = 256, 512, 1024, 8
    layers = _layers(d, nq, ni, L, seed=10)
    h0 = _vec(d, 7)
    h = h0.clone()
    ch = tp.DecodeChain(ctx, h, layers)
    (ch.record_fused if fused else ch.record_unfused)()
    href, qref = odecode.chain(h0.cpu(), [(a.cpu(), b.cpu(), c.cpu()) for a, b, c in layers])
    assert ogemm.rel_frobenius(h.cpu(), href) <= 1e-4
    assert ogemm.rel_frobenius(ch.qkv.cpu(), qref) <= 1e-4
    ch.close()


def test_fused_equals_oracle_full_dims_two_layers(ctx):
    d, nq, ni = 5120, 10240, 25600
    layers = _layers(d, nq, ni, 2, seed=20)
    h0 = _vec(d, 8)
    h = h0.clone()
    ch = tp.DecodeChain(ctx, h, layers)
    counts = torch.zeros(nq + ni, dtype=torch.int32, device="cuda")
    owner = torch.full((nq + ni,), -1, dtype=torch.int32, device="cuda")
    ex = tp.make_exec(write_counts=counts, write_owner=owner)
    tp.tp_decode_norm_qkv_gu(ctx, ch.p["qkv"], ch.p["a"], h, None, layers[0][0], layers[0][1], 1e-6, ex)
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    tp.tp_decode_down_residual(ctx, ch.p["h"], layers[0][2], ch.a)
    w1 = layers[1]
    tp.tp_decode_norm_qkv_gu(ctx, ch.p["qkv"], ch.p["a"], h, None, w1[0], w1[1], 1e-6)
    tp.tp_decode_down_residual(ctx, ch.p["h"], w1[2], ch.a)
    href, qref = odecode.chain(h0.cpu(), [(a.cpu(), b.cpu(), c.cpu()) for a, b, c in layers])
    assert ogemm.rel_frobenius(h.cpu(), href) <= 1e-4
    assert ogemm.rel_frobenius(ch.qkv.cpu(), qref) <= 1e-4
    ch.close()


def test_zero_down_projection_is_identity(ctx):
    d, nq, ni = 5120, 10240, 25600
    layers = _layers(d, nq, ni, 1, seed=30)
    layers = [(layers[0][0], layers[0][1], torch.zeros_like(layers[0][2]))]
    h0 = _vec(d, 9)
    h = h0.clone()
    ch = tp.DecodeChain(ctx, h, layers)
    ch.record_fused()
    assert torch.equal(h, h0)
    ch.close()


def test_64_layer_chain_matches_oracle_and_replay_matches_eager(ctx):
    """The full decode-shaped chain (d = 5120, QKV 10240, gate/up 2 x 25600,
    64 layers of bf16 N(0, 0.02) weights, 57 GB) as the benchmark runs it:
    the eager result matches the FP64 oracle run layer by layer on the host
    (each layer's three weight matrices copied to the host in turn) within
    1e-4 relative Frobenius error for h and for the last layer's qkv, and
    the captured graph replayed gives exactly the eager result, on every
    replay. The graph holds three kernels a layer: the fused norm + QKV +
    gate/up product, the down product over K slices, and the finish kernel
    adding the slices' partial sums to h."""
    d, nq, ni, L = 5120, 10240, 25600, 64
    g = torch.Generator(device="cuda")
    layers = []
    for i in range(L):
        g.manual_seed(100 + i)
        layers.append(tuple((torch.randn(r, k, device="cuda", generator=g) * 0.02).to(torch.bfloat16)
                            for r, k in ((nq, d), (2 * ni, d), (d, ni))))
    h0 = _vec(d, 11)
    h = h0.clone()
    ch = tp.DecodeChain(ctx, h, layers)
    ch.record_fused()
    eager = h.clone()
    eager_qkv = ch.qkv.clone()
    assert torch.isfinite(eager).all()
    # FP64 oracle, one layer at a time
    href = h0.cpu()
    qref = None
    for w_qkv, w_gu, w_down in layers:
        href, qref = odecode.layer(href, w_qkv.cpu(), w_gu.cpu(), w_down.cpu())
    err_h = ogemm.rel_frobenius(eager.cpu(), href)
    err_q = ogemm.rel_frobenius(eager_qkv.cpu(), qref)
    print(f"64-layer chain vs FP64: h {err_h:.3e}, last qkv {err_q:.3e}")
    assert err_h <= 1e-4 and err_q <= 1e-4, (err_h, err_q)
    s = torch.cuda.Stream()
    gr = tp.tp_graph_begin(ctx, s)
    ch.record_fused(tp.make_exec(mode=tp.CAPTURE, stream=s))
    tp.tp_graph_end(gr)
    assert tp.tp_graph_kernel_count(gr) == 3 * L
    for _ in range(3):
        h.copy_(h0)
        torch.cuda.synchronize()
        tp.tp_graph_replay(gr, tp.make_exec(stream=s))
        assert torch.equal(h, eager)
        assert torch.equal(ch.qkv, eager_qkv)
    tp.tp_graph_destroy(gr)
    ch.close()
    del layers
    torch.cuda.empty_cache()


@pytest.mark.parametrize("d,nq,ni", [(8, 1, 8), (264, 45, 40), (5000, 70, 24), (512, 96, 3000)])
def test_streamed_layer_ragged_shapes(ctx, d, nq, ni):
    """The TMA-fed matrix-vector kernels on ragged sizes: rows that do not
    fill a 32-row (QKV, down) or 16-pair (gate/up) unit, columns that do not
    fill a 256-column stage, and rows of 3000 (down projection) cut into K
    slices whose partial sums a finish kernel adds; every output row written
    once, h and qkv against the FP64 oracle."""
    layers = _layers(d, nq, ni, 1, seed=d + ni)
    h0 = _vec(d, 13)
    h = h0.clone()
    ch = tp.DecodeChain(ctx, h, layers)
    counts = torch.zeros(nq + ni, dtype=torch.int32, device="cuda")
    owner = torch.full((nq + ni,), -1, dtype=torch.int32, device="cuda")
    w = layers[0]
    tp.tp_decode_norm_qkv_gu(ctx, ch.p["qkv"], ch.p["a"], h, None, w[0], w[1], 1e-6,
                             tp.make_exec(write_counts=counts, write_owner=owner))
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    dcounts = torch.zeros(d, dtype=torch.int32, device="cuda")
    downer = torch.full((d,), -1, dtype=torch.int32, device="cuda")
    tp.tp_decode_down_residual(ctx, ch.p["h"], w[2], ch.a, tp.make_exec(write_counts=dcounts, write_owner=downer))
    assert opart.check_counts(dcounts.cpu().numpy())["ok"]
    href, qref = odecode.chain(h0.cpu(), [(a.cpu(), b.cpu(), c.cpu()) for a, b, c in layers])
    assert ogemm.rel_frobenius(h.cpu(), href) <= 1e-5
    assert ogemm.rel_frobenius(ch.qkv.cpu(), qref) <= 1e-5
    ch.close()


def test_unaligned_input_takes_the_per_lane_kernel(ctx):
    """An input vector that is not 16-byte aligned goes to the per-lane
    kernel (the streaming kernel reads x in 16-byte pieces): same results
    within the oracle's tolerance."""
    d, nq, ni = 264, 40, 24
    layers = _layers(d, nq, ni, 1, seed=91)
    buf = torch.zeros(d + 1, device="cuda")
    h = buf[1:]                                    # 4-byte offset
    h.copy_(_vec(d, 14))
    h0 = h.clone()
    ch = tp.DecodeChain(ctx, h, layers)
    ch.record_fused()
    href, qref = odecode.chain(h0.cpu(), [(a.cpu(), b.cpu(), c.cpu()) for a, b, c in layers])
    assert ogemm.rel_frobenius(h.cpu(), href) <= 1e-5
    assert ogemm.rel_frobenius(ch.qkv.cpu(), qref) <= 1e-5
    ch.close()


@pytest.mark.parametrize("d,nq,ni,pad", [(261, 40, 48, 3), (64, 8, 3001, 7), (64, 8, 3004, 4), (96, 8, 70000, 0)])
def test_streamed_layer_padded_weights(ctx, d, nq, ni, pad):
    """Weights that are views of wider matrices (row pitch a multiple of 8
    elements, rows of any length): an odd input length for the fused norm +
    QKV + gate/up kernel, a down projection whose input length is not a
    multiple of 4 floats (no bulk copies of its slices: the per-lane kernel
    runs it) or is one (ragged last slice), and rows of 70000 cut into
    4096-column slices. h and qkv against the FP64 oracle, every output row
    written once."""
    def wpad(rows, k, seed):
        kp = (k + pad + 7) // 8 * 8
        return _w(rows, kp, seed)[:, :k]

    layers = [(wpad(nq, d, 5), wpad(2 * ni, d, 6), wpad(d, ni, 7))]
    h0 = _vec(d, 17)
    h = h0.clone()
    ch = tp.DecodeChain(ctx, h, layers)
    counts = torch.zeros(nq + ni, dtype=torch.int32, device="cuda")
    owner = torch.full((nq + ni,), -1, dtype=torch.int32, device="cuda")
    w = layers[0]
    tp.tp_decode_norm_qkv_gu(ctx, ch.p["qkv"], ch.p["a"], h, None, w[0], w[1], 1e-6,
                             tp.make_exec(write_counts=counts, write_owner=owner))
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    dcounts = torch.zeros(d, dtype=torch.int32, device="cuda")
    downer = torch.full((d,), -1, dtype=torch.int32, device="cuda")
    tp.tp_decode_down_residual(ctx, ch.p["h"], w[2], ch.a, tp.make_exec(write_counts=dcounts, write_owner=downer))
    assert opart.check_counts(dcounts.cpu().numpy())["ok"]
    href, qref = odecode.chain(h0.cpu(), [tuple(t.cpu().contiguous() for t in lay) for lay in layers])
    assert ogemm.rel_frobenius(h.cpu(), href) <= 1e-5
    assert ogemm.rel_frobenius(ch.qkv.cpu(), qref) <= 1e-5
    ch.close()


def test_weights_written_just_before_on_the_stream(ctx):
    """A decode product whose weight matrix the previous launch on the same
    stream writes (a tensor-core GEMM, whose kernels let the next one start
    early): without TP_EXEC_STATIC_WEIGHTS the product reads the weights only
    after that GEMM completes, so qkv and a match the FP64 oracle on the
    weights the GEMM wrote. Queued with no host synchronisation between."""
    d, nq, ni = 1024, 2048, 1536
    g = torch.Generator(device="cuda")
    g.manual_seed(21)
    f = torch.randn(nq, 256, device="cuda", generator=g).to(torch.bfloat16) * 0.1
    e = torch.randn(d, 256, device="cuda", generator=g).to(torch.bfloat16) * 0.1
    w_qkv = torch.zeros(nq, d, device="cuda", dtype=torch.bfloat16)          # written by the GEMM below
    w_gu = (torch.randn(2 * ni, d, device="cuda", generator=g) * 0.02).to(torch.bfloat16)
    w_down = (torch.randn(d, ni, device="cuda", generator=g) * 0.02).to(torch.bfloat16)
    h = _vec(d, 22)
    h0 = h.clone()
    ch = tp.DecodeChain(ctx, h, [(w_qkv, w_gu, w_down)])
    s = torch.cuda.Stream()
    ev = tp.tp_event_create(ctx)
    torch.cuda.synchronize()
    pw = tp.tp_partition_create(ctx, w_qkv, (256, 256))
    tp.tp_partition_map(pw, tp.MAP_STRIDED, min(ctx.sm_count // 2, (nq // 256) * (d // 256)))
    ex = tp.make_exec(tp.ASYNC, s, ev)
    tp.tp_gemm(ctx, pw, f, e.t(), tp.gemm_config(bm=256, bn=256), ex)       # W_qkv = F E^T
    tp.tp_decode_norm_qkv_gu(ctx, ch.p["qkv"], ch.p["a"], h, None, w_qkv, w_gu, 1e-6, ex)
    tp.tp_event_wait(ev)
    href, qref = odecode.chain(h0.cpu(), [(w_qkv.cpu(), w_gu.cpu(), torch.zeros(d, ni, dtype=torch.bfloat16))])
    assert float(w_qkv.float().abs().max()) > 0
    assert ogemm.rel_frobenius(ch.qkv.cpu(), qref) <= 1e-5
    tp.tp_partition_destroy(pw)
    tp.tp_event_destroy(ev)
    ch.close()


def test_static_weights_flag_is_for_the_decode_products(ctx):
    """TP_EXEC_STATIC_WEIGHTS is accepted by the two decode products and
    refused (TP_ERR_UNSUPPORTED) by other operations."""
    x = _vec(4096, 3)
    y = torch.empty_like(x)
    p = tp.tp_partition_create(ctx, y, (4096,))
    with pytest.raises(tp.TPError) as ei:
        tp.tp_map_axpy(ctx, p, 1.0, x, x, tp.make_exec(static_weights=True))
    assert ei.value.status == tp._lib.ERR_UNSUPPORTED
    tp.tp_partition_destroy(p)
    d, nq, ni = 264, 40, 40
    layers = _layers(d, nq, ni, 1, seed=5)
    h0 = _vec(d, 6)
    h = h0.clone()
    ch = tp.DecodeChain(ctx, h, layers)
    w = layers[0]
    flag = tp.make_exec(static_weights=True)
    tp.tp_decode_norm_qkv_gu(ctx, ch.p["qkv"], ch.p["a"], h, None, w[0], w[1], 1e-6, flag)
    tp.tp_decode_down_residual(ctx, ch.p["h"], w[2], ch.a, flag)
    href, qref = odecode.chain(h0.cpu(), [(a.cpu(), b.cpu(), c.cpu()) for a, b, c in layers])
    assert ogemm.rel_frobenius(h.cpu(), href) <= 1e-5
    ch.close()
