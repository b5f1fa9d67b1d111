"""Pins for the decode-chain and MLP oracles (closed forms, finite differences, autograd)."""
import numpy as np
import torch

import synth
from oracle import decode, mlp


def test_rmsnorm_closed_forms():
    h = np.full(64, 3.0)
    assert np.allclose(decode.rmsnorm(h, eps=0.0), np.ones(64), rtol=0, atol=1e-15)
    x = synth.normal(5120, seed=1, dtype=np.float64)
    n = decode.rmsnorm(x)
    ms = np.mean(x * x)
    assert abs(np.mean(n * n) - ms / (ms + decode.EPS)) < 1e-12
    g = synth.normal(5120, seed=2, dtype=np.float64)
    assert np.allclose(decode.rmsnorm(x, g), n * g, rtol=0, atol=1e-14)


def test_silu_landmarks():
    assert decode.silu(0.0) == 0.0
    assert abs(decode.silu(40.0) - 40.0) < 1e-12
    x = synth.normal(1000, seed=3, std=4.0, dtype=np.float64)
    assert np.allclose(decode.silu(x) - decode.silu(-x), x, rtol=0, atol=1e-12)   # silu(x) - silu(-x) = x


def test_layer_zero_down_is_identity_and_brute_force():
    d, qkv, inter = 8, 6, 5
    h = synth.normal(d, seed=4, dtype=np.float64)
    wq = synth.normal(qkv * d, seed=5, dtype=np.float64).reshape(qkv, d)
    wgu = synth.normal(2 * inter * d, seed=6, dtype=np.float64).reshape(2 * inter, d)
    wd = np.zeros((d, inter))
    h2, q = decode.layer(h, wq, wgu, wd)
    assert np.array_equal(h2, h)
    # brute force with python loops
    wd = synth.normal(d * inter, seed=7, dtype=np.float64).reshape(d, inter)
    h2, q = decode.layer(h, wq, wgu, wd)
    ms = sum(v * v for v in h) / d
    n = [v / (ms + 1e-6) ** 0.5 for v in h]
    gu = [sum(wgu[i, j] * n[j] for j in range(d)) for i in range(2 * inter)]
    a = [gu[i] / (1 + np.exp(-gu[i])) * gu[inter + i] for i in range(inter)]
    ref = [h[i] + sum(wd[i, j] * a[j] for j in range(inter)) for i in range(d)]
    assert np.allclose(h2, ref, rtol=0, atol=1e-12)
    assert np.allclose(q, [sum(wq[i, j] * n[j] for j in range(d)) for i in range(qkv)], rtol=0, atol=1e-12)


def _params(F=5, H=16, C=7, seed=0):
    rng = lambda n, s: synth.normal(n, seed=seed * 10 + s, std=0.5, dtype=np.float64)
    return {"W1": rng(H * F, 1).reshape(H, F), "b1": rng(H, 2), "W2": rng(H * H, 3).reshape(H, H),
            "b2": rng(H, 4), "W3": rng(C * H, 5).reshape(C, H), "b3": rng(C, 6)}


def _batch(B=9, F=5, C=7):
    X = synth.normal(B * F, seed=50, dtype=np.float64).reshape(B, F)
    T = synth.normal(B * C, seed=51, dtype=np.float64).reshape(B, C)
    V = (synth.uniform(B * C, seed=52, lo=0, hi=1, dtype=np.float64) > 0.3).astype(np.float64).reshape(B, C)
    return X, T, V


def test_mlp_gradients_finite_differences():
    p = _params()
    X, T, V = _batch()
    Y, cache = mlp.forward(p, X)
    g = mlp.backward(p, cache, Y, T, V)
    h = 1e-6
    for k in mlp.PARAMS:
        flat = p[k].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(mlp.forward(p, X)[0], T, V)
            flat[idx] = old - h
            lm = mlp.loss(mlp.forward(p, X)[0], T, V)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[idx]) < 1e-6 * max(1.0, abs(fd))


def test_mlp_gradients_match_torch_autograd():
    p = _params()
    X, T, V = _batch()
    Y, cache = mlp.forward(p, X)
    g = mlp.backward(p, cache, Y, T, V)
    tp = {k: torch.tensor(v, requires_grad=True) for k, v in p.items()}
    x = torch.tensor(X)
    h1 = torch.relu(x @ tp["W1"].T + tp["b1"])
    h2 = torch.relu(h1 @ tp["W2"].T + tp["b2"])
    y = h2 @ tp["W3"].T + tp["b3"]
    v = torch.tensor(V)
    L = (v * (y - torch.tensor(T)) ** 2).sum() / max(1.0, float(V.sum()))
    L.backward()
    assert abs(L.item() - mlp.loss(Y, T, V)) < 1e-12
    for k in mlp.PARAMS:
        assert np.allclose(tp[k].grad.numpy(), g[k], rtol=1e-10, atol=1e-12)


def test_adam_first_step_closed_form():
    p = _params()
    g = {k: np.full_like(v, 0.25) * np.where(np.arange(v.size).reshape(v.shape) % 2, 1, -1) for k, v in p.items()}
    z = {k: np.zeros_like(v) for k, v in p.items()}
    p2, m, v = mlp.adam_step(p, g, z, z, 1, lr=0.01, eps=0.0)
    for k in mlp.PARAMS:
        assert np.allclose(p2[k], p[k] - 0.01 * np.sign(g[k]), rtol=0, atol=1e-15)
    opt = torch.optim.Adam([torch.tensor(p["W1"], requires_grad=True)], lr=0.01, eps=1e-8)
    t = opt.param_groups[0]["params"][0]
    pp, mm, vv = dict(p), {k: np.zeros_like(x) for k, x in p.items()}, {k: np.zeros_like(x) for k, x in p.items()}
    for step in range(1, 4):
        gg = {k: np.cos(step + np.arange(x.size).reshape(x.shape)) for k, x in p.items()}
        t.grad = torch.tensor(gg["W1"])
        opt.step()
        pp, mm, vv = mlp.adam_step(pp, gg, mm, vv, step, lr=0.01)
    assert np.allclose(t.detach().numpy(), pp["W1"], rtol=0, atol=1e-12)


def test_mlp_learns_separable_toy():
    p = _params(F=5, H=32, C=3, seed=3)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(x) for k, x in p.items()}
    X = synth.uniform(300 * 5, seed=60, dtype=np.float64).reshape(300, 5)
    cls = np.argmax(X[:, :3], axis=1)
    T = np.eye(3)[cls]
    V = np.ones_like(T)
    for t in range(1, 400):
        Y, cache = mlp.forward(p, X)
        g = mlp.backward(p, cache, Y, T, V)
        p, m, v = mlp.adam_step(p, g, m, v, t, lr=0.01)
    acc = np.mean(np.argmax(mlp.forward(p, X)[0], axis=1) == cls)
    assert acc > 0.95
