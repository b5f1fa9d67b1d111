"""Learned tile proposer pipeline (driver around the library's kernels).

1. collect: run the exhaustive autotuner (tp_autotune) on sampled shapes; each
   shape gives one TFLOP/s measurement per config of the space.
2. train:   fit the 3-layer MLP on the GPU with tp_mlp_train_step (the
   library's forward, backward and Adam kernels), mini-batches drawn in a
   seeded order.
3. evaluate: on held-out shapes that were tuned exhaustively, the proposal
   (tp_propose: the arg-max of the MLP's scores over the autotuner's
   single-pass configs) is charged its measured TFLOP/s; regret =
   1 - TFLOP/s(proposal) / TFLOP/s(best). The method without the MLP is a fixed
   default config (the best on average over the training shapes).
   `retimed_regret` re-times the proposal, the exhaustive pick and the default
   (median of independent timings), so that regret is not measured against
   the maximum of one noisy sample per config.

The space is the autotuner's single-pass class: every config in it computes
C bit-identically, so neither a proposal nor its fallback changes numerics.

Shapes: M, N, K log-uniform on [1, 16384]; K is rounded up to a multiple of 16
so TMA rows are 16-byte multiples in both BF16 and FP8.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

import synth

from . import (tp_autotune, tp_autotune_space, tp_autotune_time, tp_mlp_create, tp_mlp_forward, tp_mlp_features,
               tp_mlp_targets, tp_mlp_train_step)

DTYPES = ("bf16", "fp8")
HIDDEN = 64


def sample_shapes(count: int, seed: int, lo: int = 1, hi: int = 16384):
    """(M, N, K, dtype) with M, N, K log-uniform on [lo, hi], K rounded up to a
    multiple of 16, dtype alternating BF16 / FP8."""
    out = []
    for i, (m, n, k) in enumerate(synth.log_uniform_shapes(count, seed, lo, hi)):
        k = min(hi, ((k + 15) // 16) * 16)
        out.append((m, n, k, DTYPES[i % 2]))
    return out


def collect(ctx, shapes, reps: int = 0, log=None):
    """Exhaustive tables: returns X [S, 5], T [S, C], V [S, C], tflops [S, C]."""
    C = len(tp_autotune_space("bf16"))
    X = np.zeros((len(shapes), 5), np.float32)
    T = np.zeros((len(shapes), C), np.float32)
    V = np.zeros((len(shapes), C), np.float32)
    TF = np.zeros((len(shapes), C), np.float32)
    t0 = time.perf_counter()
    for i, (m, n, k, dt) in enumerate(shapes):
        _, table, _ = tp_autotune(ctx, m, n, k, dt, reps)
        X[i] = tp_mlp_features(m, n, k, dt)
        tg, mk = tp_mlp_targets(table)
        T[i], V[i], TF[i] = tg, mk, table
        if log and (i + 1) % 100 == 0:
            log(f"collected {i + 1}/{len(shapes)} shapes in {time.perf_counter() - t0:.1f} s")
    return X, T, V, TF


def init_params(F: int, H: int, C: int, seed: int = 0) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases, flat layout
    [W1, b1, W2, b2, W3, b3]."""
    parts = []
    for i, (rows, fan_in) in enumerate(((H, F), (H, H), (C, H))):
        b = 1.0 / math.sqrt(fan_in)
        parts.append(synth.uniform(rows * fan_in, seed + 2 * i, -b, b))
        parts.append(synth.uniform(rows, seed + 2 * i + 1, -b, b))
    return np.concatenate(parts).astype(np.float32)


def train(ctx, X, T, V, epochs: int = 200, batch: int = 256, lr: float = 3e-3, seed: int = 0, log=None):
    """Trains a fresh MLP on the GPU; returns (mlp, per-epoch mean loss)."""
    S, F = X.shape
    C = T.shape[1]
    batch = min(batch, S)
    mlp = tp_mlp_create(ctx, F, HIDDEN, C, max(batch, 256), init_params(F, HIDDEN, C, seed))
    Xd = torch.from_numpy(X).cuda()
    Td = torch.from_numpy(T).cuda()
    Vd = torch.from_numpy(V).cuda()
    loss = torch.zeros(1, device="cuda")
    hist = []
    nb = S // batch
    for ep in range(epochs):
        u = synth.uniform(S, seed + 1000 + ep, 0.0, 1.0, dtype=np.float64)
        order = torch.from_numpy(np.argsort(u, kind="stable")).cuda()
        tot = 0.0
        for b in range(nb):
            idx = order[b * batch:(b + 1) * batch]
            tp_mlp_train_step(mlp, Xd[idx].contiguous(), Td[idx].contiguous(), Vd[idx].contiguous(), lr, loss)
            tot += loss.item()
        hist.append(tot / max(1, nb))
        if log and (ep + 1) % 50 == 0:
            log(f"epoch {ep + 1}: loss {hist[-1]:.5f}")
    return mlp, hist


def scores(mlp, X) -> np.ndarray:
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    out = torch.empty(X.shape[0], mlp.shape[2], device="cuda")
    for s in range(0, X.shape[0], 256):
        e = min(X.shape[0], s + 256)
        part = torch.empty(e - s, mlp.shape[2], device="cuda")
        tp_mlp_forward(mlp, Xd[s:e].contiguous(), part)
        out[s:e] = part
    return out.cpu().numpy()


def config_index(space, cfg) -> int:
    """Position of a proposed config in the autotuner's space (of its dtype:
    BF16 and FP8 configs differ in bk, K blocks of 64 or 128 elements)."""
    key = (cfg.bm, cfg.bn, cfg.bk, cfg.stages, cfg.group_m, cfg.split_k, cfg.swap_ab)
    for i, c in enumerate(space):
        if (c.bm, c.bn, c.bk, c.stages, c.group_m, c.split_k, c.swap_ab) == key:
            return i
    raise ValueError(f"config {key} is not in the space")


def propose_indices(ctx, mlp, shapes) -> np.ndarray:
    """tp_propose's choice (no fallback) for each (M, N, K, dtype), as space indices."""
    from . import tp_propose
    spaces = {dt: tp_autotune_space(dt) for dt in DTYPES}
    return np.array([config_index(spaces[dt], tp_propose(ctx, mlp, m, n, k, dt, min_score=-1e9)[0])
                     for m, n, k, dt in shapes])


def evaluate(mlp, X, TF, default_index: int, min_score: float = 0.0, prop=None) -> dict:
    """Regret of the MLP's proposals (the given space indices, else the plain
    arg-max of its scores) and of the fixed default config."""
    S = scores(mlp, X)
    if prop is None:
        prop = S.argmax(axis=1)
    return regret_stats(TF, prop, default_index, S.max(axis=1), min_score)


def regret_stats(TF, prop, default_index: int, top_score=None, min_score: float = 0.0) -> dict:
    """Regret summary from exhaustive tables TF [shapes, configs] (TFLOP/s):
    regret = 1 - TF[proposal] / max TF, for the proposals `prop` and for the
    fixed config `default_index`; a shape whose top score is below
    `min_score` goes to the exhaustive fallback, whose regret is 0."""
    TF = np.asarray(TF, dtype=np.float64)
    prop = np.asarray(prop)
    best = TF.max(axis=1)
    reg = 1.0 - TF[np.arange(len(TF)), prop] / best
    reg_def = 1.0 - TF[:, default_index] / best
    fallback = (np.zeros(len(TF), bool) if top_score is None else np.asarray(top_score) < min_score)
    reg_fb = np.where(fallback, 0.0, reg)   # the exhaustive fallback has zero regret by definition
    return {"median_regret": float(np.median(reg)), "p90_regret": float(np.percentile(reg, 90)),
            "mean_regret": float(reg.mean()),
            "median_regret_default": float(np.median(reg_def)), "p90_regret_default": float(np.percentile(reg_def, 90)),
            "mean_regret_default": float(reg_def.mean()),
            "fallback_rate": float(fallback.mean()), "median_regret_with_fallback": float(np.median(reg_fb)),
            "exact_pick_rate": float((reg <= 1e-6).mean()), "shapes": int(len(TF))}


def retimed_regret(ctx, shapes, TF, prop, default_index: int, repeats: int = 3) -> dict:
    """Regret from re-timed configs. For each shape the proposal, the
    exhaustive pick (arg-max of its table) and the default config are each
    timed `repeats` times (tp_autotune_time, median); the reference is the
    fastest of them, so regret = 1 - TFLOP/s(config) / TFLOP/s(reference)."""
    spaces = {dt: tp_autotune_space(dt) for dt in DTYPES}
    reg, reg_def, beat = [], [], 0
    for i, (m, n, k, dt) in enumerate(shapes):
        best = int(np.argmax(TF[i]))
        idx = {int(prop[i]), best, int(default_index)}
        t = {j: tp_autotune_time(ctx, m, n, k, dt, spaces[dt][j], repeats=repeats) for j in sorted(idx)}
        ref = max(t.values())
        reg.append(1.0 - t[int(prop[i])] / ref)
        reg_def.append(1.0 - t[int(default_index)] / ref)
        beat += int(t[int(prop[i])] > t[best])
    reg, reg_def = np.array(reg), np.array(reg_def)
    return {"median_regret": float(np.median(reg)), "p90_regret": float(np.percentile(reg, 90)),
            "mean_regret": float(reg.mean()),
            "median_regret_default": float(np.median(reg_def)), "p90_regret_default": float(np.percentile(reg_def, 90)),
            "mean_regret_default": float(reg_def.mean()), "repeats": repeats, "shapes": len(shapes),
            "proposal_faster_than_exhaustive_pick": beat}


def default_config(T, V) -> int:
    """Index of the config with the best mean relative TFLOP/s on training shapes."""
    return int((T * V).sum(axis=0).argmax())
