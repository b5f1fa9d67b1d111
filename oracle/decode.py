"""Batch-1 decode-shaped layer chain in float64 (oracle; test infrastructure).

One layer of the graph-captured forward pass of §3.2 (Listing 3: RMSNorm, then
matrix-vector products, then a residual add), widened to the gated-MLP shape of
the decode workload:

  n   = h / sqrt(mean(h^2) + eps) * gamma          (RMSNorm over d)
  qkv = W_qkv . n                                   (computed and kept; it
                                                     stands in for attention)
  [g; u] = W_gu . n                                 (gate = first half, up = second)
  a   = silu(g) * u,  silu(g) = g / (1 + exp(-g))
  dd  = W_down . a
  h  <- h + dd

Weights are given as [out, in] matrices holding the exact bf16 values.
"""
from __future__ import annotations

import numpy as np

EPS = 1e-6


def _f64(a) -> np.ndarray:
    if hasattr(a, "detach"):
        a = a.detach().to("cpu").double().numpy()
    return np.asarray(a, dtype=np.float64)


def rmsnorm(h, gamma=None, eps: float = EPS) -> np.ndarray:
    h = _f64(h)
    r = h / np.sqrt(np.mean(h * h) + eps)
    return r if gamma is None else r * _f64(gamma)


def silu(g) -> np.ndarray:
    g = _f64(g)
    return g / (1.0 + np.exp(-g))


def layer(h, w_qkv, w_gu, w_down, gamma=None, eps: float = EPS):
    """One layer; returns (h_next, qkv)."""
    h = _f64(h)
    n = rmsnorm(h, gamma, eps)
    qkv = _f64(w_qkv) @ n
    gu = _f64(w_gu) @ n
    half = gu.shape[0] // 2
    a = silu(gu[:half]) * gu[half:]
    dd = _f64(w_down) @ a
    return h + dd, qkv


def chain(h, layers, gamma=None, eps: float = EPS):
    """Apply `layers` = [(w_qkv, w_gu, w_down), ...] in order; returns (h, last qkv)."""
    qkv = None
    for w_qkv, w_gu, w_down in layers:
        h, qkv = layer(h, w_qkv, w_gu, w_down, gamma, eps)
    return h, qkv
