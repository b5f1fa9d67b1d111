"""Three-layer MLP tile proposer in float64 (oracle; test infrastructure).

Network (the learned tile proposer; the paper has none, its GEMM tile shapes
are "tuned once per size", §5.1):
  x  (F features: log2 M, log2 N, log2 K, one-hot dtype)
  h1 = relu(W1 x + b1)      W1: H x F
  h2 = relu(W2 h1 + b2)     W2: H x H
  y  = W3 h2 + b3           W3: C x H   (one score per tile configuration)

Loss over a batch of B rows with targets T and a validity mask V (a config
that cannot run a shape has V = 0):
  L = sum_{b,c} V_bc (y_bc - T_bc)^2 / max(1, sum V)

Adam (Kingma and Ba, 2015) with bias correction, step t starting at 1:
  m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2
  p <- p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
"""
from __future__ import annotations

import numpy as np

PARAMS = ("W1", "b1", "W2", "b2", "W3", "b3")


def forward(p: dict, X):
    """Returns (Y, cache) for a batch X of shape B x F."""
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    Y = h2 @ p["W3"].T + p["b3"]
    return Y, (X, z1, h1, z2, h2)


def loss(Y, T, V) -> float:
    Y, T, V = (np.asarray(a, dtype=np.float64) for a in (Y, T, V))
    return float(np.sum(V * (Y - T) ** 2) / max(1.0, float(np.sum(V))))


def backward(p: dict, cache, Y, T, V) -> dict:
    """Gradients of `loss` w.r.t. every parameter (plain chain rule)."""
    X, z1, h1, z2, h2 = cache
    Y, T, V = (np.asarray(a, dtype=np.float64) for a in (Y, T, V))
    dY = 2.0 * V * (Y - T) / max(1.0, float(np.sum(V)))
    g = {"W3": dY.T @ h2, "b3": dY.sum(axis=0)}
    dh2 = dY @ p["W3"]
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return g


def adam_step(p: dict, g: dict, m: dict, v: dict, t: int, lr: float,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update at step t (t >= 1); returns new (p, m, v)."""
    p2, m2, v2 = {}, {}, {}
    for k in PARAMS:
        m2[k] = beta1 * m[k] + (1.0 - beta1) * g[k]
        v2[k] = beta2 * v[k] + (1.0 - beta2) * g[k] ** 2
        mh = m2[k] / (1.0 - beta1 ** t)
        vh = v2[k] / (1.0 - beta2 ** t)
        p2[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p2, m2, v2


def features(m: int, n: int, k: int, dtype_index: int, n_dtypes: int = 2) -> np.ndarray:
    """[log2 M, log2 N, log2 K, one-hot(dtype)]."""
    x = np.zeros(3 + n_dtypes)
    x[0], x[1], x[2] = np.log2(m), np.log2(n), np.log2(k)
    x[3 + dtype_index] = 1.0
    return x
