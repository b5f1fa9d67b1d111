"""Element-wise maps in float64 (oracle; test infrastructure).

Each output element depends only on the input elements at the same index, so
the plain definition is the whole computation; the tiling of the output into
disjoint partitions (§3.4) changes nothing in the values.

* axpy: z_i = alpha * x_i + y_i. The paper's element-wise add (§2, Listing 1;
  evaluated at N = 2^28 in §5.1) is the alpha = 1 case.
* gelu_mul: y_i = gelu_tanh(x_i) * w_i with the tanh form of GELU (Hendrycks
  and Gimpel, 2016): gelu_tanh(x) = 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).
* scale (y = x * g), the launch-overhead probe of §5.2.
* add_accum: c_i <- c_i + a_i + b_i, the read-modify-write map of §3.4, Listing 4.

Inputs are the exact values the kernel reads (fp32, or bf16 widened exactly).
"""
from __future__ import annotations

import math

import numpy as np

GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def _f64(a) -> np.ndarray:
    if hasattr(a, "detach"):  # torch tensor
        a = a.detach().to("cpu").double().numpy()
    return np.asarray(a, dtype=np.float64)


def axpy(alpha: float, x, y) -> np.ndarray:
    """z = alpha * x + y, element by element, in float64."""
    return float(alpha) * _f64(x) + _f64(y)


def gelu_tanh(x) -> np.ndarray:
    """0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))) in float64."""
    x = _f64(x)
    return 0.5 * x * (1.0 + np.tanh(GELU_C * (x + GELU_A * x ** 3)))


def gelu_mul(x, w) -> np.ndarray:
    """y = gelu_tanh(x) * w, element by element, in float64."""
    return gelu_tanh(x) * _f64(w)


def scale(x, g) -> np.ndarray:
    """y = x * g, element by element (the §5.2 pipeline kernel)."""
    return _f64(x) * _f64(g)


def add_accum(c, a, b) -> np.ndarray:
    """c + a + b (the new value of the read-modify-write output, §3.4 Listing 4)."""
    return _f64(c) + _f64(a) + _f64(b)
