"""GEMM in float64, with the rounding steps of the low-precision paths (oracle).

The paper's GEMM (§3.6, Listing 6; evaluated in §5.1) computes C = A . B, one
output tile per loop iteration, accumulating mma over the K tiles. Tiling and
the order of the K loop change only the rounding, so the oracle is the plain
definition C_ij = sum_k A_ik B_kj, evaluated in float64 on the exact input
values (numpy's float64 matmul serves as that sum).

Per-tensor-scaled FP8-E4M3 path (the FP8 GEMM workload; the paper has no FP8):
  1. amax_X = max |X| over the whole tensor.
  2. s_X = 448 / amax_X, in fp32 (IEEE division, round to nearest).
  3. q_X = E4M3(satfinite(RN(fp32(X) * s_X))): the product is an fp32 multiply,
     so the quantised code is decided in the precision the kernel uses.
  4. C = (q_A . q_B) * inv, inv = fp32(1 / fp32(s_A * s_B)), accumulated here
     in float64; the kernel accumulates in fp32 and rounds C to bf16.
"""
from __future__ import annotations

import numpy as np

from . import lowp


def _f64(a) -> np.ndarray:
    if hasattr(a, "detach"):
        a = a.detach().to("cpu").double().numpy()
    return np.asarray(a, dtype=np.float64)


def gemm(a, b) -> np.ndarray:
    """C = A . B in float64. A is M x K, B is K x N."""
    return _f64(a) @ _f64(b)


def gemm_tiles(a, b, tiles, bm: int, bn: int) -> dict:
    """Float64 C over selected output tiles only: {(tm, tn): C[tm*bm:.., tn*bn:..]}.

    Each tile is the plain definition restricted to its rows and columns."""
    a = _f64(a)
    b = _f64(b)
    out = {}
    for tm, tn in tiles:
        out[(tm, tn)] = a[tm * bm:(tm + 1) * bm, :] @ b[:, tn * bn:(tn + 1) * bn]
    return out


def rel_frobenius(c, c_ref) -> float:
    """||C - C_ref||_F / ||C_ref||_F (0 when both are zero)."""
    c = _f64(c)
    c_ref = _f64(c_ref)
    den = np.linalg.norm(c_ref)
    num = np.linalg.norm(c - c_ref)
    if den == 0.0:
        return 0.0 if num == 0.0 else float("inf")
    return float(num / den)


def amax(x) -> np.float32:
    """max |x| over the whole tensor (exact; returned as fp32, which holds it)."""
    return np.float32(np.max(np.abs(_f64(x))))


def fp8_scale(amax_value) -> np.float32:
    """s = 448 / amax in fp32. An all-zero tensor (amax = 0) takes s = 1."""
    a = np.float32(amax_value)
    if a == 0.0:
        return np.float32(1.0)
    return np.float32(np.float32(lowp.E4M3_MAX) / a)


def fp8_quantize(x, s) -> np.ndarray:
    """E4M3 bytes of satfinite(RN(fp32(x) * s)), the product taken in fp32."""
    xf = np.asarray(_f64(x), dtype=np.float32)
    prod = (xf * np.float32(s)).astype(np.float32)
    return lowp.e4m3_encode(lowp.round_e4m3_satfinite(prod.astype(np.float64)))


def fp8_dequant_factor(s_a, s_b) -> np.float32:
    """inv = 1 / (s_A * s_B), both steps in fp32."""
    return np.float32(np.float32(1.0) / np.float32(np.float32(s_a) * np.float32(s_b)))


def gemm_fp8(a, b):
    """Per-tensor-scaled FP8 GEMM. Returns (C_float64, qA, qB, sA, sB, inv) where
    C = (decode(qA) . decode(qB)) * inv in float64."""
    sa = fp8_scale(amax(a))
    sb = fp8_scale(amax(b))
    qa = fp8_quantize(a, sa)
    qb = fp8_quantize(b, sb)
    inv = fp8_dequant_factor(sa, sb)
    c = (lowp.e4m3_decode(qa) @ lowp.e4m3_decode(qb)) * np.float64(inv)
    return c, qa, qb, sa, sb, inv
