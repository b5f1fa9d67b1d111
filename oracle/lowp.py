"""Low-precision formats written from their definitions (oracle; test infrastructure).

bf16: 1 sign bit, 8 exponent bits (bias 127), 7 stored mantissa bits; the same
exponent range as IEEE binary32. Rounding: to nearest, ties to even.

fp8 E4M3 (the OCP 8-bit "E4M3FN" format): 1 sign bit, 4 exponent bits (bias 7),
3 stored mantissa bits, no infinities, NaN only at S.1111.111. Largest finite
magnitude 1.75 * 2^8 = 448, smallest normal 2^-6, subnormal spacing 2^-9.
Conversion used by the per-tensor-scaled GEMM: round to nearest even, then
saturate to +-448 ("satfinite").
"""
from __future__ import annotations

import numpy as np

BF16_MAX = float((2.0 - 2.0 ** -7) * 2.0 ** 127)
E4M3_MAX = 448.0
E4M3_MIN_NORMAL = 2.0 ** -6
E4M3_SUBNORMAL_STEP = 2.0 ** -9


def _quantum(x: np.ndarray, precision_bits: int, emin: int) -> np.ndarray:
    """Spacing of the representable grid around |x| for a binary format with
    `precision_bits` significand bits (including the hidden one) and minimum
    normal exponent `emin` (subnormals share the spacing at emin)."""
    ax = np.abs(x)
    _, e2 = np.frexp(np.where(ax > 0, ax, 1.0))  # ax = m * 2^e2, m in [0.5, 1)
    e = np.maximum(e2 - 1, emin)
    return np.ldexp(1.0, e - (precision_bits - 1))


def round_bf16(x) -> np.ndarray:
    """Round float64 values to the nearest bf16 value (ties to even); overflow
    past the rounding threshold gives +-inf. Returns float64."""
    x = np.asarray(x, dtype=np.float64)
    q = _quantum(x, 8, -126)
    r = np.rint(x / q) * q  # x/q is exact (power-of-two scaling); rint ties to even
    r = np.where(np.abs(r) > BF16_MAX, np.copysign(np.inf, x), r)
    return np.where(np.isfinite(x), r, x)


def round_e4m3_satfinite(x) -> np.ndarray:
    """Round float64 values to E4M3 (nearest, ties to even) and saturate to
    +-448. NaN stays NaN. Returns the E4M3 value as float64."""
    x = np.asarray(x, dtype=np.float64)
    q = _quantum(x, 4, -6)
    r = np.rint(x / q) * q
    r = np.clip(r, -E4M3_MAX, E4M3_MAX)
    return np.where(np.isnan(x), np.nan, r)


def e4m3_decode(codes) -> np.ndarray:
    """Value of each E4M3 byte (uint8) as float64 from the bit-field definition."""
    c = np.asarray(codes, dtype=np.uint8).astype(np.int64)
    s = np.where(c & 0x80, -1.0, 1.0)
    e = (c >> 3) & 0xF
    m = c & 0x7
    val = np.where(e == 0, m * 2.0 ** -9, (1.0 + m / 8.0) * np.ldexp(1.0, e - 7))
    val = np.where((e == 15) & (m == 7), np.nan, val)
    return s * val


def e4m3_encode(x) -> np.ndarray:
    """E4M3 byte of each float64 value that is already exactly representable
    (use round_e4m3_satfinite first). -0.0 encodes as 0x80."""
    x = np.asarray(x, dtype=np.float64)
    sign = np.where(np.signbit(x), 0x80, 0)
    ax = np.abs(x)
    sub = ax < E4M3_MIN_NORMAL
    _, e2 = np.frexp(np.where(ax > 0, ax, 1.0))
    e = e2 - 1
    mant_norm = np.rint((ax / np.ldexp(1.0, e) - 1.0) * 8.0)
    code_norm = ((e + 7) << 3) + mant_norm.astype(np.int64)
    code_sub = np.rint(ax / 2.0 ** -9).astype(np.int64)
    code = np.where(sub, code_sub, code_norm)
    code = np.where(np.isnan(x), 0x7F, code)
    return (code | sign).astype(np.uint8)


def bf16_bits_to_f64(bits) -> np.ndarray:
    """Value of each bf16 bit pattern (uint16) as float64 (exact widening)."""
    b = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << np.uint32(16)
    return b.view(np.float32).astype(np.float64)
