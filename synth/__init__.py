"""Seeded synthetic input generators shared by the oracle and the CUDA path.

This module holds no arithmetic of the method itself: it only draws numbers.
Every draw is a pure function of (seed, element index) through the
counter-based SplitMix64 generator (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), so the same call gives the same
values on x86 and on Arm, in any chunking.

* uniform01: the top 53 bits of SplitMix64(seed, i) scaled by 2^-53.
* normal:    Box-Muller, z = sqrt(-2 ln(1-u1)) * cos(2 pi u2), with u1 from
             counter 2i and u2 from counter 2i+1.
* bf16:      the fp32 draw rounded to nearest-even by torch's own cast (an
             input-preparation step; the method's own roundings live in the
             kernels and, independently, in the oracle).
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_SEEDMIX = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def splitmix64(counter: np.ndarray, seed: int) -> np.ndarray:
    """SplitMix64 output for each uint64 counter value under `seed`."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _SEEDMIX + (counter + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _u01(counter: np.ndarray, seed: int) -> np.ndarray:
    return (splitmix64(counter, seed) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _chunked(n: int, fn, dtype) -> np.ndarray:
    out = np.empty(n, dtype=dtype)
    starts = list(range(0, n, _CHUNK))

    def work(s):
        e = min(n, s + _CHUNK)
        out[s:e] = fn(np.arange(s, e, dtype=np.uint64))

    if len(starts) <= 1:
        for s in starts:
            work(s)
    else:
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(work, starts))
    return out


def uniform(n: int, seed: int, lo: float = -1.0, hi: float = 1.0, dtype=np.float32) -> np.ndarray:
    """n draws from U[lo, hi), rounded to `dtype`."""
    return _chunked(n, lambda c: lo + (hi - lo) * _u01(c, seed), dtype)


def normal(n: int, seed: int, mean: float = 0.0, std: float = 1.0, dtype=np.float32) -> np.ndarray:
    """n draws from N(mean, std^2) by Box-Muller, rounded to `dtype`."""
    two = np.uint64(2)

    def fn(c):
        u1 = _u01(c * two, seed)
        u2 = _u01(c * two + np.uint64(1), seed)
        r = np.sqrt(-2.0 * np.log1p(-u1))
        return mean + std * (r * np.cos(2.0 * math.pi * u2))

    return _chunked(n, fn, dtype)


def to_bf16(a: np.ndarray):
    """fp32 array -> torch.bfloat16 CPU tensor (round to nearest even)."""
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)


def tensor(a: np.ndarray, dtype: str = "f32"):
    """numpy fp32 draw -> torch CPU tensor in 'f32' or 'bf16'."""
    import torch

    if dtype == "f32":
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    if dtype == "bf16":
        return to_bf16(a)
    raise ValueError(dtype)


def integers(n: int, seed: int, lo: int, hi: int) -> np.ndarray:
    """n integers uniform on [lo, hi] inclusive (as float32; exact for |v| < 2^24)."""
    span = hi - lo + 1
    return _chunked(n, lambda c: lo + np.floor(_u01(c, seed) * span), np.float32)


def grouped_problems(count: int = 64, seed: int = 0, kn_pairs=None, m_max: int = 4096):
    """Group of GEMM problem shapes (M, N, K).

    M = clamp(round(2^(log2(m_max) * U)), 1, m_max) with U ~ U[0,1) (log-uniform on
    [1, m_max]); (K, N) is drawn uniformly from `kn_pairs`. Draw j uses counters
    2j (for M) and 2j+1 (for the pair index).
    """
    if kn_pairs is None:
        kn_pairs = [(2560, 9728), (5120, 25600), (25600, 5120), (5120, 10240)]
    c = np.arange(count, dtype=np.uint64)
    u = _u01(c * np.uint64(2), seed)
    v = _u01(c * np.uint64(2) + np.uint64(1), seed)
    lg = math.log2(m_max)
    probs = []
    for j in range(count):
        m = int(min(m_max, max(1, round(2.0 ** (lg * u[j])))))
        k, n = kn_pairs[min(len(kn_pairs) - 1, int(v[j] * len(kn_pairs)))]
        probs.append((m, n, k))
    return probs


def log_uniform_shapes(count: int, seed: int, lo: int = 1, hi: int = 16384):
    """`count` (M, N, K) triples, each log-uniform on [lo, hi] (integer, rounded)."""
    c = np.arange(3 * count, dtype=np.uint64)
    u = _u01(c, seed).reshape(count, 3)
    a, b = math.log2(lo), math.log2(hi)
    v = np.clip(np.rint(2.0 ** (a + (b - a) * u)), lo, hi).astype(np.int64)
    return [tuple(int(x) for x in row) for row in v]


def sample_tiles(grid_m: int, grid_n: int, count: int, seed: int = 0):
    """`count` distinct tile coordinates from a grid_m x grid_n grid.

    Partial Fisher-Yates over the row-major flattened grid; draw i picks
    j = i + floor(u_i * (total - i)) with u_i = uniform01(seed, i).
    Returns [(tm, tn), ...] in draw order."""
    total = grid_m * grid_n
    count = min(count, total)
    perm = np.arange(total, dtype=np.int64)
    u = _u01(np.arange(count, dtype=np.uint64), seed)
    for i in range(count):
        j = i + int(u[i] * (total - i))
        perm[i], perm[j] = perm[j], perm[i]
    return [(int(t // grid_n), int(t % grid_n)) for t in perm[:count]]
