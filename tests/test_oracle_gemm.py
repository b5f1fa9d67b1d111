"""Pins for the oracle's GEMM and FP8 path (closed forms, brute force, library casts)."""
import numpy as np
import pytest
import torch

import synth
from oracle import gemm, lowp


def _brute(a, b):
    m, k = len(a), len(a[0])
    n = len(b[0])
    return [[sum(int(a[i][t]) * int(b[t][j]) for t in range(k)) for j in range(n)] for i in range(m)]


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (3, 5, 7), (17, 13, 11), (16, 1, 9), (2, 17, 1)])
def test_gemm_brute_force_tiny(m, n, k):
    a = synth.integers(m * k, seed=m, lo=-9, hi=9).reshape(m, k)
    b = synth.integers(k * n, seed=n + 100, lo=-9, hi=9).reshape(k, n)
    assert np.array_equal(gemm.gemm(a, b), np.array(_brute(a, b), dtype=np.float64))


def test_gemm_identity_and_permutation():
    b = synth.uniform(64 * 48, seed=1).reshape(64, 48)
    assert np.array_equal(gemm.gemm(np.eye(64), b), b.astype(np.float64))
    perm = np.array([(7 * i + 3) % 64 for i in range(64)])
    p = np.zeros((64, 64))
    p[np.arange(64), perm] = 1.0
    assert np.array_equal(gemm.gemm(p, b), b[perm].astype(np.float64))


def test_gemm_rank1():
    u = synth.integers(40, seed=2, lo=-5, hi=5)
    v = synth.integers(30, seed=3, lo=-5, hi=5)
    k = 24
    a = np.repeat(u[:, None], k, axis=1)
    b = np.repeat(v[None, :], k, axis=0)
    assert np.array_equal(gemm.gemm(a, b), k * np.outer(u, v).astype(np.float64))


def test_gemm_operand_order():
    a = synth.uniform(12 * 7, seed=4).reshape(12, 7)
    b = synth.uniform(7 * 9, seed=5).reshape(7, 9)
    c = gemm.gemm(a, b)
    assert c.shape == (12, 9)
    assert np.allclose(gemm.gemm(b.T, a.T).T, c, rtol=0, atol=1e-13)
    assert abs(c[3, 4] - sum(float(a[3, t]) * float(b[t, 4]) for t in range(7))) < 1e-13


def test_rel_frobenius():
    c = np.ones((4, 4))
    assert gemm.rel_frobenius(c, c) == 0.0
    assert gemm.rel_frobenius(np.zeros((2, 2)), np.zeros((2, 2))) == 0.0
    assert abs(gemm.rel_frobenius(2 * c, c) - 1.0) < 1e-15


def test_gemm_tiles_equal_full():
    a = synth.uniform(96 * 40, seed=6).reshape(96, 40)
    b = synth.uniform(40 * 80, seed=7).reshape(40, 80)
    full = gemm.gemm(a, b)
    tiles = gemm.gemm_tiles(a, b, [(0, 0), (2, 1), (1, 4)], 32, 16)
    for (tm, tn), t in tiles.items():
        assert np.array_equal(t, full[tm * 32:(tm + 1) * 32, tn * 16:(tn + 1) * 16])


def test_fp8_integer_inputs_exact():
    # integers in [-7, 7] with amax 7 => s = 64, a power of two: every x*s is
    # representable in E4M3 and the dequantised product is exact.
    a = synth.integers(32 * 64, seed=8, lo=-7, hi=7).reshape(32, 64)
    b = synth.integers(64 * 16, seed=9, lo=-7, hi=7).reshape(64, 16)
    a[0, 0], b[0, 0] = 7.0, -7.0
    c, qa, qb, sa, sb, inv = gemm.gemm_fp8(a, b)
    assert sa == 64.0 and sb == 64.0 and inv == np.float32(2.0 ** -12)
    assert np.array_equal(lowp.e4m3_decode(qa), 64.0 * a)
    assert np.array_equal(c, gemm.gemm(a, b))


def test_fp8_identity_scale_448():
    c, qa, qb, sa, sb, inv = gemm.gemm_fp8(np.eye(16), np.eye(16))
    assert sa == 448.0 and np.all(qa[np.eye(16, dtype=bool)] == 0x7E)
    assert np.allclose(c, np.eye(16), rtol=0, atol=1e-6)


def test_fp8_quantize_matches_torch_cast():
    x = synth.normal(100000, seed=10).astype(np.float32)
    s = gemm.fp8_scale(gemm.amax(x))
    assert s == np.float32(448.0) / np.float32(np.max(np.abs(x)))
    q = gemm.fp8_quantize(x, s)
    prod = torch.from_numpy(x) * torch.tensor(float(s), dtype=torch.float32)
    ref = prod.to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(q, ref)
    assert np.max(np.abs(lowp.e4m3_decode(q))) == 448.0


def test_fp8_gemm_error_vs_fp64_within_gate():
    a = synth.normal(128 * 256, seed=20).reshape(128, 256)
    b = synth.normal(256 * 128, seed=21).reshape(256, 128)
    c = gemm.gemm_fp8(a, b)[0]
    assert gemm.rel_frobenius(c, gemm.gemm(a, b)) < 5e-2


def test_fp8_zero_tensor_scale():
    assert gemm.fp8_scale(0.0) == 1.0


def test_sample_tiles_distinct():
    t = synth.sample_tiles(64, 64, 64, seed=0)
    assert len(set(t)) == 64 and all(0 <= a < 64 and 0 <= b < 64 for a, b in t)
    assert t == synth.sample_tiles(64, 64, 64, seed=0)
