"""Pins for the oracle's element-wise maps (closed forms, identities, library GELU)."""
import math
from fractions import Fraction

import numpy as np
import torch

import synth
from oracle import maps


def test_axpy_closed_forms():
    x = synth.normal(4096, seed=1)
    y = synth.normal(4096, seed=2)
    assert np.array_equal(maps.axpy(0.0, x, y), y.astype(np.float64))   # x*0 + b
    assert np.array_equal(maps.axpy(1.0, x, np.zeros_like(y)), x.astype(np.float64))
    assert np.array_equal(maps.axpy(-1.0, x, x), np.zeros(4096))


def test_axpy_exact_rationals():
    x = synth.integers(257, seed=5, lo=-1000, hi=1000)
    y = synth.integers(257, seed=6, lo=-1000, hi=1000)
    alpha = 0.5
    z = maps.axpy(alpha, x, y)
    for i in range(257):
        assert Fraction(z[i]) == Fraction(1, 2) * Fraction(int(x[i])) + Fraction(int(y[i]))


def test_gelu_landmarks_and_odd_identity():
    assert maps.gelu_tanh(0.0) == 0.0
    x = synth.normal(10000, seed=7, std=3.0, dtype=np.float64)
    # tanh is odd => gelu(-x) = gelu(x) - x
    assert np.allclose(maps.gelu_tanh(-x), maps.gelu_tanh(x) - x, rtol=0, atol=1e-12)
    assert abs(maps.gelu_tanh(20.0) - 20.0) < 1e-12
    assert abs(maps.gelu_tanh(-20.0)) < 1e-12
    w = synth.normal(10000, seed=8)
    assert np.array_equal(maps.gelu_mul(x, np.zeros_like(w)), np.zeros(10000))


def test_gelu_matches_torch_tanh_gelu():
    x = synth.normal(100000, seed=9, std=4.0, dtype=np.float64)
    ref = torch.nn.functional.gelu(torch.from_numpy(x), approximate="tanh").numpy()
    assert np.max(np.abs(maps.gelu_tanh(x) - ref)) < 1e-14


def test_gelu_tanh_approximates_erf_gelu():
    # The tanh form approximates x * Phi(x) to about 1e-3 everywhere; a wrong
    # constant (sqrt(2/pi) or 0.044715) would break this bound.
    xs = np.linspace(-8, 8, 4001)
    exact = np.array([0.5 * v * (1.0 + math.erf(v / math.sqrt(2.0))) for v in xs])
    assert np.max(np.abs(maps.gelu_tanh(xs) - exact)) < 1e-3


def test_scale_and_add_accum():
    a = synth.integers(100, seed=1, lo=-50, hi=50)
    b = synth.integers(100, seed=2, lo=-50, hi=50)
    c = synth.integers(100, seed=3, lo=-50, hi=50)
    assert np.array_equal(maps.add_accum(c, a, b), (c.astype(int) + a.astype(int) + b.astype(int)).astype(float))
    assert np.array_equal(maps.scale(a, np.ones(100)), a.astype(float))
