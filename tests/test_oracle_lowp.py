"""Pins for the oracle's bf16 / E4M3 rounding (format definitions, library casts)."""
import numpy as np
import pytest
import torch

import synth
from oracle import lowp


def test_e4m3_code_table_landmarks():
    codes = np.arange(256, dtype=np.uint8)
    v = lowp.e4m3_decode(codes)
    assert np.isnan(v[0x7F]) and np.isnan(v[0xFF])
    assert np.sum(np.isfinite(v)) == 254
    assert v[0x7E] == 448.0 and v[0xFE] == -448.0
    assert v[0x01] == 2.0 ** -9
    assert v[0x08] == 2.0 ** -6
    assert v[0x38] == 1.0  # exponent field 7 = bias
    assert v[0x00] == 0.0 and np.signbit(v[0x80])
    # positive codes are strictly increasing in value (sign-magnitude layout)
    assert np.all(np.diff(v[0x00:0x7F]) > 0)


def test_e4m3_encode_roundtrip_all_finite_codes():
    codes = np.array([c for c in range(256) if c not in (0x7F, 0xFF)], dtype=np.uint8)
    back = lowp.e4m3_encode(lowp.e4m3_decode(codes))
    assert np.array_equal(back, codes)


def test_e4m3_rounding_ties_and_saturation():
    r = lowp.round_e4m3_satfinite
    assert r(1.0625) == 1.0          # tie between 1.0 (even) and 1.125
    assert r(1.1875) == 1.25         # tie between 1.125 and 1.25 (even)
    assert r(1000.0) == 448.0 and r(-1e9) == -448.0
    assert r(464.0) == 448.0
    assert r(2.0 ** -10) == 0.0      # half of the smallest subnormal: tie to even 0
    assert r(3 * 2.0 ** -10) == 2.0 ** -8
    assert np.isnan(r(np.nan))


def test_e4m3_matches_torch_cast():
    x = synth.normal(200000, seed=11, std=60.0, dtype=np.float64)
    x = np.clip(x, -448.0, 448.0)
    x = np.concatenate([x, synth.normal(50000, seed=12, std=0.01, dtype=np.float64)])
    x32 = x.astype(np.float32)
    ours = lowp.round_e4m3_satfinite(x32.astype(np.float64))
    ref = torch.from_numpy(x32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)


def test_bf16_ties_and_landmarks():
    r = lowp.round_bf16
    assert r(1.0 + 2.0 ** -8) == 1.0
    assert r(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert r(lowp.BF16_MAX) == lowp.BF16_MAX
    assert np.isinf(r(3.5e38))
    assert r(2.0 ** -133) == 2.0 ** -133   # smallest bf16 subnormal


@pytest.mark.parametrize("std", [1.0, 1e-20, 1e-39, 1e30])
def test_bf16_matches_torch_cast(std):
    x32 = synth.normal(100000, seed=13, std=std, dtype=np.float64).astype(np.float32)
    ours = lowp.round_bf16(x32.astype(np.float64))
    ref = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)


def test_bf16_bits_widening():
    t = synth.to_bf16(synth.normal(1000, seed=3))
    bits = t.view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(lowp.bf16_bits_to_f64(bits), t.double().numpy())
