"""The seeded input generators (no GPU): SplitMix64 against its published
output sequence, draws as pure functions of (seed, index), and the moments
and ranges of the distributions the workloads use."""
import numpy as np

import synth


def test_splitmix64_published_sequence():
    # state 0 (seed 0 here), the generator's first three outputs
    v = synth.splitmix64(np.arange(3, dtype=np.uint64), 0)
    assert [int(x) for x in v] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_draws_depend_only_on_seed_and_index():
    n = (1 << 22) + 1000                       # spans two chunks of the threaded path
    a = synth.normal(n, seed=5)
    assert np.array_equal(a[:777], synth.normal(777, seed=5))
    assert np.array_equal(a, synth.normal(n, seed=5))
    assert not np.array_equal(a[:777], synth.normal(777, seed=6))
    u = synth.uniform(n, seed=3, lo=0.0, hi=1.0, dtype=np.float64)
    assert np.array_equal(u[-1000:], 0.0 + synth._u01(np.arange(n - 1000, n, dtype=np.uint64), 3))


def test_moments_and_ranges():
    x = synth.normal(1 << 20, seed=1, dtype=np.float64)
    assert abs(x.mean()) < 5e-3 and abs(x.std() - 1.0) < 5e-3
    assert abs((x ** 3).mean()) < 1e-2 and abs((x ** 4).mean() - 3.0) < 3e-2    # symmetric, normal kurtosis
    u = synth.uniform(1 << 20, seed=2, lo=-1.0, hi=1.0, dtype=np.float64)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 5e-3 and abs(u.var() - 1.0 / 3.0) < 5e-3
    k = synth.integers(1 << 16, seed=4, lo=-4, hi=4)
    assert set(np.unique(k).tolist()) == set(range(-4, 5))
    assert all(abs((k == v).mean() - 1.0 / 9.0) < 0.01 for v in range(-4, 5))


def test_shape_samplers():
    shapes = synth.log_uniform_shapes(4000, seed=1)
    m = np.array([s[0] for s in shapes])
    assert m.min() >= 1 and m.max() <= 16384
    assert abs(np.mean(np.log2(m)) - 7.0) < 0.2          # log-uniform on [1, 2^14]: mean log2 = 7
    probs = synth.grouped_problems(64, seed=0)
    assert len(probs) == 64 and all(1 <= m <= 4096 for m, _, _ in probs)
    assert {(k, n) for _, n, k in probs} <= {(2560, 9728), (5120, 25600), (25600, 5120), (5120, 10240)}
    tiles = synth.sample_tiles(64, 64, 64, seed=0)
    assert len(set(tiles)) == 64 and all(0 <= a < 64 and 0 <= b < 64 for a, b in tiles)
    assert synth.sample_tiles(2, 3, 10, seed=1) and len(synth.sample_tiles(2, 3, 10, seed=1)) == 6
