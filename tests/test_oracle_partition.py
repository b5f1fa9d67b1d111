"""Pins for the oracle's partitions and write-count checker (paper examples, hand-built maps)."""
import os

import itertools

import numpy as np
import pytest

from oracle import grouped, partition

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = int(v)
    return vals


def test_listing1_worked_example():
    g = _golden("listing1_vec_add.txt")
    grid = partition.grid((g["n"],), (g["tile"],))
    assert grid == (g["programs"],)
    owner = partition.owner_map((g["n"],), (g["tile"],))
    assert np.array_equal(owner, np.arange(g["n"]) // g["tile"])
    assert partition.check_counts(np.bincount(np.arange(g["n"]), minlength=g["n"]))["ok"]


def test_grid_ragged_and_rejections():
    assert partition.grid((10,), (4,)) == (3,)
    assert list(partition.tile_elements((10,), (4,), (2,))) == [8, 9]
    assert partition.grid((5, 7, 3), (2, 3, 3)) == (3, 3, 1)
    with pytest.raises(ValueError):
        partition.grid((2, 2, 2, 2), (1, 1, 1, 1))
    with pytest.raises(ValueError):
        partition.grid((8,), (0,))
    with pytest.raises(ValueError):
        partition.grid((8, 8), (4,))
    assert partition.grid((0,), (4,)) == (0,)


def test_tile_elements_2d():
    e = partition.tile_elements((5, 7), (2, 3), (2, 2))
    assert list(e) == [4 * 7 + 6]   # ragged corner tile of a 5x7 output


@pytest.mark.parametrize("shape,tile", [((1000,), (64,)), ((13, 29), (4, 8)), ((5, 6, 7), (2, 4, 3))])
@pytest.mark.parametrize("kind,P", [("identity", None), ("strided", 3)])
def test_owner_map_covers_exactly_once(shape, tile, kind, P):
    owner = partition.owner_map(shape, tile, P, kind)
    assert np.all(owner >= 0)
    n = int(np.prod(shape))
    g = partition.grid(shape, tile)
    writes = []
    for p, slots in partition.program_tiles(int(np.prod(g)), P, kind).items():
        for s in slots:
            writes += [(p, int(e)) for e in partition.tile_elements(shape, tile, partition.tile_coord(s, g))]
    assert len(writes) == n
    assert partition.check_counts(partition.write_counts(n, writes))["ok"]


def test_strided_program_count_validation():
    with pytest.raises(ValueError):
        partition.program_tiles(8, 9, "strided")
    with pytest.raises(ValueError):
        partition.program_tiles(8, 0, "strided")
    assert partition.program_tiles(8, 3, "strided") == {0: [0, 3, 6], 1: [1, 4, 7], 2: [2, 5]}


def test_checker_flags_hand_built_maps():
    shape, tile = (12,), (4,)
    good = partition.writes_of_map(shape, tile, {0: [0], 1: [1], 2: [2]})
    assert partition.check_counts(partition.write_counts(12, good))["ok"]
    missing = partition.writes_of_map(shape, tile, {0: [0], 1: [2]})
    r = partition.check_counts(partition.write_counts(12, missing))
    assert not r["ok"] and list(r["missing"]) == [4, 5, 6, 7] and r["duplicate"].size == 0
    dup = partition.writes_of_map(shape, tile, {0: [0, 1], 1: [1], 2: [2]})
    r = partition.check_counts(partition.write_counts(12, dup))
    assert list(r["duplicate"]) == [4, 5, 6, 7] and r["missing"].size == 0


def test_permute_heads_race_is_flagged():
    g = _golden("permute_heads_race.txt")
    B, H, M, D = g["B"], g["H"], g["M"], g["D"]
    writes = partition.permute_heads_writes(B, H, M, D, g["BM"], g["BD"])
    counts = partition.write_counts(B * H * M * D, writes)
    assert np.all(counts == g["writes_per_element"])
    r = partition.check_counts(counts)
    assert not r["ok"] and r["duplicate"].size == B * H * M * D
    # the programs writing one destination differ only in h1
    e0 = [p for p, e in writes if e == 0]
    assert sorted(e0) == sorted(h1 * H + 0 for h1 in range(H))


def test_gemm_cut_schedule_worked_example():
    # 7 tiles of 64 columns on 5 programs: one whole round (tiles 0..4), and
    # the 2 remaining tiles cut into 2 narrow tiles of 32 columns: slots 5, 6
    # = tile 5 columns [0, 32), [32, 64) and slots 7, 8 = tile 6, run by
    # programs 0, 1, 2, 3 (program 4 idles in the last round)
    assert partition.gemm_cut_schedule(7, 5, 64, 32) == (5, 2)
    own = partition.gemm_owner_map_cut(16, 7 * 64, 16, 64, 5).reshape(16, 7 * 64)
    assert [int(own[0, c]) for c in range(0, 7 * 64, 32)] == [0, 0, 1, 1, 2, 2, 3, 3, 4, 4, 0, 1, 2, 3]


@pytest.mark.parametrize("T,P,bn,unit,limit,expect", [(5, 3, 64, 32, 4, (5, 1)),     # P // R = 1: nothing cut
                                                       (10, 3, 128, 32, 4, (9, 2)),   # 3 parts is no power of 2
                                                       (11, 5, 128, 32, 4, (10, 4)),
                                                       (11, 5, 128, 64, 4, (10, 2)),  # 64-column narrow tiles
                                                       (11, 5, 64, 64, 4, (11, 1)),
                                                       (11, 5, 128, 32, 1, (11, 1)),  # cutting disabled
                                                       (1024, 76, 256, 64, 4, (988, 2)),
                                                       (12, 4, 128, 32, 4, (12, 1))]) # no partial round
def test_gemm_cut_schedule_cases(T, P, bn, unit, limit, expect):
    assert partition.gemm_cut_schedule(T, P, bn, unit, limit) == expect


@pytest.mark.parametrize("m,n,bm,bn,P,G", [(300, 200, 32, 64, 9, 2), (1024, 640, 128, 64, 13, 1),
                                           (1024, 640, 256, 64, 13, 3), (96, 96, 32, 32, 4, 1)])
def test_gemm_owner_map_cut_partitions_the_output(m, n, bm, bn, P, G):
    own = partition.gemm_owner_map_cut(m, n, bm, bn, P, G)
    assert own.min() >= 0 and own.max() < P            # every element owned by a program
    no_cut = partition.gemm_owner_map_cut(m, n, bm, bn, P, G, limit=1)
    assert np.array_equal(no_cut, partition.gemm_owner_map(m, n, bm, bn, P, "strided", G))
    # whole tiles keep their strided owner; only the last round's tiles change
    gm, gn = -(-m // bm), -(-n // bn)
    D, S = partition.gemm_cut_schedule(gm * gn, P, bn, 64 if bm == 256 else 32)
    diff = own.reshape(m, n) != no_cut.reshape(m, n)
    for s in range(D):
        tm, tn = partition.raster_tile(s, gm, gn, G)
        assert not diff[tm * bm:(tm + 1) * bm, tn * bn:(tn + 1) * bn].any()


def test_permute_heads_worked_example():
    # B=1, H=2, M=4, BM=2, D=1: heads [0 1 2 3] and [4 5 6 7]. Destination head
    # m holds, for each source head h, source head h's sequence tile m.
    src = np.arange(8, dtype=np.float64).reshape(1, 2, 4, 1)
    dst = partition.permute_heads(src, 2)
    assert dst[0, :, :, 0].tolist() == [[0, 1, 4, 5], [2, 3, 6, 7]]


def test_permute_heads_is_an_involution_and_a_permutation():
    # swapping the head index with the sequence-tile index twice is the identity
    src = np.arange(2 * 3 * 6 * 4, dtype=np.float64).reshape(2, 3, 6, 4)
    dst = partition.permute_heads(src, 2)
    assert sorted(dst.reshape(-1)) == sorted(src.reshape(-1))
    assert not np.array_equal(dst, src)
    assert np.array_equal(partition.permute_heads(dst, 2), src)
    # element-wise definition on every index
    for b, m, r, d in itertools.product(range(2), range(3), range(6), range(4)):
        h, i = divmod(r, 2)
        assert dst[b, m, r, d] == src[b, h, m * 2 + i, d]


def test_permute_heads_race_candidates():
    src = np.arange(2 * 3 * 6 * 4, dtype=np.float64).reshape(2, 3, 6, 4)
    cand = partition.permute_heads_race_candidates(src, 2)
    good = partition.permute_heads(src, 2)
    # the correct value is among the racing candidates (candidate h1 == h2)
    assert np.any(cand == good[None], axis=0).all()
    # each destination element has H distinct candidates, one per source head
    assert all(len(set(cand[:, 0, 1, r, 2])) == 3 for r in range(6))
    # candidates of one element come from the H heads of the same sequence tile
    assert sorted(cand[:, 1, 2, 3, 1]) == sorted(src[1, h1, 2 * 2 + 1, 1] for h1 in range(3))


@pytest.mark.parametrize("gm,gn,G", [(1, 1, 1), (7, 5, 1), (7, 5, 3), (16, 16, 8), (5, 9, 16)])
def test_raster_bijection(gm, gn, G):
    seen = {partition.raster_tile(s, gm, gn, G) for s in range(gm * gn)}
    assert seen == {(i, j) for i in range(gm) for j in range(gn)}
    if G == 1:
        assert [partition.raster_tile(s, gm, gn, 1) for s in range(gm * gn)] == \
               [(i, j) for i in range(gm) for j in range(gn)]


def test_raster_band_order():
    # 4x3 grid, bands of 2 rows: first slots go down the band's rows
    assert [partition.raster_tile(s, 4, 3, 2) for s in range(6)] == \
        [(0, 0), (1, 0), (0, 1), (1, 1), (0, 2), (1, 2)]


def test_gemm_owner_map_strided():
    owner = partition.gemm_owner_map(300, 200, 128, 64, num_programs=5, kind="strided", group_m=2)
    gm, gn = 3, 4
    o = owner.reshape(300, 200)
    for s in range(gm * gn):
        tm, tn = partition.raster_tile(s, gm, gn, 2)
        assert np.all(o[tm * 128:(tm + 1) * 128, tn * 64:(tn + 1) * 64] == s % 5)


def test_grouped_queue_coverage():
    probs = [(1, 300, 64), (200, 96, 64), (65, 129, 64)]
    cfg = [(128, 16, True), (128, 64, False), (64, 32, False)]
    tc = [grouped.problem_tiles(m, n, *c)[0] for (m, n, _), c in zip(probs, cfg)]
    total = sum(tc)
    counts = grouped.element_counts(probs, cfg, range(total))
    assert all(np.all(c == 1) for c in counts)
    counts = grouped.element_counts(probs, cfg, [g for g in range(total) if g != 3])
    assert not all(np.all(c == 1) for c in counts)
    assert [grouped.queue_decode(g, tc)[0] for g in range(total)] == \
        [i for i, t in enumerate(tc) for _ in range(t)]
    with pytest.raises(ValueError):
        grouped.queue_decode(total, tc)


@pytest.mark.parametrize("T", [1, 5, 7, 33, 76, 100, 1024])
@pytest.mark.parametrize("P", [1, 3, 4, 13, 76, 152])
@pytest.mark.parametrize("bn,unit", [(64, 32), (128, 32), (256, 64), (192, 32)])
def test_gemm_cut_schedule_properties(T, P, bn, unit):
    """The cut schedule from its properties rather than its loop: whole tiles
    first (one per program per round), then each of the R = T mod P tiles of
    the partial round split into S narrow tiles with S a power of two, at
    most the limit, no more narrow tiles than programs (R S <= P), each of a
    whole number of units; and S is the largest such choice (doubling it
    breaks one of these), S = 1 meaning nothing is cut."""
    limit = 4
    D, S = partition.gemm_cut_schedule(T, P, bn, unit, limit)
    R = T % P
    assert S >= 1 and S & (S - 1) == 0 and S <= limit
    if S == 1:
        assert D == T
    else:
        assert D == T - R and R * S <= P and (bn // S) % unit == 0 and bn % S == 0
    feasible = lambda s: R > 0 and s <= limit and R * s <= P and bn % (s * unit) == 0
    assert not feasible(2 * S)
    # every slot of the schedule maps to a distinct (tile, column range) and
    # the ranges of each tile cover its columns exactly once
    cover = {}
    slots = D + (T - D) * S
    for s in range(slots):
        if s < D:
            cover.setdefault(s, []).append((0, bn))
        else:
            tile, j = D + (s - D) // S, (s - D) % S
            cover.setdefault(tile, []).append((j * bn // S, (j + 1) * bn // S))
    assert sorted(cover) == list(range(T))
    for ranges in cover.values():
        ranges.sort()
        assert ranges[0][0] == 0 and ranges[-1][1] == bn
        assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
    # the last round gives no program more than one narrow tile more than another
    per_prog = np.zeros(P, dtype=np.int64)
    for s in range(D, slots):
        per_prog[s % P] += 1
    assert per_prog.max() - per_prog.min() <= 1
