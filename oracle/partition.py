"""Partitions of a mutable output and the write-count checker (oracle).

Definitions followed (§3.4 Partitioning and Ordering, §3.6 Mapped Partitions,
Appendix A):

* A partition of an output of shape S (rank r <= 3, the CUDA grid being
  three-dimensional) into sub-tensors of shape T has the grid
  G_d = ceil(S_d / T_d). Sub-tensor t covers the elements e with
  t_d T_d <= e_d < min((t_d + 1) T_d, S_d) (the last tile of an axis is ragged).
* Plain partition: one tile program per sub-tensor. Program ids and tile ids are
  the row-major linear index over the grid (last axis fastest), and program
  p owns tile p.
* Mapped partition: P programs (P <= number of tiles), program p owning the
  bounded sequence of tiles given by the partition map. Two maps are defined:
  'strided' (program p owns schedule slots p, p + P, p + 2P, ...) and 'queue'
  (a shared counter hands out each slot once, so ownership is decided at run
  time). For a GEMM output the schedule slot s is turned into a tile (tm, tn)
  by the raster function below.
* Data-race freedom (Appendix A) needs every output element to be written by
  exactly one program; the checker counts writes per element and reports every
  element whose count differs from one.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def grid(shape, tile):
    """Partition grid: ceil(S_d / T_d) per axis. Raises on rank > 3 or a bad tile."""
    shape = tuple(int(s) for s in shape)
    tile = tuple(int(t) for t in tile)
    if len(shape) != len(tile):
        raise ValueError("tile rank differs from tensor rank")
    if not 1 <= len(shape) <= 3:
        raise ValueError("a mutable partition has rank 1..3")
    if any(t <= 0 for t in tile) or any(s < 0 for s in shape):
        raise ValueError("tile extents must be positive")
    return tuple(-(-s // t) for s, t in zip(shape, tile))


def num_tiles(shape, tile) -> int:
    return int(np.prod(grid(shape, tile), dtype=np.int64))


def tile_coord(linear: int, g):
    """Row-major (last axis fastest) coordinate of tile `linear` in grid g."""
    coord = []
    for extent in reversed(g):
        coord.append(linear % extent)
        linear //= extent
    return tuple(reversed(coord))


def tile_elements(shape, tile, coord) -> np.ndarray:
    """Flat row-major indices of the output elements covered by tile `coord`."""
    ranges = []
    for s, t, c in zip(shape, tile, coord):
        lo = c * t
        ranges.append(range(lo, min(lo + t, s)))
    strides = [int(np.prod(shape[d + 1:], dtype=np.int64)) for d in range(len(shape))]
    return np.array([sum(i * st for i, st in zip(idx, strides))
                     for idx in itertools.product(*ranges)], dtype=np.int64)


def raster_tile(s: int, gm: int, gn: int, group_m: int):
    """GEMM schedule slot s -> output tile (tm, tn).

    Slots run through bands of `group_m` tile rows; inside a band they go down
    the band's rows first, then to the next tile column. group_m = 1 is plain
    row-major order. The map is a bijection of [0, gm*gn) onto the grid."""
    per_band = group_m * gn
    band = s // per_band
    first = band * group_m
    rows = min(group_m, gm - first)
    r = s % per_band
    return first + r % rows, r // rows


def program_tiles(n_tiles: int, num_programs: int | None = None, kind: str = "identity"):
    """Schedule slots owned by each program: {p: [slots]}."""
    if kind == "identity":
        return {p: [p] for p in range(n_tiles)}
    if kind == "strided":
        if num_programs is None or num_programs <= 0:
            raise ValueError("a mapped partition needs a positive program count")
        if num_programs > max(n_tiles, 1):
            raise ValueError("more programs than tiles in the partition grid")
        return {p: list(range(p, n_tiles, num_programs)) for p in range(num_programs)}
    raise ValueError(kind)


def owner_map(shape, tile, num_programs=None, kind="identity") -> np.ndarray:
    """Program id that must write each output element (flat, row-major).

    Built by enumerating each program's tiles and their elements, independent
    of any kernel's index arithmetic."""
    g = grid(shape, tile)
    n = int(np.prod(shape, dtype=np.int64))
    owner = np.full(n, -1, dtype=np.int64)
    for p, slots in program_tiles(int(np.prod(g, dtype=np.int64)), num_programs, kind).items():
        for s in slots:
            owner[tile_elements(shape, tile, tile_coord(s, g))] = p
    return owner


def gemm_owner_map(m: int, n: int, bm: int, bn: int, num_programs=None,
                   kind="identity", group_m: int = 1) -> np.ndarray:
    """Program id per element of an M x N GEMM output with BM x BN tiles under
    the given map; slots become tiles through raster_tile."""
    gm, gn = -(-m // bm), -(-n // bn)
    owner = np.full((m, n), -1, dtype=np.int64)
    for p, slots in program_tiles(gm * gn, num_programs, kind).items():
        for s in slots:
            tm, tn = raster_tile(s, gm, gn, group_m)
            owner[tm * bm:(tm + 1) * bm, tn * bn:(tn + 1) * bn] = p
    return owner.reshape(-1)


def gemm_cut_schedule(tiles: int, programs: int, bn: int, unit: int, limit: int = 4):
    """The GEMM schedule on a strided map with the last round cut along N.
    With P programs and T tiles of BN columns, the first T - R slots
    (R = T mod P) are whole tiles, slot = tile index. When R > 0 each of the
    R remaining tiles is cut into S narrow tiles of BN / S columns, S the
    largest power of two with S <= limit, S <= P // R and BN / S a multiple
    of `unit` (nothing is cut when that S is 1): narrow tile j of remaining
    tile r is slot (T - R) + r * S + j and covers columns [j BN/S, (j+1) BN/S)
    of it. Program p runs slots p, p + P, ... Returns (whole_slots, S)."""
    R = tiles % programs
    S = 1
    while R > 0 and 2 * S <= limit and 2 * S <= programs // R and bn % (2 * S * unit) == 0:
        S *= 2
    return (tiles - R, S) if S >= 2 else (tiles, 1)


def gemm_owner_map_cut(m: int, n: int, bm: int, bn: int, programs: int, group_m: int = 1,
                       limit: int = 4) -> np.ndarray:
    """Program id per element of an M x N output under the strided map with
    the last round cut along N (narrow tiles keep 64-column multiples for
    256-row tiles, 32 otherwise); slots become tiles through raster_tile."""
    gm, gn = -(-m // bm), -(-n // bn)
    T = gm * gn
    D, S = gemm_cut_schedule(T, programs, bn, 64 if bm == 256 else 32, limit)
    owner = np.full((m, n), -1, dtype=np.int64)
    w = bn // S
    for s in range(D + (T - D) * S):
        if s < D:
            tile, c0, c1 = s, 0, bn
        else:
            tile, j = D + (s - D) // S, (s - D) % S
            c0, c1 = j * w, (j + 1) * w
        tm, tn = raster_tile(tile, gm, gn, group_m)
        owner[tm * bm:(tm + 1) * bm, tn * bn + c0:tn * bn + c1] = s % programs
    return owner.reshape(-1)


def write_counts(n_elements: int, writes) -> np.ndarray:
    """Count per element from an iterable of (program, flat element index)."""
    counts = np.zeros(n_elements, dtype=np.int64)
    for _, idx in writes:
        counts[idx] += 1
    return counts


def check_counts(counts) -> dict:
    """Every element must be written exactly once (Appendix A). Returns
    {'ok', 'missing': indices with 0 writes, 'duplicate': indices with > 1}."""
    c = np.asarray(counts).reshape(-1)
    missing = np.nonzero(c == 0)[0]
    dup = np.nonzero(c > 1)[0]
    return {"ok": missing.size == 0 and dup.size == 0, "missing": missing, "duplicate": dup}


def writes_of_map(shape, tile, assignment) -> list:
    """(program, element) writes of an explicit program -> [tile ids] assignment
    (used to build hand-made correct, missing and duplicate maps)."""
    g = grid(shape, tile)
    out = []
    for p, tiles in assignment.items():
        for t in tiles:
            for e in tile_elements(shape, tile, tile_coord(t, g)):
                out.append((p, int(e)))
    return out


def permute_heads_writes(B: int, H: int, M: int, D: int, BM: int, BD: int) -> list:
    """(program, flat dst element) writes of the index-swapped head permutation
    of §3.5, Listing 5: grid (B*H, H, 1); program (bh1, h2) with b = bh1 // H,
    h1 = bh1 % H loops m over the M/BM source tiles and stores its
    (1, 1, BM, BD) tile at destination tile index (b, m, h2, 0), the m and h2
    indices swapped. dst has shape (B, H, M, D), so the swapped store needs
    M/BM == H to stay in bounds; each destination tile is then written by the
    H programs that differ only in h1."""
    if M % BM or D != BD or M // BM != H:
        raise ValueError("this demo needs M/BM == H and BD == D")
    writes = []
    for bh1 in range(B * H):
        for h2 in range(H):
            prog = bh1 * H + h2
            b = bh1 // H
            for m in range(M // BM):
                # destination tile (b, m, h2, 0) of shape (1, 1, BM, BD)
                for i in range(BM):
                    for d in range(BD):
                        e = ((b * H + m) * M + h2 * BM + i) * D + d
                        writes.append((prog, e))
    return writes


def permute_heads(src, BM: int) -> np.ndarray:
    """The head permutation that Listing 5 means to compute (§3.5), written
    tile by tile: src has shape (B, H, M, D) with M/BM == H, and destination
    tile (b, m, h) of shape (BM, D) is source tile (b, h, m), i.e.
    dst[b, m, h*BM + i, :] = src[b, h, m*BM + i, :]."""
    src = np.asarray(src)
    B, H, M, D = src.shape
    if M % BM or M // BM != H:
        raise ValueError("needs M/BM == H")
    dst = np.empty_like(src)
    for b in range(B):
        for m in range(H):
            for h in range(H):
                dst[b, m, h * BM:(h + 1) * BM, :] = src[b, h, m * BM:(m + 1) * BM, :]
    return dst


def permute_heads_race_candidates(src, BM: int) -> np.ndarray:
    """For the index-swapped kernel of Listing 5: the H values that may land in
    each destination element, shape (H, B, H, M, D). Destination tile
    (b, m, h2) receives source tile (b, h1, m) from every h1, so candidate h1
    of element (b, m, h2*BM + i, d) is src[b, h1, m*BM + i, d], for every h2."""
    src = np.asarray(src)
    B, H, M, D = src.shape
    if M % BM or M // BM != H:
        raise ValueError("needs M/BM == H")
    out = np.empty((H,) + src.shape, src.dtype)
    for h1 in range(H):
        for b in range(B):
            for m in range(H):
                for h2 in range(H):
                    out[h1, b, m, h2 * BM:(h2 + 1) * BM, :] = src[b, h1, m * BM:(m + 1) * BM, :]
    return out


def ceil_div(a: int, b: int) -> int:
    return -(-a // b)


def gemm_grid(m: int, n: int, bm: int, bn: int):
    return math.ceil(m / bm), math.ceil(n / bn)
