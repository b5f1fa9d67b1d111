"""Grouped GEMM (oracle; test infrastructure).

A group of independent problems C_i = A_i . B_i, each reducing to the plain
GEMM definition (oracle.gemm). One persistent launch walks all output tiles of
all problems through a shared device queue (the many-uneven-GEMMs workload;
the paper's nearest setting is the bimodal GEMM queue of Appendix B). The
queue is a bijection from global slot g in [0, sum_i T_i) onto (i, local tile):
with the exclusive prefix P_i = T_0 + ... + T_{i-1}, slot g belongs to the i
with P_i <= g < P_{i+1} and is that problem's local slot g - P_i.

A problem may be computed transposed ("swap-AB": C_i^T = B_i^T . A_i^T, so the
large N fills the tensor-core M dimension); its tiles then cover C_i^T, i.e.
a (BM x BN) tile of C^T is a (BN x BM) block of C.
"""
from __future__ import annotations

import numpy as np

from .gemm import gemm


def problem_tiles(m: int, n: int, bm: int, bn: int, swap: bool):
    """Number of output tiles and the C-block of each local slot (row-major
    over the tile grid of C, or of C^T when swapped)."""
    rows, cols = (n, m) if swap else (m, n)
    gr, gc = -(-rows // bm), -(-cols // bn)
    blocks = []
    for s in range(gr * gc):
        tr, tc = s // gc, s % gc
        r0, r1 = tr * bm, min((tr + 1) * bm, rows)
        c0, c1 = tc * bn, min((tc + 1) * bn, cols)
        blocks.append(((c0, c1), (r0, r1)) if swap else ((r0, r1), (c0, c1)))
    return gr * gc, blocks


def queue_decode(g: int, tile_counts):
    """Global queue slot g -> (problem i, local slot) through the exclusive prefix."""
    prefix = np.concatenate([[0], np.cumsum(tile_counts)])
    if not 0 <= g < prefix[-1]:
        raise ValueError("slot out of range")
    i = int(np.searchsorted(prefix, g, side="right") - 1)
    return i, int(g - prefix[i])


def element_counts(problems, tile_cfg, dequeued_slots):
    """Write counts per element of every C_i when the listed global slots run.

    problems: [(M, N, K)]; tile_cfg: [(bm, bn, swap)] per problem."""
    tiles = [problem_tiles(m, n, *cfg) for (m, n, _), cfg in zip(problems, tile_cfg)]
    counts = [np.zeros((m, n), dtype=np.int64) for (m, n, _) in problems]
    tc = [t[0] for t in tiles]
    for g in dequeued_slots:
        i, s = queue_decode(int(g), tc)
        (r0, r1), (c0, c1) = tiles[i][1][s]
        counts[i][r0:r1, c0:c1] += 1
    return counts


def grouped_gemm(As, Bs):
    """[C_i = A_i . B_i] in float64."""
    return [gemm(a, b) for a, b in zip(As, Bs)]
