// Grouped persistent BF16 GEMM: many independent problems C_i = A_i . B_i of
// uneven sizes in one launch. Every output tile of every problem is a slot of
// one device queue (a mapped partition whose map is a shared counter, §3.6);
// each persistent CTA (or CTA pair) dequeues slots until the queue is empty.
// The plan's slot map orders the queue: HBM-bound and tensor-bound tiles are
// interleaved in proportion to their cost, each kind most expensive first.
//
// A problem with M <= 256 runs transposed ("swap-AB"): C^T = B^T . A^T, so
// the large N fills the 128 rows of the tensor-core tile and the small M is
// the MMA's N (rounded up to 32). Its tile is a 128-column slab of C; one pass
// streams the matching 128 rows of B_i from HBM exactly once.
//
// On CTA pairs, a larger problem whose last 256-row band is partial (M mod
// 256 <= 192) runs that band the same way: its tail rows become a swap
// problem of their own (A, C and the write counts offset to the band's first
// row), whose tile for column slab j is queued right after the normal tiles
// of column j, while their B slab is still in L2. The tail then costs MMA
// columns for its rows rounded up to 32 instead of a full 256-row tile.
//
// Roles per CTA (192 threads): warp 0 dequeues slots, publishes them through
// a 4-entry shared-memory ring and streams the tile's K slices with TMA;
// warp 1 issues tcgen05.mma into two TMEM accumulators; warps 2-5 drain TMEM
// and store. Every wait is bounded and reports TP_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "sm100_ptx.cuh"
#include "tp_internal.h"

namespace tp {

// Device-side description of one problem (tensor maps first: 64-byte aligned).
struct alignas(64) GroupedProblem {
  CUtensorMap map_x;      // MMA A operand: A_i (normal) or B_i stored N x K (swap), box 128 rows
  CUtensorMap map_y;      // MMA B operand: B_i (normal, box 256 rows) or A_i (swap, box bn rows)
  CUtensorMap map_c;      // C_i as 32 x 64 boxes (128-byte swizzle) for the epilogue's TMA stores
  __nv_bfloat16* c;
  int64_t M, N, K;
  int64_t tiles_r, tiles_c;  // tile grid in MMA orientation (rows of 128, columns of bn)
  int64_t count_base;     // offset of C_i in the write-count arrays
  int32_t swap, bn;       // bn = MMA N of every tile of this problem
  int32_t tile_rows;      // 128 (one CTA) or 256 (CTA pair), MMA orientation
  int32_t box_y;          // rows of the MMA B operand each CTA loads per stage
  int32_t c_tma;          // 1: normal orientation with 16-byte aligned C rows (map_c is valid)
  int32_t stream_x;       // swap tile whose B slab no other tile reads (loaded evict-first)
  int32_t kc;             // K blocks per ring stage: the ring's count (3-D maps) when K % 64 == 0, else 1;
                          // 3 for a swap problem on pairs with at most 32 B-operand rows per CTA
};

}  // namespace tp

struct tp_grouped_plan {
  tp_ctx* ctx = nullptr;
  int32_t n = 0;
  int64_t total_tiles = 0;
  tp::GroupedProblem* d_probs = nullptr;   // device table (input order)
  int64_t* d_slots = nullptr;              // queue slot -> (problem << 32) | local tile
  std::vector<tp_partition*> outs;         // one partition per C_i (busy tracking)
  std::vector<tp_tensor> ins;              // A_i and B_i views (alias checks)
  std::vector<int32_t> order;              // queue position -> problem index
  int64_t total_elems = 0;
  bool pair = true;                        // 256-row tiles on CTA pairs
};

namespace tp {
namespace {

using namespace sm100;

constexpr int kThreads = 192;
constexpr int kRing = 4;
constexpr int kMaxProblems = 1 << 16;
constexpr uint32_t kStageX = 128 * 128;   // 128 rows x 128 bytes per CTA
// B-operand rows per CTA, K blocks per stage and stage count: one CTA holds
// up to 256 rows, one K block per stage (4 stages of 48 KB); a CTA of a pair
// holds up to 128 rows, two K blocks per stage (3 stages of 64 KB), so each
// operand arrives as one 3-D TMA box of two K blocks. A TMA copy costs about
// the same time whatever its size, so a swap tile streams its B slab in
// 32 KB copies at twice the rate of 16 KB ones.
#ifndef TP_GROUPED_PAIR_KC
#define TP_GROUPED_PAIR_KC 2
#endif
template <bool kPair> struct Ring {
  static constexpr uint32_t kStageY = kPair ? 128 * 128 : 256 * 128;  // per K block
  static constexpr int kKc = kPair ? TP_GROUPED_PAIR_KC : 1;
  static constexpr int kStages = kPair ? 6 / TP_GROUPED_PAIR_KC : 4;
};
constexpr size_t kWordsBytes = 8 + 8 * kRing;
constexpr int kWideKc = 3;  // K blocks per stage of a swap problem with few B rows (pairs)
constexpr uint32_t kStageC = 4u * 2u * 4096u;  // epilogue staging: 4 warps x 2 buffers x (32 rows x 128 B)
// Longest partial last 256-row band of a normal problem that CTA pairs run
// as a swap-AB tail (0 = never)
#ifndef TP_GROUPED_TAIL_MAX
#define TP_GROUPED_TAIL_MAX 192
#endif
constexpr int64_t kTailMax = TP_GROUPED_TAIL_MAX;

struct GroupedArgs {
  const GroupedProblem* probs;
  const int64_t* slot_map;   // queue slot -> (problem << 32) | local tile
  int32_t n;
  int64_t total;
  unsigned* queue;
  int* err;
  uint32_t* counts;
  int32_t* owner;
};

template <bool kPair, bool kCount>
__global__ void __launch_bounds__(kThreads, 1) grouped_kernel(const __grid_constant__ GroupedArgs p) {
  constexpr int kKc = Ring<kPair>::kKc;
  constexpr uint32_t kStageY = Ring<kPair>::kStageY * kKc;  // a stage: kKc K blocks of each operand
  constexpr uint32_t kStageXs = kStageX * kKc;
  constexpr int kStages = Ring<kPair>::kStages;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const int warp = threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  // On a pair, the even CTA dequeues slots and issues the MMAs; both CTAs
  // load their half of each operand and store their half of each tile.
  const uint32_t rank = kPair ? cluster_ctarank() : 0u;
  const bool leader = rank == 0;
  const int32_t prog = kPair ? (int32_t)(blockIdx.x / 2) : (int32_t)blockIdx.x;

  // stage s: [A-operand K blocks][B-operand K blocks], the B blocks right
  // after the problem's kc A blocks (so a swap problem with few B rows fits
  // 3 K blocks of each in one stage)
  constexpr uint32_t kStageBytes = kStageXs + kStageY;
  auto stage_at = [&](int s) { return base + kStageBytes * (uint32_t)s; };
  const uint32_t cst = base + kStageBytes * kStages;  // epilogue staging
  const uint32_t bars = cst + kStageC;
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 64u + 8u * s; };
  auto tfull_bar = [&](int b) { return bars + 128u + 8u * b; };
  auto tempty_bar = [&](int b) { return bars + 144u + 8u * b; };
  auto rfull_bar = [&](int r) { return bars + 160u + 8u * r; };
  auto rempty_bar = [&](int r) { return bars + 192u + 8u * r; };
  const uint32_t drain_bar = bars + 224u;
  uint8_t* words = gbase + (bars - base) + 232u;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(words);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(words + 4);
  volatile int64_t* ring = reinterpret_cast<volatile int64_t*>(words + 8);          // kRing slots

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), kPair ? 8 : 4);  // epilogue warps (of both CTAs)
    }
    for (int r = 0; r < kRing; ++r) {
      mbar_init(rfull_bar(r), 1);
      // readers of a slot: the MMA thread and 4 epilogue warps (+ the odd
      // CTA's 4 epilogue warps and producer on a pair)
      mbar_init(rempty_bar(r), kPair ? 10 : 5);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    if constexpr (kPair) {
      tmem_alloc_pair(smem_u32(tmem_slot), 512);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(smem_u32(tmem_slot), 512);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  if constexpr (kPair) cluster_sync();
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  // decode a queue slot into (problem, tile row, tile column) through the
  // plan's slot map; a problem's tiles are column-major over its tile grid so
  // consecutive tiles share a B slab while the problem's A stays in L2
  auto decode = [&](int64_t g, const GroupedProblem** pr, int64_t* tr, int64_t* tc) {
    const int64_t e = p.slot_map[g];
    *pr = p.probs + (e >> 32);
    const int64_t local = e & 0xffffffffll;
    *tr = local % (*pr)->tiles_r;
    *tc = local / (*pr)->tiles_r;
  };
  // wait for a ring slot's value; on a pair it may come from the peer CTA
  auto ring_wait = [&](uint32_t bar, uint32_t parity) {
    return kPair ? mbar_wait_cluster(bar, parity, abort_flag, p.err) : mbar_wait(bar, parity, abort_flag, p.err);
  };
  auto ring_release = [&](int r) {
    if constexpr (kPair) mbar_arrive_cluster(mapa(rempty_bar(r), 0));
    else mbar_arrive(rempty_bar(r));
  };

  if (warp == 0) {
    if (lane == 0) {
      const uint64_t pol_stream = policy_evict_first();
      const uint64_t pol_keep = policy_evict_last();
      uint32_t fills[8] = {};
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t j = 0; ok; ++j) {
        const int r = (int)(j % kRing);
        const uint32_t par = (uint32_t)((j / kRing) & 1);
        int64_t g;
        if (leader) {
          if (!ring_wait(rempty_bar(r), par ^ 1u)) { ok = false; break; }
          const int64_t d = (int64_t)atomicAdd(p.queue, 1u);
          g = d < p.total ? d : -1;
          ring[r] = g;
          if constexpr (kPair) {
            st_cluster_u64(mapa(smem_u32(const_cast<int64_t*>(ring + r)), 1), g);
            mbar_arrive(rfull_bar(r));
            mbar_arrive_cluster(mapa(rfull_bar(r), 1));
          } else {
            mbar_arrive(rfull_bar(r));
          }
        } else {
          if (!ring_wait(rfull_bar(r), par)) { ok = false; break; }
          g = ring[r];
          ring_release(r);
        }
        if (g < 0) break;
        const GroupedProblem* pr;
        int64_t tr, tc;
        decode(g, &pr, &tr, &tc);
        const int32_t xrow = (int32_t)(tr * pr->tile_rows + rank * 128);
        const int32_t yrow = (int32_t)(tc * pr->bn + rank * pr->box_y);
        const int32_t pkc = pr->kc;
        const uint32_t tx = (kStageX + (uint32_t)pr->box_y * 128u) * (uint32_t)pkc;
        const int64_t nk = (pr->K + 63) / 64;
        for (int64_t kb = 0; kb < nk; kb += pkc) {
          if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, p.err)) { ok = false; break; }
          // 2-D maps take K at element kb * 64; 3-D maps take K block kb (a
          // block past the last is zero-filled and never multiplied)
          const int32_t kx = pkc > 1 ? 0 : (int32_t)(kb * 64);
          // streamed swap: x = B_i slab (read once), y = A_i (reused by every tile)
          const uint64_t px = pr->stream_x ? pol_stream : pol_keep;
          if constexpr (kPair) {
            const uint32_t fb = mapa(full_bar(stage), 0);  // both halves complete on the even CTA's barrier
            if (leader) mbar_arrive_expect_tx(full_bar(stage), 2 * tx);
            if (pkc > 1) {
              tma_load_3d_pair(stage_at(stage), &pr->map_x, 0, xrow, (int32_t)kb, fb, px);
              tma_load_3d_pair(stage_at(stage) + kStageX * (uint32_t)pkc, &pr->map_y, 0, yrow, (int32_t)kb, fb,
                               pol_keep);
            } else {
              tma_load_2d_pair(stage_at(stage), &pr->map_x, kx, xrow, fb, px);
              tma_load_2d_pair(stage_at(stage) + kStageX, &pr->map_y, kx, yrow, fb, pol_keep);
            }
          } else {
            mbar_arrive_expect_tx(full_bar(stage), tx);
            tma_load_2d(stage_at(stage), &pr->map_x, kx, xrow, full_bar(stage), px);
            tma_load_2d(stage_at(stage) + kStageX, &pr->map_y, kx, yrow, full_bar(stage), pol_keep);
          }
          fills[stage]++;
          if (++stage == kStages) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok && leader) {
        for (int s2 = 0; s2 < kStages; ++s2)
          if (fills[s2]) mbar_wait(full_bar(s2), (fills[s2] - 1u) & 1u, nullptr, nullptr, 200000000ull);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t j = 0; ok; ++j) {
        const int r = (int)(j % kRing);
        if (!mbar_wait(rfull_bar(r), (uint32_t)((j / kRing) & 1), abort_flag, p.err)) { ok = false; break; }
        const int64_t g = ring[r];
        ring_release(r);
        if (g < 0) break;
        const GroupedProblem* pr;
        int64_t tr, tc;
        decode(g, &pr, &tr, &tc);
        const int acc = (int)(j & 1);
        const uint32_t use = (uint32_t)((j >> 1) & 1);
        if (!mbar_wait(tempty_bar(acc), use ^ 1u, abort_flag, p.err)) { ok = false; break; }
        tc_fence_after();
        const uint32_t idesc = idesc_f32acc(kPair ? 256 : 128, (uint32_t)pr->bn, false);
        const uint32_t d = tmem_base + (uint32_t)(acc * 256);
        const int64_t nk = (pr->K + 63) / 64;
        const int32_t pkc = pr->kc;
        const uint32_t y_blk = (uint32_t)pr->box_y * 128u;  // one K block of the B operand
        for (int64_t kb = 0; kb < nk; kb += pkc) {
          if (!mbar_wait(full_bar(stage), phase, abort_flag, p.err)) { ok = false; break; }
          tc_fence_after();
          // the stage's K blocks in K order (blocks past the last are not multiplied)
          for (int32_t jb = 0; jb < pkc && kb + jb < nk; ++jb) {
            const uint64_t ad = desc_kmajor_sw128(stage_at(stage) + kStageX * (uint32_t)jb);
            const uint64_t bd = desc_kmajor_sw128(stage_at(stage) + kStageX * (uint32_t)pkc + y_blk * (uint32_t)jb);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint32_t accum = (kb + jb > 0 || k > 0) ? 1u : 0u;
              if constexpr (kPair) mma_pair<false>(d, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc, accum);
              else mma<false>(d, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc, accum);
            }
          }
          if constexpr (kPair) mma_commit_pair(empty_bar(stage), 0x3);
          else mma_commit(empty_bar(stage));
          if (++stage == kStages) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        if constexpr (kPair) mma_commit_pair(tfull_bar(acc), 0x3);
        else mma_commit(tfull_bar(acc));
      }
      if (!ok) {
        if constexpr (kPair) mma_commit_pair(drain_bar, 0x1);
        else mma_commit(drain_bar);
        mbar_wait(drain_bar, 0, nullptr, nullptr, 200000000ull);
      }
    }
    __syncwarp();
  } else {
    const int quad = warp & 3;
    const int lane_row = (int)rank * 128 + quad * 32 + lane;  // tile row (MMA orientation) of this TMEM lane
    const uint32_t stg = cst + (uint32_t)quad * 8192u;       // this warp's two 4 KB staging buffers
    uint32_t nstaged = 0;
    for (int64_t j = 0;; ++j) {
      const int r = (int)(j % kRing);
      const bool got = ring_wait(rfull_bar(r), (uint32_t)((j / kRing) & 1));
      if (!__all_sync(0xffffffffu, got)) break;  // leave together (tcgen05.ld below is warp-collective)
      const int64_t g = ring[r];
      __syncwarp();
      if (lane == 0) ring_release(r);
      if (g < 0) break;
      const GroupedProblem* pr;
      int64_t tr, tc;
      decode(g, &pr, &tr, &tc);
      const int acc = (int)(j & 1);
      const uint32_t use = (uint32_t)((j >> 1) & 1);
      const bool ready = mbar_wait(tfull_bar(acc), use, abort_flag, p.err);
      if (!__all_sync(0xffffffffu, ready)) break;
      tc_fence_after();
      const int64_t N = pr->N, M = pr->M;
      const int64_t rr = tr * pr->tile_rows + lane_row;  // row of C (normal) or column of C (swap)
      int ch0 = 0;
      if (!kCount && pr->c_tma) {
        // normal orientation, 16-byte aligned C rows: 32 x 64 blocks staged
        // with 16-byte piece u of row `lane` at piece u ^ (lane & 7) and
        // written by one TMA store each, clipped to C_i's bounds by its
        // tensor map (bn = 256: four blocks per tile row slice)
        const int64_t row0 = rr - lane;
        for (; ch0 + 1 < pr->bn / 32; ch0 += 2) {
          uint32_t v0[32], v1[32];
          tmem_ld32(tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * 256 + ch0 * 32), v0);
          tmem_ld32(tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * 256 + ch0 * 32 + 32), v1);
          tmem_ld_wait();
          const int64_t c0 = tc * pr->bn + ch0 * 32;
          if (row0 >= M || c0 >= N) continue;  // warp-uniform
          const uint32_t buf = stg + (nstaged & 1u) * 4096u;
          if (lane == 0 && nstaged >= 2) bulk_wait_read<1>();  // the store from this buffer two blocks ago has read it
          __syncwarp();
          uint32_t w[32];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            __nv_bfloat162 h = __floats2bfloat162_rn(__uint_as_float(v0[2 * i]), __uint_as_float(v0[2 * i + 1]));
            w[i] = *reinterpret_cast<uint32_t*>(&h);
            h = __floats2bfloat162_rn(__uint_as_float(v1[2 * i]), __uint_as_float(v1[2 * i + 1]));
            w[16 + i] = *reinterpret_cast<uint32_t*>(&h);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u)
            st_shared_v4(buf + (uint32_t)lane * 128u + ((uint32_t)(u ^ (lane & 7)) << 4), w[4 * u], w[4 * u + 1],
                         w[4 * u + 2], w[4 * u + 3]);
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) {
            tma_store_2d(&pr->map_c, buf, (int32_t)c0, (int32_t)row0);
            bulk_commit();
          }
          ++nstaged;
        }
      }
      for (int ch = ch0; ch < pr->bn / 32; ++ch) {
        uint32_t v[32];
        tmem_ld32(tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * 256 + ch * 32), v);
        tmem_ld_wait();
        const int64_t c0 = tc * pr->bn + ch * 32;  // first column of the chunk (MMA orientation)
        if (!pr->swap) {
          if (rr >= M || c0 >= N) continue;
          __nv_bfloat16* crow = pr->c + rr * N;
          if ((N & 7) == 0 && c0 + 32 <= N) {
            uint4 w[4];
            __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(w);
#pragma unroll
            for (int i = 0; i < 16; ++i) h[i] = __floats2bfloat162_rn(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
            uint4* dst = reinterpret_cast<uint4*>(crow + c0);
#pragma unroll
            for (int i = 0; i < 4; ++i) dst[i] = w[i];
          } else {
            for (int i = 0; i < 32; ++i)
              if (c0 + i < N) crow[c0 + i] = __float2bfloat16_rn(__uint_as_float(v[i]));
          }
          if constexpr (kCount) {
            for (int i = 0; i < 32; ++i)
              if (c0 + i < N) {
                const int64_t e = pr->count_base + rr * N + c0 + i;
                atomicAdd(p.counts + e, 1u);
                p.owner[e] = prog;
              }
          }
        } else {
          // swap: TMEM lane = column n of C, TMEM column = row m of C
          if (rr >= N) continue;
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int64_t m = c0 + i;
            if (m < M) {
              pr->c[m * N + rr] = __float2bfloat16_rn(__uint_as_float(v[i]));
              if constexpr (kCount) {
                const int64_t e = pr->count_base + m * N + rr;
                atomicAdd(p.counts + e, 1u);
                p.owner[e] = prog;
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if constexpr (kPair) mbar_arrive_cluster(mapa(tempty_bar(acc), 0));
        else mbar_arrive(tempty_bar(acc));
      }
    }
    if (lane == 0) bulk_wait_all();  // C written before the CTA retires
    __syncwarp();
  }
  if constexpr (kPair) settle_after_abort(abort_flag);
  tc_fence_before();
  if constexpr (kPair) cluster_sync();  // the peer no longer touches our shared memory / TMEM
  else __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    if constexpr (kPair) tmem_dealloc_pair(tmem_base, 512);
    else tmem_dealloc(tmem_base, 512);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  return fn;
}

// C_i (bf16, N columns, row stride N) as 32 x 64 boxes with the 128-byte
// swizzle of the epilogue's staging layout.
tp_status c_map(CUtensorMap* map, void* ptr, int64_t M, int64_t N) {
  auto fn = encode();
  if (!fn) return fail(TP_ERR_CUDA, "cuTensorMapEncodeTiled unavailable from the driver");
  cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)M};
  cuuint64_t strides[1] = {(cuuint64_t)(N * 2)};
  cuuint32_t box[2] = {64, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(TP_ERR_CUDA, "cuTensorMapEncodeTiled (C) failed (" + std::to_string((int)r) + ")");
  return TP_OK;
}

// K-major bf16 operand, boxes of box_rows rows x 64 elements (128 bytes,
// 128-byte swizzle); with kc > 1 (K a multiple of 64) seen as 3-D {64, rows,
// K / 64} so that one box brings kc consecutive K blocks, stacked in shared
// memory as kc K-major tiles.
tp_status kmajor_map(CUtensorMap* map, const void* ptr, int64_t rows, int64_t k, int64_t ld, int box_rows, int kc) {
  auto fn = encode();
  if (!fn) return fail(TP_ERR_CUDA, "cuTensorMapEncodeTiled unavailable from the driver");
  const cuuint32_t rank = kc > 1 ? 3 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)rows, 1};
  cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), 0};
  cuuint32_t box[3] = {64, (cuuint32_t)box_rows, 1};
  if (kc > 1) {
    dims[0] = 64;
    dims[2] = (cuuint64_t)(k / 64);
    strides[1] = 128;
    box[2] = (cuuint32_t)kc;
  }
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(TP_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return TP_OK;
}

}  // namespace
}  // namespace tp

using namespace tp;

extern "C" {

tp_status tp_grouped_plan_create(tp_ctx* ctx, const tp_gemm_problem* probs, int32_t n, int32_t swap_max_m,
                                 int32_t cta_pair, tp_grouped_plan** out) {
  if (!ctx || !probs || !out) return fail(TP_ERR_INVALID, "null argument");
  *out = nullptr;
  DeviceGuard guard(ctx);
  if (n < 1 || n > kMaxProblems) return fail(TP_ERR_INVALID, "group size must be 1..65536");
  if (swap_max_m < 0) swap_max_m = 256;
  if (swap_max_m > 256) return fail(TP_ERR_INVALID, "swap_max_m must be <= 256");
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->capturing) return fail(TP_ERR_CAPTURE, "a plan allocates device memory: build it before capture");
  }
  std::vector<GroupedProblem> host(n);
  host.reserve(2 * (size_t)n);  // tails are appended: no reallocation under the references below
  std::vector<double> cost(n);
  // tails[j] = (parent problem, table entry); tail entries follow the n
  // problems in the device table
  std::vector<std::pair<int, int>> tails;
  auto* plan = new tp_grouped_plan();
  plan->ctx = ctx;
  plan->n = n;
  plan->pair = cta_pair != 0;
  const int32_t trows = plan->pair ? 256 : 128;
  auto cleanup = [&](tp_status s) {
    for (auto* q : plan->outs) tp_partition_destroy(q);
    delete plan;
    return s;
  };
  // K blocks per ring stage of a problem: the ring's count when K is a
  // multiple of the 64-element K block (3-D maps), else one
  const int ring_kc = plan->pair ? Ring<true>::kKc : Ring<false>::kKc;
  auto kc_of = [&](int64_t K) { return K % 64 == 0 ? ring_kc : 1; };
  // a swap-orientation entry: C rows [0, M) of `c` (row stride N) from A rows
  // of `a` (row stride lda) and B (N x K, row stride ldb)
  auto make_swap = [&](GroupedProblem& g, const void* a, const void* b, void* c, int64_t M, int64_t N, int64_t K,
                       int64_t lda, int64_t ldb) {
    g.c = static_cast<__nv_bfloat16*>(c);
    g.M = M;
    g.N = N;
    g.K = K;
    g.swap = 1;
    g.tile_rows = trows;
    g.bn = (int32_t)(((M + 31) / 32) * 32);
    g.box_y = plan->pair ? g.bn / 2 : g.bn;
    g.tiles_r = (N + trows - 1) / trows;
    g.tiles_c = 1;
    g.kc = kc_of(K);
    // few B rows (M <= 64 on a pair): a stage holds 3 K blocks of each
    // operand (48 KB of the streamed slab instead of 32 KB), so the slab
    // streams with more bytes in flight and fewer copies per byte
    constexpr uint32_t kPairStage = (kStageX + Ring<true>::kStageY) * Ring<true>::kKc;
    if (plan->pair && K % 64 == 0 && (uint32_t)kWideKc * (kStageX + (uint32_t)g.box_y * 128u) <= kPairStage)
      g.kc = kWideKc;
    tp_status s = kmajor_map(&g.map_x, b, N, K, ldb, 128, g.kc);
    if (s == TP_OK) s = kmajor_map(&g.map_y, a, M, K, lda, g.box_y, g.kc);
    return s;
  };
  int64_t elems = 0;
  for (int i = 0; i < n; ++i) {
    const tp_tensor& a = probs[i].a;
    const tp_tensor& b = probs[i].b;
    const tp_tensor& c = probs[i].c;
    if (a.rank != 2 || b.rank != 2 || c.rank != 2) return cleanup(fail(TP_ERR_RANK, "grouped operands are rank 2"));
    const int64_t M = a.shape[0], K = a.shape[1], N = b.shape[1];
    if (b.shape[0] != K || c.shape[0] != M || c.shape[1] != N)
      return cleanup(fail(TP_ERR_SHAPE, "problem " + std::to_string(i) + ": need A M x K, B K x N, C M x N"));
    if (a.dtype != TP_BF16 || b.dtype != TP_BF16 || c.dtype != TP_BF16)
      return cleanup(fail(TP_ERR_UNSUPPORTED, "grouped GEMM is BF16 x BF16 -> BF16"));
    if (a.strides[1] != 1 || b.strides[0] != 1 || !is_contiguous(c))
      return cleanup(fail(TP_ERR_UNSUPPORTED, "grouped GEMM needs K-major A and B and a contiguous C"));
    if (M < 1 || N < 1 || K < 1) return cleanup(fail(TP_ERR_SHAPE, "empty problem"));
    const int64_t lda = a.strides[0], ldb = b.strides[1];
    if (((uintptr_t)a.ptr & 15) || ((uintptr_t)b.ptr & 15) || ((lda * 2) & 15) || ((ldb * 2) & 15) || (K * 2) % 16)
      return cleanup(fail(TP_ERR_ALIGN, "TMA needs 16-byte aligned bases and row strides (K % 8 == 0)"));
    GroupedProblem& g = host[i];
    std::memset(&g, 0, sizeof(g));
    tp_status s;
    int64_t tile_rows, tile_cols;
    if (M <= swap_max_m) {
      s = make_swap(g, a.ptr, b.ptr, c.ptr, M, N, K, lda, ldb);
      g.stream_x = 1;
      tile_rows = M;
      tile_cols = trows;
      cost[i] = trows * (double)K * 2.0 / 44e9 + 2.0 * trows * g.bn * K / 1.2e13;
    } else {
      // on CTA pairs, a partial last band of at most 192 rows runs as a swap
      // tail (below); the normal tiles cover the whole bands above it
      const int64_t tail = plan->pair ? M % 256 : 0;
      const bool split = tail > 0 && tail <= kTailMax;
      const int64_t M0 = split ? M - tail : M;
      g.c = static_cast<__nv_bfloat16*>(c.ptr);
      g.M = M0;
      g.N = N;
      g.K = K;
      g.swap = 0;
      g.tile_rows = trows;
      g.bn = 256;
      g.box_y = plan->pair ? 128 : 256;
      g.tiles_r = (M0 + trows - 1) / trows;
      g.tiles_c = (N + 255) / 256;
      g.kc = kc_of(K);
      s = kmajor_map(&g.map_x, a.ptr, M0, K, lda, 128, g.kc);
      if (s == TP_OK) s = kmajor_map(&g.map_y, b.ptr, N, K, ldb, g.box_y, g.kc);
      if (s == TP_OK && N % 8 == 0 && ((uintptr_t)c.ptr & 15) == 0) {
        s = c_map(&g.map_c, c.ptr, M0, N);
        g.c_tma = 1;
      }
      tile_rows = trows;
      tile_cols = 256;
      cost[i] = 2.0 * trows * 256 * (double)K / (plan->pair ? 2.4e13 : 1.2e13);
      if (s == TP_OK && split) {
        GroupedProblem t;
        std::memset(&t, 0, sizeof(t));
        const char* a_tail = static_cast<const char*>(a.ptr) + M0 * lda * 2;
        char* c_tail = static_cast<char*>(c.ptr) + M0 * N * 2;
        s = make_swap(t, a_tail, b.ptr, c_tail, tail, N, K, lda, ldb);
        t.stream_x = 0;  // its B slab was just read by the normal tiles of that column
        t.count_base = elems + M0 * N;
        tails.push_back({i, (int)(n + tails.size())});
        host.push_back(t);
        cost.push_back(2.0 * trows * t.bn * (double)K / 2.4e13);
      }
    }
    if (s != TP_OK) return cleanup(s);
    host[i].count_base = elems;
    elems += M * N;
    tp_partition* part = nullptr;
    int64_t tile[2] = {tile_rows, tile_cols};
    s = tp_partition_create(ctx, &c, tile, &part);
    if (s != TP_OK) return cleanup(s);
    s = tp_partition_map(part, TP_MAP_QUEUE, 1);
    if (s != TP_OK) {
      tp_partition_destroy(part);
      return cleanup(s);
    }
    plan->outs.push_back(part);
    plan->ins.push_back(a);
    plan->ins.push_back(b);
  }
  std::vector<int> tail_of(n, -1);
  for (auto& t : tails) tail_of[t.first] = t.second;
  // Queue order. Tiles of swapped problems stream B from HBM, the others are
  // tensor-core bound; each stream is ordered most expensive problem first
  // (longest processing time first) and the two are merged in proportion to
  // their total cost, so that tiles running at the same time use both HBM
  // and the tensor cores. A normal problem's tiles go column by column, each
  // column followed by its tail tile.
  std::vector<int> mem_p, comp_p;
  for (int i = 0; i < n; ++i) (host[i].swap ? mem_p : comp_p).push_back(i);
  auto by_cost = [&](int x, int y) { return cost[x] > cost[y]; };
  std::stable_sort(mem_p.begin(), mem_p.end(), by_cost);
  std::stable_sort(comp_p.begin(), comp_p.end(), by_cost);
  auto expand = [&](const std::vector<int>& ps, std::vector<std::pair<int64_t, double>>& out) {
    for (int i : ps) {
      const GroupedProblem& g = host[i];
      for (int64_t tc = 0; tc < g.tiles_c; ++tc) {
        for (int64_t tr = 0; tr < g.tiles_r; ++tr) out.push_back({((int64_t)i << 32) | (tc * g.tiles_r + tr), cost[i]});
        const int t = tail_of[i];
        if (t >= 0) out.push_back({((int64_t)t << 32) | tc, cost[t]});
      }
    }
  };
  std::vector<std::pair<int64_t, double>> mem_t, comp_t;
  expand(mem_p, mem_t);
  expand(comp_p, comp_t);
  double mem_total = 0, comp_total = 0;
  for (auto& x : mem_t) mem_total += x.second;
  for (auto& x : comp_t) comp_total += x.second;
  std::vector<int64_t> slots;
  slots.reserve(mem_t.size() + comp_t.size());
  size_t im = 0, ic = 0;
  double dm = 0, dc = 0;
  while (im < mem_t.size() || ic < comp_t.size()) {
    const bool take_mem = ic >= comp_t.size() ||
                          (im < mem_t.size() && dm / std::max(mem_total, 1e-30) <= dc / std::max(comp_total, 1e-30));
    if (take_mem) {
      dm += mem_t[im].second;
      slots.push_back(mem_t[im++].first);
    } else {
      dc += comp_t[ic].second;
      slots.push_back(comp_t[ic++].first);
    }
  }
  plan->order.resize(n);
  std::iota(plan->order.begin(), plan->order.end(), 0);
  int64_t slot = (int64_t)slots.size();
  std::vector<GroupedProblem>& ordered = host;
  plan->total_tiles = slot;
  plan->total_elems = elems;
  if (slot >= (int64_t(1) << 31)) return cleanup(fail(TP_ERR_UNSUPPORTED, "more than 2^31 tiles in a group"));
  cudaError_t e = cudaMalloc(&plan->d_probs, sizeof(GroupedProblem) * ordered.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(plan->d_probs, ordered.data(), sizeof(GroupedProblem) * ordered.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&plan->d_slots, sizeof(int64_t) * std::max<int64_t>(slot, 1));
  if (e == cudaSuccess)
    e = cudaMemcpy(plan->d_slots, slots.data(), sizeof(int64_t) * slot, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(plan->d_probs);
    cudaFree(plan->d_slots);
    return cleanup(cuda_fail(e, "uploading the problem table"));
  }
  *out = plan;
  return TP_OK;
}

tp_status tp_grouped_plan_info(const tp_grouped_plan* plan, int64_t* total_tiles, int32_t* swapped) {
  if (!plan) return fail(TP_ERR_INVALID, "null plan");
  if (total_tiles) *total_tiles = plan->total_tiles;
  if (swapped) {
    std::vector<GroupedProblem> h(plan->n);
    cudaError_t e = cudaMemcpy(h.data(), plan->d_probs, sizeof(GroupedProblem) * plan->n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the problem table");
    for (int q = 0; q < plan->n; ++q) swapped[plan->order[q]] = h[q].swap;
  }
  return TP_OK;
}

tp_status tp_grouped_plan_destroy(tp_grouped_plan* plan) {
  if (!plan) return fail(TP_ERR_INVALID, "null plan");
  for (auto* q : plan->outs)
    if (q->busy.load()) return fail(TP_ERR_BUSY, "the group has work in flight");
  for (auto* q : plan->outs) tp_partition_destroy(q);
  cudaFree(plan->d_probs);
  cudaFree(plan->d_slots);
  delete plan;
  return TP_OK;
}

tp_status tp_grouped_gemm(tp_ctx* ctx, tp_grouped_plan* plan, int32_t num_programs, const tp_exec* ex) {
  if (!ctx || !plan || !ex) return fail(TP_ERR_INVALID, "null argument");
  if (plan->ctx != ctx) return fail(TP_ERR_INVALID, "plan belongs to another context");
  if ((ex->write_counts == nullptr) != (ex->write_owner == nullptr))
    return fail(TP_ERR_INVALID, "write_counts and write_owner must be given together");
  Op o(__func__);
  tp_status s = o.begin_lists(ctx, ex, plan->outs, plan->ins);
  if (s != TP_OK) return s;
  o.check_err = true;
  unsigned* q = nullptr;
  s = queue_counter(ctx, o.stream, &q);
  if (s != TP_OK) {
    o.abort();
    return s;
  }
  GroupedArgs a{};
  a.probs = plan->d_probs;
  a.slot_map = plan->d_slots;
  a.n = plan->n;
  a.total = plan->total_tiles;
  a.queue = q;
  a.err = ctx->d_err;
  a.counts = ex->write_counts;
  a.owner = ex->write_owner;
  const bool pair = plan->pair;
  int64_t programs = num_programs > 0 ? num_programs : (pair ? ctx->sm_count / 2 : ctx->sm_count);
  if (programs > plan->total_tiles) programs = plan->total_tiles;
  if (programs < 1) {
    o.abort();
    return fail(TP_ERR_INVALID, "the plan has no tiles");
  }
  const int grid = (int)(pair ? 2 * programs : programs);
  size_t smem;
  cudaError_t e;
  auto launch = [&](auto kernel, size_t bytes, int cluster) {
    cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (err != cudaSuccess) return err;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3(kThreads);
    lc.dynamicSmemBytes = bytes;
    lc.stream = o.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, kernel, a);
  };
  if (pair) {
    smem = 1024 + (kStageX + Ring<true>::kStageY) * Ring<true>::kKc * Ring<true>::kStages + kStageC + 232 +
           kWordsBytes;
    e = a.counts ? launch(grouped_kernel<true, true>, smem, 2) : launch(grouped_kernel<true, false>, smem, 2);
  } else {
    smem = 1024 + (kStageX + Ring<false>::kStageY) * Ring<false>::kKc * Ring<false>::kStages + kStageC + 232 +
           kWordsBytes;
    e = a.counts ? launch(grouped_kernel<false, true>, smem, 1) : launch(grouped_kernel<false, false>, smem, 1);
  }
  return o.end(e);
}

}  // extern "C"
