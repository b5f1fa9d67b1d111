// Tensor-core GEMM for sm_103a: C (bf16) = A . B with BF16 (kind::f16) or
// FP8-E4M3 (kind::f8f6f4) operands and FP32 accumulation in TMEM.
//
// One output tile of 64 x BN or 128 x BN (one CTA) or 256 x BN (a CTA pair
// running cta_group::2 MMAs) per tile program step, with a K loop (§3.6, Listing 6:
// the program walks its mapped sequence of output tiles and, for each,
// accumulates mma over the K tiles). On a strided map the tiles of the last,
// partial round may be cut along N into narrow tiles for programs that would
// otherwise idle. With split_k = S > 1 a program is a cluster of S CTAs that
// each accumulate one contiguous slice of the K blocks of the program's
// (single) tile; the partial sums then meet through distributed shared
// memory, CTA j adding the S partials of column slice j in slice order
// (a fixed order, so C is bit-reproducible) and storing that slice.
// A persistent CTA (or CTA pair) runs one program:
//   warp 0   TMA producer: streams (A, B) K-slices into a ring of shared-
//            memory stages (128-byte swizzle), guarded by full/empty mbarriers;
//   warp 1   MMA issuer: one thread issues tcgen05.mma into one of two TMEM
//            accumulators and commits each consumed stage back to the producer;
//   warps 2-5 epilogue: tcgen05.ld the finished accumulator (each warp owns the
//            32 TMEM lanes its warp index selects: tile rows 32q..32q+31 of a
//            128-row MMA, or in lanes 0-15 rows 16q..16q+15 of a 64-row MMA,
//            whose D rows occupy lanes 32(r/16) + r%16), scale, round to
//            bf16 and store only inside this program's tile (32 x 64 blocks,
//            or 32 x 32 for an odd last chunk, staged in shared memory and
//            written by TMA stores, or per-row stores when C rows are not
//            16-byte aligned), while the MMA warp already fills the other
//            accumulator.
// Every mbarrier wait is bounded; on timeout the kernel records an error,
// drains its in-flight copies and MMAs, frees TMEM and returns. The checked
// build (TP_EXEC_CHECKED) validates and claims every tile before storing it;
// the write-count build records each stored element's writer.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "sm100_ptx.cuh"
#include "tile_claim.cuh"
#include "tp_internal.h"

namespace tp {
namespace {

using namespace sm100;

constexpr int BM = 128;
constexpr int kThreads = 192;
constexpr int kMaxStages = 16;
constexpr uint32_t kStageC = 4u * 2u * 4096u;  // epilogue staging: 4 warps x 2 buffers x (32 rows x 128 B)

struct TcArgs {
  int64_t M, N, K;
  int32_t gm, gn;       // tile grid (gm * gn < 2^31)
  int32_t rows;         // MMA rows of one CTA: 64 or 128 (a CTA pair: 128 each, 256 per tile; swap: 64 each)
  int32_t bn;           // tile columns (32..256, multiple of 32)
  int32_t stages;
  int32_t kind;         // tp_map_kind (IDENTITY or STRIDED)
  int32_t group_m;
  int32_t tmem_cols;    // allocated TMEM columns (2 * bn rounded to a power of two)
  int32_t c_vec;        // C rows are 16-byte aligned (N % 8 == 0, aligned base)
  int32_t kblk;         // K elements per K block: 128 bytes (64 bf16 / 128 fp8)
  int32_t nk;           // K blocks per tile: ceil(K / kblk)
  int32_t kc;           // K blocks per ring stage; > 1: each operand arrives as one 3-D box per stage
  int32_t split;        // K slices per tile (cluster size of a split program); 1 = none
  int32_t stage_c;      // epilogue writes C by TMA stores of 32 x 32 blocks staged in shared memory
  int32_t body_bytes;   // shared memory before the staging area: max(ring, split receive buffer)
  int32_t parts;        // claim parts per tile: narrow tiles (ncut) or K slices (split)
  int32_t inject;       // failure-path test: each program's first K block is never loaded
  uint64_t wait_ns;     // limit of every bounded wait (ns)
  __nv_bfloat16* c;
  const float* scale_a; // optional (FP8): C = acc * 1 / (*scale_a * *scale_b)
  const float* scale_b;
  int* err;             // context error word
  uint32_t* counts;     // write-count instrumentation (optional)
  int32_t* owner;
  uint32_t* claims;     // checked launch: tile-claim bitmap (kChecked)
  unsigned* claim_done; // checked launch: finished-CTA counter
  int64_t claim_bits;   // bits this launch may set
  // Schedule: slots [0, dp_slots) are whole tiles (slot = tile index); each
  // remaining tile dp_slots + r is cut along N into ncut narrow tiles of
  // bn_cut columns, narrow tile j being slot dp_slots + r * ncut + j.
  int32_t dp_slots;
  int32_t total_slots;  // dp_slots + (tiles - dp_slots) * ncut (< 2^31)
  int32_t ncut;         // 1 = no tile is cut
  int32_t bn_cut;       // bn / ncut
};

// The work of one slot: a tile and the columns [col, col + width) of it.
struct Unit {
  int32_t tile;
  int32_t col, width, part;
  bool cut;
};

__device__ __forceinline__ Unit unit_of(int32_t s, const TcArgs& p) {
  Unit u;
  if (s < p.dp_slots) {
    u.tile = s;
    u.col = 0;
    u.width = p.bn;
    u.part = 0;
    u.cut = false;
  } else {
    const int32_t q = s - p.dp_slots;
    u.tile = p.dp_slots + q / p.ncut;
    u.part = q % p.ncut;
    u.col = u.part * p.bn_cut;
    u.width = p.bn_cut;
    u.cut = true;
  }
  return u;
}

// Band raster: bands of g tile rows, column-major inside a band (32-bit
// arithmetic: the host keeps the tile count below 2^31 and g <= gm).
__device__ __forceinline__ void raster(uint32_t s, uint32_t gm, uint32_t gn, uint32_t g, int32_t* tm, int32_t* tn) {
  const uint32_t per = g * gn;
  const uint32_t band = s / per;
  const uint32_t first = band * g;
  const uint32_t rows = min(g, gm - first);
  const uint32_t r = s - band * per;
  const uint32_t col = r / rows;
  *tm = (int32_t)(first + (r - col * rows));
  *tn = (int32_t)col;
}

// kSwap (BF16 CTA pairs only): swap-AB tiles, the MMA computing C^T = B^T A^T
// with its rows on C's columns.
template <bool kF8, bool kPair, bool kCount, bool kChecked, bool kSwap = false>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                   const __grid_constant__ CUtensorMap map_b_cut, const __grid_constant__ CUtensorMap map_c,
                   const __grid_constant__ CUtensorMap map_c64, const __grid_constant__ TcArgs p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);

  const int warp = threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  // A CTA pair computes a 256-row tile: this CTA holds rows [rank*128, +128)
  // of A and of the accumulator, and B rows (tile columns) [rank*bn/2, +bn/2).
  // A split program (cluster of S single CTAs) gives CTA `kslice` the K
  // blocks [kslice*nk/S, (kslice+1)*nk/S) of the tile.
  const int32_t S = kPair ? 1 : p.split;
  const uint32_t crank = (kPair || S > 1) ? cluster_ctarank() : 0u;
  const uint32_t rank = kPair ? crank : 0u;
  const uint32_t kslice = kPair ? 0u : crank;
  const bool leader = rank == 0;
  const int32_t csize = kPair ? 2 : S;
  const int32_t prog = (int32_t)blockIdx.x / csize;
  const int32_t nprog = (int32_t)gridDim.x / csize;
  const int tile_m = kPair ? 2 * p.rows : p.rows;  // MMA rows of a tile
  const int b_rows = kPair ? p.bn / 2 : p.bn;
  // a stage holds kc K blocks of each operand, stacked: block j of A at
  // j * a_blk, of B at j * (its box rows * 128), each a 128-byte-swizzled
  // K-major tile
  const uint32_t a_blk = (uint32_t)p.rows * 128;
  const uint32_t a_stage = a_blk * (uint32_t)p.kc;
  const uint32_t b_stage = (uint32_t)b_rows * 128 * (uint32_t)p.kc;
  const uint32_t a0 = base;
  const uint32_t b0 = base + a_stage * p.stages;
  const uint32_t cst = base + (uint32_t)p.body_bytes;           // epilogue staging
  const uint32_t bars = cst + (p.stage_c ? kStageC : 0u);
  // barrier block: full[16], empty[16], tfull[2], tempty[2], drain, two
  // words, recv (split-K)
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 128u + 8u * s; };
  auto tfull_bar = [&](int b) { return bars + 256u + 8u * b; };
  auto tempty_bar = [&](int b) { return bars + 272u + 8u * b; };
  const uint32_t drain_bar = bars + 288u;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + (bars - base) + 296u);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + (bars - base) + 300u);
  const uint32_t recv_bar = bars + 304u;

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), kPair ? 8 : 4);  // one arrive per epilogue warp (of both CTAs)
    }
    mbar_init(drain_bar, 1);
    mbar_init(recv_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
    tma_prefetch_desc(&map_a);
    tma_prefetch_desc(&map_b);
    if (p.ncut > 1) tma_prefetch_desc(&map_b_cut);
    if (p.stage_c) {
      tma_prefetch_desc(&map_c);
      tma_prefetch_desc(&map_c64);
    }
  }
  if (warp == 1) {
    if constexpr (kPair) {
      tmem_alloc_pair(smem_u32(tmem_slot), (uint32_t)p.tmem_cols);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(smem_u32(tmem_slot), (uint32_t)p.tmem_cols);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  if constexpr (kPair) cluster_sync();  // peer barriers initialised before any remote signal
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  // The prologue above touches no global memory, so it may overlap the tail
  // of the grid this launch depends on (programmatic dependent launch).
  grid_dependency_wait();
  allow_dependents();

  const int32_t TS = p.total_slots;
  const int32_t step = p.kind == TP_MAP_IDENTITY ? p.gm * p.gn : nprog;
  // S is a power of two and kslice * nk < 2^31 (nk < 2^25), so the slice
  // bounds are shifts rather than 64-bit divisions (hundreds of cycles)
  const int lgS = __ffs(S) - 1;
  const int32_t kb0 = ((int32_t)kslice * p.nk) >> lgS;
  const int32_t kb1 = ((int32_t)(kslice + 1) * p.nk) >> lgS;
  // split programs: the tile this CTA accumulated and whether its partial sum is complete
  int32_t sp_tm = 0, sp_tn = 0;
  bool sp_have = false;

  if (warp == 0) {
    // ---------------- TMA producer (one thread; the rest of the warp waits)
    if (lane == 0) {
      const uint64_t pol_a = policy_evict_last();
      const uint64_t pol_b = policy_evict_last();
      uint32_t fills[kMaxStages] = {};
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int32_t s = prog; s < TS && ok; s += step) {
        const Unit u = unit_of(s, p);
        int32_t tm, tn;
        raster((uint32_t)u.tile, (uint32_t)p.gm, (uint32_t)p.gn, (uint32_t)p.group_m, &tm, &tn);
        // a narrow tile loads only its own columns of B, through the map whose
        // box has that many rows
        const int ub_rows = kPair ? u.width / 2 : u.width;
        const CUtensorMap* mb = u.cut ? &map_b_cut : &map_b;
        const uint32_t utx = a_stage + (uint32_t)ub_rows * 128 * (uint32_t)p.kc;
        // swap-AB: the MMA's A operand is B^T (rows = C columns, tile column
        // tn) and its B operand is A (rows = C rows, tile row tm)
        const int32_t arow = (kSwap ? tn : tm) * tile_m + (int32_t)rank * p.rows;
        const int32_t brow = (kSwap ? tm : tn) * p.bn + u.col + (int32_t)rank * ub_rows;
        for (int32_t kb = kb0; kb < kb1; kb += p.kc) {
          if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, p.err, p.wait_ns)) { ok = false; break; }
          if (p.inject && s == prog && kb == kb0) {
            // test hook: this stage is never armed or filled, so its
            // consumer's bounded wait runs out
            if (++stage == p.stages) { stage = 0; phase ^= 1u; }
            continue;
          }
          // 2-D boxes take K at element kb * kblk; 3-D boxes take K block kb
          // (blocks past the last one are zero-filled and never multiplied)
          const int32_t kx = p.kc > 1 ? 0 : kb * p.kblk;
          if constexpr (kPair) {
            // both CTAs' copies complete on the even CTA's full barrier
            const uint32_t fb = mapa(full_bar(stage), 0);
            if (leader) mbar_arrive_expect_tx(full_bar(stage), 2 * utx);
            if (p.kc > 1) {
              tma_load_3d_pair(a0 + a_stage * stage, &map_a, 0, arow, kb, fb, pol_a);
              tma_load_3d_pair(b0 + b_stage * stage, mb, 0, brow, kb, fb, pol_b);
            } else {
              tma_load_2d_pair(a0 + a_stage * stage, &map_a, kx, arow, fb, pol_a);
              tma_load_2d_pair(b0 + b_stage * stage, mb, kx, brow, fb, pol_b);
            }
          } else {
            mbar_arrive_expect_tx(full_bar(stage), utx);
            if (p.kc > 1) {
              tma_load_3d(a0 + a_stage * stage, &map_a, 0, arow, kb, full_bar(stage), pol_a);
              tma_load_3d(b0 + b_stage * stage, mb, 0, brow, kb, full_bar(stage), pol_b);
            } else {
              tma_load_2d(a0 + a_stage * stage, &map_a, kx, arow, full_bar(stage), pol_a);
              tma_load_2d(b0 + b_stage * stage, mb, kx, brow, full_bar(stage), pol_b);
            }
          }
          fills[stage]++;
          if (++stage == p.stages) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok && (!kPair || leader)) {
        // drain: wait (bounded) until every copy signalled on our full
        // barriers landed (the odd CTA's copies signal the even CTA's)
        for (int s2 = 0; s2 < p.stages; ++s2)
          if (fills[s2]) mbar_wait(full_bar(s2), (fills[s2] - 1u) & 1u, nullptr, nullptr, 200000000ull);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer (one thread of the even CTA)
    if (lane == 0 && leader) {
      const uint32_t idesc_full = idesc_f32acc((uint32_t)tile_m, (uint32_t)p.bn, kF8);
      const uint32_t idesc_cut = idesc_f32acc((uint32_t)tile_m, (uint32_t)p.bn_cut, kF8);
      int stage = 0;
      uint32_t phase = 0;
      int32_t t = 0;
      bool ok = true;
      for (int32_t s = prog; s < TS && ok; s += step, ++t) {
        const Unit u = unit_of(s, p);
        const uint32_t idesc = u.cut ? idesc_cut : idesc_full;
        const uint32_t b_blk = (uint32_t)(kPair ? u.width / 2 : u.width) * 128;  // B box rows * 128
        const int acc = t & 1;
        const uint32_t use = (uint32_t)((t >> 1) & 1);
        if (!mbar_wait(tempty_bar(acc), use ^ 1u, abort_flag, p.err, p.wait_ns)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(acc * p.bn);
        for (int32_t kb = kb0; kb < kb1; kb += p.kc) {
          if (!mbar_wait(full_bar(stage), phase, abort_flag, p.err, p.wait_ns)) { ok = false; break; }
          tc_fence_after();
          // the stage's K blocks in K order, the same MMAs as one block per
          // stage (blocks past the tile's last are not multiplied)
          for (int32_t j = 0; j < p.kc && kb + j < kb1; ++j) {
            const uint64_t ad = desc_kmajor_sw128(a0 + a_stage * stage + a_blk * (uint32_t)j);
            const uint64_t bd = desc_kmajor_sw128(b0 + b_stage * stage + b_blk * (uint32_t)j);
            // 128-byte K slice = 4 MMAs of K = 16 (bf16) or K = 32 (fp8), 32
            // bytes apart inside the swizzle atom (start address advances by 32 >> 4).
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint32_t accum = (kb + j > kb0 || k > 0) ? 1u : 0u;
              if constexpr (kPair) mma_pair<kF8>(d, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc, accum);
              else mma<kF8>(d, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc, accum);
            }
          }
          if constexpr (kPair) mma_commit_pair(empty_bar(stage), 0x3);
          else mma_commit(empty_bar(stage));
          if (++stage == p.stages) { stage = 0; phase ^= 1u; }
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
  }

  // ------------------------------------------------------------ epilogue
  // (warps 2..5 -> TMEM lane quadrants 2,3,0,1)
  const int quad = warp & 3;
  // rows of this warp: 32 of a 128-row MMA, 16 (in lanes 0-15) of a 64-row
  // one
  int wrows = p.rows == BM ? 32 : 16;
  int32_t warp_row0 = (int32_t)rank * p.rows + quad * wrows;  // first tile row (MMA orientation) of this warp
  int32_t swap_col = 0;  // swap-AB: first MMA column of this warp
  if constexpr (kSwap) {
    // an M = 128 MMA on a CTA pair leaves each CTA 64 D rows: columns
    // [0, N/2) in TMEM lanes 0-63, columns [N/2, N) in lanes 64-127 (at TMEM
    // columns 0..N/2-1), so each warp holds 32 rows x N/2 columns
    wrows = 32;
    warp_row0 = (int32_t)rank * p.rows + (quad & 1) * 32;
    swap_col = (quad >> 1) * (p.bn / 2);
  }
  const uint32_t tlane = (uint32_t)(quad * 32) << 16;         // TMEM lane offset of this warp
  // FP8 dequantisation factor 1 / (s_A * s_B), both steps in fp32
  const float scale = (p.scale_a && p.scale_b) ? 1.f / (*p.scale_a * *p.scale_b) : 1.f;
  // this warp's two 4 KB staging buffers: 32 rows x 128 bytes (128-byte
  // swizzle) for a 64-column block, or 32 rows x 64 bytes (64-byte swizzle)
  // for a 32-column block
  const uint32_t stg = cst + (uint32_t)quad * 8192u;
  uint32_t nstaged = 0;
  // one row's 32 columns [c0, c0 + 32) of C from FP32 values f (plain stores)
  auto store_chunk = [&](const float* f, int64_t row, int64_t c0) {
    if (row >= p.M || c0 >= p.N) return;
    __nv_bfloat16* crow = p.c + row * p.N;
    if (p.c_vec != 0 && c0 + 32 <= p.N) {
      uint4 v[4];
      __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(v);
#pragma unroll
      for (int i = 0; i < 16; ++i) h[i] = __floats2bfloat162_rn(f[2 * i] * scale, f[2 * i + 1] * scale);
      uint4* dst = reinterpret_cast<uint4*>(crow + c0);
#pragma unroll
      for (int i = 0; i < 4; ++i) dst[i] = v[i];
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (c0 + i < p.N) crow[c0 + i] = __float2bfloat16_rn(f[i] * scale);
    }
    if constexpr (kCount) {
      for (int i = 0; i < 32; ++i)
        if (c0 + i < p.N) {
          atomicAdd(p.counts + row * p.N + c0 + i, 1u);
          p.owner[row * p.N + c0 + i] = (int32_t)prog;
        }
    }
  };
  // the wrows x 32 block of C at rows [row0, +wrows), columns [c0, +32):
  // lane i < wrows holds row row0 + i in f. Staged in shared memory and
  // written by one TMA store (the tensor map's box has wrows rows and is
  // clipped to C's bounds), or by per-row stores.
  auto store_block = [&](const float* f, int64_t row0, int64_t c0) {
    if (!kCount && p.stage_c) {
      if (row0 >= p.M || c0 >= p.N) return;  // warp-uniform: the block lies outside C
      const uint32_t buf = stg + (nstaged & 1u) * 4096u;
      if (lane == 0 && nstaged >= 2) bulk_wait_read<1>();  // the store issued from this buffer two blocks ago has read it
      __syncwarp();
      uint32_t w[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * i] * scale, f[2 * i + 1] * scale);
        w[i] = *reinterpret_cast<uint32_t*>(&h);
      }
      // 16-byte piece u of row `lane` sits at piece u ^ ((lane >> 1) & 3)
#pragma unroll
      for (int u = 0; u < 4; ++u)
        st_shared_v4(buf + (uint32_t)lane * 64u + ((uint32_t)(u ^ ((lane >> 1) & 3)) << 4), w[4 * u], w[4 * u + 1],
                     w[4 * u + 2], w[4 * u + 3]);
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        tma_store_2d(&map_c, buf, (int32_t)c0, (int32_t)row0);
        bulk_commit();
      }
      ++nstaged;
    } else {
      if (lane < wrows) store_chunk(f, row0 + lane, c0);
    }
  };
  // the wrows x 64 block at rows [row0, +wrows), columns [c0, +64) from two
  // TMEM chunks (lane i holds row row0 + i): staged with 16-byte piece u of
  // row `lane` at piece u ^ (lane & 7) and written by one TMA store (lanes
  // past wrows stage rows that the store's box leaves out)
  auto store_block64 = [&](const uint32_t* r0, const uint32_t* r1, int64_t row0, int64_t c0) {
    if (row0 >= p.M || c0 >= p.N) return;  // warp-uniform: the block lies outside C
    const uint32_t buf = stg + (nstaged & 1u) * 4096u;
    if (lane == 0 && nstaged >= 2) bulk_wait_read<1>();  // as in store_block
    __syncwarp();
    uint32_t w[32];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      __nv_bfloat162 h = __floats2bfloat162_rn(__uint_as_float(r0[2 * i]) * scale, __uint_as_float(r0[2 * i + 1]) * scale);
      w[i] = *reinterpret_cast<uint32_t*>(&h);
      h = __floats2bfloat162_rn(__uint_as_float(r1[2 * i]) * scale, __uint_as_float(r1[2 * i + 1]) * scale);
      w[16 + i] = *reinterpret_cast<uint32_t*>(&h);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      st_shared_v4(buf + (uint32_t)lane * 128u + ((uint32_t)(u ^ (lane & 7)) << 4), w[4 * u], w[4 * u + 1],
                   w[4 * u + 2], w[4 * u + 3]);
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
      tma_store_2d(&map_c64, buf, (int32_t)c0, (int32_t)row0);
      bulk_commit();
    }
    ++nstaged;
  };
  // swap-AB: lane i holds the MMA row n0 + i, i.e. column n0 + i of C, and
  // r its FP32 values in C rows [m0, m0 + cols): 2-byte stores, consecutive
  // lanes on consecutive columns
  auto store_swap = [&](const uint32_t* r, int64_t n0, int64_t m0, int cols) {
    const int64_t n = n0 + lane;
    if (n >= p.N || m0 >= p.M) return;
    const int lim = (int)min((int64_t)cols, p.M - m0);
    __nv_bfloat16* dst = p.c + m0 * p.N + n;
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if (i < lim) dst[(int64_t)i * p.N] = __float2bfloat16_rn(__uint_as_float(r[i]) * scale);
    if constexpr (kCount) {
      for (int i = 0; i < lim; ++i) {
        atomicAdd(p.counts + (m0 + i) * p.N + n, 1u);
        p.owner[(m0 + i) * p.N + n] = (int32_t)prog;
      }
    }
  };
  bool counted = false;
  // Checked launch: each epilogue warp counts itself done right after its
  // last claim (still ahead of its last accumulator); the warp that counts
  // last clears the bitmap for the next launch. A warp that leaves its loop
  // early counts itself at the exit.
  auto finish_claims = [&]() {
    if (counted) return;
    counted = true;
    int last = 0;
    if (lane == 0) {
      __threadfence();
      last = atomicAdd(p.claim_done, 1u) == gridDim.x * 4u - 1u ? 1 : 0;
    }
    if (__shfl_sync(0xffffffffu, last, 0)) {
      __threadfence();
      const int64_t words = (p.claim_bits + 31) / 32;
      for (int64_t i = lane; i < words; i += 32) p.claims[i] = 0u;
      if (lane == 0) *p.claim_done = 0u;
    }
  };
  if (warp >= 2) {
    const uint32_t tempty_remote = kPair ? mapa(tempty_bar(0), 0) : 0u;
    int32_t t = 0;
    // validate a store against the map (the slot is this program's and its
    // tile lies in the grid), then claim this warp's 32-row slice of the
    // (narrow) tile or K-slice part: (tile, part, CTA of the pair, lane
    // quadrant); warp-uniform result
    auto claim = [&](int32_t s, int32_t tm, int32_t tn, int32_t part) -> bool {
      int ok = 1;
      if (lane == 0) {
        const bool on_map = s < TS && (s - prog) % step == 0 && tm >= 0 && tm < p.gm && tn >= 0 && tn < p.gn;
        if (!on_map) {
          record_device_error(p.err, kDevRace);
          ok = 0;
        } else {
          const int64_t id = ((((int64_t)tm * p.gn + tn) * p.parts + part) * (kPair ? 2 : 1) + rank) * 4 + quad;
          ok = claim_tile(p.claims, id, p.err) ? 1 : 0;
        }
      }
      return __shfl_sync(0xffffffffu, ok, 0) != 0;
    };
    auto release_acc = [&](int acc) {
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if constexpr (kPair) mbar_arrive_cluster(tempty_remote + 8u * acc);
        else mbar_arrive(tempty_bar(acc));
      }
    };
    for (int32_t s = prog; s < TS; s += step, ++t) {
      const Unit u = unit_of(s, p);
      const int acc = t & 1;
      const uint32_t use = (uint32_t)((t >> 1) & 1);
      int32_t tm, tn;
      raster((uint32_t)u.tile, (uint32_t)p.gm, (uint32_t)p.gn, (uint32_t)p.group_m, &tm, &tn);
      bool store_ok = true;
      // claimed before the accumulator is ready, so the atomic's latency
      // hides behind the K loop
      if constexpr (kChecked) {
        store_ok = claim(s, tm, tn, S > 1 ? (int32_t)kslice : u.part);
        if (s + step >= TS) finish_claims();
      }
      const bool ready = mbar_wait(tfull_bar(acc), use, abort_flag, p.err, p.wait_ns);
      if (!__all_sync(0xffffffffu, ready)) break;  // leave together (tcgen05.ld is warp-collective)
      tc_fence_after();
      if (S > 1) {
        // split program: the partial sum meets the others' below
        sp_have = store_ok;
        sp_tm = tm;
        sp_tn = tn;
        break;
      }
      // first tile row and column of this warp in MMA orientation (swap-AB:
      // rows are C columns, columns C rows)
      const int64_t row0 = (int64_t)(kSwap ? tn : tm) * tile_m + warp_row0;
      const int64_t col0 = (int64_t)(kSwap ? tm : tn) * p.bn + u.col;
      const uint32_t tacc = tmem_base + tlane + (uint32_t)(acc * p.bn);
      if constexpr (kSwap) {
        // this warp's N/2 MMA columns (C rows) in chunks of 32
        const int half = p.bn / 2;
#pragma unroll 1
        for (int ch = 0; ch * 32 < half && store_ok; ++ch) {
          uint32_t r[32];
          tmem_ld32(tacc + (uint32_t)(ch * 32), r);
          tmem_ld_wait();
          store_swap(r, row0, col0 + swap_col + ch * 32, min(32, half - ch * 32));
        }
        release_acc(acc);
        continue;
      }
      const int nch = u.width / 32;
      int ch = 0;
      if (!kCount && p.stage_c) {
        for (; ch + 1 < nch && store_ok; ch += 2) {
          uint32_t r0[32], r1[32];
          tmem_ld32(tacc + (uint32_t)(ch * 32), r0);
          tmem_ld32(tacc + (uint32_t)(ch * 32 + 32), r1);
          tmem_ld_wait();
          store_block64(r0, r1, row0, col0 + ch * 32);
        }
      }
      for (; ch < nch && store_ok; ++ch) {
        uint32_t r[32];
        tmem_ld32(tacc + (uint32_t)(ch * 32), r);
        tmem_ld_wait();
        float f[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) f[i] = __uint_as_float(r[i]);
        store_block(f, row0, col0 + ch * 32);
      }
      release_acc(acc);
    }
  }

  if (!kPair && S > 1) {
    // ---------------- split-K reduction across the cluster's CTAs
    // Column slice j (width w = bn / S) of the tile belongs to CTA j. Every
    // CTA copies its partial sums of the other slices, as 4 KB blocks (one
    // lane quadrant x 32 columns, 16-byte pieces lane-major), from a send
    // area into the owners' receive areas; both areas overlay the operand
    // ring, idle once every CTA's MMAs have completed. The copies complete on
    // the owner's recv barrier; the owner then adds the S partials of its
    // slice in slice order 0..S-1 and stores the slice.
    const int32_t w = p.bn / S;
    const int32_t nch = w / 32;
    const uint32_t slot_bytes = 128u * (uint32_t)w * 4u;  // one source's partial of one slice
    const uint32_t send0 = a0 + (uint32_t)(S - 1) * slot_bytes;
    const bool tile = prog < TS;  // the same for every CTA of the cluster
    auto block = [&](uint32_t area, int32_t slot, int32_t ch) {
      return area + (uint32_t)((slot * 4 + quad) * nch + ch) * 4096u;
    };
    if (warp == 2 && lane == 0 && tile) mbar_arrive_expect_tx(recv_bar, (uint32_t)(S - 1) * slot_bytes);
    cluster_sync();  // (1) every CTA's accumulator is final and its ring is free
    if (warp >= 2 && tile) {
      for (int32_t j = 0; j < S; ++j) {
        if (j == (int32_t)kslice) continue;
        const int32_t dslot = j < (int32_t)kslice ? j : j - 1;                  // among this CTA's destinations
        const int32_t rslot = (int32_t)kslice < j ? (int32_t)kslice : (int32_t)kslice - 1;  // at the owner
        for (int32_t ch = 0; ch < nch; ++ch) {
          uint32_t r[32];
          tmem_ld32(tmem_base + tlane + (uint32_t)(j * w + ch * 32), r);
          tmem_ld_wait();
          const uint32_t src = block(send0, dslot, ch);
#pragma unroll
          for (uint32_t q = 0; q < 8; ++q)
            st_shared_v4(src + q * 512u + (uint32_t)lane * 16u, r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0)
            bulk_copy_to_cluster(mapa(block(a0, rslot, ch), (uint32_t)j), src, 4096u, mapa(recv_bar, (uint32_t)j));
        }
      }
    }
    if (warp >= 2 && tile) {
      // not cut short by the abort flag: the peers' copies into this CTA's
      // shared memory must land before it can retire (they are issued right
      // after barrier (1), so the bounded wait ends well within its limit)
      const bool got = mbar_wait(recv_bar, 0, nullptr, p.err, p.wait_ns);
      if (__all_sync(0xffffffffu, got) && sp_have) {
        const int64_t row0 = (int64_t)sp_tm * tile_m + warp_row0;
        const int64_t col0 = (int64_t)sp_tn * p.bn + (int64_t)kslice * w;
        for (int32_t ch = 0; ch < nch; ++ch) {
          float f[32];
          for (int32_t src = 0; src < S; ++src) {
            uint32_t v[32];
            if (src == (int32_t)kslice) {
              tmem_ld32(tmem_base + tlane + (uint32_t)((int32_t)kslice * w + ch * 32), v);
              tmem_ld_wait();
            } else {
              const uint32_t at = block(a0, src < (int32_t)kslice ? src : src - 1, ch);
#pragma unroll
              for (uint32_t q = 0; q < 8; ++q) ld_shared_v4(at + q * 512u + (uint32_t)lane * 16u, v + 4 * q);
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) f[i] = src == 0 ? __uint_as_float(v[i]) : f[i] + __uint_as_float(v[i]);
          }
          store_block(f, row0, col0 + ch * 32);
        }
      }
    }
    cluster_sync();  // (2) every copy into every CTA of the cluster has completed (sources read)
  }
  if (warp >= 2) {
    if constexpr (kChecked) finish_claims();
    if (!kCount && p.stage_c && lane == 0) bulk_wait_all();  // C written before the CTA retires
    __syncwarp();
  }
  if constexpr (kPair) settle_after_abort(abort_flag);
  tc_fence_before();
  if constexpr (kPair) cluster_sync();  // the peer no longer touches our shared memory / TMEM
  else __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    if constexpr (kPair) tmem_dealloc_pair(tmem_base, (uint32_t)p.tmem_cols);
    else tmem_dealloc(tmem_base, (uint32_t)p.tmem_cols);
  }
}

// ---------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

// K-major operand: `rows` rows of `k` elements, row stride `ld` elements,
// box of `box_rows` rows x 128 bytes, 128-byte swizzle, zero fill out of bounds.
tp_status make_map(CUtensorMap* map, const void* ptr, int64_t rows, int64_t k, int64_t ld, int esize,
                   int box_rows) {
  auto fn = encode_fn();
  if (!fn) return fail(TP_ERR_CUDA, "cuTensorMapEncodeTiled unavailable from the driver");
  cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * esize)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / esize), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                  const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(TP_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return TP_OK;
}

// K-major operand seen as 3-D {K block element, row, K block}: a box of
// {128 bytes, box_rows, kc} brings kc consecutive K blocks of box_rows rows
// in one copy, stacked in shared memory as kc 128-byte-swizzled K-major
// tiles. Needs k a multiple of the K block (128 bytes).
tp_status make_map3(CUtensorMap* map, const void* ptr, int64_t rows, int64_t k, int64_t ld, int esize, int box_rows,
                    int kc) {
  auto fn = encode_fn();
  if (!fn) return fail(TP_ERR_CUDA, "cuTensorMapEncodeTiled unavailable from the driver");
  const int kblk = 128 / esize;
  cuuint64_t dims[3] = {(cuuint64_t)kblk, (cuuint64_t)rows, (cuuint64_t)(k / kblk)};
  cuuint64_t strides[2] = {(cuuint64_t)(ld * esize), 128};
  cuuint32_t box[3] = {(cuuint32_t)kblk, (cuuint32_t)box_rows, (cuuint32_t)kc};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 3,
                  const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(TP_ERR_CUDA, "cuTensorMapEncodeTiled (3-D) failed (" + std::to_string((int)r) + ")");
  return TP_OK;
}

// The tensor maps of a launch: A, B, B for narrow tiles, C in 32- and
// 64-column boxes (TMA stores).
struct Maps {
  CUtensorMap a, b, b_cut, c, c64;
};

template <bool kF8, bool kPair, bool kCount, bool kChecked, bool kSwap = false>
cudaError_t launch_kernel(const Maps& m, const TcArgs& p, int grid, int csize, size_t smem, cudaStream_t st) {
  auto k = gemm_tc_kernel<kF8, kPair, kCount, kChecked, kSwap>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k, m.a, m.b, m.b_cut, m.c, m.c64, p);
}

template <bool kF8, bool kPair>
cudaError_t launch_inst(bool count, bool checked, const Maps& m, const TcArgs& p, int grid, int csize, size_t smem,
                        cudaStream_t st) {
  if (checked) return count ? launch_kernel<kF8, kPair, true, true>(m, p, grid, csize, smem, st)
                            : launch_kernel<kF8, kPair, false, true>(m, p, grid, csize, smem, st);
  return count ? launch_kernel<kF8, kPair, true, false>(m, p, grid, csize, smem, st)
               : launch_kernel<kF8, kPair, false, false>(m, p, grid, csize, smem, st);
}

// swap-AB tiles: BF16 on CTA pairs
cudaError_t launch_swap(bool count, bool checked, const Maps& m, const TcArgs& p, int grid, size_t smem,
                        cudaStream_t st) {
  if (checked) return count ? launch_kernel<false, true, true, true, true>(m, p, grid, 2, smem, st)
                            : launch_kernel<false, true, false, true, true>(m, p, grid, 2, smem, st);
  return count ? launch_kernel<false, true, true, false, true>(m, p, grid, 2, smem, st)
               : launch_kernel<false, true, false, false, true>(m, p, grid, 2, smem, st);
}

template <bool kF8>
cudaError_t launch_any(bool pair, bool count, bool checked, const Maps& m, const TcArgs& p, int grid, int csize,
                       size_t smem, cudaStream_t st) {
  return pair ? launch_inst<kF8, true>(count, checked, m, p, grid, csize, smem, st)
              : launch_inst<kF8, false>(count, checked, m, p, grid, csize, smem, st);
}

// Clusters of `csize` CTAs (a CTA pair, a split program, or single CTAs) of
// the kernel that can be resident at once (0 when the query fails).
template <bool kPair>
int max_active_clusters(int csize, size_t smem) {
  auto k = gemm_tc_kernel<false, kPair, false, false>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448) != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)csize);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// Shared-memory plan of a launch: ring stages, the region before the
// epilogue staging (the ring, or the larger split-K receive buffer), whether
// the epilogue stages C blocks, and the dynamic size requested.
struct SmemPlan {
  int kc = 1;  // K blocks per stage
  int stages = 0;
  size_t body = 0;
  bool stage_c = false;
  size_t smem = 0;
};

constexpr size_t kSmemFixed = 1024 + 320;  // alignment slack + barriers (312 bytes)
constexpr size_t kSmemBudget = 232448;     // 227 KB opt-in

// stages_req = 0 asks for the deepest ring that fits beside the staging
// area. The staging area is dropped (per-row stores) when an explicitly
// requested ring leaves no room for it.
// kc_req: K blocks per stage asked for; the plan takes the largest count up
// to it that leaves room for two stages, preferring a plan that keeps the
// epilogue's staging area.
tp_status plan_smem(bool pair, int rows, int bn, int kc_req, int split, int stages_req, bool want_stage_c,
                    SmemPlan* out) {
  // split-K: receive and send areas of (split - 1) slice partials each
  const size_t recv = split > 1 ? 2 * (size_t)(split - 1) * 128 * (size_t)(bn / split) * 4 : 0;
  for (int stage_c = want_stage_c ? 1 : 0; stage_c >= 0; --stage_c) {
    const size_t stg = stage_c ? kStageC : 0;
    for (int kc = kc_req; kc >= 1; kc /= 2) {
      const size_t stage_bytes = ((size_t)rows * 128 + (size_t)(pair ? bn / 2 : bn) * 128) * (size_t)kc;
      int stages = stages_req > 0 ? stages_req : (int)((kSmemBudget - kSmemFixed - stg) / stage_bytes);
      stages = stages > kMaxStages ? kMaxStages : stages;
      if (stages < 2) continue;
      size_t body = std::max((size_t)stages * stage_bytes, recv);
      body = (body + 1023) & ~(size_t)1023;
      if (kSmemFixed + body + stg > kSmemBudget) continue;
      out->kc = kc;
      out->stages = stages;
      out->body = body;
      out->stage_c = stage_c != 0;
      out->smem = kSmemFixed + body + stg;
      return TP_OK;
    }
  }
  return fail(TP_ERR_UNSUPPORTED, "shared memory too small for the requested stages");
}

// C (bf16, N columns, row stride N) as boxes of `rows` (16 or 32) rows x
// `cols` columns (32: 64-byte swizzle, 64: 128-byte swizzle) matching the
// epilogue's staging layouts.
tp_status make_map_c(CUtensorMap* map, void* ptr, int64_t M, int64_t N, int cols, int rows) {
  auto fn = encode_fn();
  if (!fn) return fail(TP_ERR_CUDA, "cuTensorMapEncodeTiled unavailable from the driver");
  cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)M};
  cuuint64_t strides[1] = {(cuuint64_t)(N * 2)};
  cuuint32_t box[2] = {(cuuint32_t)cols, (cuuint32_t)rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, cols == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(TP_ERR_CUDA, "cuTensorMapEncodeTiled (C) failed (" + std::to_string((int)r) + ")");
  return TP_OK;
}

}  // namespace

// Shared by the BF16 and FP8 entry points. esize = 2 (bf16) or 1 (fp8).
tp_status launch_gemm_tc_impl(tp_ctx* ctx, tp_partition* c, const tp_tensor* a, const tp_tensor* b,
                              const tp_gemm_config* cfg, const tp_exec* ex, cudaStream_t stream, int esize,
                              const float* scale_a, const float* scale_b) {
  const int64_t M = a->shape[0], K = a->shape[1], N = b->shape[1];
  if ((ex->write_counts == nullptr) != (ex->write_owner == nullptr))
    return fail(TP_ERR_INVALID, "write_counts and write_owner must be given together");
  if (c->kind == TP_MAP_QUEUE) return fail(TP_ERR_UNSUPPORTED, "the tensor-core GEMM maps tiles by slot (identity/strided)");
  const int tile_r = (int)c->tile[0], tile_c = (int)c->tile[1];  // the partition's tile of C
  if (cfg && cfg->bm && cfg->bm != tile_r) return fail(TP_ERR_SHAPE, "cfg.bm differs from the partition's tile");
  if (cfg && cfg->bn && cfg->bn != tile_c) return fail(TP_ERR_SHAPE, "cfg.bn differs from the partition's tile");
  // swap-AB (cfg.swap_ab): a C tile of W rows x 128 columns is computed as
  // C^T = B^T A^T by a CTA pair, the MMA's 128 rows being C's columns (64
  // per CTA) and its W columns C's rows (W/2 rows of A per CTA)
  if (cfg && (cfg->swap_ab < 0 || cfg->swap_ab > 1)) return fail(TP_ERR_INVALID, "swap_ab must be 0 or 1");
  const bool swap = cfg && cfg->swap_ab == 1;
  int bm, bn;  // MMA tile: rows (256 = CTA pair) and columns
  if (swap) {
    if (esize != 2) return fail(TP_ERR_UNSUPPORTED, "swap_ab applies to the BF16 GEMM");
    if (tile_c != BM || (tile_r != 32 && tile_r != 64 && tile_r != 128))
      return fail(TP_ERR_UNSUPPORTED, "swap_ab tiles have 32, 64 or 128 rows and 128 columns");
    if (cfg->split_k > 1) return fail(TP_ERR_UNSUPPORTED, "swap_ab and split_k do not combine");
    if (ex->flags & TP_EXEC_INJECT_TIMEOUT) return fail(TP_ERR_UNSUPPORTED, "TP_EXEC_INJECT_TIMEOUT applies to 128-row tiles");
    bm = 2 * BM;  // a CTA pair
    bn = tile_r;
  } else {
    bm = tile_r;
    bn = tile_c;
    if (bm != BM / 2 && bm != BM && bm != 2 * BM)
      return fail(TP_ERR_UNSUPPORTED, "tensor-core GEMM tiles have 64 or 128 rows (one CTA) or 256 rows (CTA pair)");
    if (bn < 32 || bn > 256 || bn % 32 || (bm == 2 * BM && bn % 64))
      return fail(TP_ERR_UNSUPPORTED, "tile columns must be 32..256, a multiple of 32 (of 64 for 256-row tiles)");
  }
  const bool pair = bm == 2 * BM;
  const int rows = swap ? BM / 2 : pair ? BM : bm;  // MMA rows per CTA and stage
  // K-major operands: A row-major (stride along K = 1), B stored N x K.
  if (a->strides[1] != 1 || b->strides[0] != 1)
    return fail(TP_ERR_UNSUPPORTED, "tensor-core GEMM needs K-major A (row-major M x K) and K-major B (stored N x K)");
  const int64_t lda = a->strides[0], ldb = b->strides[1];
  if (((uintptr_t)a->ptr & 15) || ((uintptr_t)b->ptr & 15) || ((lda * esize) & 15) || ((ldb * esize) & 15) ||
      (K * esize) % 16)
    return fail(TP_ERR_ALIGN, "TMA needs 16-byte aligned bases and row strides (K a multiple of 16 bytes)");
  if (M == 0 || N == 0) return TP_OK;
  if (K == 0) return fail(TP_ERR_UNSUPPORTED, "K = 0");
  const int64_t T = c->num_tiles;
  // slots (tiles, or narrow tiles: up to 8 per tile) are counted in 32 bits
  if (T >= ((int64_t)1 << 28) || M >= ((int64_t)1 << 31) || N >= ((int64_t)1 << 31) || K >= ((int64_t)1 << 31))
    return fail(TP_ERR_UNSUPPORTED, "tensor-core GEMM: 2^28 tiles or more, or an extent of 2^31");
  const int64_t progs = c->kind == TP_MAP_IDENTITY ? T : c->num_programs;
  const int kblk = 128 / esize;
  const int64_t nk = (K + kblk - 1) / kblk;
  const int32_t split = (cfg && cfg->split_k > 1) ? cfg->split_k : 1;
  if (cfg && (cfg->split_k < 0 || cfg->split_k > 8 || (split > 1 && (split & (split - 1)))))
    return fail(TP_ERR_INVALID, "split_k must be 0, 1, 2, 4 or 8");
  if (split > 1) {
    if (bm != BM) return fail(TP_ERR_UNSUPPORTED, "split_k applies to 128-row tiles (one CTA per K slice)");
    if (bn % (32 * split)) return fail(TP_ERR_UNSUPPORTED, "split_k needs tile columns a multiple of 32 * split_k");
    if (nk < split) return fail(TP_ERR_UNSUPPORTED, "split_k exceeds the number of K blocks");
    if (progs < T) return fail(TP_ERR_UNSUPPORTED, "split_k needs at most one tile per program");
  }
  // K blocks per stage from cfg->bk (a multiple of the K block); one block
  // per stage (2-D boxes) when K is not a multiple of the K block or the
  // program splits K
  int32_t kc = 1;
  if (cfg && cfg->bk > 0) {
    if (cfg->bk % kblk || (cfg->bk / kblk != 1 && cfg->bk / kblk != 2 && cfg->bk / kblk != 4))
      return fail(TP_ERR_INVALID, "bk must be 1, 2 or 4 K blocks (64 bf16 / 128 fp8 elements each)");
    kc = cfg->bk / kblk;
  }
  if (K % kblk || split > 1) kc = 1;
  const int32_t limit = (cfg && cfg->cut_limit > 0) ? cfg->cut_limit : 4;
  if (cfg && (cfg->cut_limit < 0 || cfg->cut_limit > 8)) return fail(TP_ERR_INVALID, "cut_limit must be 0..8");
  const bool count = ex->write_counts != nullptr;
  const bool checked = (ex->flags & TP_EXEC_CHECKED) != 0;
  Maps maps;
  tp_status s = TP_OK;
  TcArgs p{};
  p.M = M;
  p.N = N;
  p.K = K;
  p.gm = (int32_t)c->grid[0];
  p.gn = (int32_t)c->grid[1];
  p.rows = rows;
  p.bn = bn;
  p.kind = c->kind;
  p.group_m = (c->kind != TP_MAP_IDENTITY && cfg && cfg->group_m > 0) ? cfg->group_m : 1;
  if (p.group_m > p.gm) p.group_m = p.gm;
  p.kblk = kblk;
  p.nk = (int32_t)nk;

  p.split = split;
  p.c_vec = (N % 8 == 0) && (((uintptr_t)c->t.ptr & 15) == 0);
  p.c = static_cast<__nv_bfloat16*>(c->t.ptr);
  p.scale_a = scale_a;
  p.scale_b = scale_b;
  p.err = ctx->d_err;
  p.counts = ex->write_counts;
  p.owner = ex->write_owner;
  int cols = 32;
  while (cols < 2 * bn) cols *= 2;
  p.tmem_cols = cols;
  SmemPlan plan;
  // swap-AB tiles store C with plain stores: no staging area
  s = plan_smem(pair, rows, bn, kc, split, cfg ? cfg->stages : 0, p.c_vec && !count && !swap, &plan);
  if (s != TP_OK) return s;
  kc = plan.kc;
  p.kc = kc;
  auto operand_map = [&](CUtensorMap* m, const void* ptr, int64_t rws, int64_t ld, int box_rows) {
    return kc > 1 ? make_map3(m, ptr, rws, K, ld, esize, box_rows, kc) : make_map(m, ptr, rws, K, ld, esize, box_rows);
  };
  // the MMA's operands: A (rows of A) and B (rows of B^T), or swapped
  s = swap ? operand_map(&maps.a, b->ptr, N, ldb, rows) : operand_map(&maps.a, a->ptr, M, lda, rows);
  if (s != TP_OK) return s;
  s = swap ? operand_map(&maps.b, a->ptr, M, lda, bn / 2) : operand_map(&maps.b, b->ptr, N, ldb, pair ? bn / 2 : bn);
  if (s != TP_OK) return s;
  maps.b_cut = maps.b;
  p.stages = plan.stages;
  p.body_bytes = (int32_t)plan.body;
  p.stage_c = plan.stage_c ? 1 : 0;
  if (plan.stage_c) {
    const int store_rows = rows == BM / 2 ? 16 : 32;  // rows of C one epilogue warp holds
    s = make_map_c(&maps.c, c->t.ptr, M, N, 32, store_rows);
    if (s == TP_OK) s = make_map_c(&maps.c64, c->t.ptr, M, N, 64, store_rows);
    if (s != TP_OK) return s;
  } else {
    maps.c = maps.c64 = maps.a;  // unused
  }
  const int csize = pair ? 2 : split;
  const int64_t grid = progs * csize;
  if (grid >= ((int64_t)1 << 31)) return fail(TP_ERR_UNSUPPORTED, "grid too large");
  // Schedule: whole tiles, except that on a strided map the R = T mod P tiles
  // of the last, partial round may each be cut along N into S narrow tiles
  // run by the programs that would otherwise sit idle in that round (not in
  // split-K programs, which hold one tile each).
  p.dp_slots = (int32_t)T;
  p.total_slots = (int32_t)T;
  p.ncut = 1;
  p.bn_cut = bn;
  if (c->kind == TP_MAP_STRIDED && split == 1 && !swap) {
    const int64_t R = T % progs;
    const int unit = pair ? 64 : 32;  // narrow tiles keep whole 32-row B boxes per CTA
    int64_t S = 1;
    while (R > 0 && 2 * S <= limit && 2 * S <= progs / R && bn % (2 * S * unit) == 0) S *= 2;
    if (S >= 2) {
      p.ncut = (int32_t)S;
      p.bn_cut = (int32_t)(bn / S);
      p.dp_slots = (int32_t)(T - R);
      p.total_slots = (int32_t)(T - R + R * S);
      s = operand_map(&maps.b_cut, b->ptr, N, ldb, pair ? p.bn_cut / 2 : p.bn_cut);
      if (s != TP_OK) return s;
    }
  }
  p.parts = p.ncut * split;
  p.wait_ns = 2000000000ull;
  if (ex->flags & TP_EXEC_INJECT_TIMEOUT) {
    if (pair) return fail(TP_ERR_UNSUPPORTED, "TP_EXEC_INJECT_TIMEOUT applies to 128-row tiles");
    p.inject = 1;
    p.wait_ns = 50000000ull;
  }
  if (checked) {
    p.claim_bits = T * p.parts * (pair ? 8 : 4);
    s = claims_for(ctx, p.claim_bits, &p.claims, &p.claim_done);
    if (s != TP_OK) return s;
  }
  cudaError_t e = swap         ? launch_swap(count, checked, maps, p, (int)grid, plan.smem, stream)
                 : esize == 2 ? launch_any<false>(pair, count, checked, maps, p, (int)grid, csize, plan.smem, stream)
                              : launch_any<true>(pair, count, checked, maps, p, (int)grid, csize, plan.smem, stream);
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core GEMM launch");
  return TP_OK;
}

tp_status gemm_tc_resident(tp_ctx* ctx, const tp_gemm_config* cfg, int32_t* programs) {
  const int kc = cfg->bk >= 256 ? 4 : cfg->bk >= 128 ? 2 : 1;  // K blocks per stage (bf16 K blocks of 64)
  (void)ctx;
  if (cfg->swap_ab < 0 || cfg->swap_ab > 1) return fail(TP_ERR_INVALID, "swap_ab must be 0 or 1");
  if (cfg->swap_ab) {
    // swap-AB tiles: CTA pairs, each CTA holding 64 rows of B^T and W/2 rows
    // of A per K block, no staging area
    const int w = cfg->bm ? cfg->bm : BM;
    if ((w != 32 && w != 64 && w != 128) || (cfg->bn && cfg->bn != BM))
      return fail(TP_ERR_UNSUPPORTED, "swap_ab tiles have 32, 64 or 128 rows and 128 columns");
    if (cfg->split_k > 1) return fail(TP_ERR_UNSUPPORTED, "swap_ab and split_k do not combine");
    SmemPlan plan;
    tp_status s = plan_smem(true, BM / 2, w, kc, 1, cfg->stages, false, &plan);
    if (s != TP_OK) return s;
    const int pairs = max_active_clusters<true>(2, plan.smem);
    if (pairs <= 0) return fail(TP_ERR_CUDA, "cudaOccupancyMaxActiveClusters failed");
    *programs = pairs;
    return TP_OK;
  }
  const int bm = cfg->bm ? cfg->bm : BM, bn = cfg->bn ? cfg->bn : 256;
  if (bm != BM / 2 && bm != BM && bm != 2 * BM) return fail(TP_ERR_UNSUPPORTED, "tiles have 64, 128 or 256 rows");
  const bool pair = bm == 2 * BM;
  const int split = cfg->split_k > 1 ? cfg->split_k : 1;
  if (split > 8 || (split & (split - 1))) return fail(TP_ERR_INVALID, "split_k must be 0, 1, 2, 4 or 8");
  if (split > 1 && bm != BM) return fail(TP_ERR_UNSUPPORTED, "split_k applies to 128-row tiles");
  SmemPlan plan;
  tp_status s = plan_smem(pair, pair ? BM : bm, bn, kc, split, cfg->stages, true, &plan);
  if (s != TP_OK) return s;
  const int csize = pair ? 2 : split;
  const int clusters = pair ? max_active_clusters<true>(csize, plan.smem) : max_active_clusters<false>(csize, plan.smem);
  if (clusters <= 0) return fail(TP_ERR_CUDA, "cudaOccupancyMaxActiveClusters failed");
  *programs = clusters;  // CTA pairs (256-row tiles), split programs, or CTAs
  return TP_OK;
}

tp_status launch_gemm_tc(tp_ctx* ctx, tp_partition* c, const tp_tensor* a, const tp_tensor* b,
                         const tp_gemm_config* cfg, const tp_exec* ex, cudaStream_t stream, unsigned* queue) {
  (void)queue;
  return launch_gemm_tc_impl(ctx, c, a, b, cfg, ex, stream, 2, nullptr, nullptr);
}

}  // namespace tp
