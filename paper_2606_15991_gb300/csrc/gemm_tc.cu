// Tensor-core GEMM for sm_103a: C (bf16) = A . B with BF16 (kind::f16) or
// FP8-E4M3 (kind::f8f6f4) operands and FP32 accumulation in TMEM.
//
// One output tile of 128 x BN (one CTA) or 256 x BN (a CTA pair running
// cta_group::2 MMAs) per tile program step, with a K loop (§3.6, Listing 6:
// the program walks its mapped sequence of output tiles and, for each,
// accumulates mma over the K tiles). On a strided map the tiles of the last,
// partial round may be cut along N into narrow tiles for programs that would
// otherwise idle. A persistent CTA (or CTA pair) runs one program:
//   warp 0   TMA producer: streams (A, B) K-slices into a ring of shared-
//            memory stages (128-byte swizzle), guarded by full/empty mbarriers;
//   warp 1   MMA issuer: one thread issues tcgen05.mma into one of two TMEM
//            accumulators and commits each consumed stage back to the producer;
//   warps 2-5 epilogue: tcgen05.ld the finished accumulator (each warp owns the
//            32 TMEM lanes = tile rows its warp index selects), scale, round to
//            bf16 and store only inside this program's tile, while the MMA
//            warp already fills the other accumulator.
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
constexpr int kMaxStages = 8;

struct TcArgs {
  int64_t M, N, K;
  int64_t gm, gn;       // tile grid
  int32_t bn;           // tile columns (32..256, multiple of 32)
  int32_t stages;
  int32_t kind;         // tp_map_kind (IDENTITY or STRIDED)
  int32_t group_m;
  int32_t tmem_cols;    // allocated TMEM columns (2 * bn rounded to a power of two)
  int32_t c_vec;        // C rows are 16-byte aligned (N % 8 == 0, aligned base)
  int32_t kblk;         // K elements per stage (64 bf16 / 128 fp8)
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
  int64_t dp_slots;
  int64_t total_slots;  // dp_slots + (tiles - dp_slots) * ncut
  int32_t ncut;         // 1 = no tile is cut
  int32_t bn_cut;       // bn / ncut
};

// The work of one slot: a tile and the columns [col, col + width) of it.
struct Unit {
  int64_t tile;
  int32_t col, width, part;
  bool cut;
};

__device__ __forceinline__ Unit unit_of(int64_t s, const TcArgs& p) {
  Unit u;
  if (s < p.dp_slots) {
    u.tile = s;
    u.col = 0;
    u.width = p.bn;
    u.part = 0;
    u.cut = false;
  } else {
    const int64_t q = s - p.dp_slots;
    u.tile = p.dp_slots + q / p.ncut;
    u.part = (int32_t)(q % p.ncut);
    u.col = u.part * p.bn_cut;
    u.width = p.bn_cut;
    u.cut = true;
  }
  return u;
}

__device__ __forceinline__ void raster(int64_t s, int64_t gm, int64_t gn, int64_t g, int64_t* tm, int64_t* tn) {
  const int64_t per = g * gn;
  const int64_t first = (s / per) * g;
  const int64_t rows = min(g, gm - first);
  const int64_t r = s % per;
  *tm = first + r % rows;
  *tn = r / rows;
}

template <bool kF8, bool kPair, bool kCount, bool kChecked>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                   const __grid_constant__ CUtensorMap map_b_cut, const __grid_constant__ TcArgs p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);

  const int warp = threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  // A CTA pair computes a 256-row tile: this CTA holds rows [rank*128, +128)
  // of A and of the accumulator, and B rows (tile columns) [rank*bn/2, +bn/2).
  const uint32_t rank = kPair ? cluster_ctarank() : 0u;
  const bool leader = rank == 0;
  const int64_t prog = kPair ? (int64_t)(blockIdx.x / 2) : (int64_t)blockIdx.x;
  const int64_t nprog = kPair ? (int64_t)(gridDim.x / 2) : (int64_t)gridDim.x;
  const int tile_m = kPair ? 2 * BM : BM;
  const int b_rows = kPair ? p.bn / 2 : p.bn;
  const uint32_t a_stage = BM * 128;
  const uint32_t b_stage = (uint32_t)b_rows * 128;
  const uint32_t a0 = base;
  const uint32_t b0 = base + a_stage * p.stages;
  const uint32_t bars = b0 + b_stage * p.stages;
  // barrier block: full[8], empty[8], tfull[2], tempty[2], drain, then words
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 64u + 8u * s; };
  auto tfull_bar = [&](int b) { return bars + 128u + 8u * b; };
  auto tempty_bar = [&](int b) { return bars + 144u + 8u * b; };
  const uint32_t drain_bar = bars + 160u;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + (bars - base) + 168u);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + (bars - base) + 172u);

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
    *abort_flag = 0;
    fence_mbar_init();
    tma_prefetch_desc(&map_a);
    tma_prefetch_desc(&map_b);
    if (p.ncut > 1) tma_prefetch_desc(&map_b_cut);
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

  const int64_t T = p.gm * p.gn;
  const int64_t TS = p.total_slots;
  const int64_t step = p.kind == TP_MAP_IDENTITY ? T : nprog;
  const int64_t nk = (p.K + p.kblk - 1) / p.kblk;

  if (warp == 0) {
    // ---------------- TMA producer (one thread; the rest of the warp waits)
    if (lane == 0) {
      const uint64_t pol_a = policy_evict_last();
      const uint64_t pol_b = policy_evict_last();
      uint32_t fills[kMaxStages] = {};
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t s = prog; s < TS && ok; s += step) {
        const Unit u = unit_of(s, p);
        int64_t tm, tn;
        raster(u.tile, p.gm, p.gn, p.group_m, &tm, &tn);
        // a narrow tile loads only its own columns of B, through the map whose
        // box has that many rows
        const int ub_rows = kPair ? u.width / 2 : u.width;
        const CUtensorMap* mb = u.cut ? &map_b_cut : &map_b;
        const uint32_t utx = a_stage + (uint32_t)ub_rows * 128;
        const int32_t arow = (int32_t)(tm * tile_m + rank * BM);
        const int32_t brow = (int32_t)(tn * p.bn + u.col + rank * ub_rows);
        for (int64_t kb = 0; kb < nk; ++kb) {
          if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, p.err)) { ok = false; break; }
          const int32_t kc = (int32_t)(kb * p.kblk);
          if constexpr (kPair) {
            // both CTAs' copies complete on the even CTA's full barrier
            const uint32_t fb = mapa(full_bar(stage), 0);
            if (leader) mbar_arrive_expect_tx(full_bar(stage), 2 * utx);
            tma_load_2d_pair(a0 + a_stage * stage, &map_a, kc, arow, fb, pol_a);
            tma_load_2d_pair(b0 + b_stage * stage, mb, kc, brow, fb, pol_b);
          } else {
            mbar_arrive_expect_tx(full_bar(stage), utx);
            tma_load_2d(a0 + a_stage * stage, &map_a, kc, arow, full_bar(stage), pol_a);
            tma_load_2d(b0 + b_stage * stage, mb, kc, brow, full_bar(stage), pol_b);
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
      int64_t t = 0;
      bool ok = true;
      for (int64_t s = prog; s < TS && ok; s += step, ++t) {
        const Unit u = unit_of(s, p);
        const uint32_t idesc = u.cut ? idesc_cut : idesc_full;
        const int acc = (int)(t & 1);
        const uint32_t use = (uint32_t)((t >> 1) & 1);
        if (!mbar_wait(tempty_bar(acc), use ^ 1u, abort_flag, p.err)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(acc * p.bn);
        for (int64_t kb = 0; kb < nk; ++kb) {
          if (!mbar_wait(full_bar(stage), phase, abort_flag, p.err)) { ok = false; break; }
          tc_fence_after();
          const uint64_t ad = desc_kmajor_sw128(a0 + a_stage * stage);
          const uint64_t bd = desc_kmajor_sw128(b0 + b_stage * stage);
          // 128-byte K slice = 4 MMAs of K = 16 (bf16) or K = 32 (fp8), 32 bytes
          // apart inside the swizzle atom (start address advances by 32 >> 4).
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t accum = (kb > 0 || k > 0) ? 1u : 0u;
            if constexpr (kPair) mma_pair<kF8>(d, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc, accum);
            else mma<kF8>(d, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc, accum);
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
  } else {
    // ---------------- epilogue (warps 2..5 -> TMEM lane quadrants 2,3,0,1)
    const int quad = warp & 3;
    const int row_in_tile = (int)rank * BM + quad * 32 + lane;
    // FP8 dequantisation factor 1 / (s_A * s_B), both steps in fp32
    const float scale = (p.scale_a && p.scale_b) ? 1.f / (*p.scale_a * *p.scale_b) : 1.f;
    const uint32_t tempty_remote = kPair ? mapa(tempty_bar(0), 0) : 0u;
    int64_t t = 0;
    // validate a store against the map (the slot is this program's and its
    // tile lies in the grid), then claim this warp's 32-row slice of the
    // (narrow) tile: (tile, narrow part, CTA of the pair, lane quadrant);
    // warp-uniform result
    auto claim = [&](int64_t s, int64_t tm, int64_t tn, int32_t part) -> bool {
      int ok = 1;
      if (lane == 0) {
        const bool on_map = s < TS && (s - prog) % step == 0 && tm >= 0 && tm < p.gm && tn >= 0 && tn < p.gn;
        if (!on_map) {
          record_device_error(p.err, kDevRace);
          ok = 0;
        } else {
          const int64_t id = (((tm * p.gn + tn) * p.ncut + part) * (kPair ? 2 : 1) + rank) * 4 + quad;
          ok = claim_tile(p.claims, id, p.err) ? 1 : 0;
        }
      }
      return __shfl_sync(0xffffffffu, ok, 0) != 0;
    };
    // one row's 32 columns [c0, c0 + 32) of C from FP32 values f
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
    auto release_acc = [&](int acc) {
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if constexpr (kPair) mbar_arrive_cluster(tempty_remote + 8u * acc);
        else mbar_arrive(tempty_bar(acc));
      }
    };
    // Checked launch: each epilogue warp counts itself done right after its
    // last claim (still ahead of its last accumulator); the warp that counts
    // last clears the bitmap for the next launch. A warp that leaves its loop
    // early counts itself at the exit.
    bool counted = false;
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
    for (int64_t s = prog; s < TS; s += step, ++t) {
      const Unit u = unit_of(s, p);
      const int acc = (int)(t & 1);
      const uint32_t use = (uint32_t)((t >> 1) & 1);
      int64_t tm, tn;
      raster(u.tile, p.gm, p.gn, p.group_m, &tm, &tn);
      bool store_ok = true;
      // claimed before the accumulator is ready, so the atomic's latency
      // hides behind the K loop
      if constexpr (kChecked) {
        store_ok = claim(s, tm, tn, u.part);
        if (s + step >= TS) finish_claims();
      }
      const bool ready = mbar_wait(tfull_bar(acc), use, abort_flag, p.err);
      if (!__all_sync(0xffffffffu, ready)) break;  // leave together (tcgen05.ld is warp-collective)
      tc_fence_after();
      const int64_t row = tm * tile_m + row_in_tile;
      const int64_t col0 = tn * p.bn + u.col;
      const uint32_t tacc = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * p.bn);
      for (int ch = 0; ch < u.width / 32 && store_ok; ++ch) {
        uint32_t r[32];
        tmem_ld32(tacc + (uint32_t)(ch * 32), r);
        tmem_ld_wait();
        float f[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) f[i] = __uint_as_float(r[i]);
        store_chunk(f, row, col0 + ch * 32);
      }
      release_acc(acc);
    }
    if constexpr (kChecked) finish_claims();
  }
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

template <bool kF8, bool kPair, bool kCount, bool kChecked>
cudaError_t launch_kernel(const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mbc, const TcArgs& p,
                          int grid, size_t smem, cudaStream_t st) {
  auto k = gemm_tc_kernel<kF8, kPair, kCount, kChecked>;
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
  attr[0].val.clusterDim.x = kPair ? 2 : 1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k, ma, mb, mbc, p);
}

template <bool kF8, bool kPair>
cudaError_t launch_inst(bool count, bool checked, const CUtensorMap& ma, const CUtensorMap& mb,
                        const CUtensorMap& mbc, const TcArgs& p, int grid, size_t smem, cudaStream_t st) {
  if (checked) return count ? launch_kernel<kF8, kPair, true, true>(ma, mb, mbc, p, grid, smem, st)
                            : launch_kernel<kF8, kPair, false, true>(ma, mb, mbc, p, grid, smem, st);
  return count ? launch_kernel<kF8, kPair, true, false>(ma, mb, mbc, p, grid, smem, st)
               : launch_kernel<kF8, kPair, false, false>(ma, mb, mbc, p, grid, smem, st);
}

template <bool kF8>
cudaError_t launch_any(bool pair, bool count, bool checked, const CUtensorMap& ma, const CUtensorMap& mb,
                       const CUtensorMap& mbc, const TcArgs& p, int grid, size_t smem, cudaStream_t st) {
  return pair ? launch_inst<kF8, true>(count, checked, ma, mb, mbc, p, grid, smem, st)
              : launch_inst<kF8, false>(count, checked, ma, mb, mbc, p, grid, smem, st);
}

// Clusters (CTA pairs, or single CTAs) of the kernel that can be resident at
// once (0 when the query fails).
template <bool kPair>
int max_active_clusters(size_t smem) {
  auto k = gemm_tc_kernel<false, kPair, false, false>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448) != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kPair ? 2 : 1);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kPair ? 2 : 1;
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

}  // namespace

// Shared by the BF16 and FP8 entry points. esize = 2 (bf16) or 1 (fp8).
tp_status launch_gemm_tc_impl(tp_ctx* ctx, tp_partition* c, const tp_tensor* a, const tp_tensor* b,
                              const tp_gemm_config* cfg, const tp_exec* ex, cudaStream_t stream, int esize,
                              const float* scale_a, const float* scale_b) {
  const int64_t M = a->shape[0], K = a->shape[1], N = b->shape[1];
  if ((ex->write_counts == nullptr) != (ex->write_owner == nullptr))
    return fail(TP_ERR_INVALID, "write_counts and write_owner must be given together");
  if (c->kind == TP_MAP_QUEUE) return fail(TP_ERR_UNSUPPORTED, "the tensor-core GEMM maps tiles by slot (identity/strided)");
  const int bm = (int)c->tile[0], bn = (int)c->tile[1];
  if (bm != BM && bm != 2 * BM)
    return fail(TP_ERR_UNSUPPORTED, "tensor-core GEMM tiles have 128 rows (one CTA) or 256 rows (CTA pair)");
  const bool pair = bm == 2 * BM;
  if (bn < 32 || bn > 256 || bn % 32 || (pair && bn % 64))
    return fail(TP_ERR_UNSUPPORTED, "tile columns must be 32..256, a multiple of 32 (of 64 for 256-row tiles)");
  if (cfg && cfg->bm && cfg->bm != bm) return fail(TP_ERR_SHAPE, "cfg.bm differs from the partition's tile");
  if (cfg && cfg->bn && cfg->bn != bn) return fail(TP_ERR_SHAPE, "cfg.bn differs from the partition's tile");
  // K-major operands: A row-major (stride along K = 1), B stored N x K.
  if (a->strides[1] != 1 || b->strides[0] != 1)
    return fail(TP_ERR_UNSUPPORTED, "tensor-core GEMM needs K-major A (row-major M x K) and K-major B (stored N x K)");
  const int64_t lda = a->strides[0], ldb = b->strides[1];
  if (((uintptr_t)a->ptr & 15) || ((uintptr_t)b->ptr & 15) || ((lda * esize) & 15) || ((ldb * esize) & 15) ||
      (K * esize) % 16)
    return fail(TP_ERR_ALIGN, "TMA needs 16-byte aligned bases and row strides (K a multiple of 16 bytes)");
  if (M == 0 || N == 0) return TP_OK;
  if (K == 0) return fail(TP_ERR_UNSUPPORTED, "K = 0");
  CUtensorMap ma, mb;
  tp_status s = make_map(&ma, a->ptr, M, K, lda, esize, BM);
  if (s != TP_OK) return s;
  s = make_map(&mb, b->ptr, N, K, ldb, esize, pair ? bn / 2 : bn);
  if (s != TP_OK) return s;
  TcArgs p{};
  p.M = M;
  p.N = N;
  p.K = K;
  p.gm = c->grid[0];
  p.gn = c->grid[1];
  p.bn = bn;
  p.kind = c->kind;
  p.group_m = (c->kind != TP_MAP_IDENTITY && cfg && cfg->group_m > 0) ? cfg->group_m : 1;
  p.kblk = 128 / esize;
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
  const size_t stage_bytes = (size_t)BM * 128 + (size_t)(pair ? bn / 2 : bn) * 128;
  const size_t fixed = 1024 + 256;  // alignment slack + barriers
  const size_t budget = 232448;     // 227 KB opt-in
  int stages = (cfg && cfg->stages > 0) ? cfg->stages : (int)((budget - fixed) / stage_bytes);
  stages = stages > kMaxStages ? kMaxStages : stages;
  if (stages < 2 || fixed + stages * stage_bytes > budget)
    return fail(TP_ERR_UNSUPPORTED, "shared memory too small for the requested stages");
  p.stages = stages;
  const size_t smem = fixed + stages * stage_bytes;
  const int64_t progs = c->kind == TP_MAP_IDENTITY ? c->num_tiles : c->num_programs;
  const int64_t grid = pair ? 2 * progs : progs;
  // Schedule: whole tiles, except that on a strided map the R = T mod P tiles
  // of the last, partial round may each be cut along N into S narrow tiles
  // run by the programs that would otherwise sit idle in that round.
  const int64_t T = c->num_tiles;
  p.dp_slots = T;
  p.total_slots = T;
  p.ncut = 1;
  p.bn_cut = bn;
  const int32_t limit = (cfg && cfg->split_k > 0) ? cfg->split_k : 4;
  if (limit > 8) return fail(TP_ERR_INVALID, "split_k must be 0..8");
  CUtensorMap mb_cut = mb;
  if (c->kind == TP_MAP_STRIDED) {
    const int64_t R = T % progs;
    const int unit = pair ? 64 : 32;  // narrow tiles keep whole 32-row B boxes per CTA
    int64_t S = 1;
    while (R > 0 && 2 * S <= limit && 2 * S <= progs / R && bn % (2 * S * unit) == 0) S *= 2;
    if (S >= 2) {
      p.ncut = (int32_t)S;
      p.bn_cut = (int32_t)(bn / S);
      p.dp_slots = T - R;
      p.total_slots = T - R + R * S;
      s = make_map(&mb_cut, b->ptr, N, K, ldb, esize, pair ? p.bn_cut / 2 : p.bn_cut);
      if (s != TP_OK) return s;
    }
  }
  const bool count = ex->write_counts != nullptr;
  const bool checked = (ex->flags & TP_EXEC_CHECKED) != 0;
  if (checked) {
    p.claim_bits = c->num_tiles * p.ncut * (pair ? 8 : 4);
    s = claims_for(ctx, p.claim_bits, &p.claims, &p.claim_done);
    if (s != TP_OK) return s;
  }
  cudaError_t e = esize == 2 ? launch_any<false>(pair, count, checked, ma, mb, mb_cut, p, (int)grid, smem, stream)
                             : launch_any<true>(pair, count, checked, ma, mb, mb_cut, p, (int)grid, smem, stream);
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core GEMM launch");
  return TP_OK;
}

tp_status gemm_tc_resident(tp_ctx* ctx, const tp_gemm_config* cfg, int32_t* programs) {
  const int bm = cfg->bm ? cfg->bm : BM, bn = cfg->bn ? cfg->bn : 256;
  if (bm != BM && bm != 2 * BM) return fail(TP_ERR_UNSUPPORTED, "tiles have 128 or 256 rows");
  const bool pair = bm == 2 * BM;
  const size_t stage_bytes = (size_t)BM * 128 + (size_t)(pair ? bn / 2 : bn) * 128;
  const size_t fixed = 1024 + 256, budget = 232448;
  int stages = cfg->stages > 0 ? cfg->stages : (int)((budget - fixed) / stage_bytes);
  stages = stages > kMaxStages ? kMaxStages : stages;
  if (stages < 2 || fixed + stages * stage_bytes > budget)
    return fail(TP_ERR_UNSUPPORTED, "shared memory too small for the requested stages");
  const size_t smem = fixed + stages * stage_bytes;
  (void)ctx;
  const int clusters = pair ? max_active_clusters<true>(smem) : max_active_clusters<false>(smem);
  if (clusters <= 0) return fail(TP_ERR_CUDA, "cudaOccupancyMaxActiveClusters failed");
  *programs = clusters;  // CTA pairs (256-row tiles) or CTAs
  return TP_OK;
}

tp_status launch_gemm_tc(tp_ctx* ctx, tp_partition* c, const tp_tensor* a, const tp_tensor* b,
                         const tp_gemm_config* cfg, const tp_exec* ex, cudaStream_t stream, unsigned* queue) {
  (void)queue;
  return launch_gemm_tc_impl(ctx, c, a, b, cfg, ex, stream, 2, nullptr, nullptr);
}

}  // namespace tp
