// FP32 GEMM on the CUDA cores (FFMA, FP32 accumulation, no TF32): one 64x64
// C tile per tile program with a K loop (§3.6, Listing 6). Plain partitions
// launch one program per tile; mapped partitions launch persistent programs
// that walk their tiles (strided slots or a device queue), slots being turned
// into tiles by the band raster shared with the tensor-core GEMM.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "sm100_ptx.cuh"
#include "tp_internal.h"

namespace tp {
namespace {

constexpr int BM = 64, BN = 64, TH = 256;

struct SimtArgs {
  const float* a;
  const float* b;
  float* c;
  int64_t M, N, K;
  int64_t sam, sak, sbk, sbn;  // element strides of A (m, k) and B (k, n)
  int64_t gm, gn;              // tile grid
  int32_t kind, group_m;
  int32_t split;               // K slices per tile (cluster size); 1 = none
  unsigned* queue;
  uint32_t* counts;
  int32_t* owner;
};

// Schedule slot -> (tm, tn): bands of group_m tile rows, column by column
// inside a band (group_m = 1 is row-major).
__device__ __forceinline__ void raster(int64_t s, int64_t gm, int64_t gn, int64_t g, int64_t* tm,
                                       int64_t* tn) {
  const int64_t per = g * gn;
  const int64_t first = (s / per) * g;
  const int64_t rows = min(g, gm - first);
  const int64_t r = s % per;
  *tm = first + r % rows;
  *tn = r / rows;
}

// Each of the 256 threads owns a 4 x 4 block of the tile: rows 4*ty..4*ty+3
// and columns 4*tx..4*tx+3 (ty = tid / 16, tx = tid % 16). Shared memory
// holds the A slice K-major (As[k][m]) and the B slice as stored (Bs[k][n]),
// rows padded by 4 floats, so one 16-byte load gives a thread its 4 A or 4 B
// values of a k step. The next K slice is loaded into registers while the
// current one is multiplied (register-staged double buffering), so the
// global-memory latency overlaps the FFMAs.
// With split = S > 1 a tile program is a cluster of S CTAs: CTA r runs the
// K slices [r*nk/S, (r+1)*nk/S) and keeps its partial 64 x 64 block in
// shared memory; after a cluster barrier CTA r adds, for rows
// [r*64/S, (r+1)*64/S), the S partials in slice order 0..S-1 (reading the
// others through distributed shared memory) and stores them, so every
// element still has one writer and C is bit-reproducible.
template <int BK, bool COUNT>
__global__ void __launch_bounds__(TH, 1) gemm_f32_kernel(const __grid_constant__ SimtArgs p) {
  constexpr int PA = BM * BK / TH;  // A elements per thread per K slice
  constexpr int PB = BK * BN / TH;
  // the operand buffers; a split program's partial block overlays them once
  // its K loop has ended
  constexpr int kAB = 2 * BK * (BM + 4) + 2 * BK * (BN + 4);
  __shared__ __align__(16) float raw[kAB > BM * BN ? kAB : BM * BN];
  auto As = reinterpret_cast<float(*)[BK][BM + 4]>(raw);
  auto Bs = reinterpret_cast<float(*)[BK][BN + 4]>(raw + 2 * BK * (BM + 4));
  auto Ps = reinterpret_cast<float(*)[BN]>(raw);
  __shared__ int64_t slot;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t T = p.gm * p.gn;
  const int S = p.split;
  const uint32_t r = S > 1 ? sm100::cluster_ctarank() : 0u;
  int64_t s = S > 1 ? (int64_t)(blockIdx.x / S) : (int64_t)blockIdx.x;
  if (p.kind == TP_MAP_QUEUE) {
    if (tid == 0) slot = atomicAdd(p.queue, 1u);
    __syncthreads();
    s = slot;
  }
  while (s < T) {
    int64_t tm, tn;
    raster(s, p.gm, p.gn, p.group_m, &tm, &tn);
    const int64_t m0 = tm * BM, n0 = tn * BN;
    float acc[4][4] = {};
    const int64_t nk_all = (p.K + BK - 1) / BK;
    const int64_t kt0 = (int64_t)r * nk_all / S, kt1 = (int64_t)(r + 1) * nk_all / S;
    const int64_t nk = kt1 - kt0;
    float ra[PA], rb[PB];
    // element e of this thread's share: A (row e*TH/BK + tid/BK, k tid%BK),
    // B (k e*TH/BN + tid/BN, column tid%BN): consecutive threads read
    // consecutive k of A and consecutive n of B
    auto fetch = [&](int64_t k0) {
#pragma unroll
      for (int e = 0; e < PA; ++e) {
        const int i = e * TH + tid;
        const int64_t gm_ = m0 + i / BK, gk = k0 + i % BK;
        ra[e] = (gm_ < p.M && gk < p.K) ? p.a[gm_ * p.sam + gk * p.sak] : 0.f;
      }
#pragma unroll
      for (int e = 0; e < PB; ++e) {
        const int i = e * TH + tid;
        const int64_t gk = k0 + i / BN, gn_ = n0 + i % BN;
        rb[e] = (gk < p.K && gn_ < p.N) ? p.b[gk * p.sbk + gn_ * p.sbn] : 0.f;
      }
    };
    auto stash = [&](int buf) {
#pragma unroll
      for (int e = 0; e < PA; ++e) {
        const int i = e * TH + tid;
        As[buf][i % BK][i / BK] = ra[e];
      }
#pragma unroll
      for (int e = 0; e < PB; ++e) {
        const int i = e * TH + tid;
        Bs[buf][i / BN][i % BN] = rb[e];
      }
    };
    if (nk > 0) {
      fetch(kt0 * BK);
      stash(0);
    }
    __syncthreads();
    for (int64_t kt = 0; kt < nk; ++kt) {
      const int buf = kt & 1;
      if (kt + 1 < nk) fetch((kt0 + kt + 1) * BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        const float4 a4 = *reinterpret_cast<const float4*>(&As[buf][kk][4 * ty]);
        const float4 b4 = *reinterpret_cast<const float4*>(&Bs[buf][kk][4 * tx]);
        const float av[4] = {a4.x, a4.y, a4.z, a4.w};
        const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      if (kt + 1 < nk) stash(buf ^ 1);  // the other buffer's readers passed the barrier below last step
      __syncthreads();
    }
    bool mine = true;  // this thread's rows are stored by this CTA
    if (S > 1) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        *reinterpret_cast<float4*>(&Ps[4 * ty + i][4 * tx]) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      sm100::cluster_sync();  // every CTA's partial is in its shared memory
      mine = (4 * ty) / (BM / S) == (int)r;
      if (mine) {
        float sum[4][4];
        for (int src = 0; src < S; ++src) {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            float4 v;
            if (src == (int)r) {
              v = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
            } else {
              const uint32_t at = sm100::mapa(sm100::smem_u32(&Ps[4 * ty + i][4 * tx]), (uint32_t)src);
              asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                           : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                           : "r"(at)
                           : "memory");
            }
            const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) sum[i][j] = src == 0 ? vv[j] : sum[i][j] + vv[j];
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = sum[i][j];
      }
      sm100::cluster_sync();  // the peers' reads of this CTA's partial are done
    }
    const bool vec = (p.N % 4 == 0) && ((reinterpret_cast<uintptr_t>(p.c) & 15) == 0);
#pragma unroll
    for (int i = 0; i < 4 && mine; ++i) {
      const int64_t r = m0 + 4 * ty + i;
      if (r >= p.M) continue;
      const int64_t c0 = n0 + 4 * tx;
      if (vec && c0 + 4 <= p.N) {
        *reinterpret_cast<float4*>(p.c + r * p.N + c0) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (c0 + j < p.N) p.c[r * p.N + c0 + j] = acc[i][j];
      }
      if constexpr (COUNT) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (c0 + j < p.N) {
            atomicAdd(p.counts + r * p.N + c0 + j, 1u);
            p.owner[r * p.N + c0 + j] = (int32_t)(blockIdx.x / S);
          }
      }
    }
    if (p.kind == TP_MAP_IDENTITY) break;
    if (p.kind == TP_MAP_STRIDED) {
      s += gridDim.x / S;
    } else {
      __syncthreads();
      if (tid == 0) slot = atomicAdd(p.queue, 1u);
      __syncthreads();
      s = slot;
    }
  }
}

template <int BK>
cudaError_t launch_bk(const SimtArgs& p, bool count, int64_t grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(grid * p.split));
  cfg.blockDim = dim3(TH);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)p.split;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return count ? cudaLaunchKernelEx(&cfg, gemm_f32_kernel<BK, true>, p)
               : cudaLaunchKernelEx(&cfg, gemm_f32_kernel<BK, false>, p);
}

// ------------------------------------------------ TMA-fed FP32 GEMM
// The same tiles, thread blocking, K order and split-K reduction as
// gemm_f32_kernel (so the same C bit for bit), with the operands brought by
// TMA: a producer thread copies each 32-wide K chunk of the tile's A rows
// (64 x 32 floats, 128-byte rows, 128-byte swizzle) and B columns (32 x 64
// floats, 256-byte rows) into a ring of 16 KB stages while eight compute
// warps multiply the chunks already landed; no register staging, no block
// barrier per K step. Used for identity and strided maps with unit-stride,
// 16-byte-aligned operands (and split-K only when each program holds one
// tile); other launches take gemm_f32_kernel.
constexpr int kFChunk = 32;
constexpr int kFStages = 8;
constexpr uint32_t kFChunkA = BM * kFChunk * 4;  // 8 KB
constexpr uint32_t kFChunkB = kFChunk * BN * 4;  // 8 KB
constexpr uint32_t kFStageBytes = kFChunkA + kFChunkB;
constexpr int kFThreads = TH + 32;               // eight compute warps + the producer warp
constexpr size_t kFSmem = 1024 + (size_t)kFStages * kFStageBytes + BM * BN * 4 + 8 * (2 * kFStages) + 16;

struct F32TmaArgs {
  float* c;
  int64_t M, N, K;
  int64_t gm, gn;
  int32_t kind, group_m, split;
  int32_t nchunks;  // K chunks of 32
  uint32_t* counts;
  int32_t* owner;
  int* err;
  uint64_t wait_ns;
};

template <bool COUNT>
__global__ void __launch_bounds__(kFThreads, 1)
    gemm_f32_tma_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                        const __grid_constant__ F32TmaArgs p) {
  using namespace sm100;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // 128-byte swizzle: 1024-byte aligned stages
  uint8_t* gbase = smem_raw + (base - raw);
  auto Ps = reinterpret_cast<float(*)[BN]>(gbase + (size_t)kFStages * kFStageBytes);
  const uint32_t bars = base + kFStages * kFStageBytes + BM * BN * 4;
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 8u * (kFStages + s); };
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + (bars - base) + 8 * 2 * kFStages);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int S = p.split;
  const uint32_t r = S > 1 ? cluster_ctarank() : 0u;
  if (tid == 0) {
    for (int s = 0; s < kFStages; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), TH / 32);
    }
    *abort_flag = 0;
    fence_mbar_init();
    tma_prefetch_desc(&map_a);
    tma_prefetch_desc(&map_b);
  }
  __syncthreads();
  // A and B may be the previous kernel's output, and C its input
  grid_dependency_wait();
  allow_dependents();
  const int64_t T = p.gm * p.gn;
  const int64_t s0 = (int64_t)(blockIdx.x / S);
  const int64_t step = p.kind == TP_MAP_IDENTITY ? T : (int64_t)(gridDim.x / S);
  const int32_t c0 = (int32_t)(((int64_t)r * p.nchunks) / S), c1 = (int32_t)(((int64_t)(r + 1) * p.nchunks) / S);
  if (warp == TH / 32) {
    // ---------------- producer
    if (lane == 0) {
      uint32_t fills[kFStages] = {};
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t s = s0; s < T && ok; s += step) {
        int64_t tm, tn;
        raster(s, p.gm, p.gn, p.group_m, &tm, &tn);
        for (int32_t ch = c0; ch < c1; ++ch) {
          if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, p.err, p.wait_ns)) { ok = false; break; }
          const uint32_t dst = base + kFStageBytes * (uint32_t)stage;
          mbar_arrive_expect_tx(full_bar(stage), kFStageBytes);
          tma_load_2d(dst, &map_a, ch * kFChunk, (int32_t)(tm * BM), full_bar(stage), policy_evict_last());
          tma_load_2d(dst + kFChunkA, &map_b, (int32_t)(tn * BN), ch * kFChunk, full_bar(stage), policy_evict_last());
          fills[stage]++;
          if (++stage == kFStages) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok)  // every copy this thread issued lands before the CTA retires
        for (int s2 = 0; s2 < kFStages; ++s2)
          if (fills[s2]) mbar_wait(full_bar(s2), (fills[s2] - 1u) & 1u, nullptr, nullptr, 200000000ull);
    }
    __syncwarp();
    // split programs hold one tile: the producer warp joins the two
    // cluster barriers of the epilogue below
    if (S > 1) {
      cluster_sync();
      cluster_sync();
    }
    return;
  }
  // ---------------- compute warps: thread (tx, ty) owns rows 4ty..4ty+3 and
  // columns 4tx..4tx+3 of the tile, as in gemm_f32_kernel
  const int tx = tid % 16, ty = tid / 16;
  int stage = 0;
  uint32_t phase = 0;
  bool ok = true;
  for (int64_t s = s0; s < T || (S > 1 && s == s0); s += step) {
    const bool have = s < T;  // a split cluster without a tile still joins the cluster barriers
    int64_t tm = 0, tn = 0;
    if (have) raster(s, p.gm, p.gn, p.group_m, &tm, &tn);
    float acc[4][4] = {};
    for (int32_t ch = c0; have && ok && ch < c1; ++ch) {
      const bool got = mbar_wait(full_bar(stage), phase, abort_flag, p.err, p.wait_ns);
      if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
      const uint32_t sa = base + kFStageBytes * (uint32_t)stage;
      const uint32_t sb = sa + kFChunkA;
#pragma unroll
      for (int g = 0; g < kFChunk / 4; ++g) {
        // A rows 4ty+i, k = 4g..4g+3 (16-byte piece g of a 128-byte row,
        // stored at piece g ^ (row & 7)); B rows k = 4g+j, columns 4tx..
        float av[4][4], bv[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const uint32_t row = (uint32_t)(4 * ty + i);
          uint32_t w[4];
          ld_shared_v4(sa + row * 128u + ((((uint32_t)g) ^ (row & 7u)) << 4), w);
#pragma unroll
          for (int q = 0; q < 4; ++q) av[i][q] = __uint_as_float(w[q]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          uint32_t w[4];
          ld_shared_v4(sb + (uint32_t)(4 * g + j) * 256u + (uint32_t)tx * 16u, w);
#pragma unroll
          for (int q = 0; q < 4; ++q) bv[j][q] = __uint_as_float(w[q]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][q] = fmaf(av[i][j], bv[j][q], acc[i][q]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty_bar(stage));
      if (++stage == kFStages) { stage = 0; phase ^= 1u; }
    }
    const int64_t m0 = tm * BM, n0 = tn * BN;
    bool mine = have;  // this thread's rows are stored by this CTA
    if (S > 1) {
      // partial blocks in shared memory, summed in slice order by the CTA
      // that owns the rows (peers read through distributed shared memory)
      if (have) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          *reinterpret_cast<float4*>(&Ps[4 * ty + i][4 * tx]) =
              make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      }
      cluster_sync();
      mine = have && (4 * ty) / (BM / S) == (int)r;
      if (mine) {
        float sum[4][4];
        for (int src = 0; src < S; ++src) {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            float4 v;
            if (src == (int)r) {
              v = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
            } else {
              const uint32_t at = mapa(smem_u32(&Ps[4 * ty + i][4 * tx]), (uint32_t)src);
              asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                           : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                           : "r"(at)
                           : "memory");
            }
            const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) sum[i][q] = src == 0 ? vv[q] : sum[i][q] + vv[q];
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[i][q] = sum[i][q];
      }
      cluster_sync();  // the peers' reads of this CTA's partial are done
    }
    if (!ok) mine = false;
    const bool vec = (p.N % 4 == 0) && ((reinterpret_cast<uintptr_t>(p.c) & 15) == 0);
#pragma unroll
    for (int i = 0; i < 4 && mine; ++i) {
      const int64_t row = m0 + 4 * ty + i;
      if (row >= p.M) continue;
      const int64_t col = n0 + 4 * tx;
      if (vec && col + 4 <= p.N) {
        *reinterpret_cast<float4*>(p.c + row * p.N + col) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (col + q < p.N) p.c[row * p.N + col + q] = acc[i][q];
      }
      if constexpr (COUNT) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (col + q < p.N) {
            atomicAdd(p.counts + row * p.N + col + q, 1u);
            p.owner[row * p.N + col + q] = (int32_t)(blockIdx.x / S);
          }
      }
    }
    if (S > 1 || !ok) break;
  }
}

template <bool COUNT>
cudaError_t launch_f32_tma(const CUtensorMap& ma, const CUtensorMap& mb, const F32TmaArgs& p, int64_t programs,
                           cudaStream_t st) {
  auto k = gemm_f32_tma_kernel<COUNT>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(programs * p.split));
  cfg.blockDim = dim3(kFThreads);
  cfg.dynamicSmemBytes = kFSmem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)p.split;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k, ma, mb, p);
}

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

// fp32 [rows, cols] row-major (row pitch ld floats) in boxes of box_cols x
// box_rows, zero fill past the edges
bool f32_map(CUtensorMap* map, const float* ptr, int64_t rows, int64_t cols, int64_t ld, int box_cols, int box_rows,
             bool swizzle) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

tp_status launch_gemm_simt(tp_ctx* ctx, tp_partition* c, const tp_tensor* a, const tp_tensor* b,
                           const tp_gemm_config* cfg, const tp_exec* ex, cudaStream_t stream,
                           unsigned* queue) {
  if (c->tile[0] != BM || c->tile[1] != BN)
    return fail(TP_ERR_UNSUPPORTED, "the FP32 GEMM uses 64 x 64 output tiles");
  if ((ex->write_counts == nullptr) != (ex->write_owner == nullptr))
    return fail(TP_ERR_INVALID, "write_counts and write_owner must be given together");
  SimtArgs p{};
  p.a = static_cast<const float*>(a->ptr);
  p.b = static_cast<const float*>(b->ptr);
  p.c = static_cast<float*>(c->t.ptr);
  p.M = a->shape[0];
  p.K = a->shape[1];
  p.N = b->shape[1];
  p.sam = a->strides[0];
  p.sak = a->strides[1];
  p.sbk = b->strides[0];
  p.sbn = b->strides[1];
  p.gm = c->grid[0];
  p.gn = c->grid[1];
  p.kind = c->kind;
  // a plain partition is program p -> tile p in row-major order (§3.4)
  p.group_m = (c->kind != TP_MAP_IDENTITY && cfg && cfg->group_m > 0) ? cfg->group_m : 1;
  p.queue = queue;
  p.counts = ex->write_counts;
  p.owner = ex->write_owner;
  if (p.M == 0 || p.N == 0) return TP_OK;
  const int64_t grid = c->kind == TP_MAP_IDENTITY ? c->num_tiles : c->num_programs;
  const int bk = (cfg && cfg->bk > 0) ? cfg->bk : 32;  // 32: fewest barriers per K (fastest at 512^3)
  p.split = (cfg && cfg->split_k > 1) ? cfg->split_k : 1;
  if (cfg && (cfg->split_k < 0 || cfg->split_k > 4 || (p.split & (p.split - 1))))
    return fail(TP_ERR_INVALID, "FP32 GEMM split_k must be 0, 1, 2 or 4");
  if (p.split > 1 && c->kind == TP_MAP_QUEUE)
    return fail(TP_ERR_UNSUPPORTED, "FP32 GEMM split_k with a queue map (each CTA would dequeue its own tile)");
  const bool count = p.counts != nullptr;
  cudaError_t e;
  // TMA-fed kernel: unit-stride rows 16-byte aligned, K chunks of 32 (the
  // bk = 32 schedule), identity or strided maps, split programs one tile each
  const int64_t T = p.gm * p.gn;
  const bool tma_ok = bk == 32 && p.sak == 1 && p.sbn == 1 && p.sam % 4 == 0 && p.sbk % 4 == 0 &&
                      ((reinterpret_cast<uintptr_t>(p.a) | reinterpret_cast<uintptr_t>(p.b)) & 15) == 0 &&
                      p.K > 0 && p.K < ((int64_t)1 << 30) && p.M < ((int64_t)1 << 31) && p.N < ((int64_t)1 << 31) &&
                      c->kind != TP_MAP_QUEUE && (p.split == 1 || grid >= T);
  if (tma_ok) {
    CUtensorMap ma, mb;
    if (f32_map(&ma, p.a, p.M, p.K, p.sam, kFChunk, BM, true) && f32_map(&mb, p.b, p.K, p.N, p.sbk, BN, kFChunk, false)) {
      F32TmaArgs t{};
      t.c = p.c;
      t.M = p.M;
      t.N = p.N;
      t.K = p.K;
      t.gm = p.gm;
      t.gn = p.gn;
      t.kind = p.kind;
      t.group_m = p.group_m;
      t.split = p.split;
      t.nchunks = (int32_t)((p.K + kFChunk - 1) / kFChunk);
      t.counts = p.counts;
      t.owner = p.owner;
      t.err = ctx->d_err;
      t.wait_ns = 2000000000ull;
      e = count ? launch_f32_tma<true>(ma, mb, t, grid, stream) : launch_f32_tma<false>(ma, mb, t, grid, stream);
      if (e != cudaSuccess) return cuda_fail(e, "FP32 GEMM launch");
      return TP_OK;
    }
  }
  switch (bk) {
    case 8: e = launch_bk<8>(p, count, grid, stream); break;
    case 16: e = launch_bk<16>(p, count, grid, stream); break;
    case 32: e = launch_bk<32>(p, count, grid, stream); break;
    default: return fail(TP_ERR_UNSUPPORTED, "FP32 GEMM bk must be 8, 16 or 32");
  }
  if (e != cudaSuccess) return cuda_fail(e, "FP32 GEMM launch");
  return TP_OK;
}

}  // namespace tp
