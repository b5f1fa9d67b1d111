// Batch-1 decode-shaped layer chain (one layer of the graph-captured forward
// pass of §3.2, Listing 3: RMSNorm, matrix-vector products, residual add,
// widened to a gated MLP):
//   n = h / sqrt(mean(h^2) + eps) * gamma
//   qkv = W_qkv n;  [g; u] = W_gu n;  a = silu(g) * u;  h <- h + W_down a
// Weights are BF16 [out, in] row-major; activations and h are FP32.
//
// Every step streams weights once from HBM, so the kernels are matrix-vector
// products built for bandwidth: the input vector sits in shared memory (fp32),
// each group of warps owns whole output rows (a plain partition of the output
// vector into row tiles) and reads its rows with 16-byte loads, several in
// flight per lane; a row's dot product is reduced in a fixed order, so replays
// are bit-reproducible.
//
// Fused kernels (the graph-replayed path): norm + QKV + gate/up with SiLU*mul
// in the epilogue, and down projection + residual add. Unfused kernels (one
// per step, the plain per-call path): rmsnorm, gemv, silu_mul, residual_add.
//
// The fused path streams the weights through TMA (gemv_stream_kernel): a
// producer thread copies blocks of 32 rows x 256 columns (16 KB per box; a
// 3-D box brings 16 gate rows with their 16 up partners) into a ring of
// shared-memory stages, and eight consumer warps take four rows each; every
// lane multiplies 8 consecutive weights of a row by the matching 8 entries of
// x, which sits in shared memory (whole, or one K slice at a time brought by
// bulk copies), into four fixed-order accumulators. A TMA copy into one SM
// costs about the same time whatever its size, so a few large copies keep a
// stream going at the DRAM read rate, above what per-lane 16-byte loads reach
// here.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "sm100_ptx.cuh"
#include "tp_internal.h"

namespace tp {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Sum of squares of h[0..d) by the whole block; returns rsqrt(mean + eps).
__device__ float block_rms_scale(const float* __restrict__ h, int64_t d, float eps, float* red) {
  float s = 0.f;
  for (int64_t i = threadIdx.x; i < d; i += kThreads) s = fmaf(h[i], h[i], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  float t = 0.f;
  for (int w = 0; w < kWarps; ++w) t += red[w];  // fixed order
  __syncthreads();
  return rsqrtf(t / (float)d + eps);
}

// Dot product of one bf16 row (length k, 16-byte aligned) with x (fp32, in
// shared memory) by the lanes of one warp, lane-partial then shuffle tree.
// Warps of a group split the row into `parts` contiguous pieces; each lane
// keeps kUnroll 16-byte weight loads in flight.
template <int kUnroll>
__device__ __forceinline__ float row_dot(const __nv_bfloat16* __restrict__ w, const float* __restrict__ xs,
                                         int64_t k, int part, int parts) {
  const int lane = threadIdx.x & 31;
  const int64_t nv = k / 8;  // 16-byte vectors
  const int64_t per = (nv + parts - 1) / parts;
  const int64_t v0 = part * per, v1 = min(nv, v0 + per);
  const uint4* wv = reinterpret_cast<const uint4*>(w);
  float acc0 = 0.f, acc1 = 0.f;
  // kUnroll vectors per lane in flight per round; a row's last round is
  // predicated rather than handled one vector at a time, so every round costs
  // one DRAM round trip. A lane's vectors are consumed in the same order as
  // an unrolled-then-tail loop would, so the sums are unchanged.
  for (int64_t v = v0 + lane; v < v1; v += 32 * kUnroll) {
    uint4 q[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) q[u] = v + 32 * u < v1 ? __ldcs(wv + v + 32 * u) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (v + 32 * u >= v1) break;
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q[u]);
      const float4* xv = reinterpret_cast<const float4*>(xs + (v + 32 * u) * 8);
      const float4 xa = xv[0], xb = xv[1];
      float2 f0 = __bfloat1622float2(h[0]), f1 = __bfloat1622float2(h[1]);
      float2 f2 = __bfloat1622float2(h[2]), f3 = __bfloat1622float2(h[3]);
      acc0 = fmaf(f0.x, xa.x, acc0); acc1 = fmaf(f0.y, xa.y, acc1);
      acc0 = fmaf(f1.x, xa.z, acc0); acc1 = fmaf(f1.y, xa.w, acc1);
      acc0 = fmaf(f2.x, xb.x, acc0); acc1 = fmaf(f2.y, xb.y, acc1);
      acc0 = fmaf(f3.x, xb.z, acc0); acc1 = fmaf(f3.y, xb.w, acc1);
    }
  }
  // elements past the last full vector (k % 8), handled by the last part
  if (part == parts - 1)
    for (int64_t i = nv * 8 + lane; i < k; i += 32) acc0 = fmaf(__bfloat162float(w[i]), xs[i], acc0);
  float s = acc0 + acc1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

__device__ __forceinline__ float silu(float g) { return g / (1.f + __expf(-g)); }

enum Epi : int { kPlain = 0, kResidual = 1, kSiluPair = 2 };

struct GemvArgs {
  const __nv_bfloat16* w;   // [rows, k]
  const float* x;           // [k]
  float* y;                 // output vector
  int64_t rows;             // output rows (kSiluPair: pairs)
  int64_t k;
  int64_t ld;               // row stride of w (elements)
  int64_t pair_offset;      // kSiluPair: row offset of u relative to g
  // fused RMSNorm of x on load (norm + gemv kernels)
  int32_t norm;
  float eps;
  const float* gamma;
  // second problem of the fused norm kernel (rows after `rows` go to w2/y2)
  const __nv_bfloat16* w2;
  float* y2;
  int64_t rows2;
  int64_t ld2;
  int64_t pair_offset2;
  int32_t epi2;
  uint32_t* counts;
  int32_t* owner;
};

template <int kEpi, int kParts, int kUnroll, bool kCount>
__global__ void __launch_bounds__(kThreads) gemv_kernel(const __grid_constant__ GemvArgs p) {
  extern __shared__ float xs[];  // k floats (+ reduction scratch)
  float* red = xs + ((p.k + 3) & ~int64_t(3));
  // stage x (optionally normalised) in shared memory
  float scale = 1.f;
  if (p.norm) scale = block_rms_scale(p.x, p.k, p.eps, red);
  for (int64_t i = threadIdx.x; i < p.k; i += kThreads) {
    float v = p.x[i];
    if (p.norm) v = v * scale * (p.gamma ? p.gamma[i] : 1.f);
    xs[i] = v;
  }
  __syncthreads();
  constexpr int kGroups = kWarps / kParts;
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int group = warp / kParts, part = warp % kParts;
  const int64_t units = p.rows + p.rows2;
  const int64_t gstride = (int64_t)gridDim.x * kGroups;
  // the trip count depends on the block only, so the block-wide barriers
  // below are reached by every thread the same number of times
  for (int64_t base = (int64_t)blockIdx.x * kGroups; base < units; base += gstride) {
    const int64_t u = base + group;
    const bool valid = u < units;
    const bool second = u >= p.rows;
    const int64_t r = second ? u - p.rows : u;
    const int epi = second ? p.epi2 : kEpi;
    float s0 = 0.f, s1 = 0.f;
    float* y = second ? p.y2 : p.y;
    if (valid) {
      const __nv_bfloat16* w = second ? p.w2 : p.w;
      const int64_t ld = second ? p.ld2 : p.ld;
      s0 = row_dot<kUnroll>(w + r * ld, xs, p.k, part, kParts);
      if (epi == kSiluPair)
        s1 = row_dot<kUnroll>(w + (r + (second ? p.pair_offset2 : p.pair_offset)) * ld, xs, p.k, part, kParts);
    }
    if constexpr (kParts > 1) {
      // combine the warps of a group in a fixed order
      float* slot = red + 16 + (warp * 2);
      if (lane == 0) {
        slot[0] = s0;
        slot[1] = s1;
      }
      __syncthreads();
      if (part == 0) {
        s0 = 0.f;
        s1 = 0.f;
        for (int q = 0; q < kParts; ++q) {
          s0 += red[16 + (group * kParts + q) * 2];
          s1 += red[16 + (group * kParts + q) * 2 + 1];
        }
      }
      __syncthreads();
    }
    if (valid && part == 0 && lane == 0) {
      float out;
      if (epi == kSiluPair) out = silu(s0) * s1;
      else if (epi == kResidual) out = y[r] + s0;
      else out = s0;
      y[r] = out;
      if constexpr (kCount) {
        const int64_t e = second ? p.rows + r : r;
        atomicAdd(p.counts + e, 1u);
        p.owner[e] = (int32_t)(blockIdx.x * kGroups + group);
      }
    }
  }
}

// Split-K matrix-vector product for long rows: CTA b works on column slice
// part = b % parts of every row, so it stages only that slice of x in shared
// memory (several CTAs fit per SM); each warp computes (row, slice) dot
// products with no block barrier and writes one partial per unit. The finish
// kernel adds a row's partials in slice order (deterministic) to h.
template <int kUnroll>
__global__ void __launch_bounds__(kThreads) gemv_partial_kernel(const __grid_constant__ GemvArgs p, int parts,
                                                                float* __restrict__ partial) {
  extern __shared__ float xs[];
  const int part = (int)(blockIdx.x % parts);
  const int64_t nv = p.k / 8;
  const int64_t per = (nv + parts - 1) / parts;
  const int64_t k0 = min(nv, part * per) * 8;
  const int64_t k1 = part == parts - 1 ? p.k : min(nv, (part + 1) * per) * 8;
  for (int64_t i = threadIdx.x; i < k1 - k0; i += kThreads) xs[i] = p.x[k0 + i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t ctas = gridDim.x / parts;  // CTAs working on this slice
  const int64_t nwarps = ctas * kWarps;
  for (int64_t r = (int64_t)(blockIdx.x / parts) * kWarps + threadIdx.x / 32; r < p.rows; r += nwarps) {
    const float s = row_dot<kUnroll>(p.w + r * p.ld, xs - k0, p.k, part, parts);
    if (lane == 0) partial[(int64_t)part * p.rows + r] = s;
  }
}

template <bool kCount>
__global__ void __launch_bounds__(kThreads) residual_finish_kernel(float* __restrict__ h, const float* __restrict__ partial,
                                                                   int64_t rows, int parts, uint32_t* counts,
                                                                   int32_t* owner) {
  // launched as a programmatic dependent of the kernel that wrote the partial
  // sums: let the next kernel be scheduled at once, then wait for them
  sm100::allow_dependents();
  sm100::grid_dependency_wait();
  const int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (r >= rows) return;
  float s = 0.f;
  for (int q = 0; q < parts; ++q) s += partial[(int64_t)q * rows + r];
  h[r] = h[r] + s;
  if constexpr (kCount) {
    atomicAdd(counts + r, 1u);
    owner[r] = (int32_t)blockIdx.x;
  }
}

// ------------------------------------------------ TMA-fed matrix-vector products
constexpr int kSCols = 256;                       // columns per stage (512 bytes of bf16)
constexpr int kSRows = 32;                        // rows of a plain unit (one 16 KB box)
constexpr int kSPairRows = 16;                    // row pairs of a SiLU unit (one 16 KB 3-D box)
constexpr int kSStage = kSRows * kSCols * 2;      // 16 KB per stage
constexpr int kSConsumers = 8;                    // consumer warps
constexpr int kSThreads = (kSConsumers + 1) * 32; // + the producer warp
constexpr int kSStages = 12;                      // ring stages at most (StreamArgs::stages)
constexpr int kSMaxXCols = 8192;                  // x (or a slice of it) kept in shared memory, fp32
constexpr int kSXVec = kSMaxXCols / (kSConsumers * 32 * 4);  // 16-byte pieces of x per consumer thread
constexpr int kSMaxXBufs = 4;                     // x slice buffers (sliced mode)
constexpr int kSOBuf = 32;                        // units whose outputs are held in shared memory
constexpr size_t kSSmemMax = 232448;              // opt-in shared memory per CTA
// shared memory beside the x buffers: alignment slack, ring, barriers, abort word, reduction scratch
// alignment slack, barriers, abort word, reduction scratch, output buffer (+ the ring and x)
constexpr size_t kSSmemFixed = 1024 + 8 * (2 * kSStages + 2 * kSMaxXBufs) + 16 + 64 + (size_t)kSOBuf * kSRows * 4;

// Units of equal work (32 rows x one K slice): a plain unit is 32 rows of its
// problem, a SiLU-pair unit 16 rows g = [r0, +16) of the first half of its
// weight matrix and their partners u, the same rows of the second half. Problem 0 has units0
// units, problem 1 the rest. With slices > 1 (long rows) a unit is (row
// block, K slice), its dot products go to partial[slice * rows + r], and the
// producer brings each unit's slice of x into one of xbufs x buffers (2-4,
// as many as shared memory holds).
struct StreamArgs {
  int64_t k;                // columns (x length)
  int32_t slices;           // K slices (1, or > 1 with partial sums)
  int32_t xbufs;            // x slice buffers when slices > 1 (2..kSMaxXBufs)
  int32_t stages;           // ring stages (2..kSStages)
  int32_t early_weights;    // weights may be copied before the dependency wait (TP_EXEC_STATIC_WEIGHTS)
  int64_t slice_cols;       // columns per slice, a multiple of kSCols, <= kSMaxXCols
  int64_t units0, units;    // units of problem 0, total units
  int64_t rows0, rows1;
  int32_t epi0, epi1;       // kPlain / kSiluPair / kResidual (partial sums when slices > 1)
  float* y0;
  float* y1;
  float* partial;
  const float* x;           // 16-byte aligned
  int32_t norm;             // x = rmsnorm(x) * gamma (slices == 1 only)
  float eps;
  const float* gamma;
  int* err;
  uint64_t wait_ns;
  uint32_t* counts;
  int32_t* owner;
};

template <bool kCount>
__global__ void __launch_bounds__(kSThreads, 1)
    gemv_stream_kernel(const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1,
                       const __grid_constant__ StreamArgs p) {
  using namespace sm100;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  // [ring: stages x 16 KB][x: one buffer of slice_cols floats, xbufs when sliced][barriers]
  const int nst = p.stages;
  const uint32_t xcols = (uint32_t)p.slice_cols;
  const uint32_t xstride = (xcols + 3u) & ~3u;  // floats per x buffer: 16-byte multiples
  const int xbufs = p.slices > 1 ? p.xbufs : 1;
  const uint32_t xs0 = base + (uint32_t)kSStage * nst;
  float* xsp = reinterpret_cast<float*>(gbase + (size_t)kSStage * nst);
  const uint32_t bars = xs0 + 4u * xstride * (uint32_t)xbufs;
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 8u * (kSStages + s); };
  auto xfull_bar = [&](int b) { return bars + 8u * (2 * kSStages + b); };
  auto xempty_bar = [&](int b) { return bars + 8u * (2 * kSStages + kSMaxXBufs + b); };
  const uint32_t words = 8u * (2 * kSStages + 2 * kSMaxXBufs);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + (bars - base) + words);
  float* red = reinterpret_cast<float*>(gbase + (bars - base) + words + 16u);
  // outputs of the last kSOBuf units: slot t mod kSOBuf holds unit t's 32
  // values (warp w's at [4w, 4w + 4)), written to global memory kSOBuf units
  // at a time and at the end
  float* obuf = red + 16;
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), kSConsumers);
    }
    for (int b = 0; b < kSMaxXBufs; ++b) {
      mbar_init(xfull_bar(b), 1);
      mbar_init(xempty_bar(b), kSConsumers);
    }
    *abort_flag = 0;
    fence_mbar_init();
    if (p.units0 > 0) tma_prefetch_desc(&map0);
    if (p.units > p.units0) tma_prefetch_desc(&map1);
  }
  __syncthreads();
  // Programmatic dependent launch: when the caller vouches that the weights
  // are not written by the grids before this one (early_weights), the
  // producer streams them at once, overlapping the previous kernel's tail;
  // otherwise it waits for those grids first. x (written by the previous
  // kernels) is read only after the dependency wait (consumers; the
  // producer before its first copy of an x slice).
  allow_dependents();
  // consumers only (warps 0-7): named barrier 1
  auto consumers_sync = [] { asm volatile("bar.sync 1, %0;" ::"n"(kSConsumers * 32) : "memory"); };
  if (warp < kSConsumers) {
    grid_dependency_wait();
    if (p.slices == 1) {
      // The whole of x (normalised) in shared memory. Each consumer thread
      // loads its 16-byte pieces of x (and of gamma) at once, up to
      // kSXVec of them, so the prologue waits about one memory latency,
      // not one per element.
      constexpr int kT = kSConsumers * 32;
      const int64_t n4 = p.k / 4;   // whole 16-byte pieces
      const int tail = (int)(p.k - 4 * n4);
      const float4* x4 = reinterpret_cast<const float4*>(p.x);
      float4 xv[kSXVec];
#pragma unroll
      for (int j = 0; j < kSXVec; ++j) {
        const int64_t i4 = threadIdx.x + (int64_t)j * kT;
        xv[j] = i4 < n4 ? x4[i4] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      const float xt = threadIdx.x < tail ? p.x[4 * n4 + threadIdx.x] : 0.f;
      float gv[kSXVec][4];
      float gt = 1.f;
#pragma unroll
      for (int j = 0; j < kSXVec; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) gv[j][c] = 1.f;
      if (p.norm && p.gamma) {
#pragma unroll
        for (int j = 0; j < kSXVec; ++j) {
          const int64_t i4 = threadIdx.x + (int64_t)j * kT;
          if (i4 < n4)
#pragma unroll
            for (int c = 0; c < 4; ++c) gv[j][c] = p.gamma[4 * i4 + c];
        }
        if (threadIdx.x < tail) gt = p.gamma[4 * n4 + threadIdx.x];
      }
      float scale = 1.f;
      if (p.norm) {
        float sq = xt * xt;
#pragma unroll
        for (int j = 0; j < kSXVec; ++j) {
          sq = fmaf(xv[j].x, xv[j].x, sq);
          sq = fmaf(xv[j].y, xv[j].y, sq);
          sq = fmaf(xv[j].z, xv[j].z, sq);
          sq = fmaf(xv[j].w, xv[j].w, sq);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (lane == 0) red[warp] = sq;
        consumers_sync();
        float t = 0.f;
        for (int w = 0; w < kSConsumers; ++w) t += red[w];  // fixed order
        scale = rsqrtf(t / (float)p.k + p.eps);
      }
      float4* xs4 = reinterpret_cast<float4*>(xsp);
#pragma unroll
      for (int j = 0; j < kSXVec; ++j) {
        const int64_t i4 = threadIdx.x + (int64_t)j * kT;
        if (i4 < n4) {
          float4 v = xv[j];
          if (p.norm) {
            v.x = v.x * scale * gv[j][0];
            v.y = v.y * scale * gv[j][1];
            v.z = v.z * scale * gv[j][2];
            v.w = v.w * scale * gv[j][3];
          }
          xs4[i4] = v;
        }
      }
      if (threadIdx.x < tail) xsp[4 * n4 + threadIdx.x] = p.norm ? xt * scale * gt : xt;
      consumers_sync();
    }
  }
  const int64_t stages_per_unit = (p.slice_cols + kSCols - 1) / kSCols;
  // unit u -> problem, row block, K slice
  auto decode_unit = [&](int64_t u, bool* second, int64_t* rb, int32_t* slice) {
    *second = u >= p.units0;
    const int64_t ub = *second ? u - p.units0 : u;
    *rb = p.slices > 1 ? ub / p.slices : ub;
    *slice = p.slices > 1 ? (int32_t)(ub % p.slices) : 0;
  };
  if (warp == kSConsumers) {
    // ---------------- producer: one thread issues every copy. With K
    // slices, unit t's x slice goes to buffer t mod xbufs; the first unit's
    // weight stages (as many as the ring holds) are issued before the
    // dependency wait, the x slices only after it.
    if (lane == 0) {
      uint32_t fills[kSStages] = {};
      uint32_t xfills[kSMaxXBufs] = {};
      int stage = 0;
      uint32_t phase = 0;
      int64_t t = 0;  // units taken by this CTA
      bool ok = true;
      const uint64_t pol = policy_evict_first();  // weights are read once
      if (!p.early_weights) grid_dependency_wait();
      for (int64_t u = blockIdx.x; u < p.units && ok; u += gridDim.x, ++t) {
        bool second;
        int64_t rb;
        int32_t slice;
        decode_unit(u, &second, &rb, &slice);
        const bool pair = (second ? p.epi1 : p.epi0) == kSiluPair;
        const CUtensorMap* m = second ? &map1 : &map0;
        const int32_t r0 = (int32_t)(rb * (pair ? kSPairRows : kSRows));
        auto issue = [&](int64_t st) {
          if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, p.err, p.wait_ns)) return false;
          const int32_t c0 = (int32_t)(slice * p.slice_cols + st * kSCols);  // 512-byte aligned
          const uint32_t dst = base + (uint32_t)kSStage * stage;
          mbar_arrive_expect_tx(full_bar(stage), (uint32_t)kSStage);
          if (pair) tma_load_3d(dst, m, c0, r0, 0, full_bar(stage), pol);  // g rows, then their u rows
          else tma_load_2d(dst, m, c0, r0, full_bar(stage), pol);
          fills[stage]++;
          if (++stage == nst) { stage = 0; phase ^= 1u; }
          return true;
        };
        int64_t st = 0;
        if (p.slices > 1) {
          if (t == 0) {
            // consumers start on x only after this copy, so at most a ring's
            // worth of stages goes first
            if (p.early_weights)
              for (; st < stages_per_unit && st < nst && ok; ++st) ok = issue(st);
            if (!ok) break;
            grid_dependency_wait();  // x is the previous kernels' output
          }
          // this unit's slice of x (whole 8-float pieces: k is a multiple of 8)
          const int xb = (int)(t % xbufs);
          if (!mbar_wait(xempty_bar(xb), (uint32_t)(((t / xbufs) & 1) ^ 1), abort_flag, p.err, p.wait_ns)) {
            ok = false;
            break;
          }
          const int64_t c0 = (int64_t)slice * p.slice_cols;
          const uint32_t bytes = (uint32_t)(min(p.slice_cols, p.k - c0) * 4);
          mbar_arrive_expect_tx(xfull_bar(xb), bytes);
          bulk_copy_g2s(xs0 + 4u * xstride * (uint32_t)xb, p.x + c0, bytes, xfull_bar(xb));
          xfills[xb]++;
        }
        for (; st < stages_per_unit && ok; ++st) ok = issue(st);
      }
      if (!ok) {
        // every copy this thread issued lands before the CTA retires
        for (int s2 = 0; s2 < nst; ++s2)
          if (fills[s2]) mbar_wait(full_bar(s2), (fills[s2] - 1u) & 1u, nullptr, nullptr, 200000000ull);
        for (int b = 0; b < kSMaxXBufs; ++b)
          if (xfills[b]) mbar_wait(xfull_bar(b), (xfills[b] - 1u) & 1u, nullptr, nullptr, 200000000ull);
      }
    }
    __syncwarp();
  } else {
    // ---------------- consumers: warp w owns rows [4w, 4w + 4) of a plain
    // unit, or row pairs [2w, 2w + 2) of a SiLU-pair unit (g in the stage's
    // first half, u in its second)
    int stage = 0;
    uint32_t phase = 0;
    int64_t t = 0, done = 0;
    bool ok = true;
    // Writes this warp's outputs of the CTA's units [t0, t1) (at most kSOBuf),
    // 8 units per round, lane l taking value l % 4 of unit t0 + l / 4 (a
    // SiLU-pair unit has 2 values per warp, the others 4). Stores of a unit
    // leave at once in a batch instead of holding up the next stage's
    // release of its ring slot.
    auto flush = [&](int64_t t0, int64_t t1) {
      __syncwarp();
      for (int64_t b0 = t0; b0 < t1; b0 += 8) {
        const int64_t tt = b0 + lane / 4;
        const int q = lane & 3;
        if (tt >= t1) continue;
        bool sec;
        int64_t rbb;
        int32_t sl;
        decode_unit(blockIdx.x + tt * (int64_t)gridDim.x, &sec, &rbb, &sl);
        const int ep = sec ? p.epi1 : p.epi0;
        const bool pr = ep == kSiluPair;
        if (pr && q >= 2) continue;
        const int64_t rows = sec ? p.rows1 : p.rows0;
        const int64_t r = pr ? rbb * kSPairRows + 2 * warp + q : rbb * kSRows + 4 * warp + q;
        if (r >= rows) continue;
        const float v = obuf[(tt % kSOBuf) * kSRows + 4 * warp + q];
        if (p.slices > 1) {
          p.partial[(int64_t)sl * rows + r] = v;
          continue;
        }
        float* y = sec ? p.y1 : p.y0;
        y[r] = ep == kResidual ? y[r] + v : v;
        if constexpr (kCount) {
          const int64_t e = sec ? p.rows0 + r : r;
          atomicAdd(p.counts + e, 1u);
          p.owner[e] = (int32_t)blockIdx.x;
        }
      }
      __syncwarp();
    };
    for (int64_t u = blockIdx.x; u < p.units && ok; u += gridDim.x, ++t) {
      bool second;
      int64_t rb;
      int32_t slice;
      decode_unit(u, &second, &rb, &slice);
      const int epi = second ? p.epi1 : p.epi0;
      const bool pair = epi == kSiluPair;
      const int xb = p.slices > 1 ? (int)(t % xbufs) : 0;
      const float* xs = xsp + (size_t)xstride * xb;
      const int64_t lim = min(p.k - (int64_t)slice * p.slice_cols, p.slice_cols);  // valid x in this slice
      if (p.slices > 1) {
        const bool got = mbar_wait(xfull_bar(xb), (uint32_t)((t / xbufs) & 1), abort_flag, p.err, p.wait_ns);
        if (!__all_sync(0xffffffffu, got)) break;
      }
      // acc[q][j]: q = row (plain) or 2 * half + pair (SiLU); j = lane slot
      float acc[4][4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[q][j] = 0.f;
      for (int64_t st = 0; st < stages_per_unit; ++st) {
        // this lane's 8 columns of x (zero past the valid part of the buffer)
        const int64_t cx = st * kSCols + lane * 8;
        float xv[8];
        if (cx + 8 <= lim) {
          const float4 a = *reinterpret_cast<const float4*>(xs + cx);
          const float4 b = *reinterpret_cast<const float4*>(xs + cx + 4);
          xv[0] = a.x; xv[1] = a.y; xv[2] = a.z; xv[3] = a.w;
          xv[4] = b.x; xv[5] = b.y; xv[6] = b.z; xv[7] = b.w;
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) xv[j] = cx + j < lim ? xs[cx + j] : 0.f;
        }
        const bool got = mbar_wait(full_bar(stage), phase, abort_flag, p.err, p.wait_ns);
        if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
        const uint32_t src = base + (uint32_t)kSStage * stage;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          // smem row of slot q: plain row 4w + q; SiLU half q / 2, pair 2w + q % 2
          const uint32_t row = pair ? (uint32_t)((q >> 1) * kSPairRows + 2 * warp + (q & 1)) : (uint32_t)(4 * warp + q);
          uint32_t w4[4];
          ld_shared_v4(src + row * (kSCols * 2) + (uint32_t)lane * 16u, w4);
          const __nv_bfloat162* w2 = reinterpret_cast<const __nv_bfloat162*>(w4);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float2 f = __bfloat1622float2(w2[j]);
            acc[q][j] = fmaf(f.x, xv[2 * j], acc[q][j]);
            acc[q][j] = fmaf(f.y, xv[2 * j + 1], acc[q][j]);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty_bar(stage));
        if (++stage == nst) { stage = 0; phase ^= 1u; }
      }
      if (p.slices > 1 && ok) {
        __syncwarp();
        if (lane == 0) mbar_arrive(xempty_bar(xb));  // this warp is done with the x buffer
      }
      if (!ok) break;
      // fixed-order reductions: the lane's four slots, then a butterfly
      float sum[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float tq = (acc[q][0] + acc[q][1]) + (acc[q][2] + acc[q][3]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tq += __shfl_xor_sync(0xffffffffu, tq, o);
        sum[q] = tq;
      }
      if (lane == 0) {
        float* ob = obuf + (t % kSOBuf) * kSRows + 4 * warp;
        if (pair && p.slices == 1) {
          ob[0] = silu(sum[0]) * sum[2];
          ob[1] = silu(sum[1]) * sum[3];
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) ob[q] = sum[q];
        }
      }
      done = t + 1;
      if (done % kSOBuf == 0) flush(done - kSOBuf, done);
    }
    if (ok && done % kSOBuf) flush(done - done % kSOBuf, done);
  }
}

struct VecArgs {
  const float* a;
  const float* b;
  float* y;
  int64_t n;
  float eps;
  int32_t op;  // 0 rmsnorm (a = h, b = gamma), 1 silu_mul (a = gu), 2 residual add (y += a)
  uint32_t* counts;
  int32_t* owner;
};

template <bool kCount>
__global__ void __launch_bounds__(kThreads) vec_kernel(const __grid_constant__ VecArgs p) {
  __shared__ float red[kWarps];
  float scale = 1.f;
  if (p.op == 0) scale = block_rms_scale(p.a, p.n, p.eps, red);
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < p.n; i += stride) {
    float v;
    if (p.op == 0) v = p.a[i] * scale * (p.b ? p.b[i] : 1.f);
    else if (p.op == 1) v = silu(p.a[i]) * p.a[i + p.n];
    else v = p.y[i] + p.a[i];
    p.y[i] = v;
    if constexpr (kCount) {
      atomicAdd(p.counts + i, 1u);
      p.owner[i] = (int32_t)blockIdx.x;
    }
  }
}

bool vec_f32(const tp_tensor* t, int64_t n) {
  return t && t->dtype == TP_F32 && t->rank == 1 && t->shape[0] == n && (t->strides[0] == 1 || n <= 1);
}

bool weights(const tp_tensor* w, int64_t rows, int64_t k) {
  return w && w->dtype == TP_BF16 && w->rank == 2 && w->shape[0] == rows && w->shape[1] == k &&
         w->strides[1] == 1 && (w->strides[0] % 8) == 0 && ((uintptr_t)w->ptr & 15) == 0;
}

bool vec_out(const tp_partition* p, int64_t n) {
  return p && p->t.dtype == TP_F32 && p->rank == 1 && p->shape[0] == n;
}

template <int kEpi, int kParts, int kUnroll>
cudaError_t launch_gemv(const GemvArgs& a, int grid, cudaStream_t st) {
  const size_t smem = (((a.k + 3) & ~int64_t(3)) + 16 + 2 * kWarps) * sizeof(float);
  auto k = a.counts ? gemv_kernel<kEpi, kParts, kUnroll, true> : gemv_kernel<kEpi, kParts, kUnroll, false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

int gemv_grid(tp_ctx* ctx, int64_t k) {
  // shared memory holds the input vector; 2 CTAs per SM for 100 KB vectors
  const size_t smem = (size_t)k * 4 + 256;
  const int per_sm = smem > 110 * 1024 ? 1 : (smem > 70 * 1024 ? 2 : 4);
  return ctx->sm_count * per_sm;
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

// Weights [rows, k] bf16 (row stride ld) as boxes of 32 rows x 256 columns,
// no swizzle (each row's 512 bytes contiguous in shared memory), zero fill
// past the edges. A SiLU-pair matrix ([2 n, k]: g rows, then u rows) is seen
// as 3-D {k, n, 2} and boxed {256, 16, 2}, so one copy brings 16 g rows and
// their 16 u partners (16 KB, g first).
tp_status weight_map(CUtensorMap* map, const tp_tensor* w, bool pair) {
  auto fn = encode_fn();
  if (!fn) return fail(TP_ERR_CUDA, "cuTensorMapEncodeTiled unavailable from the driver");
  const int64_t half = w->shape[0] / 2;
  cuuint64_t dims[3] = {(cuuint64_t)w->shape[1], (cuuint64_t)(pair ? half : w->shape[0]), 2};
  cuuint64_t strides[2] = {(cuuint64_t)(w->strides[0] * 2), (cuuint64_t)(half * w->strides[0] * 2)};
  cuuint32_t box[3] = {(cuuint32_t)kSCols, (cuuint32_t)(pair ? kSPairRows : kSRows), 2};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, pair ? 3 : 2, w->ptr, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(TP_ERR_CUDA, "cuTensorMapEncodeTiled (weights) failed (" + std::to_string((int)r) + ")");
  return TP_OK;
}

// Ring depth of the streaming kernel: 10 stages of 16 KB per SM. Deeper
// rings were measured slower (a 10240 x 5120 + 51200 x 5120 product: 89.4 us
// at 10 stages, 92.6 at 12; 8 stages: 89.7), the DRAM queues fuller for no
// more bandwidth.
constexpr int kSRingStages = 10;
int stream_stages() { return kSRingStages; }

// The longest K slice (whole stages) of which two x buffers fit beside the ring.
int64_t stream_max_slice_cols() {
  const size_t fixed = kSSmemFixed + (size_t)kSStage * stream_stages();
  return (int64_t)((kSSmemMax - fixed) / 8 / kSCols * kSCols);
}

// The streaming kernel on w0 (problem 0) and w1 (problem 1, may equal w0):
// one persistent CTA per SM, or one per unit when there are fewer units.
tp_status launch_stream(tp_ctx* ctx, StreamArgs a, const tp_tensor* w0, bool pair0, const tp_tensor* w1, bool pair1,
                        cudaStream_t st) {
  // a problem without units has no map (and its descriptor is never touched)
  CUtensorMap m0 = {}, m1 = {};
  tp_status s = a.units0 > 0 ? weight_map(&m0, w0, pair0) : TP_OK;
  if (s == TP_OK && a.units > a.units0) s = weight_map(&m1, w1, pair1);
  if (s != TP_OK) return s;
  a.err = ctx->d_err;
  a.wait_ns = 2000000000ull;
  // x: one buffer, or with K slices as many (2..kSMaxXBufs) as fit
  a.stages = stream_stages();
  const size_t fixed = kSSmemFixed + (size_t)kSStage * a.stages;
  const size_t xbuf = (size_t)((a.slice_cols + 3) & ~int64_t(3)) * 4;
  a.xbufs = a.slices > 1 ? (int32_t)std::min<size_t>(kSMaxXBufs, (kSSmemMax - fixed) / xbuf) : 1;
  if (a.slices > 1 && a.xbufs < 2) return fail(TP_ERR_INVALID, "streaming matrix-vector kernel: K slice too long");
  const size_t smem = fixed + xbuf * (size_t)a.xbufs;
  auto k = a.counts ? gemv_stream_kernel<true> : gemv_stream_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "streaming matrix-vector kernel attributes");
  // the fewest CTAs (at most one per SM) that take as many units each as
  // one per SM would: every CTA gets the same count, give or take one
  int grid = (int)std::min<int64_t>(a.units, ctx->sm_count);
  if (grid > 0) {
    const int64_t per = (a.units + grid - 1) / grid;
    grid = (int)((a.units + per - 1) / per);
  }
  if (grid > 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kSThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k, m0, m1, a);
    if (e != cudaSuccess) return cuda_fail(e, "streaming matrix-vector kernel launch");
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "streaming matrix-vector kernel launch");
  return TP_OK;
}

// Whether the streaming kernel takes x: 16-byte aligned fp32 (copied to
// shared memory in bulk, read in 16-byte pieces).
bool stream_ok(const tp_tensor* x) { return ((uintptr_t)x->ptr & 15) == 0; }

tp_status check_counts(const tp_exec* ex) {
  if ((ex->write_counts == nullptr) != (ex->write_owner == nullptr))
    return fail(TP_ERR_INVALID, "write_counts and write_owner must be given together");
  return TP_OK;
}

}  // namespace
}  // namespace tp

using namespace tp;

extern "C" {

tp_status tp_rmsnorm(tp_ctx* ctx, tp_partition* n_out, const tp_tensor* h, const tp_tensor* gamma, float eps,
                     const tp_exec* ex) {
  if (!ctx || !n_out || !h || !ex) return fail(TP_ERR_INVALID, "null argument");
  const int64_t d = n_out->shape[0];
  if (!vec_out(n_out, d) || !vec_f32(h, d) || (gamma && !vec_f32(gamma, d)))
    return fail(TP_ERR_SHAPE, "rmsnorm takes fp32 vectors of one length");
  tp_status s = check_counts(ex);
  if (s != TP_OK) return s;
  Op o(__func__);
  s = gamma ? o.begin(ctx, ex, {n_out}, {h, gamma}) : o.begin(ctx, ex, {n_out}, {h});
  if (s != TP_OK) return s;
  VecArgs a{h ? static_cast<const float*>(h->ptr) : nullptr, gamma ? static_cast<const float*>(gamma->ptr) : nullptr,
            static_cast<float*>(n_out->t.ptr), d, eps, 0, ex->write_counts, ex->write_owner};
  // the scale needs the whole vector: one CTA (d is a hidden size, tiny)
  if (d > 0) {
    if (a.counts) vec_kernel<true><<<1, kThreads, 0, o.stream>>>(a);
    else vec_kernel<false><<<1, kThreads, 0, o.stream>>>(a);
  }
  return o.end(cudaGetLastError());
}

tp_status tp_gemv(tp_ctx* ctx, tp_partition* y, const tp_tensor* w, const tp_tensor* x, const tp_exec* ex) {
  if (!ctx || !y || !w || !x || !ex) return fail(TP_ERR_INVALID, "null argument");
  const int64_t rows = y->shape[0], k = x->shape[0];
  if (!vec_out(y, rows) || !vec_f32(x, k)) return fail(TP_ERR_SHAPE, "gemv: y [rows] and x [k] fp32");
  if (!weights(w, rows, k)) return fail(TP_ERR_SHAPE, "gemv: W must be bf16 [rows, k], rows 16-byte aligned");
  tp_status s = check_counts(ex);
  if (s != TP_OK) return s;
  Op o(__func__);
  s = o.begin(ctx, ex, {y}, {w, x});
  if (s != TP_OK) return s;
  GemvArgs a{};
  a.w = static_cast<const __nv_bfloat16*>(w->ptr);
  a.x = static_cast<const float*>(x->ptr);
  a.y = static_cast<float*>(y->t.ptr);
  a.rows = rows;
  a.k = k;
  a.ld = w->strides[0];
  a.counts = ex->write_counts;
  a.owner = ex->write_owner;
  cudaError_t e = cudaSuccess;
  if (rows > 0 && k > 0) e = launch_gemv<kPlain, 1, 4>(a, gemv_grid(ctx, k), o.stream);
  return o.end(e);
}

tp_status tp_silu_mul(tp_ctx* ctx, tp_partition* a_out, const tp_tensor* gu, const tp_exec* ex) {
  if (!ctx || !a_out || !gu || !ex) return fail(TP_ERR_INVALID, "null argument");
  const int64_t n = a_out->shape[0];
  if (!vec_out(a_out, n) || !vec_f32(gu, 2 * n)) return fail(TP_ERR_SHAPE, "silu_mul: a [n], gu [2n] fp32");
  tp_status s = check_counts(ex);
  if (s != TP_OK) return s;
  Op o(__func__);
  s = o.begin(ctx, ex, {a_out}, {gu});
  if (s != TP_OK) return s;
  VecArgs a{static_cast<const float*>(gu->ptr), nullptr, static_cast<float*>(a_out->t.ptr), n, 0.f, 1,
            ex->write_counts, ex->write_owner};
  if (n > 0) {
    const int grid = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 4 * ctx->sm_count);
    if (a.counts) vec_kernel<true><<<grid, kThreads, 0, o.stream>>>(a);
    else vec_kernel<false><<<grid, kThreads, 0, o.stream>>>(a);
  }
  return o.end(cudaGetLastError());
}

tp_status tp_residual_add(tp_ctx* ctx, tp_partition* h, const tp_tensor* d, const tp_exec* ex) {
  if (!ctx || !h || !d || !ex) return fail(TP_ERR_INVALID, "null argument");
  const int64_t n = h->shape[0];
  if (!vec_out(h, n) || !vec_f32(d, n)) return fail(TP_ERR_SHAPE, "residual_add: h [n], d [n] fp32");
  tp_status s = check_counts(ex);
  if (s != TP_OK) return s;
  Op o(__func__);
  s = o.begin(ctx, ex, {h}, {d});
  if (s != TP_OK) return s;
  VecArgs a{static_cast<const float*>(d->ptr), nullptr, static_cast<float*>(h->t.ptr), n, 0.f, 2,
            ex->write_counts, ex->write_owner};
  if (n > 0) {
    const int grid = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 4 * ctx->sm_count);
    if (a.counts) vec_kernel<true><<<grid, kThreads, 0, o.stream>>>(a);
    else vec_kernel<false><<<grid, kThreads, 0, o.stream>>>(a);
  }
  return o.end(cudaGetLastError());
}

tp_status tp_decode_norm_qkv_gu(tp_ctx* ctx, tp_partition* qkv, tp_partition* a_out, const tp_tensor* h,
                                const tp_tensor* gamma, const tp_tensor* w_qkv, const tp_tensor* w_gu, float eps,
                                const tp_exec* ex) {
  if (!ctx || !qkv || !a_out || !h || !w_qkv || !w_gu || !ex) return fail(TP_ERR_INVALID, "null argument");
  const int64_t d = h->shape[0], nq = qkv->shape[0], ni = a_out->shape[0];
  if (!vec_f32(h, d) || !vec_out(qkv, nq) || !vec_out(a_out, ni) || (gamma && !vec_f32(gamma, d)))
    return fail(TP_ERR_SHAPE, "norm_qkv_gu: fp32 h [d], qkv [nq], a [ni]");
  if (!weights(w_qkv, nq, d) || !weights(w_gu, 2 * ni, d))
    return fail(TP_ERR_SHAPE, "norm_qkv_gu: W_qkv bf16 [nq, d], W_gu bf16 [2 ni, d]");
  tp_status s = check_counts(ex);
  if (s != TP_OK) return s;
  Op o(__func__);
  o.allow_static_weights = true;
  s = gamma ? o.begin(ctx, ex, {qkv, a_out}, {h, gamma, w_qkv, w_gu}) : o.begin(ctx, ex, {qkv, a_out}, {h, w_qkv, w_gu});
  if (s != TP_OK) return s;
  GemvArgs a{};
  a.w = static_cast<const __nv_bfloat16*>(w_qkv->ptr);
  a.x = static_cast<const float*>(h->ptr);
  a.y = static_cast<float*>(qkv->t.ptr);
  a.rows = nq;
  a.k = d;
  a.ld = w_qkv->strides[0];
  a.norm = 1;
  a.eps = eps;
  a.gamma = gamma ? static_cast<const float*>(gamma->ptr) : nullptr;
  a.w2 = static_cast<const __nv_bfloat16*>(w_gu->ptr);
  a.y2 = static_cast<float*>(a_out->t.ptr);
  a.rows2 = ni;
  a.ld2 = w_gu->strides[0];
  a.pair_offset2 = ni;
  a.epi2 = kSiluPair;
  a.counts = ex->write_counts;
  a.owner = ex->write_owner;
  cudaError_t e = cudaSuccess;
  if (d > 0 && nq + ni > 0) {
    if (stream_ok(h) && d <= kSMaxXCols) {
      // QKV rows in 32-row units, then gate/up pairs in 16-pair units
      o.check_err = true;  // its waits are bounded: a timeout lands in the error word
      StreamArgs sa{};
      sa.k = d;
      sa.slices = 1;
      sa.slice_cols = d;
      sa.units0 = (nq + kSRows - 1) / kSRows;
      sa.units = sa.units0 + (ni + kSPairRows - 1) / kSPairRows;
      sa.rows0 = nq;
      sa.rows1 = ni;
      sa.epi0 = kPlain;
      sa.epi1 = kSiluPair;
      sa.y0 = a.y;
      sa.y1 = a.y2;
      sa.x = a.x;
      sa.norm = 1;
      sa.eps = eps;
      sa.gamma = a.gamma;
      sa.counts = a.counts;
      sa.owner = a.owner;
      sa.early_weights = (ex->flags & TP_EXEC_STATIC_WEIGHTS) ? 1 : 0;
      tp_status ls = launch_stream(ctx, sa, w_qkv, false, w_gu, true, o.stream);
      if (ls != TP_OK) {
        o.abort();
        return ls;
      }
    } else {
      e = launch_gemv<kPlain, 1, 4>(a, gemv_grid(ctx, d), o.stream);
    }
  }
  return o.end(e);
}

tp_status tp_decode_down_residual(tp_ctx* ctx, tp_partition* h, const tp_tensor* w_down, const tp_tensor* a_in,
                                  const tp_exec* ex) {
  if (!ctx || !h || !w_down || !a_in || !ex) return fail(TP_ERR_INVALID, "null argument");
  const int64_t d = h->shape[0], ni = a_in->shape[0];
  if (!vec_out(h, d) || !vec_f32(a_in, ni)) return fail(TP_ERR_SHAPE, "down_residual: fp32 h [d], a [ni]");
  if (!weights(w_down, d, ni)) return fail(TP_ERR_SHAPE, "down_residual: W_down bf16 [d, ni]");
  tp_status s = check_counts(ex);
  if (s != TP_OK) return s;
  Op o(__func__);
  o.allow_static_weights = true;
  s = o.begin(ctx, ex, {h}, {w_down, a_in});
  if (s != TP_OK) return s;
  GemvArgs a{};
  a.w = static_cast<const __nv_bfloat16*>(w_down->ptr);
  a.x = static_cast<const float*>(a_in->ptr);
  a.y = static_cast<float*>(h->t.ptr);
  a.rows = d;
  a.k = ni;
  a.ld = w_down->strides[0];
  a.counts = ex->write_counts;
  a.owner = ex->write_owner;
  cudaError_t e = cudaSuccess;
  // Streamed in K slices as long as two x buffers of one fit beside the
  // ring, and more of them (down to 2048 columns) while the units (32-row
  // block x slice) number under four per SM; slices of equal whole stages.
  // Few long units beat many short ones (measured: a 5120 x 25600 product
  // takes 43.4 us in 4 slices, 44.7 us in 10, 52 us in 15). One slice (x
  // whole in shared memory, no finish kernel) when that is all it takes.
  const int64_t row_blocks = (d + kSRows - 1) / kSRows;
  const int64_t max_cols = stream_max_slice_cols();
  int64_t slices64 = (ni + max_cols - 1) / max_cols;
  while (row_blocks * slices64 < 4 * (int64_t)ctx->sm_count && ni / (slices64 + 1) >= 2048) ++slices64;
  int32_t slices = (int32_t)slices64;
  int64_t slice_cols = slices == 1 ? ni : ((ni + slices - 1) / slices + kSCols - 1) / kSCols * kSCols;
  if (slices > 1) slices = (int32_t)((ni + slice_cols - 1) / slice_cols);
  // (x slices arrive by bulk copies, whose sizes are multiples of 16 bytes)
  const bool streamed = stream_ok(a_in) && (slices == 1 || ni % 4 == 0) && d * slices <= tp_ctx::kPartialFloats;
  if (d > 0 && ni > 0 && streamed) {
    o.check_err = true;  // the streaming kernel's waits are bounded
    // 32-row units; with slices, a finish kernel adds the partial sums to h
    // in slice order
    StreamArgs sa{};
    sa.k = ni;
    sa.slices = slices;
    sa.slice_cols = slice_cols;
    sa.units0 = (d + kSRows - 1) / kSRows * sa.slices;
    sa.units = sa.units0;
    sa.rows0 = d;
    sa.rows1 = d;
    sa.epi0 = kResidual;
    sa.epi1 = kResidual;
    sa.y0 = a.y;
    sa.y1 = a.y;
    sa.partial = ctx->d_partial;
    sa.x = a.x;
    sa.early_weights = (ex->flags & TP_EXEC_STATIC_WEIGHTS) ? 1 : 0;
    sa.counts = sa.slices > 1 ? nullptr : a.counts;
    sa.owner = sa.slices > 1 ? nullptr : a.owner;
    tp_status ls = launch_stream(ctx, sa, w_down, false, w_down, false, o.stream);
    if (ls != TP_OK) {
      o.abort();
      return ls;
    }
    if (sa.slices > 1) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)((d + kThreads - 1) / kThreads));
      cfg.blockDim = dim3(kThreads);
      cfg.stream = o.stream;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      e = a.counts ? cudaLaunchKernelEx(&cfg, residual_finish_kernel<true>, a.y, (const float*)ctx->d_partial, d,
                                        (int)sa.slices, a.counts, a.owner)
                   : cudaLaunchKernelEx(&cfg, residual_finish_kernel<false>, a.y, (const float*)ctx->d_partial, d,
                                        (int)sa.slices, (uint32_t*)nullptr, (int32_t*)nullptr);
      if (e == cudaSuccess) e = cudaGetLastError();
    }
    return o.end(e);
  }
  // few long rows: split K into 8 slices, one slice per CTA (so 4 CTAs fit
  // per SM); partial sums go to context scratch allocated once, and a
  // finish kernel adds them to h in slice order
  const int parts = 8;
  if (d > 0 && ni > 0) {
    if (d * parts > tp_ctx::kPartialFloats || ni < 8 * parts) e = launch_gemv<kResidual, 4, 4>(a, gemv_grid(ctx, ni), o.stream);
    else {
      const int64_t slice = ((ni / 8 + parts - 1) / parts) * 8 + 8;
      const size_t smem = (size_t)((slice + 3) & ~int64_t(3)) * sizeof(float);
      auto k = gemv_partial_kernel<8>;
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) {
        const int grid = ctx->sm_count * 4;  // a multiple of `parts` on every GB300 SM count used (152)
        k<<<(grid / parts) * parts, kThreads, smem, o.stream>>>(a, parts, ctx->d_partial);
        const unsigned fg = (unsigned)((d + kThreads - 1) / kThreads);
        if (a.counts)
          residual_finish_kernel<true><<<fg, kThreads, 0, o.stream>>>(a.y, ctx->d_partial, d, parts, a.counts, a.owner);
        else
          residual_finish_kernel<false><<<fg, kThreads, 0, o.stream>>>(a.y, ctx->d_partial, d, parts, nullptr, nullptr);
        e = cudaGetLastError();
      }
    }
  }
  return o.end(e);
}

}  // extern "C"
