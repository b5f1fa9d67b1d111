// FP32 GEMM on the CUDA cores (FFMA, FP32 accumulation, no TF32): one 64x64
// C tile per tile program with a K loop (§3.6, Listing 6). Plain partitions
// launch one program per tile; mapped partitions launch persistent programs
// that walk their tiles (strided slots or a device queue), slots being turned
// into tiles by the band raster shared with the tensor-core GEMM.
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

template <int BK, bool COUNT>
__global__ void __launch_bounds__(TH) gemm_f32_kernel(const __grid_constant__ SimtArgs p) {
  __shared__ float As[2][BK][BM + 4];
  __shared__ float Bs[2][BK][BN + 4];
  __shared__ int64_t slot;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t T = p.gm * p.gn;
  int64_t s = blockIdx.x;
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
    const int64_t nk = (p.K + BK - 1) / BK;
    auto load = [&](int buf, int64_t k0) {
      for (int i = tid; i < BM * BK; i += TH) {
        const int r = i / BK, kk = i % BK;
        const int64_t gm_ = m0 + r, gk = k0 + kk;
        As[buf][kk][r] = (gm_ < p.M && gk < p.K) ? p.a[gm_ * p.sam + gk * p.sak] : 0.f;
      }
      for (int i = tid; i < BK * BN; i += TH) {
        const int kk = i / BN, c = i % BN;
        const int64_t gk = k0 + kk, gn_ = n0 + c;
        Bs[buf][kk][c] = (gk < p.K && gn_ < p.N) ? p.b[gk * p.sbk + gn_ * p.sbn] : 0.f;
      }
    };
    if (nk > 0) load(0, 0);
    __syncthreads();
    for (int64_t kt = 0; kt < nk; ++kt) {
      const int buf = kt & 1;
      if (kt + 1 < nk) load(buf ^ 1, (kt + 1) * BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        float av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bv[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t r = m0 + ty + 16 * i;
      if (r >= p.M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t c = n0 + tx + 16 * j;
        if (c < p.N) {
          p.c[r * p.N + c] = acc[i][j];
          if constexpr (COUNT) {
            atomicAdd(p.counts + r * p.N + c, 1u);
            p.owner[r * p.N + c] = (int32_t)blockIdx.x;
          }
        }
      }
    }
    if (p.kind == TP_MAP_IDENTITY) break;
    if (p.kind == TP_MAP_STRIDED) {
      s += gridDim.x;
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
  if (count) gemm_f32_kernel<BK, true><<<(unsigned)grid, TH, 0, st>>>(p);
  else gemm_f32_kernel<BK, false><<<(unsigned)grid, TH, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

tp_status launch_gemm_simt(tp_ctx* ctx, tp_partition* c, const tp_tensor* a, const tp_tensor* b,
                           const tp_gemm_config* cfg, const tp_exec* ex, cudaStream_t stream,
                           unsigned* queue) {
  (void)ctx;
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
  const int bk = (cfg && cfg->bk > 0) ? cfg->bk : 16;
  const bool count = p.counts != nullptr;
  cudaError_t e;
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
