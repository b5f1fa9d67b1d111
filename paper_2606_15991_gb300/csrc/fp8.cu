// Per-tensor-scaled FP8-E4M3 path: amax reduction, quantisation to E4M3 and
// the scaled tensor-core GEMM entry point.
//
//   amax = max |x| over the whole tensor
//   s    = 448 / amax in fp32 (s = 1 for an all-zero tensor)
//   q    = E4M3(satfinite(RN(x * s)))  (the product in fp32)
//   C    = (qA . qB) * 1 / (s_A * s_B), FP32 accumulation, bf16 output
#include <cuda_bf16.h>

#include "tp_internal.h"

namespace tp {
namespace {

constexpr int kThreads = 256;

template <typename T> struct In;
template <> struct In<float> {
  static __device__ __forceinline__ void load16(const float* p, float* f) {
    const float4* v = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float4 t = __ldcs(v + i);
      f[4 * i] = t.x; f[4 * i + 1] = t.y; f[4 * i + 2] = t.z; f[4 * i + 3] = t.w;
    }
  }
};
template <> struct In<__nv_bfloat16> {
  static __device__ __forceinline__ void load16(const __nv_bfloat16* p, float* f) {
    const uint4* v = reinterpret_cast<const uint4*>(p);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      uint4 t = __ldcs(v + i);
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&t);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float2 q = __bfloat1622float2(h[j]);
        f[8 * i + 2 * j] = q.x;
        f[8 * i + 2 * j + 1] = q.y;
      }
    }
  }
};

__device__ __forceinline__ float ld_f(const float* p) { return *p; }
__device__ __forceinline__ float ld_f(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// Non-negative floats order like their bit patterns, so max |x| can be taken
// with an unsigned atomicMax on the bits.
template <typename T>
__global__ void __launch_bounds__(kThreads) amax_kernel(const T* __restrict__ x, int64_t n, bool vec,
                                                        unsigned* out_bits) {
  float m = 0.f;
  const int64_t tid = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * kThreads;
  int64_t done = 0;
  if (vec) {
    const int64_t nv = n / 16;
    for (int64_t v = tid; v < nv; v += nthreads) {
      float f[16];
      In<T>::load16(x + v * 16, f);
#pragma unroll
      for (int i = 0; i < 16; ++i) m = fmaxf(m, fabsf(f[i]));
    }
    done = nv * 16;
  }
  for (int64_t i = done + tid; i < n; i += nthreads) m = fmaxf(m, fabsf(ld_f(x + i)));
  unsigned b = __float_as_uint(m);
  b = __reduce_max_sync(0xffffffffu, b);
  if ((threadIdx.x & 31) == 0 && b != 0) atomicMax(out_bits, b);
}

// Two E4M3 codes from two fp32 values, round to nearest even with
// saturation to +-448; `lo` lands in the low byte.
__device__ __forceinline__ uint16_t cvt_e4m3x2(float lo, float hi) {
  uint16_t r;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ float scale_from_amax(const float* amax) {
  const float a = *amax;
  return a > 0.f ? 448.f / a : 1.f;
}

struct QuantArgs {
  const void* x;
  uint8_t* q;
  int64_t n;
  int64_t tile;      // elements per tile (contiguous)
  int64_t ntiles;
  int32_t kind;      // identity or strided
  const float* amax;
  float* scale;
  uint32_t* counts;
  int32_t* owner;
};

template <typename T, bool kCount>
__global__ void __launch_bounds__(kThreads) quantize_kernel(const __grid_constant__ QuantArgs a) {
  const float s = scale_from_amax(a.amax);
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.scale = s;
  const T* x = static_cast<const T*>(a.x);
  const bool vec = (a.tile % 16) == 0 && ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(a.q)) & 15) == 0;
  const int64_t step = a.kind == TP_MAP_IDENTITY ? a.ntiles : (int64_t)gridDim.x;
  for (int64_t t = blockIdx.x; t < a.ntiles; t += step) {
    const int64_t start = t * a.tile;
    const int64_t len = min(a.tile, a.n - start);
    int64_t done = 0;
    if (vec) {
      const int64_t nv = len / 16;
      for (int64_t v = threadIdx.x; v < nv; v += kThreads) {
        float f[16];
        In<T>::load16(x + start + v * 16, f);
        uint4 out;
        uint16_t* h = reinterpret_cast<uint16_t*>(&out);
#pragma unroll
        for (int i = 0; i < 8; ++i) h[i] = cvt_e4m3x2(f[2 * i] * s, f[2 * i + 1] * s);
        *reinterpret_cast<uint4*>(a.q + start + v * 16) = out;
        if constexpr (kCount) {
          for (int i = 0; i < 16; ++i) {
            atomicAdd(a.counts + start + v * 16 + i, 1u);
            a.owner[start + v * 16 + i] = (int32_t)blockIdx.x;
          }
        }
      }
      done = nv * 16;
    }
    for (int64_t i = done + threadIdx.x; i < len; i += kThreads) {
      const int64_t g = start + i;
      a.q[g] = (uint8_t)(cvt_e4m3x2(ld_f(x + g) * s, 0.f) & 0xFF);
      if constexpr (kCount) {
        atomicAdd(a.counts + g, 1u);
        a.owner[g] = (int32_t)blockIdx.x;
      }
    }
  }
}

}  // namespace
}  // namespace tp

using namespace tp;

extern "C" {

tp_status tp_amax(tp_ctx* ctx, const tp_tensor* x, float* amax, const tp_exec* ex) {
  if (!ctx || !x || !amax || !ex) return fail(TP_ERR_INVALID, "null argument");
  if (x->dtype != TP_F32 && x->dtype != TP_BF16) return fail(TP_ERR_UNSUPPORTED, "amax supports F32 and BF16");
  if (!is_contiguous(*x)) return fail(TP_ERR_UNSUPPORTED, "amax input must be contiguous");
  Op o(__func__);
  tp_status s = o.begin(ctx, ex, {}, {x});
  if (s != TP_OK) return s;
  cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(float), o.stream);
  if (e != cudaSuccess) {
    o.abort();
    return cuda_fail(e, "clearing amax");
  }
  const int64_t n = numel(*x);
  if (n > 0) {
    const bool vec = (reinterpret_cast<uintptr_t>(x->ptr) & 15) == 0;
    const int grid = ctx->sm_count * 4;
    unsigned* bits = reinterpret_cast<unsigned*>(amax);
    if (x->dtype == TP_F32)
      amax_kernel<float><<<grid, kThreads, 0, o.stream>>>(static_cast<const float*>(x->ptr), n, vec, bits);
    else
      amax_kernel<__nv_bfloat16><<<grid, kThreads, 0, o.stream>>>(static_cast<const __nv_bfloat16*>(x->ptr), n,
                                                                   vec, bits);
  }
  return o.end(cudaGetLastError());
}

tp_status tp_quantize_fp8(tp_ctx* ctx, tp_partition* q, const tp_tensor* x, const float* amax, float* scale,
                          const tp_exec* ex) {
  if (!ctx || !q || !x || !amax || !scale || !ex) return fail(TP_ERR_INVALID, "null argument");
  if (x->dtype != TP_F32 && x->dtype != TP_BF16) return fail(TP_ERR_UNSUPPORTED, "quantize input must be F32 or BF16");
  if (q->t.dtype != TP_F8E4M3 && q->t.dtype != TP_U8) return fail(TP_ERR_SHAPE, "quantize output must be F8E4M3");
  if (x->rank != q->rank) return fail(TP_ERR_SHAPE, "input rank differs from output rank");
  for (int i = 0; i < q->rank; ++i)
    if (x->shape[i] != q->shape[i]) return fail(TP_ERR_SHAPE, "input shape differs from output shape");
  if (!is_contiguous(*x)) return fail(TP_ERR_UNSUPPORTED, "quantize input must be contiguous");
  // each tile must be one contiguous run of elements: full rows beyond axis 0
  int64_t tile = q->tile[0];
  for (int i = 1; i < q->rank; ++i) {
    if (q->tile[i] != q->shape[i]) return fail(TP_ERR_UNSUPPORTED, "quantize tiles must span whole rows");
    tile *= q->shape[i];
  }
  if (q->kind == TP_MAP_QUEUE) return fail(TP_ERR_UNSUPPORTED, "quantize maps tiles by slot (identity/strided)");
  if ((ex->write_counts == nullptr) != (ex->write_owner == nullptr))
    return fail(TP_ERR_INVALID, "write_counts and write_owner must be given together");
  Op o(__func__);
  tp_status s = o.begin(ctx, ex, {q}, {x});
  if (s != TP_OK) return s;
  QuantArgs a{};
  a.x = x->ptr;
  a.q = static_cast<uint8_t*>(q->t.ptr);
  a.n = numel(*x);
  a.tile = tile;
  a.ntiles = q->num_tiles;
  a.kind = q->kind;
  a.amax = amax;
  a.scale = scale;
  a.counts = ex->write_counts;
  a.owner = ex->write_owner;
  const int64_t grid = q->kind == TP_MAP_IDENTITY ? q->num_tiles : q->num_programs;
  if (grid > 0x7fffffff) {
    o.abort();
    return fail(TP_ERR_UNSUPPORTED, "too many tile programs");
  }
  if (a.n > 0) {
    const bool count = a.counts != nullptr;
    if (x->dtype == TP_F32) {
      if (count) quantize_kernel<float, true><<<(unsigned)grid, kThreads, 0, o.stream>>>(a);
      else quantize_kernel<float, false><<<(unsigned)grid, kThreads, 0, o.stream>>>(a);
    } else {
      if (count) quantize_kernel<__nv_bfloat16, true><<<(unsigned)grid, kThreads, 0, o.stream>>>(a);
      else quantize_kernel<__nv_bfloat16, false><<<(unsigned)grid, kThreads, 0, o.stream>>>(a);
    }
  }
  return o.end(cudaGetLastError());
}

tp_status tp_gemm_fp8(tp_ctx* ctx, tp_partition* c, const tp_tensor* qa, const tp_tensor* qb,
                      const float* scale_a, const float* scale_b, const tp_gemm_config* cfg, const tp_exec* ex) {
  if (!ctx || !c || !qa || !qb || !scale_a || !scale_b || !ex) return fail(TP_ERR_INVALID, "null argument");
  if (qa->rank != 2 || qb->rank != 2 || c->rank != 2) return fail(TP_ERR_RANK, "GEMM operands are rank 2");
  const int64_t M = qa->shape[0], K = qa->shape[1], N = qb->shape[1];
  if (qb->shape[0] != K || c->shape[0] != M || c->shape[1] != N)
    return fail(TP_ERR_SHAPE, "need A: M x K, B: K x N, C: M x N");
  auto f8 = [](int32_t d) { return d == TP_F8E4M3 || d == TP_U8; };
  if (!f8(qa->dtype) || !f8(qb->dtype) || c->t.dtype != TP_BF16)
    return fail(TP_ERR_UNSUPPORTED, "tp_gemm_fp8 takes E4M3 A and B and a BF16 C");
  Op o(__func__);
  o.allow_checked = true;
  tp_status s = o.begin(ctx, ex, {c}, {qa, qb});
  if (s != TP_OK) return s;
  o.check_err = true;
  s = launch_gemm_tc_impl(ctx, c, qa, qb, cfg, ex, o.stream, 1, scale_a, scale_b);
  if (s != TP_OK) {
    o.abort();
    return s;
  }
  return o.end(cudaGetLastError());
}

}  // extern "C"
