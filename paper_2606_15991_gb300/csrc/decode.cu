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
#include <cuda_bf16.h>

#include <algorithm>

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
  if (d > 0 && nq + ni > 0) e = launch_gemv<kPlain, 1, 4>(a, gemv_grid(ctx, d), o.stream);
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
