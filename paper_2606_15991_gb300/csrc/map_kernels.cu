// Element-wise map kernels: one tile program per output tile (plain
// partition, §3.4) or persistent programs walking a bounded sequence of tiles
// (mapped partition, §3.6). The rank-1 path moves 16 bytes per load/store
// (4 fp32 or 8 bf16) with streaming cache hints; other shapes use a scalar
// path over the tile's elements. Each program stores only inside its tile.
#include <cuda_bf16.h>

#include "tile_claim.cuh"
#include "tp_internal.h"

namespace tp {
namespace {

constexpr int kThreads = 256;

struct MapArgs {
  void* out;
  const void* x;
  const void* y;
  float alpha;
  int32_t kind;      // tp_map_kind
  int64_t n;         // elements of the output
  int64_t ntiles;
  int64_t tile;      // rank-1 tile length
  unsigned* queue;   // TP_MAP_QUEUE counter
  uint32_t* counts;  // write-count instrumentation (optional)
  int32_t* owner;
  int64_t shape[3];  // general path, padded to rank 3 (leading 1s)
  int64_t tshape[3];
  int64_t grid[3];
  uint32_t* claims;      // checked launch: tile-claim bitmap (null = release)
  unsigned* claim_done;  // checked launch: finished-CTA counter
  int* err;              // context error word
};

// 2^a by the hardware base-2 exponential (flush-to-zero).
__device__ __forceinline__ float ex2_approx(float a) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}

// gelu_tanh(x) = 0.5 x (1 + tanh(u)), u = sqrt(2/pi) (x + 0.044715 x^3),
// evaluated as x / (1 + exp(-2u)) (0.5 (1 + tanh u) = 1 / (1 + exp(-2u))),
// with exp(-2u) = 2^t, t = -2 log2(e) u = x (c0 + c1 x^2): one polynomial,
// one base-2 exponential, one fast division. t is capped at 125 so 1 + 2^t
// stays below 2^126, the range where the fast division is defined; the
// result there is ~0.
__device__ __forceinline__ float gelu_tanh(float x) {
  const float c0 = -2.f * 1.4426950408889634f * 0.7978845608028654f;  // -2 log2(e) sqrt(2/pi)
  const float c1 = c0 * 0.044715f;
  const float t = fminf(x * fmaf(c1, x * x, c0), 125.f);
  return __fdividef(x, 1.f + ex2_approx(t));
}

template <int OP>
__device__ __forceinline__ float apply(float x, float y, float c, float alpha) {
  if constexpr (OP == kMapAxpy) return fmaf(alpha, x, y);
  else if constexpr (OP == kMapGeluMul) return gelu_tanh(x) * y;
  else if constexpr (OP == kMapScale) return x * y;
  else return c + x + y;  // kMapAddAccum: c <- c + a + b
}

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// Tile -> program schedule of §3.4 / §3.6. Returns the next tile of this
// program or -1 when its sequence is exhausted.
struct Schedule {
  int64_t cur;
  __device__ __forceinline__ int64_t first(const MapArgs& a, int64_t* smem_slot) {
    if (a.kind == TP_MAP_QUEUE) return dequeue(a, smem_slot);
    cur = blockIdx.x;
    return cur < a.ntiles ? cur : -1;
  }
  __device__ __forceinline__ int64_t next(const MapArgs& a, int64_t* smem_slot) {
    if (a.kind == TP_MAP_QUEUE) return dequeue(a, smem_slot);
    if (a.kind == TP_MAP_IDENTITY) return -1;
    cur += gridDim.x;
    return cur < a.ntiles ? cur : -1;
  }
  __device__ __forceinline__ int64_t dequeue(const MapArgs& a, int64_t* smem_slot) {
    __syncthreads();  // everyone has read the previous slot
    if (threadIdx.x == 0) *smem_slot = (int64_t)atomicAdd(a.queue, 1u);
    __syncthreads();
    int64_t t = *smem_slot;
    return t < a.ntiles ? t : -1;
  }
};

template <bool COUNT>
__device__ __forceinline__ void count_write(const MapArgs& a, int64_t i) {
  if constexpr (COUNT) {
    atomicAdd(a.counts + i, 1u);
    a.owner[i] = (int32_t)blockIdx.x;
  }
}

// Checked launch: before storing tile t the program validates it against
// the map (a tile of the grid, and for a strided map one of this program's
// slots) and claims it; a refused claim skips the tile. Block-uniform.
template <bool kCheck = true>
__device__ __forceinline__ bool claim_map_tile(const MapArgs& a, int64_t t) {
  if constexpr (!kCheck) return true;
  if (a.claims == nullptr) return true;
  int won = 0;
  if (threadIdx.x == 0) {
    bool on_map = t >= 0 && t < a.ntiles;
    if (a.kind == TP_MAP_IDENTITY) on_map = on_map && t == (int64_t)blockIdx.x;
    if (a.kind == TP_MAP_STRIDED) on_map = on_map && (t - (int64_t)blockIdx.x) % gridDim.x == 0;
    if (!on_map) record_device_error(a.err, kDevRace);
    won = on_map && claim_tile(a.claims, t, a.err) ? 1 : 0;
  }
  return __syncthreads_or(won) != 0;
}

template <bool kCheck = true>
__device__ __forceinline__ void finish_map_claims(const MapArgs& a) {
  if constexpr (kCheck) {
    if (a.claims != nullptr) claims_finish(a.claims, a.ntiles, a.claim_done, gridDim.x);
  }
}

template <typename T> struct Vec;
template <> struct Vec<float> { using V = float4; static constexpr int N = 4; };
template <> struct Vec<__nv_bfloat16> { using V = uint4; static constexpr int N = 8; };

template <typename T>
__device__ __forceinline__ void unpack(const typename Vec<T>::V& v, float* f) {
  if constexpr (sizeof(T) == 4) {
    f[0] = v.x; f[1] = v.y; f[2] = v.z; f[3] = v.w;
  } else {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float2 t = __bfloat1622float2(h[i]);
      f[2 * i] = t.x;
      f[2 * i + 1] = t.y;
    }
  }
}

template <typename T>
__device__ __forceinline__ typename Vec<T>::V pack(const float* f) {
  typename Vec<T>::V v;
  if constexpr (sizeof(T) == 4) {
    v.x = f[0]; v.y = f[1]; v.z = f[2]; v.w = f[3];
  } else {
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&v);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
  }
  return v;
}

// Rank-1 path: tile length is a multiple of the vector width and all three
// pointers are 16-byte aligned, so every tile starts on a vector boundary.
// Programmatic dependent launch: map launches carry the programmatic
// stream-serialization attribute, so the next launch on the stream may be
// scheduled while this one runs. Each map kernel first waits until the grid
// it depends on has completed and its memory is visible (a no-op when it was
// not launched early), then lets its own dependents be scheduled.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <int OP, typename T, bool COUNT, bool CHECKED>
__global__ void __launch_bounds__(kThreads) map_vec_kernel(const __grid_constant__ MapArgs a) {
  using V = typename Vec<T>::V;
  constexpr int W = Vec<T>::N;
  constexpr int U = 16 / W > 1 ? 16 / W : 1;  // vectors per thread per round: 4 (f32), 2 (bf16)
  __shared__ int64_t slot;
  pdl_enter();
  T* __restrict__ out = static_cast<T*>(a.out);
  const T* __restrict__ x = static_cast<const T*>(a.x);
  const T* __restrict__ y = static_cast<const T*>(a.y);
  Schedule s;
  for (int64_t t = s.first(a, &slot); t >= 0; t = s.next(a, &slot)) {
    if (!claim_map_tile<CHECKED>(a, t)) continue;
    const int64_t start = t * a.tile;
    const int64_t len = min(a.tile, a.n - start);
    const int64_t nv = len / W;
    const V* xv = reinterpret_cast<const V*>(x + start);
    const V* yv = reinterpret_cast<const V*>(y + start);
    V* ov = reinterpret_cast<V*>(out + start);
    int64_t v = threadIdx.x;
    for (; v + (U - 1) * kThreads < nv; v += U * kThreads) {
      V xr[U], yr[U], cr[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        xr[u] = __ldcs(xv + v + u * kThreads);
        yr[u] = __ldcs(yv + v + u * kThreads);
        if constexpr (OP == kMapAddAccum) cr[u] = ov[v + u * kThreads];
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        float fx[W], fy[W], fc[W], fo[W];
        unpack<T>(xr[u], fx);
        unpack<T>(yr[u], fy);
        if constexpr (OP == kMapAddAccum) unpack<T>(cr[u], fc);
#pragma unroll
        for (int i = 0; i < W; ++i) fo[i] = apply<OP>(fx[i], fy[i], OP == kMapAddAccum ? fc[i] : 0.f, a.alpha);
        __stcs(ov + v + u * kThreads, pack<T>(fo));
        if constexpr (COUNT) {
#pragma unroll
          for (int i = 0; i < W; ++i) count_write<COUNT>(a, start + (v + u * kThreads) * W + i);
        }
      }
    }
    for (; v < nv; v += kThreads) {
      float fx[W], fy[W], fc[W], fo[W];
      unpack<T>(__ldcs(xv + v), fx);
      unpack<T>(__ldcs(yv + v), fy);
      if constexpr (OP == kMapAddAccum) unpack<T>(ov[v], fc);
#pragma unroll
      for (int i = 0; i < W; ++i) fo[i] = apply<OP>(fx[i], fy[i], OP == kMapAddAccum ? fc[i] : 0.f, a.alpha);
      __stcs(ov + v, pack<T>(fo));
      if constexpr (COUNT) {
#pragma unroll
        for (int i = 0; i < W; ++i) count_write<COUNT>(a, start + v * W + i);
      }
    }
    // ragged tail of the last tile (fewer than W elements)
    for (int64_t i = nv * W + threadIdx.x; i < len; i += kThreads) {
      const int64_t g = start + i;
      float c = OP == kMapAddAccum ? to_f<T>(out[g]) : 0.f;
      out[g] = from_f<T>(apply<OP>(to_f<T>(x[g]), to_f<T>(y[g]), c, a.alpha));
      count_write<COUNT>(a, g);
    }
  }
  finish_map_claims<CHECKED>(a);
}

// General path: any rank-1..3 partition of a contiguous output, scalar
// accesses, elements of the tile outside the tensor are skipped.
template <int OP, typename T, bool COUNT>
__global__ void __launch_bounds__(kThreads) map_generic_kernel(const __grid_constant__ MapArgs a) {
  __shared__ int64_t slot;
  pdl_enter();
  T* out = static_cast<T*>(a.out);
  const T* x = static_cast<const T*>(a.x);
  const T* y = static_cast<const T*>(a.y);
  const int64_t tile_elems = a.tshape[0] * a.tshape[1] * a.tshape[2];
  Schedule s;
  for (int64_t t = s.first(a, &slot); t >= 0; t = s.next(a, &slot)) {
    if (!claim_map_tile(a, t)) continue;
    const int64_t t2 = t % a.grid[2];
    const int64_t t1 = (t / a.grid[2]) % a.grid[1];
    const int64_t t0 = t / (a.grid[2] * a.grid[1]);
    for (int64_t e = threadIdx.x; e < tile_elems; e += kThreads) {
      const int64_t l2 = e % a.tshape[2];
      const int64_t l1 = (e / a.tshape[2]) % a.tshape[1];
      const int64_t l0 = e / (a.tshape[2] * a.tshape[1]);
      const int64_t g0 = t0 * a.tshape[0] + l0, g1 = t1 * a.tshape[1] + l1, g2 = t2 * a.tshape[2] + l2;
      if (g0 >= a.shape[0] || g1 >= a.shape[1] || g2 >= a.shape[2]) continue;
      const int64_t g = (g0 * a.shape[1] + g1) * a.shape[2] + g2;
      float c = OP == kMapAddAccum ? to_f<T>(out[g]) : 0.f;
      out[g] = from_f<T>(apply<OP>(to_f<T>(x[g]), to_f<T>(y[g]), c, a.alpha));
      count_write<COUNT>(a, g);
    }
  }
  finish_map_claims(a);
}

template <typename K>
cudaError_t launch_pdl(K kernel, const MapArgs& a, int64_t grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, a);
}

template <int OP, typename T>
cudaError_t launch_typed(const MapArgs& a, bool vec, bool count, int64_t grid, cudaStream_t st) {
  const bool checked = a.claims != nullptr;
  if (vec && checked) return count ? launch_pdl(map_vec_kernel<OP, T, true, true>, a, grid, st)
                                   : launch_pdl(map_vec_kernel<OP, T, false, true>, a, grid, st);
  if (vec) return count ? launch_pdl(map_vec_kernel<OP, T, true, false>, a, grid, st)
                        : launch_pdl(map_vec_kernel<OP, T, false, false>, a, grid, st);
  return count ? launch_pdl(map_generic_kernel<OP, T, true>, a, grid, st)
               : launch_pdl(map_generic_kernel<OP, T, false>, a, grid, st);
}

template <typename T>
cudaError_t launch_op(int op, const MapArgs& a, bool vec, bool count, int64_t grid, cudaStream_t st) {
  switch (op) {
    case kMapAxpy: return launch_typed<kMapAxpy, T>(a, vec, count, grid, st);
    case kMapGeluMul: return launch_typed<kMapGeluMul, T>(a, vec, count, grid, st);
    case kMapScale: return launch_typed<kMapScale, T>(a, vec, count, grid, st);
    default: return launch_typed<kMapAddAccum, T>(a, vec, count, grid, st);
  }
}

}  // namespace

tp_status launch_map(tp_ctx* ctx, tp_partition* out, int op, float alpha, const tp_tensor* x,
                     const tp_tensor* y, const tp_exec* ex, cudaStream_t stream, unsigned* queue) {
  MapArgs a{};
  a.out = out->t.ptr;
  a.x = x->ptr;
  a.y = y->ptr;
  a.alpha = alpha;
  a.kind = out->kind;
  a.n = numel(out->t);
  a.ntiles = out->num_tiles;
  a.tile = out->tile[0];
  a.queue = queue;
  a.counts = ex->write_counts;
  a.owner = ex->write_owner;
  if ((a.counts == nullptr) != (a.owner == nullptr))
    return fail(TP_ERR_INVALID, "write_counts and write_owner must be given together");
  if (ex->flags & TP_EXEC_CHECKED) {
    tp_status cs = claims_for(ctx, out->num_tiles, &a.claims, &a.claim_done);
    if (cs != TP_OK) return cs;
    a.err = ctx->d_err;
  }
  const int pad = 3 - out->rank;
  for (int i = 0; i < 3; ++i) {
    a.shape[i] = i < pad ? 1 : out->shape[i - pad];
    a.tshape[i] = i < pad ? 1 : out->tile[i - pad];
    a.grid[i] = i < pad ? 1 : out->grid[i - pad];
  }
  if (a.n == 0 || a.ntiles == 0) return TP_OK;
  const int w = out->t.dtype == TP_F32 ? 4 : 8;
  auto aligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  const bool vec = out->rank == 1 && (a.tile % w) == 0 && aligned(a.out) && aligned(a.x) && aligned(a.y);
  const int64_t grid = out->kind == TP_MAP_IDENTITY ? out->num_tiles : out->num_programs;
  if (grid > 0x7fffffff) return fail(TP_ERR_UNSUPPORTED, "more than 2^31-1 tile programs");
  const bool count = a.counts != nullptr;
  cudaError_t e = out->t.dtype == TP_F32 ? launch_op<float>(op, a, vec, count, grid, stream)
                                         : launch_op<__nv_bfloat16>(op, a, vec, count, grid, stream);
  if (e != cudaSuccess) return cuda_fail(e, "map kernel launch");
  return TP_OK;
}

}  // namespace tp

// ---------------------------------------------------------------------------
// Allocation-free queue-mapped axpy (tp_map_axpy_queue_noalloc).
//
// Its only scratch is the device queue's tile counter. It lives in the static
// device array below, so the entry point needs no context and allocates
// nothing; every GPU that loads this library holds the array until exit.
#include <mutex>

namespace tp {
namespace {

constexpr int64_t kNoallocMaxTiles = int64_t(1) << 31;  // the 32-bit counter never wraps
constexpr int kNoallocMaxDevices = 64;

// One 32-bit tile counter (4 bytes used of a 256-byte-aligned array).
static __device__ __align__(256) unsigned int g_noalloc_tile_queue[1];

// Device address of g_noalloc_tile_queue per device, looked up once per
// device with that device current. In host code the array's name is only a
// host-side stand-in; only this looked-up address may be given to a kernel.
void* g_noalloc_queue_addr[kNoallocMaxDevices] = {};
std::mutex g_noalloc_mu;

// Set-up of a device, on the entry point's first call there: the scratch
// array's device address, and every kernel instance the entry point can
// launch loaded now (with lazy module loading a kernel is otherwise loaded
// at its first launch), so later calls only enqueue work.
tp_status noalloc_queue_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(TP_ERR_UNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_queue_addr[dev]) {
    const void* kernels[4] = {reinterpret_cast<const void*>(map_vec_kernel<kMapAxpy, float, false, false>),
                              reinterpret_cast<const void*>(map_vec_kernel<kMapAxpy, __nv_bfloat16, false, false>),
                              reinterpret_cast<const void*>(map_generic_kernel<kMapAxpy, float, false>),
                              reinterpret_cast<const void*>(map_generic_kernel<kMapAxpy, __nv_bfloat16, false>)};
    for (const void* k : kernels) {
      cudaFuncAttributes fa;
      e = cudaFuncGetAttributes(&fa, k);
      if (e != cudaSuccess) return cuda_fail(e, "loading the queue-mapped axpy kernels");
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_tile_queue);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the tile-queue scratch");
    g_noalloc_queue_addr[dev] = p;
  }
  *out = g_noalloc_queue_addr[dev];
  return TP_OK;
}

}  // namespace
}  // namespace tp

extern "C" tp_status tp_map_axpy_queue_noalloc(void* z, const void* x, const void* y, int32_t dtype, int64_t n,
                                               int64_t tile, int32_t num_programs, float alpha, void* stream) {
  using namespace tp;
  if (dtype != TP_F32 && dtype != TP_BF16) return fail(TP_ERR_UNSUPPORTED, "dtype must be TP_F32 or TP_BF16");
  if (n < 0 || tile < 1) return fail(TP_ERR_INVALID, "need n >= 0 and tile >= 1");
  const int64_t ntiles = (n + tile - 1) / tile;
  if (ntiles > kNoallocMaxTiles)
    return fail(TP_ERR_INVALID, "more than 2^31 tiles: the allocation-free tile queue holds a 32-bit counter");
  if (n == 0) return TP_OK;
  if (!z || !x || !y) return fail(TP_ERR_INVALID, "null pointer");
  if (num_programs < 1 || num_programs > ntiles)
    return fail(TP_ERR_INVALID, "num_programs must be 1..number of tiles");
  const size_t es = dtype_size(dtype);
  const uintptr_t z0 = reinterpret_cast<uintptr_t>(z), z1 = z0 + (uintptr_t)n * es;
  for (const void* in : {x, y}) {
    const uintptr_t i0 = reinterpret_cast<uintptr_t>(in), i1 = i0 + (uintptr_t)n * es;
    if (i0 < z1 && z0 < i1) return fail(TP_ERR_ALIAS, "an input overlaps the output");
  }
  void* queue = nullptr;
  tp_status s = noalloc_queue_address(&queue);
  if (s != TP_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned int), st);  // the queue starts at slot 0
  if (e != cudaSuccess) return cuda_fail(e, "clearing the tile-queue scratch");
  MapArgs a{};
  a.out = z;
  a.x = x;
  a.y = y;
  a.alpha = alpha;
  a.kind = TP_MAP_QUEUE;
  a.n = n;
  a.ntiles = ntiles;
  a.tile = tile;
  a.queue = static_cast<unsigned*>(queue);
  for (int i = 0; i < 3; ++i) {
    a.shape[i] = i < 2 ? 1 : n;
    a.tshape[i] = i < 2 ? 1 : tile;
    a.grid[i] = i < 2 ? 1 : ntiles;
  }
  const int w = dtype == TP_F32 ? 4 : 8;
  auto aligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  const bool vec = (tile % w) == 0 && aligned(z) && aligned(x) && aligned(y);
  e = dtype == TP_F32 ? launch_op<float>(kMapAxpy, a, vec, false, num_programs, st)
                      : launch_op<__nv_bfloat16>(kMapAxpy, a, vec, false, num_programs, st);
  if (e != cudaSuccess) return cuda_fail(e, "map kernel launch");
  return TP_OK;
}
