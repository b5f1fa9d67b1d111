// Head permutation of §3.5 (Listing 5): dst[b, m, h, :] = src[b, h, m, :] in
// units of (BM x D) tiles, i.e. the (head, sequence-tile) transpose of a
// (B, H, M, D) tensor with M / BM == H.
//
// tp_permute_heads is the partitioned form: dst, viewed as (B*H, M, D), is
// partitioned into (1, BM, D) tiles and each tile program stores only its own
// tile, loading the source tile it needs; no destination index is chosen by
// the program, so the race below cannot be written (§3.5).
//
// tp_permute_heads_unchecked is the raw-pointer escape hatch (§3.6 "escape
// hatches") with the grid of Listing 5, (B*H, H, 1): program (bh1, h2) with
// b = bh1 / H, h1 = bh1 % H walks m and stores the source tile (b, h1, m) at
// destination tile (b, m, h2 if swap_bug else h1). With swap_bug the H
// programs that differ in h1 store to the same tile: a data race, which the
// write-count instrumentation reports deterministically (H writes per
// element). The racing stores are plain aligned word stores: the GPU does not
// fault, only the surviving values are unordered. Its checked launch
// (TP_EXEC_CHECKED) claims each destination tile before storing it: the first
// claimer stores, every later one is refused and the op reports TP_ERR_RACE.
#include <cuda_bf16.h>

#include "tile_claim.cuh"
#include "tp_internal.h"

namespace tp {
namespace {

constexpr int kThreads = 256;

template <bool kCount>
__global__ void permute_safe_kernel(float* __restrict__ dst, const float* __restrict__ src, int64_t B, int64_t H,
                                    int64_t M, int64_t D, int64_t BM, uint32_t* counts, int32_t* owner) {
  // program = dst tile (b*H + i, j): rows [j*BM, (j+1)*BM) of dst[b, i]
  const int64_t tiles_m = M / BM;
  const int64_t t = blockIdx.x;
  const int64_t bi = t / tiles_m, j = t % tiles_m;
  const int64_t b = bi / H, i = bi % H;
  // dst tile (b, i, j) holds src tile (b, j, i): head j, sequence tile i
  const float* s = src + ((b * H + j) * M + i * BM) * D;
  float* d = dst + ((b * H + i) * M + j * BM) * D;
  for (int64_t e = threadIdx.x; e < BM * D; e += kThreads) {
    d[e] = s[e];
    if constexpr (kCount) {
      const int64_t g = ((b * H + i) * M + j * BM) * D + e;
      atomicAdd(counts + g, 1u);
      owner[g] = (int32_t)t;
    }
  }
}

template <bool kCount, bool kChecked>
__global__ void permute_raw_kernel(float* dst, const float* __restrict__ src, int64_t B, int64_t H, int64_t M,
                                   int64_t D, int64_t BM, int swap_bug, uint32_t* counts, int32_t* owner,
                                   uint32_t* claims, unsigned* claim_done, int* err) {
  const int64_t bh1 = blockIdx.x, h2 = blockIdx.y;
  const int64_t b = bh1 / H, h1 = bh1 % H;
  const int64_t hd = swap_bug ? h2 : h1;
  // the corrected kernel needs one program per (b, h1): the others store nothing
  const bool active = swap_bug || h2 == 0;
  for (int64_t m = 0; active && m < M / BM; ++m) {
    const float* s = src + ((b * H + h1) * M + m * BM) * D;
    const int64_t base = ((b * H + m) * M + hd * BM) * D;  // destination tile (b, m, hd)
    if constexpr (kChecked) {
      // one claim per destination tile; the block agrees on the outcome
      const int won = threadIdx.x == 0 ? (claim_tile(claims, (b * H + m) * H + hd, err) ? 1 : 0) : 0;
      if (!__syncthreads_or(won)) continue;
    }
    for (int64_t e = threadIdx.x; e < BM * D; e += kThreads) {
      dst[base + e] = s[e];
      if constexpr (kCount) {
        atomicAdd(counts + base + e, 1u);
        owner[base + e] = (int32_t)(bh1 * gridDim.y + h2);
      }
    }
  }
  if constexpr (kChecked) claims_finish(claims, B * H * H, claim_done, gridDim.x * gridDim.y);
}

tp_status check_shape(int64_t B, int64_t H, int64_t M, int64_t D, int64_t BM) {
  if (B < 1 || H < 1 || M < 1 || D < 1 || BM < 1 || M % BM || M / BM != H)
    return fail(TP_ERR_SHAPE, "need M divisible by BM and M / BM == H (the swapped store stays in bounds)");
  if (H > 65535 || B * H * H > INT32_MAX) return fail(TP_ERR_SHAPE, "grid too large");
  return TP_OK;
}

}  // namespace
}  // namespace tp

using namespace tp;

extern "C" {

tp_status tp_permute_heads(tp_ctx* ctx, tp_partition* dst, const tp_tensor* src, int64_t H, const tp_exec* ex) {
  if (!ctx || !dst || !src || !ex) return fail(TP_ERR_INVALID, "null argument");
  if (dst->t.dtype != TP_F32 || src->dtype != TP_F32 || src->rank != 4 || dst->rank != 3)
    return fail(TP_ERR_SHAPE, "src: F32 (B, H, M, D); dst: F32 (B*H, M, D) partition");
  const int64_t B = src->shape[0], M = src->shape[2], D = src->shape[3];
  if (src->shape[1] != H || dst->shape[0] != B * H || dst->shape[1] != M || dst->shape[2] != D)
    return fail(TP_ERR_SHAPE, "dst must be src viewed as (B*H, M, D)");
  if (dst->tile[0] != 1 || dst->tile[2] != D) return fail(TP_ERR_SHAPE, "dst tiles are (1, BM, D)");
  const int64_t BM = dst->tile[1];
  tp_status s = check_shape(B, H, M, D, BM);
  if (s != TP_OK) return s;
  if (!is_contiguous(*src)) return fail(TP_ERR_UNSUPPORTED, "src must be contiguous");
  if (dst->kind != TP_MAP_IDENTITY) return fail(TP_ERR_UNSUPPORTED, "plain partition only");
  if ((ex->write_counts == nullptr) != (ex->write_owner == nullptr))
    return fail(TP_ERR_INVALID, "write_counts and write_owner must be given together");
  Op o(__func__);
  s = o.begin(ctx, ex, {dst}, {src});
  if (s != TP_OK) return s;
  float* d = static_cast<float*>(dst->t.ptr);
  const float* sp = static_cast<const float*>(src->ptr);
  const unsigned grid = (unsigned)dst->num_tiles;
  if (ex->write_counts)
    permute_safe_kernel<true><<<grid, kThreads, 0, o.stream>>>(d, sp, B, H, M, D, BM, ex->write_counts, ex->write_owner);
  else
    permute_safe_kernel<false><<<grid, kThreads, 0, o.stream>>>(d, sp, B, H, M, D, BM, nullptr, nullptr);
  return o.end(cudaGetLastError());
}

tp_status tp_permute_heads_unchecked(tp_ctx* ctx, void* dst, const void* src, int64_t B, int64_t H, int64_t M,
                                     int64_t D, int64_t BM, int32_t swap_bug, const tp_exec* ex) {
  if (!ctx || !dst || !src || !ex) return fail(TP_ERR_INVALID, "null argument");
  tp_status s = check_shape(B, H, M, D, BM);
  if (s != TP_OK) return s;
  if ((ex->write_counts == nullptr) != (ex->write_owner == nullptr))
    return fail(TP_ERR_INVALID, "write_counts and write_owner must be given together");
  const uintptr_t d0 = reinterpret_cast<uintptr_t>(dst), s0 = reinterpret_cast<uintptr_t>(src);
  const uintptr_t bytes = (uintptr_t)(B * H * M * D) * 4;
  if (d0 < s0 + bytes && s0 < d0 + bytes) return fail(TP_ERR_ALIAS, "src overlaps dst");
  // raw pointers: no partition is held, so the op tracks no busy state
  Op o(__func__);
  o.allow_checked = true;
  s = o.begin(ctx, ex, {}, {});
  if (s != TP_OK) return s;
  const bool checked = (ex->flags & TP_EXEC_CHECKED) != 0;
  uint32_t* claims = nullptr;
  unsigned* done = nullptr;
  if (checked) {
    s = claims_for(ctx, B * H * H, &claims, &done);
    if (s != TP_OK) {
      o.abort();
      return s;
    }
    o.check_err = true;
  }
  dim3 grid((unsigned)(B * H), (unsigned)H, 1);
  float* d = static_cast<float*>(dst);
  const float* sp = static_cast<const float*>(src);
  uint32_t* wc = ex->write_counts;
  int32_t* wo = ex->write_owner;
  if (wc && checked)
    permute_raw_kernel<true, true><<<grid, kThreads, 0, o.stream>>>(d, sp, B, H, M, D, BM, swap_bug, wc, wo, claims,
                                                                     done, ctx->d_err);
  else if (wc)
    permute_raw_kernel<true, false><<<grid, kThreads, 0, o.stream>>>(d, sp, B, H, M, D, BM, swap_bug, wc, wo, nullptr,
                                                                      nullptr, nullptr);
  else if (checked)
    permute_raw_kernel<false, true><<<grid, kThreads, 0, o.stream>>>(d, sp, B, H, M, D, BM, swap_bug, nullptr,
                                                                      nullptr, claims, done, ctx->d_err);
  else
    permute_raw_kernel<false, false><<<grid, kThreads, 0, o.stream>>>(d, sp, B, H, M, D, BM, swap_bug, nullptr,
                                                                       nullptr, nullptr, nullptr, nullptr);
  return o.end(cudaGetLastError());
}

}  // extern "C"
