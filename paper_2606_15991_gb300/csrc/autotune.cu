// Exhaustive autotuner for the tensor-core GEMM (§5.1 tunes tile shapes once
// per size; here the search is automatic). The config space enumerates tile
// rows (64 or 128 on one CTA, 256 on a CTA pair), tile columns, K blocks per
// ring stage and raster band height; each config is timed with CUDA events on a device
// workspace of the requested shape and the fastest wins (ties within 1% go to
// the earlier, smaller config). Results are cached per (M, N, K, dtype,
// search flags) and can be saved to / loaded from a versioned text file.
//
// Numerics classes. Every config without split-K computes each C element as
// one accumulation over K, in K order, by the one program that owns its
// tile, so all of them give bit-identical C: choosing among them is a pure
// performance decision (§5.1 tunes only the tile shape). A split-K config
// adds S slice partials in slice order: reproducible, but rounded
// differently. The default search is therefore the single-pass class only;
// split-K configs are timed only when the caller opts in (TP_TUNE_SPLIT_K).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "tp_internal.h"

namespace tp {
namespace {

struct TuneKey {
  int64_t m, n, k;
  int32_t dtype;
  int32_t flags;  // TP_TUNE_* bits of the search that produced the entry
  bool operator<(const TuneKey& o) const {
    return std::tie(m, n, k, dtype, flags) < std::tie(o.m, o.n, o.k, o.dtype, o.flags);
  }
};

struct TuneState {
  std::mutex mu;
  std::map<TuneKey, std::pair<tp_gemm_config, float>> cache;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t stream = nullptr;
};

constexpr int32_t kTuneFlags = TP_TUNE_SPLIT_K | TP_TUNE_SWAP_AB;

std::mutex g_states_mu;
std::map<tp_ctx*, TuneState*> g_states;

TuneState* state(tp_ctx* ctx) {
  std::lock_guard<std::mutex> lk(g_states_mu);
  auto& s = g_states[ctx];
  if (!s) s = new TuneState();
  return s;
}

// The single-pass configs (one numerics class), then, with TP_TUNE_SWAP_AB,
// swap-AB tiles of W x 128 on CTA pairs (the same class: every C element is
// accumulated in the same K order), then, with TP_TUNE_SPLIT_K, the split-K
// configs. K per stage is 1, 2 or 4 K blocks of 128 bytes (64 bf16 / 128 fp8
// elements), the deepest ring that fits.
std::vector<tp_gemm_config> space(int32_t dtype, int32_t flags) {
  std::vector<tp_gemm_config> v;
  const int kblk = dtype == TP_F8E4M3 ? 128 : 64;
  for (int bm : {64, 128, 256})
    for (int bn : {64, 128, 192, 256})
      for (int kb : {1, 2, 4})
        for (int gm : {1, 8}) {
          tp_gemm_config c{};
          c.bm = bm;
          c.bn = bn;
          c.bk = kb * kblk;
          c.group_m = gm;
          v.push_back(c);
        }
  // swap-AB (BF16, short M): C tiles of W rows x 128 columns, stages of 2 or
  // 4 K blocks (one block per stage streams B at two thirds of the rate)
  if (flags & TP_TUNE_SWAP_AB)
    for (int w : {32, 64, 128})
      for (int kb : {2, 4}) {
        tp_gemm_config c{};
        c.bm = w;
        c.bn = 128;
        c.bk = kb * kblk;
        c.group_m = 1;
        c.swap_ab = 1;
        v.push_back(c);
      }
  if (!(flags & TP_TUNE_SPLIT_K)) return v;
  // split-K programs (128-row tiles; a cluster of split_k CTAs per tile) for
  // shapes with fewer tiles than SMs
  for (int bn : {128, 256})
    for (int sk : {2, 4, 8}) {
      if (bn % (32 * sk)) continue;
      tp_gemm_config c{};
      c.bm = 128;
      c.bn = bn;
      c.group_m = 1;
      c.split_k = sk;
      v.push_back(c);
    }
  return v;
}

}  // namespace

// Whether config c of the space is tried on an M x N x K problem: swap-AB
// tiles serve BF16 problems that one row of tiles covers (M <= W, so B is
// read once); a split program holds one tile and needs at least split_k K
// blocks, and past two waves of clusters it cannot win.
bool autotune_config_runs(const tp_ctx* ctx, int64_t M, int64_t N, int64_t K, int32_t dtype,
                          const tp_gemm_config& c) {
  if (c.swap_ab) return dtype == TP_BF16 && M <= c.bm;
  if (c.split_k <= 1) return true;
  const int64_t tiles = ((M + c.bm - 1) / c.bm) * ((N + c.bn - 1) / c.bn);
  const int64_t kblk = dtype == TP_F8E4M3 ? 128 : 64;
  return (K + kblk - 1) / kblk >= c.split_k && tiles * c.split_k <= 2 * (int64_t)ctx->sm_count;
}

namespace {

// Fills a workspace with finite values that exercise the tensor cores the
// way real data does (a hash of the index, small magnitudes).
__global__ void fill_kernel(uint16_t* p, int64_t n16, int fp8) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)(i * 2654435761u) ^ (uint32_t)(i >> 13);
    h ^= h >> 15;
    h *= 0x2c1b3c6du;
    h ^= h >> 12;
    if (fp8) p[i] = (uint16_t)(h & 0x3737);         // two E4M3 codes of magnitude < 2
    else p[i] = (uint16_t)(0x3c00 | (h & 0x807f));  // bf16, magnitude in [2^-7, 2^-6)
  }
}

// Holds the stream for `ns` nanoseconds (bounded by the wall clock) so the
// host can queue every timed launch before the first one starts: the events
// then bracket back-to-back device execution, not host launch overhead.
__global__ void delay_kernel(uint64_t ns) {
  uint64_t t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  do {
    __nanosleep(1000);
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  } while (t - t0 < ns);
}

tp_status ensure_ws(tp_ctx* ctx, TuneState* st, size_t bytes) {
  if (st->ws_bytes >= bytes) return TP_OK;
  if (st->ws) cudaFree(st->ws);
  st->ws = nullptr;
  st->ws_bytes = 0;
  cudaError_t e = cudaMalloc(&st->ws, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "autotune workspace");
  st->ws_bytes = bytes;
  fill_kernel<<<ctx->sm_count * 8, 256, 0, st->stream>>>(static_cast<uint16_t*>(st->ws), (int64_t)(bytes / 2), 0);
  e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(e, "autotune workspace fill");
  return TP_OK;
}

}  // namespace
}  // namespace tp

namespace tp {
namespace {

// The autotuner's problem of one shape: A (M x K, row-major) and B (stored
// N x K, viewed as K x N) in the context's workspace, C behind them; FP8
// scales of 1 in the context's scratch.
struct TuneProblem {
  int64_t M = 0, N = 0, K = 0;
  int esize = 2;
  tp_tensor a{}, b{};
  void* c = nullptr;
  float* one = nullptr;
  tp_exec ex{};
};

tp_status prepare(tp_ctx* ctx, TuneState* st, int64_t M, int64_t N, int64_t K, int32_t dtype, TuneProblem* pb) {
  if (!st->stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&st->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "autotune stream");
  }
  pb->M = M;
  pb->N = N;
  pb->K = K;
  pb->esize = dtype == TP_BF16 ? 2 : 1;
  const int esize = pb->esize;
  auto align = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t ab = align((size_t)M * K * esize), bb = align((size_t)N * K * esize), cb = align((size_t)M * N * 2);
  tp_status s = ensure_ws(ctx, st, ab + bb + cb);
  if (s != TP_OK) return s;
  char* ws = static_cast<char*>(st->ws);
  pb->a.ptr = ws;
  pb->a.dtype = dtype;
  pb->a.rank = 2;
  pb->a.shape[0] = M;
  pb->a.shape[1] = K;
  pb->a.strides[0] = K;
  pb->a.strides[1] = 1;
  pb->b.ptr = ws + ab;  // stored N x K, viewed as K x N
  pb->b.dtype = dtype;
  pb->b.rank = 2;
  pb->b.shape[0] = K;
  pb->b.shape[1] = N;
  pb->b.strides[0] = 1;
  pb->b.strides[1] = K;
  pb->c = ws + ab + bb;
  pb->ex = tp_exec{};
  pb->ex.stream = st->stream;
  pb->one = nullptr;
  if (dtype == TP_F8E4M3) {
    const float ones[2] = {1.f, 1.f};
    cudaError_t e = cudaMemcpy(ctx->d_scratch, ones, sizeof(ones), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "fp8 unit scales");
    pb->one = ctx->d_scratch;
  }
  return TP_OK;
}

// Launches per timing: enough that the timed span is well above the event
// resolution.
int default_reps(int64_t M, int64_t N, int64_t K) {
  const double est_us = 2.0 * (double)M * (double)N * (double)K / 1.0e9;  // at 1 PFLOP/s
  return est_us > 2000 ? 2 : est_us > 200 ? 4 : 10;
}

// One timing of config c: `r` back-to-back launches queued behind a delay
// kernel and bracketed by CUDA events. *tf = TFLOP/s, 0 when the config
// cannot run on the shape (the returned status says why) or did not run.
tp_status time_config(tp_ctx* ctx, TuneState* st, const TuneProblem& pb, const tp_gemm_config& c, int r,
                      cudaEvent_t e0, cudaEvent_t e1, float* tf) {
  *tf = 0.f;
  tp_partition part{};
  part.ctx = ctx;
  part.t.ptr = pb.c;
  part.t.dtype = TP_BF16;
  part.t.rank = 2;
  part.t.shape[0] = pb.M;
  part.t.shape[1] = pb.N;
  part.t.strides[0] = pb.N;
  part.t.strides[1] = 1;
  part.rank = 2;
  part.shape[0] = pb.M;
  part.shape[1] = pb.N;
  part.tile[0] = c.bm;
  part.tile[1] = c.bn;
  part.grid[0] = (pb.M + c.bm - 1) / c.bm;
  part.grid[1] = (pb.N + c.bn - 1) / c.bn;
  part.num_tiles = part.grid[0] * part.grid[1];
  const int64_t cap = (c.bm == 256 || c.swap_ab) ? ctx->sm_count / 2 : ctx->sm_count;  // CTA pairs, or CTAs
  part.kind = TP_MAP_STRIDED;
  part.num_programs = std::min<int64_t>(part.num_tiles, cap);
  if (c.num_programs > 0) part.num_programs = std::min<int64_t>(part.num_tiles, c.num_programs);
  if (c.split_k > 1) part.num_programs = part.num_tiles;  // a split program holds one tile
  tp_status ls = launch_gemm_tc_impl(ctx, &part, &pb.a, &pb.b, &c, &pb.ex, st->stream, pb.esize, pb.one, pb.one);
  if (ls != TP_OK) return ls;
  delay_kernel<<<1, 32, 0, st->stream>>>(20000ull + 30000ull * (uint64_t)r);
  cudaEventRecord(e0, st->stream);
  for (int j = 0; j < r && ls == TP_OK; ++j)
    ls = launch_gemm_tc_impl(ctx, &part, &pb.a, &pb.b, &c, &pb.ex, st->stream, pb.esize, pb.one, pb.one);
  cudaEventRecord(e1, st->stream);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  if (ls == TP_OK && ms > 0.f) *tf = (float)(2.0 * (double)pb.M * (double)pb.N * (double)pb.K * r / (ms * 1e-3) / 1e12);
  return ls;
}

tp_status check_args(tp_ctx* ctx, int64_t M, int64_t N, int64_t K, int32_t dtype, int32_t flags) {
  if (!ctx) return fail(TP_ERR_INVALID, "null context");
  if (dtype != TP_BF16 && dtype != TP_F8E4M3) return fail(TP_ERR_UNSUPPORTED, "dtype must be BF16 or F8E4M3");
  if (flags & ~kTuneFlags) return fail(TP_ERR_INVALID, "undefined TP_TUNE_* flag bits");
  const int esize = dtype == TP_BF16 ? 2 : 1;
  if (M < 1 || N < 1 || K < 1 || (K * esize) % 16) return fail(TP_ERR_SHAPE, "need M, N, K >= 1 and K*esize % 16 == 0");
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->capturing) return fail(TP_ERR_CAPTURE, "autotuning allocates and synchronises: not during capture");
  return TP_OK;
}

}  // namespace
}  // namespace tp

using namespace tp;

extern "C" {

tp_status tp_autotune_space(int32_t dtype, int32_t flags, tp_gemm_config* out, int32_t cap, int32_t* count) {
  if (!count) return fail(TP_ERR_INVALID, "null count");
  if (dtype != TP_BF16 && dtype != TP_F8E4M3) return fail(TP_ERR_UNSUPPORTED, "dtype must be BF16 or F8E4M3");
  if (flags & ~kTuneFlags) return fail(TP_ERR_INVALID, "undefined TP_TUNE_* flag bits");
  auto v = space(dtype, flags);
  *count = (int32_t)v.size();
  if (out)
    for (int i = 0; i < (int)v.size() && i < cap; ++i) out[i] = v[i];
  return TP_OK;
}

tp_status tp_autotune(tp_ctx* ctx, int64_t M, int64_t N, int64_t K, int32_t dtype, int32_t reps, int32_t flags,
                      tp_gemm_config* best, float* tflops_per_config, float* best_tflops) {
  tp_status s = check_args(ctx, M, N, K, dtype, flags);
  if (s != TP_OK) return s;
  DeviceGuard guard(ctx);
  TuneState* st = state(ctx);
  std::lock_guard<std::mutex> lk(st->mu);
  TuneProblem pb;
  s = prepare(ctx, st, M, N, K, dtype, &pb);
  if (s != TP_OK) return s;
  auto cfgs = space(dtype, flags);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int r = reps > 0 ? reps : default_reps(M, N, K);
  int best_i = -1;
  float best_tf = 0.f;
  for (size_t i = 0; i < cfgs.size(); ++i) {
    float tf = 0.f;
    if (autotune_config_runs(ctx, M, N, K, dtype, cfgs[i])) {
      s = time_config(ctx, st, pb, cfgs[i], r, e0, e1, &tf);
      if (s == TP_ERR_CUDA) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return s;
      }
    }
    if (tflops_per_config) tflops_per_config[i] = tf;
    if (tf > best_tf * 1.01f) {
      best_tf = tf;
      best_i = (int)i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  tp_status es = read_device_error(ctx);
  if (es != TP_OK) return es;
  if (best_i < 0) return fail(TP_ERR_CUDA, "no configuration ran");
  st->cache[TuneKey{M, N, K, dtype, flags}] = {cfgs[best_i], best_tf};
  if (best) *best = cfgs[best_i];
  if (best_tflops) *best_tflops = best_tf;
  return TP_OK;
}

tp_status tp_autotune_time(tp_ctx* ctx, int64_t M, int64_t N, int64_t K, int32_t dtype, const tp_gemm_config* cfg,
                           int32_t reps, int32_t repeats, float* tflops_median) {
  if (!cfg || !tflops_median) return fail(TP_ERR_INVALID, "null argument");
  if (repeats < 1 || repeats > 64) return fail(TP_ERR_INVALID, "repeats must be 1..64");
  tp_status s = check_args(ctx, M, N, K, dtype, 0);
  if (s != TP_OK) return s;
  DeviceGuard guard(ctx);
  TuneState* st = state(ctx);
  std::lock_guard<std::mutex> lk(st->mu);
  TuneProblem pb;
  s = prepare(ctx, st, M, N, K, dtype, &pb);
  if (s != TP_OK) return s;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int r = reps > 0 ? reps : default_reps(M, N, K);
  std::vector<float> tf(repeats, 0.f);
  for (int i = 0; i < repeats && s == TP_OK; ++i) s = time_config(ctx, st, pb, *cfg, r, e0, e1, &tf[i]);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != TP_OK) return s;
  tp_status es = read_device_error(ctx);
  if (es != TP_OK) return es;
  std::sort(tf.begin(), tf.end());
  *tflops_median = repeats % 2 ? tf[repeats / 2] : 0.5f * (tf[repeats / 2 - 1] + tf[repeats / 2]);
  return TP_OK;
}

tp_status tp_autotune_lookup(tp_ctx* ctx, int64_t M, int64_t N, int64_t K, int32_t dtype, int32_t flags,
                             tp_gemm_config* out, int32_t* found) {
  if (!ctx || !found) return fail(TP_ERR_INVALID, "null argument");
  if (flags & ~kTuneFlags) return fail(TP_ERR_INVALID, "undefined TP_TUNE_* flag bits");
  TuneState* st = state(ctx);
  std::lock_guard<std::mutex> lk(st->mu);
  auto it = st->cache.find(TuneKey{M, N, K, dtype, flags});
  *found = it != st->cache.end();
  if (*found && out) *out = it->second.first;
  return TP_OK;
}

tp_status tp_autotune_save(tp_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(TP_ERR_INVALID, "null argument");
  TuneState* st = state(ctx);
  std::lock_guard<std::mutex> lk(st->mu);
  FILE* f = std::fopen(path, "w");
  if (!f) return fail(TP_ERR_INVALID, std::string("cannot write ") + path);
  std::fprintf(f, "tp-autotune-cache v5\n");
  for (auto& kv : st->cache) {
    const auto& c = kv.second.first;
    std::fprintf(f, "%lld %lld %lld %d %d %d %d %d %d %d %d %d %d %.3f\n", (long long)kv.first.m,
                 (long long)kv.first.n, (long long)kv.first.k, kv.first.dtype, kv.first.flags, c.bm, c.bn, c.bk,
                 c.stages, c.group_m, c.num_programs, c.split_k, c.swap_ab, kv.second.second);
  }
  std::fclose(f);
  return TP_OK;
}

tp_status tp_autotune_load(tp_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(TP_ERR_INVALID, "null argument");
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(TP_ERR_INVALID, std::string("cannot read ") + path);
  // v5 lines carry swap_ab; v4 lines the search flags and bk; v3 lines lack
  // bk; v2 and v1 entries came from searches that included split-K (v1 lines
  // also lack the split_k column)
  char magic[64] = {};
  const bool ok = std::fgets(magic, sizeof magic, f) != nullptr;
  auto is = [&](const char* m) { return ok && std::string(magic).rfind(m, 0) == 0; };
  const int ver = is("tp-autotune-cache v5")   ? 5
                  : is("tp-autotune-cache v4") ? 4
                  : is("tp-autotune-cache v3") ? 3
                  : is("tp-autotune-cache v2") ? 2
                  : is("tp-autotune-cache v1") ? 1
                                               : 0;
  if (!ver) {
    std::fclose(f);
    return fail(TP_ERR_INVALID, "not an autotune cache (v1 to v5)");
  }
  TuneState* st = state(ctx);
  std::lock_guard<std::mutex> lk(st->mu);
  long long m, n, k;
  int dt, fl = TP_TUNE_SPLIT_K, bm, bn, bk = 0, stages, gm, np, sk = 0, sw = 0;
  float tf;
  for (;;) {
    int got, want;
    if (ver == 5) {
      got = std::fscanf(f, "%lld %lld %lld %d %d %d %d %d %d %d %d %d %d %f", &m, &n, &k, &dt, &fl, &bm, &bn, &bk,
                        &stages, &gm, &np, &sk, &sw, &tf);
      want = 14;
    } else if (ver == 4) {
      got = std::fscanf(f, "%lld %lld %lld %d %d %d %d %d %d %d %d %d %f", &m, &n, &k, &dt, &fl, &bm, &bn, &bk,
                        &stages, &gm, &np, &sk, &tf);
      want = 13;
    } else if (ver == 3) {
      got = std::fscanf(f, "%lld %lld %lld %d %d %d %d %d %d %d %d %f", &m, &n, &k, &dt, &fl, &bm, &bn, &stages, &gm,
                        &np, &sk, &tf);
      want = 12;
    } else if (ver == 2) {
      got = std::fscanf(f, "%lld %lld %lld %d %d %d %d %d %d %d %f", &m, &n, &k, &dt, &bm, &bn, &stages, &gm, &np,
                        &sk, &tf);
      want = 11;
    } else {
      got = std::fscanf(f, "%lld %lld %lld %d %d %d %d %d %d %f", &m, &n, &k, &dt, &bm, &bn, &stages, &gm, &np, &tf);
      want = 10;
    }
    if (got != want) break;
    if ((fl & ~kTuneFlags) || (sk > 1 && !(fl & TP_TUNE_SPLIT_K)) || (sw && !(fl & TP_TUNE_SWAP_AB)))
      continue;  // not a winner of such a search
    tp_gemm_config c{};
    c.bm = bm;
    c.bn = bn;
    c.bk = bk;
    c.stages = stages;
    c.group_m = gm;
    c.num_programs = np;
    c.split_k = sk;
    c.swap_ab = sw;
    st->cache[TuneKey{m, n, k, dt, fl}] = {c, tf};
    // an older search over the whole space that picked a single-pass config
    // also holds the single-pass class's winner
    if (ver < 3 && sk <= 1) st->cache[TuneKey{m, n, k, dt, 0}] = {c, tf};
  }
  std::fclose(f);
  return TP_OK;
}

}  // extern "C"
