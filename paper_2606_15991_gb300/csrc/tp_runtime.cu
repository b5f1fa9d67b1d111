// Host runtime of libtp: errors, contexts, tensor views, partitions, the
// launch protocol (SYNC / ASYNC / CAPTURE, §3.2), events and graphs.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "tp_internal.h"

namespace tp {

static thread_local std::string g_detail;

void set_detail(const std::string& s) { g_detail = s; }

tp_status fail(tp_status s, const std::string& detail) {
  g_detail = detail;
  return s;
}

tp_status cuda_fail(cudaError_t e, const char* what) {
  g_detail = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return TP_ERR_CUDA;
}

size_t dtype_size(int32_t d) {
  switch (d) {
    case TP_F32: return 4;
    case TP_BF16: return 2;
    case TP_F8E4M3: return 1;
    case TP_F64: return 8;
    case TP_I32: return 4;
    case TP_U32: return 4;
    case TP_U8: return 1;
    default: return 0;
  }
}

int64_t numel(const tp_tensor& t) {
  int64_t n = 1;
  for (int i = 0; i < t.rank; ++i) n *= t.shape[i];
  return n;
}

bool is_contiguous(const tp_tensor& t) {
  if (numel(t) == 0) return true;  // an empty view has no layout to violate
  int64_t expect = 1;
  for (int i = t.rank - 1; i >= 0; --i) {
    if (t.shape[i] != 1 && t.strides[i] != expect) return false;
    expect *= t.shape[i];
  }
  return true;
}

void byte_range(const tp_tensor& t, uintptr_t* lo, uintptr_t* hi) {
  uintptr_t base = reinterpret_cast<uintptr_t>(t.ptr);
  if (numel(t) == 0) {
    *lo = *hi = base;
    return;
  }
  int64_t mn = 0, mx = 0;
  for (int i = 0; i < t.rank; ++i) {
    int64_t span = (t.shape[i] - 1) * t.strides[i];
    if (span < 0) mn += span; else mx += span;
  }
  size_t es = dtype_size(t.dtype);
  *lo = base + mn * (int64_t)es;
  *hi = base + (mx + 1) * (int64_t)es;
}

static bool overlaps(uintptr_t a0, uintptr_t a1, uintptr_t b0, uintptr_t b1) {
  return a0 < a1 && b0 < b1 && a0 < b1 && b0 < a1;
}

// Byte intervals sorted by start, with the running maximum of their ends:
// "does [lo, hi) overlap any of them" in O(log n).
struct Spans {
  std::vector<std::pair<uintptr_t, uintptr_t>> v;
  std::vector<uintptr_t> max_hi;
  void add(uintptr_t lo, uintptr_t hi) {
    if (lo < hi) v.push_back({lo, hi});
  }
  void build() {
    std::sort(v.begin(), v.end());
    max_hi.resize(v.size());
    uintptr_t m = 0;
    for (size_t i = 0; i < v.size(); ++i) max_hi[i] = m = std::max(m, v[i].second);
  }
  bool hit(uintptr_t lo, uintptr_t hi) const {
    if (lo >= hi || v.empty()) return false;
    // intervals starting before hi, then whether any of them ends after lo
    auto it = std::lower_bound(v.begin(), v.end(), std::make_pair(hi, uintptr_t(0)));
    if (it == v.begin()) return false;
    return max_hi[(size_t)(it - v.begin()) - 1] > lo;
  }
  // some two of the intervals overlap
  bool self_overlap() const {
    for (size_t i = 1; i < v.size(); ++i)
      if (v[i].first < max_hi[i - 1]) return true;
    return false;
  }
};

// Bytes of partitions held by in-flight work on streams other than `stream`
// (every stream when `all_streams`).
static void busy_spans(tp_ctx* ctx, cudaStream_t stream, bool all_streams, Spans* out) {
  for (auto& kv : ctx->busy)
    if (all_streams || kv.first.second != stream) out->add(kv.first.first->lo, kv.first.first->hi);
  out->build();
}

static void release_locked(tp_ctx* ctx, tp_partition* p, cudaStream_t st, int64_t n = 1) {
  auto it = ctx->busy.find({p, st});
  if (it == ctx->busy.end()) return;
  const int64_t k = n < it->second ? n : it->second;
  it->second -= k;
  p->busy.fetch_sub((int)k);
  if (it->second == 0) ctx->busy.erase(it);
}

static void release(tp_ctx* ctx, const std::vector<tp_partition*>& ps, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  for (auto* p : ps) release_locked(ctx, p, st);
}

static void hold_locked(tp_ctx* ctx, tp_partition* p, cudaStream_t st) {
  p->busy.fetch_add(1);
  ++ctx->busy[{p, st}];
}

static tp_status error_status(int h) {
  if (h == kDevTimeout) return fail(TP_ERR_TIMEOUT, "a device-side wait hit its iteration cap");
  if (h == kDevRace)
    return fail(TP_ERR_RACE, "checked launch: a tile was stored twice or outside the storing program's map");
  return fail(TP_ERR_INVALID, "device bounds check failed");
}

tp_status read_device_error(tp_ctx* ctx) {
  int h = 0;
  cudaError_t e = cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "reading device error word");
  return take_device_error(ctx, h);
}

cudaError_t stage_device_error(tp_ctx* ctx, cudaStream_t stream, int* slot) {
  *slot = 0;
  return cudaMemcpyAsync(slot, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, stream);
}

tp_status take_device_error(tp_ctx* ctx, int h) {
  if (h == kDevOk) return TP_OK;
  int zero = 0;
  cudaMemcpy(ctx->d_err, &zero, sizeof(int), cudaMemcpyHostToDevice);
  // a checked launch that gave up part-way may have left claim state
  // behind; the next launch must start from zero
  if (h == kDevTimeout) {
    cudaMemset(ctx->d_claim_done, 0, 256);
    cudaMemset(ctx->d_claims, 0, (size_t)tp_ctx::kClaimBits / 8);
  }
  return error_status(h);
}

tp_status claims_for(tp_ctx* ctx, int64_t bits, uint32_t** claims, unsigned** done) {
  if (bits > tp_ctx::kClaimBits) return fail(TP_ERR_UNSUPPORTED, "too many tiles for a checked launch");
  *claims = ctx->d_claims;
  *done = ctx->d_claim_done;
  return TP_OK;
}

tp_status queue_counter(tp_ctx* ctx, cudaStream_t stream, unsigned** out) {
  uint32_t slot = ctx->queue_slot.fetch_add(1) % tp_ctx::kQueueSlots;
  unsigned* q = ctx->d_queue + slot;
  cudaError_t e = cudaMemsetAsync(q, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return cuda_fail(e, "resetting tile-queue counter");
  *out = q;
  return TP_OK;
}

// TP_LOG (any value but empty or 0): one line per operation on stderr.
static bool trace_on() {
  static const bool on = [] {
    const char* v = std::getenv("TP_LOG");
    return v && *v && std::strcmp(v, "0") != 0;
  }();
  return on;
}

static void trace(const Op& o, const char* event, tp_status st) {
  if (!trace_on()) return;
  static const char* const kModes[] = {"SYNC", "ASYNC", "CAPTURE"};
  const int mode = o.ex ? o.ex->mode : -1;
  char part[96] = "";
  if (!o.outs.empty() && o.outs[0])
    std::snprintf(part, sizeof part, " tiles=%lld programs=%lld map=%d outputs=%zu", (long long)o.outs[0]->num_tiles,
                  (long long)o.outs[0]->num_programs, (int)o.outs[0]->kind, o.outs.size());
  std::fprintf(stderr, "[tp] %s %s mode=%s stream=%p%s checked=%d status=%s%s%s\n", o.name, event,
               mode >= 0 && mode <= 2 ? kModes[mode] : "?", (void*)o.stream, part,
               o.ex ? (o.ex->flags & TP_EXEC_CHECKED ? 1 : 0) : 0, tp_error_string(st), st ? " detail=" : "",
               st ? g_detail.c_str() : "");
}

tp_status Op::begin(tp_ctx* c, const tp_exec* e, std::initializer_list<tp_partition*> outputs,
                    std::initializer_list<const tp_tensor*> inputs) {
  tp_status s = begin_impl(c, e, std::vector<tp_partition*>(outputs), std::vector<const tp_tensor*>(inputs));
  if (s != TP_OK) trace(*this, "refused", s);
  return s;
}

tp_status Op::begin_lists(tp_ctx* c, const tp_exec* e, const std::vector<tp_partition*>& outputs,
                          const std::vector<tp_tensor>& inputs) {
  std::vector<const tp_tensor*> in;
  for (const auto& t : inputs) in.push_back(&t);
  tp_status s = begin_impl(c, e, outputs, in);
  if (s != TP_OK) trace(*this, "refused", s);
  return s;
}

tp_status Op::begin_impl(tp_ctx* c, const tp_exec* e, const std::vector<tp_partition*>& outputs,
                         const std::vector<const tp_tensor*>& inputs) {
  ctx = c;
  ex = e;
  if (!ctx) return fail(TP_ERR_INVALID, "null context");
  device.bind(ctx);
  if (!ex) return fail(TP_ERR_INVALID, "null tp_exec");
  if (ex->mode < TP_SYNC || ex->mode > TP_CAPTURE)
    return fail(TP_ERR_INVALID, "tp_exec.mode must be TP_SYNC, TP_ASYNC or TP_CAPTURE");
  if (ex->flags & ~(TP_EXEC_CHECKED | TP_EXEC_INJECT_TIMEOUT | TP_EXEC_STATIC_WEIGHTS))
    return fail(TP_ERR_INVALID, "undefined tp_exec.flags bits");
  if ((ex->flags & TP_EXEC_STATIC_WEIGHTS) && !allow_static_weights)
    return fail(TP_ERR_UNSUPPORTED, "TP_EXEC_STATIC_WEIGHTS applies to the decode products only");
  if ((ex->flags & TP_EXEC_CHECKED) && !allow_checked)
    return fail(TP_ERR_UNSUPPORTED, "this operation has no device-checked launch (TP_EXEC_CHECKED)");
  if ((ex->flags & TP_EXEC_INJECT_TIMEOUT) && !allow_inject)
    return fail(TP_ERR_UNSUPPORTED, "this operation has no injected-timeout hook (TP_EXEC_INJECT_TIMEOUT)");
  if (ex->mode == TP_ASYNC && !ex->event) return fail(TP_ERR_INVALID, "TP_ASYNC needs tp_exec.event");
  if (ex->mode == TP_ASYNC && ex->event->ctx != ctx)
    return fail(TP_ERR_INVALID, "event belongs to another context");
  stream = static_cast<cudaStream_t>(ex->stream);
  if (ex->mode == TP_ASYNC) {
    tp_status es = event_claim(ex->event, stream);
    if (es != TP_OK) return es;
  }
  for (auto* p : outputs) {
    if (!p) return fail(TP_ERR_INVALID, "null output partition");
    if (p->ctx != ctx) return fail(TP_ERR_INVALID, "partition belongs to another context");
    outs.push_back(p);
  }
  for (auto* t : inputs) {
    if (!t) return fail(TP_ERR_INVALID, "null input tensor");
  }
  if (ex->mode == TP_CAPTURE) {
    cudaStreamCaptureStatus st;
    cudaError_t ce = cudaStreamIsCapturing(stream, &st);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamIsCapturing");
    if (st != cudaStreamCaptureStatusActive || !ctx->capturing || ctx->capturing->stream != stream)
      return fail(TP_ERR_CAPTURE, "TP_CAPTURE needs the stream of the graph opened by tp_graph_begin");
  }
  // Alias-XOR-mutability at the launch boundary (§3.3, Appendix A): inputs
  // must not overlap an output, outputs must not overlap each other.
  std::vector<std::pair<uintptr_t, uintptr_t>> in_bytes(inputs.size());
  for (size_t i = 0; i < inputs.size(); ++i) byte_range(*inputs[i], &in_bytes[i].first, &in_bytes[i].second);
  if (!outs.empty()) {
    Spans out_spans;
    for (auto* p : outs) out_spans.add(p->lo, p->hi);
    out_spans.build();
    if (out_spans.self_overlap()) return fail(TP_ERR_ALIAS, "two output partitions overlap");
    for (auto& r : in_bytes)
      if (out_spans.hit(r.first, r.second)) return fail(TP_ERR_ALIAS, "an input tensor overlaps the output partition");
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  // In-flight work holds its output exclusively (§3.2: host access is given
  // up until the stream completes). Work queued on the same stream runs after
  // it in stream order and may read or rewrite it: the C analogue of chaining
  // dependent operations with `then` (§3.2). Other streams conflict.
  if (!ctx->busy.empty()) {
    Spans held;
    busy_spans(ctx, stream, ex->mode == TP_CAPTURE, &held);
    for (auto* p : outs)
      if (held.hit(p->lo, p->hi))
        return fail(TP_ERR_BUSY, "output partition has work in flight on another stream");
    for (auto& r : in_bytes)
      if (held.hit(r.first, r.second))
        return fail(TP_ERR_BUSY, "an input reads bytes of a partition with work in flight on another stream");
  }
  if (ex->mode == TP_CAPTURE) {
    for (auto* p : outs) {
      auto& v = ctx->capturing->parts;
      if (std::find(v.begin(), v.end(), p) == v.end()) v.push_back(p);
    }
  } else {
    for (auto* p : outs) hold_locked(ctx, p, stream);
    marked = true;
  }
  return TP_OK;
}

void Op::abort() {
  if (marked) release(ctx, outs, stream);
  marked = false;
  trace(*this, "aborted", TP_ERR_INVALID);
}

tp_status Op::end(cudaError_t launch_err) {
  tp_status s = end_impl(launch_err);
  trace(*this, ex && ex->mode == TP_CAPTURE ? "recorded" : (ex && ex->mode == TP_ASYNC ? "enqueued" : "done"), s);
  return s;
}

tp_status Op::end_impl(cudaError_t launch_err) {
  if (launch_err != cudaSuccess) {
    if (marked) release(ctx, outs, stream);
    return cuda_fail(launch_err, "kernel launch");
  }
  if (ex->mode == TP_CAPTURE) {
    if (check_err) ctx->capturing->check_err = true;
    return TP_OK;
  }
  if (ex->mode == TP_SYNC) {
    int* slot = nullptr;
    cudaError_t e = cudaSuccess;
    if (check_err) {
      slot = ctx->h_err_slots + ctx->err_slot.fetch_add(1) % tp_ctx::kErrSlots;
      e = stage_device_error(ctx, stream, slot);
    }
    cudaError_t e2 = cudaStreamSynchronize(stream);
    release(ctx, outs, stream);
    if (e != cudaSuccess) return cuda_fail(e, "staging the device error word");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamSynchronize");
    return check_err ? take_device_error(ctx, *slot) : TP_OK;
  }
  tp_event* ev = ex->event;
  cudaError_t e = check_err ? stage_device_error(ctx, stream, ev->h_err) : cudaSuccess;
  if (e == cudaSuccess) e = cudaEventRecord(ev->ev, stream);
  if (e != cudaSuccess) {
    release(ctx, outs, stream);
    return cuda_fail(e, "cudaEventRecord");
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  ev->recorded = true;
  ev->stream = stream;
  ev->check_err |= check_err;
  for (auto* p : outs) ev->held.push_back({p, stream, 1});
  return TP_OK;
}

}  // namespace tp

using namespace tp;

extern "C" {

const char* tp_error_string(tp_status s) {
  switch (s) {
    case TP_OK: return "ok";
    case TP_ERR_INVALID: return "invalid argument";
    case TP_ERR_RANK: return "unsupported rank";
    case TP_ERR_ALIGN: return "misaligned pointer or stride";
    case TP_ERR_ALIAS: return "input aliases output";
    case TP_ERR_BUSY: return "partition busy (work in flight)";
    case TP_ERR_CAPTURE: return "not allowed during graph capture";
    case TP_ERR_UNSUPPORTED: return "unsupported";
    case TP_ERR_CUDA: return "CUDA error";
    case TP_ERR_TIMEOUT: return "device wait timed out";
    case TP_ERR_SHAPE: return "shape mismatch";
    case TP_ERR_RACE: return "checked launch found a tile stored twice or off the map";
  }
  return "unknown status";
}

const char* tp_last_error_detail(void) { return g_detail.c_str(); }

tp_status tp_version(int32_t* major, int32_t* minor) {
  if (!major || !minor) return fail(TP_ERR_INVALID, "null output");
  *major = 0;
  *minor = 2;  // 0.2: tp_gemm_config gained cut_limit; split_k selects split-K programs
  return TP_OK;
}

tp_status tp_ctx_create(int32_t device, tp_ctx** out) {
  if (!out) return fail(TP_ERR_INVALID, "null output");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= n) return fail(TP_ERR_INVALID, "no such CUDA device");
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  auto* c = new tp_ctx();
  c->device = device;
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&c->cc_major, cudaDevAttrComputeCapabilityMajor, device);
  cudaDeviceGetAttribute(&c->cc_minor, cudaDevAttrComputeCapabilityMinor, device);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  c->smem_optin = optin;
  if (c->cc_major != 10) {
    delete c;
    return fail(TP_ERR_UNSUPPORTED, "this library is built for sm_103a (Blackwell) only");
  }
  e = cudaMalloc(&c->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_queue, sizeof(unsigned) * tp_ctx::kQueueSlots);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_scratch, sizeof(float) * tp_ctx::kScratchFloats);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_partial, sizeof(float) * tp_ctx::kPartialFloats);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_claims, (size_t)tp_ctx::kClaimBits / 8);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_claim_done, 256);
  if (e == cudaSuccess) e = cudaMemset(c->d_claims, 0, (size_t)tp_ctx::kClaimBits / 8);
  if (e == cudaSuccess) e = cudaMemset(c->d_claim_done, 0, 256);
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_err_slots, sizeof(int) * tp_ctx::kErrSlots);
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_queue, 0, sizeof(unsigned) * tp_ctx::kQueueSlots);
  if (e != cudaSuccess) {
    cudaFree(c->d_err);
    cudaFree(c->d_queue);
    cudaFree(c->d_scratch);
    cudaFree(c->d_partial);
    cudaFree(c->d_claims);
    cudaFree(c->d_claim_done);
    cudaFreeHost(c->h_err_slots);
    delete c;
    return cuda_fail(e, "allocating context workspace");
  }
  *out = c;
  return TP_OK;
}

tp_status tp_ctx_destroy(tp_ctx* ctx) {
  if (!ctx) return fail(TP_ERR_INVALID, "null context");
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->busy.empty()) return fail(TP_ERR_BUSY, "context still has work in flight");
    if (ctx->capturing) return fail(TP_ERR_BUSY, "context is capturing a graph");
  }
  cudaFree(ctx->d_err);
  cudaFree(ctx->d_queue);
  cudaFree(ctx->d_scratch);
  cudaFree(ctx->d_partial);
  cudaFree(ctx->d_claims);
  cudaFree(ctx->d_claim_done);
  cudaFreeHost(ctx->h_err_slots);
  delete ctx;
  return TP_OK;
}

tp_status tp_ctx_info(tp_ctx* ctx, int32_t* sm_count, int32_t* cc_major, int32_t* cc_minor) {
  if (!ctx) return fail(TP_ERR_INVALID, "null context");
  if (sm_count) *sm_count = ctx->sm_count;
  if (cc_major) *cc_major = ctx->cc_major;
  if (cc_minor) *cc_minor = ctx->cc_minor;
  return TP_OK;
}

tp_status tp_tensor_init(tp_tensor* t, void* ptr, int32_t dtype, int32_t rank, const int64_t* shape,
                         const int64_t* strides) {
  if (!t) return fail(TP_ERR_INVALID, "null tensor");
  if (rank < 0 || rank > TP_MAX_RANK) return fail(TP_ERR_RANK, "rank must be 0..8");
  if (dtype_size(dtype) == 0) return fail(TP_ERR_INVALID, "unknown dtype");
  if (rank > 0 && !shape) return fail(TP_ERR_INVALID, "null shape");
  std::memset(t, 0, sizeof(*t));
  t->ptr = ptr;
  t->dtype = dtype;
  t->rank = rank;
  int64_t expect = 1;
  for (int i = rank - 1; i >= 0; --i) {
    if (shape[i] < 0) return fail(TP_ERR_INVALID, "negative extent");
    t->shape[i] = shape[i];
    t->strides[i] = strides ? strides[i] : expect;
    expect *= shape[i];
  }
  return TP_OK;
}

tp_status tp_tensor_view(const tp_tensor* base, int64_t offset, int32_t rank, const int64_t* shape,
                         const int64_t* strides, tp_tensor* out) {
  if (!base || !out) return fail(TP_ERR_INVALID, "null tensor");
  size_t es = dtype_size(base->dtype);
  tp_tensor v;
  tp_status s = tp_tensor_init(&v, static_cast<char*>(base->ptr) + offset * (int64_t)es, base->dtype,
                               rank, shape, strides);
  if (s != TP_OK) return s;
  uintptr_t blo, bhi, vlo, vhi;
  byte_range(*base, &blo, &bhi);
  byte_range(v, &vlo, &vhi);
  if (numel(v) > 0 && (vlo < blo || vhi > bhi))
    return fail(TP_ERR_INVALID, "view reaches outside its base tensor");
  *out = v;
  return TP_OK;
}

tp_status tp_partition_create(tp_ctx* ctx, const tp_tensor* out, const int64_t* tile, tp_partition** p) {
  if (!out || !tile || !p) return fail(TP_ERR_INVALID, "null argument");
  *p = nullptr;
  if (out->rank < 1 || out->rank > 3)
    return fail(TP_ERR_RANK, "a mutable partition has rank 1..3 (the launch grid is three-dimensional)");
  if (dtype_size(out->dtype) == 0) return fail(TP_ERR_INVALID, "unknown dtype");
  if (!is_contiguous(*out)) return fail(TP_ERR_UNSUPPORTED, "partitioned outputs must be contiguous");
  auto* q = new tp_partition();
  q->ctx = ctx;
  q->t = *out;
  q->rank = out->rank;
  q->num_tiles = 1;
  for (int i = 0; i < out->rank; ++i) {
    if (tile[i] < 1) {
      delete q;
      return fail(TP_ERR_INVALID, "tile extents must be >= 1");
    }
    q->shape[i] = out->shape[i];
    q->tile[i] = tile[i];
    q->grid[i] = (out->shape[i] + tile[i] - 1) / tile[i];
    q->num_tiles *= q->grid[i];
  }
  q->num_programs = q->num_tiles;
  byte_range(*out, &q->lo, &q->hi);
  *p = q;
  return TP_OK;
}

tp_status tp_partition_map(tp_partition* p, int32_t kind, int64_t num_programs) {
  if (!p) return fail(TP_ERR_INVALID, "null partition");
  if (p->busy.load()) return fail(TP_ERR_BUSY, "partition has work in flight");
  if (kind == TP_MAP_IDENTITY) {
    p->kind = kind;
    p->num_programs = p->num_tiles;
    return TP_OK;
  }
  if (kind != TP_MAP_STRIDED && kind != TP_MAP_QUEUE) return fail(TP_ERR_INVALID, "unknown map kind");
  if (num_programs < 1 || num_programs > std::max<int64_t>(p->num_tiles, 1))
    return fail(TP_ERR_INVALID, "program count must be 1..number of tiles in the partition grid");
  p->kind = kind;
  p->num_programs = num_programs;
  return TP_OK;
}

tp_status tp_partition_query(const tp_partition* p, tp_partition_info* info) {
  if (!p || !info) return fail(TP_ERR_INVALID, "null argument");
  std::memset(info, 0, sizeof(*info));
  info->rank = p->rank;
  info->map_kind = p->kind;
  for (int i = 0; i < 3; ++i) {
    info->shape[i] = p->shape[i];
    info->tile[i] = p->tile[i];
    info->grid[i] = p->grid[i];
  }
  info->num_tiles = p->num_tiles;
  info->num_programs = p->num_programs;
  info->busy = p->busy.load() > 0 ? 1 : 0;
  return TP_OK;
}

tp_status tp_partition_destroy(tp_partition* p) {
  if (!p) return fail(TP_ERR_INVALID, "null partition");
  if (p->busy.load()) return fail(TP_ERR_BUSY, "partition has work in flight");
  if (p->ctx) {
    std::lock_guard<std::mutex> lk(p->ctx->mu);
    if (p->ctx->capturing) {
      auto& v = p->ctx->capturing->parts;
      v.erase(std::remove(v.begin(), v.end(), p), v.end());
    }
  }
  delete p;
  return TP_OK;
}

tp_status tp_event_create(tp_ctx* ctx, tp_event** out) {
  if (!ctx || !out) return fail(TP_ERR_INVALID, "null argument");
  DeviceGuard guard(ctx);
  auto* ev = new tp_event();
  ev->ctx = ctx;
  cudaError_t e = cudaEventCreateWithFlags(&ev->ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    delete ev;
    return cuda_fail(e, "cudaEventCreate");
  }
  e = cudaMallocHost(&ev->h_err, sizeof(int));
  if (e != cudaSuccess) {
    cudaEventDestroy(ev->ev);
    delete ev;
    return cuda_fail(e, "cudaMallocHost");
  }
  *ev->h_err = 0;
  *out = ev;
  return TP_OK;
}

static tp_status event_complete(tp_event* ev) {
  std::vector<Hold> held;
  bool chk;
  {
    std::lock_guard<std::mutex> lk(ev->ctx->mu);
    held.swap(ev->held);
    chk = ev->check_err;
    ev->check_err = false;
    ev->recorded = false;
    for (auto& h : held) release_locked(ev->ctx, h.p, h.stream, h.count);
  }
  return chk ? take_device_error(ev->ctx, *ev->h_err) : TP_OK;
}

}  // extern "C"

tp_status tp::event_claim(tp_event* ev, cudaStream_t stream) {
  if (!ev->recorded || ev->stream == stream) return TP_OK;
  // the event still tracks work on another stream: re-recording it here
  // would release that work's holds when this stream's work completes
  cudaError_t e = cudaEventQuery(ev->ev);
  if (e == cudaErrorNotReady)
    return fail(TP_ERR_BUSY, "the event tracks unfinished work on another stream; wait for it or use another event");
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventQuery");
  return event_complete(ev);
}

extern "C" {

tp_status tp_event_query(tp_event* ev, int32_t* done) {
  if (!ev || !done) return fail(TP_ERR_INVALID, "null argument");
  if (!ev->recorded) {
    *done = 1;
    return TP_OK;
  }
  cudaError_t e = cudaEventQuery(ev->ev);
  if (e == cudaErrorNotReady) {
    *done = 0;
    return TP_OK;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventQuery");
  *done = 1;
  return event_complete(ev);
}

tp_status tp_event_wait(tp_event* ev) {
  if (!ev) return fail(TP_ERR_INVALID, "null event");
  if (!ev->recorded) return TP_OK;
  cudaError_t e = cudaEventSynchronize(ev->ev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
  return event_complete(ev);
}

tp_status tp_event_destroy(tp_event* ev) {
  if (!ev) return fail(TP_ERR_INVALID, "null event");
  if (ev->recorded && !ev->held.empty()) {
    if (cudaEventQuery(ev->ev) == cudaErrorNotReady)
      return fail(TP_ERR_BUSY, "event still holds partitions of unfinished work");
    event_complete(ev);
  }
  cudaEventDestroy(ev->ev);
  cudaFreeHost(ev->h_err);
  delete ev;
  return TP_OK;
}

tp_status tp_graph_begin(tp_ctx* ctx, void* stream, tp_graph** out) {
  if (!ctx || !out) return fail(TP_ERR_INVALID, "null argument");
  DeviceGuard guard(ctx);
  if (!stream) return fail(TP_ERR_INVALID, "graph capture needs a non-default stream");
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->capturing) return fail(TP_ERR_CAPTURE, "this context is already capturing a graph");
  auto* g = new tp_graph();
  g->ctx = ctx;
  g->stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    delete g;
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  ctx->capturing = g;
  *out = g;
  return TP_OK;
}

tp_status tp_graph_end(tp_graph* g) {
  if (!g) return fail(TP_ERR_INVALID, "null graph");
  if (g->ended) return fail(TP_ERR_INVALID, "graph already ended");
  {
    std::lock_guard<std::mutex> lk(g->ctx->mu);
    g->ctx->capturing = nullptr;
  }
  g->ended = true;
  cudaError_t e = cudaStreamEndCapture(g->stream, &g->graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return TP_OK;
}

tp_status tp_graph_replay(tp_graph* g, const tp_exec* ex) {
  if (!g || !ex) return fail(TP_ERR_INVALID, "null argument");
  if (!g->ended || !g->exec) return fail(TP_ERR_INVALID, "graph not ended/instantiated");
  if (ex->mode == TP_CAPTURE) return fail(TP_ERR_CAPTURE, "a replay cannot itself be captured here");
  if (ex->mode == TP_ASYNC && (!ex->event || ex->event->ctx != g->ctx))
    return fail(TP_ERR_INVALID, "TP_ASYNC needs an event of the graph's context");
  tp_ctx* ctx = g->ctx;
  cudaStream_t stream = static_cast<cudaStream_t>(ex->stream);
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->busy.empty()) {
      Spans held;
      busy_spans(ctx, stream, false, &held);
      for (auto* p : g->parts)
        if (held.hit(p->lo, p->hi))
          return fail(TP_ERR_BUSY, "a partition of the graph has work in flight on another stream");
    }
    for (auto* p : g->parts) hold_locked(ctx, p, stream);
  }
  if (ex->mode == TP_ASYNC) {
    tp_status es = event_claim(ex->event, stream);
    if (es != TP_OK) {
      release(ctx, g->parts, stream);
      return es;
    }
  }
  cudaError_t e = cudaGraphLaunch(g->exec, stream);
  if (e != cudaSuccess) {
    release(ctx, g->parts, stream);
    return cuda_fail(e, "cudaGraphLaunch");
  }
  if (ex->mode == TP_SYNC) {
    int* slot = nullptr;
    if (g->check_err) {
      slot = ctx->h_err_slots + ctx->err_slot.fetch_add(1) % tp_ctx::kErrSlots;
      e = stage_device_error(ctx, stream, slot);
    }
    cudaError_t e2 = cudaStreamSynchronize(stream);
    release(ctx, g->parts, stream);
    if (e != cudaSuccess) return cuda_fail(e, "staging the device error word");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamSynchronize");
    return g->check_err ? take_device_error(ctx, *slot) : TP_OK;
  }
  e = g->check_err ? stage_device_error(ctx, stream, ex->event->h_err) : cudaSuccess;
  if (e == cudaSuccess) e = cudaEventRecord(ex->event->ev, stream);
  if (e != cudaSuccess) {
    release(ctx, g->parts, stream);
    return cuda_fail(e, "cudaEventRecord");
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  ex->event->recorded = true;
  ex->event->stream = stream;
  ex->event->check_err |= g->check_err;
  for (auto* p : g->parts) ex->event->held.push_back({p, stream, 1});
  return TP_OK;
}

tp_status tp_graph_kernel_count(tp_graph* g, int64_t* count) {
  if (!g || !count) return fail(TP_ERR_INVALID, "null argument");
  if (!g->ended || !g->graph) return fail(TP_ERR_INVALID, "graph not ended");
  size_t n = 0;
  cudaError_t e = cudaGraphGetNodes(g->graph, nullptr, &n);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphGetNodes");
  std::vector<cudaGraphNode_t> nodes(n);
  if (n > 0) e = cudaGraphGetNodes(g->graph, nodes.data(), &n);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphGetNodes");
  int64_t k = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    e = cudaGraphNodeGetType(nodes[i], &t);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphNodeGetType");
    k += t == cudaGraphNodeTypeKernel;
  }
  *count = k;
  return TP_OK;
}

tp_status tp_graph_destroy(tp_graph* g) {
  if (!g) return fail(TP_ERR_INVALID, "null graph");
  {
    std::lock_guard<std::mutex> lk(g->ctx->mu);
    for (auto* p : g->parts)
      if (p->busy.load()) return fail(TP_ERR_BUSY, "graph replay still in flight");
    if (g->ctx->capturing == g) return fail(TP_ERR_BUSY, "graph still capturing; call tp_graph_end");
  }
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return TP_OK;
}

// ----------------------------------------------------------------- ops

static tp_status check_elementwise(const tp_partition* out, const tp_tensor* x, const tp_tensor* y) {
  for (const tp_tensor* t : {x, y}) {
    if (t->dtype != out->t.dtype) return fail(TP_ERR_SHAPE, "input dtype differs from output dtype");
    if (t->rank != out->rank) return fail(TP_ERR_SHAPE, "input rank differs from output rank");
    for (int i = 0; i < out->rank; ++i)
      if (t->shape[i] != out->shape[i]) return fail(TP_ERR_SHAPE, "input shape differs from output shape");
    if (!is_contiguous(*t)) return fail(TP_ERR_UNSUPPORTED, "map inputs must be contiguous");
  }
  if (out->t.dtype != TP_F32 && out->t.dtype != TP_BF16)
    return fail(TP_ERR_UNSUPPORTED, "maps support F32 and BF16");
  return TP_OK;
}

static tp_status map_op(tp_ctx* ctx, tp_partition* out, int op, float alpha, const tp_tensor* x,
                        const tp_tensor* y, const tp_exec* ex) {
  if (!ctx || !out || !x || !y || !ex) return fail(TP_ERR_INVALID, "null argument");
  tp_status s = check_elementwise(out, x, y);
  if (s != TP_OK) return s;
  static const char* const kNames[] = {"tp_map_axpy", "tp_map_gelu_mul", "tp_map_scale", "tp_map_add_accum"};
  Op o(kNames[op & 3]);
  o.allow_checked = true;
  s = o.begin(ctx, ex, {out}, {x, y});
  if (s != TP_OK) return s;
  o.check_err = (ex->flags & TP_EXEC_CHECKED) != 0;
  unsigned* q = nullptr;
  if (out->kind == TP_MAP_QUEUE) {
    s = queue_counter(ctx, o.stream, &q);
    if (s != TP_OK) {
      o.abort();
      return s;
    }
  }
  s = launch_map(ctx, out, op, alpha, x, y, ex, o.stream, q);
  if (s != TP_OK) {
    o.abort();
    return s;
  }
  return o.end(cudaGetLastError());
}

tp_status tp_map_axpy(tp_ctx* ctx, tp_partition* z, float alpha, const tp_tensor* x, const tp_tensor* y,
                      const tp_exec* ex) {
  return map_op(ctx, z, kMapAxpy, alpha, x, y, ex);
}

tp_status tp_map_gelu_mul(tp_ctx* ctx, tp_partition* y, const tp_tensor* x, const tp_tensor* w,
                          const tp_exec* ex) {
  return map_op(ctx, y, kMapGeluMul, 0.f, x, w, ex);
}

tp_status tp_map_scale(tp_ctx* ctx, tp_partition* y, const tp_tensor* x, const tp_tensor* g,
                       const tp_exec* ex) {
  return map_op(ctx, y, kMapScale, 0.f, x, g, ex);
}

tp_status tp_map_add_accum(tp_ctx* ctx, tp_partition* c, const tp_tensor* a, const tp_tensor* b,
                           const tp_exec* ex) {
  return map_op(ctx, c, kMapAddAccum, 0.f, a, b, ex);
}

tp_status tp_gemm(tp_ctx* ctx, tp_partition* c, const tp_tensor* a, const tp_tensor* b,
                  const tp_gemm_config* cfg, const tp_exec* ex) {
  if (!ctx || !c || !a || !b || !ex) return fail(TP_ERR_INVALID, "null argument");
  if (a->rank != 2 || b->rank != 2 || c->rank != 2) return fail(TP_ERR_RANK, "GEMM operands are rank 2");
  const int64_t M = a->shape[0], K = a->shape[1], N = b->shape[1];
  if (b->shape[0] != K || c->shape[0] != M || c->shape[1] != N)
    return fail(TP_ERR_SHAPE, "need A: M x K, B: K x N, C: M x N");
  if (a->dtype != b->dtype) return fail(TP_ERR_SHAPE, "A and B must have the same dtype");
  bool simt = a->dtype == TP_F32 && c->t.dtype == TP_F32;
  bool tc = a->dtype == TP_BF16 && c->t.dtype == TP_BF16;
  if (!simt && !tc) return fail(TP_ERR_UNSUPPORTED, "tp_gemm supports F32xF32->F32 and BF16xBF16->BF16");
  Op o(__func__);
  o.allow_checked = tc;
  o.allow_inject = tc;
  tp_status s = o.begin(ctx, ex, {c}, {a, b});
  if (s != TP_OK) return s;
  unsigned* q = nullptr;
  if (c->kind == TP_MAP_QUEUE) {
    s = queue_counter(ctx, o.stream, &q);
    if (s != TP_OK) {
      o.abort();
      return s;
    }
  }
  o.check_err = true;  // the tensor-core and TMA-fed FP32 kernels' waits are bounded
  s = simt ? launch_gemm_simt(ctx, c, a, b, cfg, ex, o.stream, q)
           : launch_gemm_tc(ctx, c, a, b, cfg, ex, o.stream, q);
  if (s != TP_OK) {
    o.abort();
    return s;
  }
  return o.end(cudaGetLastError());
}

tp_status tp_gemm_resident_programs(tp_ctx* ctx, const tp_gemm_config* cfg, int32_t* programs) {
  if (!ctx || !cfg || !programs) return fail(TP_ERR_INVALID, "null argument");
  DeviceGuard guard(ctx);
  return gemm_tc_resident(ctx, cfg, programs);
}

tp_status tp_gemm_unchecked(tp_ctx* ctx, void* c, const tp_tensor* a, const tp_tensor* b, const tp_gemm_config* cfg,
                            void* stream) {
  if (!ctx || !c || !a || !b || !cfg) return fail(TP_ERR_INVALID, "null argument");
  DeviceGuard guard(ctx);
  if (a->rank != 2 || b->rank != 2) return fail(TP_ERR_RANK, "GEMM operands are rank 2");
  if (a->dtype != TP_BF16 || b->dtype != TP_BF16) return fail(TP_ERR_UNSUPPORTED, "BF16 operands only");
  const int64_t M = a->shape[0], K = a->shape[1], N = b->shape[1];
  if (b->shape[0] != K) return fail(TP_ERR_SHAPE, "need A: M x K, B: K x N");
  if (cfg->swap_ab ? (cfg->bm != 32 && cfg->bm != 64 && cfg->bm != 128)
                   : (cfg->bm != 64 && cfg->bm != 128 && cfg->bm != 256))
    return fail(TP_ERR_INVALID, "cfg.bm must be 64, 128 or 256 (swap_ab: 32, 64 or 128)");
  if (cfg->bn <= 0) return fail(TP_ERR_INVALID, "cfg.bn must be given");
  // a stack descriptor of C's tiling; nothing is registered with the context
  tp_partition p;
  p.ctx = ctx;
  p.t.ptr = c;
  p.t.dtype = TP_BF16;
  p.t.rank = 2;
  p.t.shape[0] = M;
  p.t.shape[1] = N;
  p.t.strides[0] = N;
  p.t.strides[1] = 1;
  p.rank = 2;
  p.shape[0] = M;
  p.shape[1] = N;
  p.tile[0] = cfg->bm;
  p.tile[1] = cfg->bn;
  p.grid[0] = (M + cfg->bm - 1) / cfg->bm;
  p.grid[1] = (N + cfg->bn - 1) / cfg->bn;
  p.num_tiles = p.grid[0] * p.grid[1];
  if (cfg->num_programs > 0) {
    p.kind = TP_MAP_STRIDED;
    p.num_programs = cfg->num_programs < p.num_tiles ? cfg->num_programs : p.num_tiles;
  } else {
    p.kind = TP_MAP_IDENTITY;
    p.num_programs = p.num_tiles;
  }
  tp_exec ex{};
  ex.mode = TP_SYNC;
  ex.stream = stream;
  return launch_gemm_tc(ctx, &p, a, b, cfg, &ex, static_cast<cudaStream_t>(stream), nullptr);
}

}  // extern "C"
