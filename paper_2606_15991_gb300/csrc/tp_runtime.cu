// Host runtime of libtp: errors, contexts, tensor views, partitions, the
// launch protocol (SYNC / ASYNC / CAPTURE, §3.2), events and graphs.
#include <algorithm>
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

static void release_locked(tp_ctx* ctx, tp_partition* p) {
  p->busy.store(0);
  auto& v = ctx->busy;
  auto it = std::find(v.begin(), v.end(), p);
  if (it != v.end()) v.erase(it);
}

static void release(tp_ctx* ctx, const std::vector<tp_partition*>& ps) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  for (auto* p : ps) release_locked(ctx, p);
}

tp_status read_device_error(tp_ctx* ctx) {
  int h = 0;
  cudaError_t e = cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "reading device error word");
  if (h != kDevOk) {
    int zero = 0;
    cudaMemcpy(ctx->d_err, &zero, sizeof(int), cudaMemcpyHostToDevice);
    if (h == kDevTimeout) return fail(TP_ERR_TIMEOUT, "a device-side wait hit its iteration cap");
    return fail(TP_ERR_INVALID, "device bounds check failed");
  }
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

tp_status Op::begin(tp_ctx* c, const tp_exec* e, std::initializer_list<tp_partition*> outputs,
                    std::initializer_list<const tp_tensor*> inputs) {
  return begin_impl(c, e, std::vector<tp_partition*>(outputs), std::vector<const tp_tensor*>(inputs));
}

tp_status Op::begin_lists(tp_ctx* c, const tp_exec* e, const std::vector<tp_partition*>& outputs,
                          const std::vector<tp_tensor>& inputs) {
  std::vector<const tp_tensor*> in;
  for (const auto& t : inputs) in.push_back(&t);
  return begin_impl(c, e, outputs, in);
}

tp_status Op::begin_impl(tp_ctx* c, const tp_exec* e, const std::vector<tp_partition*>& outputs,
                         const std::vector<const tp_tensor*>& inputs) {
  ctx = c;
  ex = e;
  if (!ctx) return fail(TP_ERR_INVALID, "null context");
  if (!ex) return fail(TP_ERR_INVALID, "null tp_exec");
  if (ex->mode < TP_SYNC || ex->mode > TP_CAPTURE || ex->reserved != 0)
    return fail(TP_ERR_INVALID, "tp_exec.mode must be TP_SYNC, TP_ASYNC or TP_CAPTURE");
  if (ex->mode == TP_ASYNC && !ex->event) return fail(TP_ERR_INVALID, "TP_ASYNC needs tp_exec.event");
  if (ex->mode == TP_ASYNC && ex->event->ctx != ctx)
    return fail(TP_ERR_INVALID, "event belongs to another context");
  stream = static_cast<cudaStream_t>(ex->stream);
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
  std::lock_guard<std::mutex> lk(ctx->mu);
  // Alias-XOR-mutability at the launch boundary (§3.3, Appendix A): inputs
  // must not overlap an output, outputs must not overlap each other.
  for (size_t i = 0; i < outs.size(); ++i) {
    for (auto* t : inputs) {
      uintptr_t lo, hi;
      byte_range(*t, &lo, &hi);
      if (overlaps(lo, hi, outs[i]->lo, outs[i]->hi))
        return fail(TP_ERR_ALIAS, "an input tensor overlaps the output partition");
    }
    for (size_t j = i + 1; j < outs.size(); ++j)
      if (overlaps(outs[i]->lo, outs[i]->hi, outs[j]->lo, outs[j]->hi))
        return fail(TP_ERR_ALIAS, "two output partitions overlap");
  }
  // In-flight work holds its output exclusively (§3.2: host access is given
  // up until the stream completes).
  for (auto* b : ctx->busy) {
    for (auto* p : outs)
      if (p == b || overlaps(p->lo, p->hi, b->lo, b->hi))
        return fail(TP_ERR_BUSY, "output partition has work in flight");
    for (auto* t : inputs) {
      uintptr_t lo, hi;
      byte_range(*t, &lo, &hi);
      if (overlaps(lo, hi, b->lo, b->hi))
        return fail(TP_ERR_BUSY, "an input reads bytes of a partition with work in flight");
    }
  }
  if (ex->mode == TP_CAPTURE) {
    for (auto* p : outs) {
      auto& v = ctx->capturing->parts;
      if (std::find(v.begin(), v.end(), p) == v.end()) v.push_back(p);
    }
  } else {
    for (auto* p : outs) {
      p->busy.store(1);
      ctx->busy.push_back(p);
    }
    marked = true;
  }
  return TP_OK;
}

void Op::abort() {
  if (marked) release(ctx, outs);
  marked = false;
}

tp_status Op::end(cudaError_t launch_err) {
  if (launch_err != cudaSuccess) {
    if (marked) release(ctx, outs);
    return cuda_fail(launch_err, "kernel launch");
  }
  if (ex->mode == TP_CAPTURE) {
    if (check_err) ctx->capturing->check_err = true;
    return TP_OK;
  }
  if (ex->mode == TP_SYNC) {
    cudaError_t e = cudaStreamSynchronize(stream);
    release(ctx, outs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return check_err ? read_device_error(ctx) : TP_OK;
  }
  tp_event* ev = ex->event;
  cudaError_t e = cudaEventRecord(ev->ev, stream);
  if (e != cudaSuccess) {
    release(ctx, outs);
    return cuda_fail(e, "cudaEventRecord");
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  ev->recorded = true;
  ev->check_err |= check_err;
  for (auto* p : outs) ev->held.push_back(p);
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
  }
  return "unknown status";
}

const char* tp_last_error_detail(void) { return g_detail.c_str(); }

tp_status tp_version(int32_t* major, int32_t* minor) {
  if (!major || !minor) return fail(TP_ERR_INVALID, "null output");
  *major = 0;
  *minor = 1;
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
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_queue, 0, sizeof(unsigned) * tp_ctx::kQueueSlots);
  if (e != cudaSuccess) {
    cudaFree(c->d_err);
    cudaFree(c->d_queue);
    cudaFree(c->d_scratch);
    cudaFree(c->d_partial);
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
  info->busy = p->busy.load();
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
  auto* ev = new tp_event();
  ev->ctx = ctx;
  cudaError_t e = cudaEventCreateWithFlags(&ev->ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    delete ev;
    return cuda_fail(e, "cudaEventCreate");
  }
  *out = ev;
  return TP_OK;
}

static tp_status event_complete(tp_event* ev) {
  std::vector<tp_partition*> held;
  bool chk;
  {
    std::lock_guard<std::mutex> lk(ev->ctx->mu);
    held.swap(ev->held);
    chk = ev->check_err;
    ev->check_err = false;
    ev->recorded = false;
    for (auto* p : held) release_locked(ev->ctx, p);
  }
  return chk ? read_device_error(ev->ctx) : TP_OK;
}

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
  delete ev;
  return TP_OK;
}

tp_status tp_graph_begin(tp_ctx* ctx, void* stream, tp_graph** out) {
  if (!ctx || !out) return fail(TP_ERR_INVALID, "null argument");
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
    for (auto* p : g->parts)
      if (p->busy.load()) return fail(TP_ERR_BUSY, "a partition of the graph has work in flight");
    for (auto* p : g->parts) {
      p->busy.store(1);
      ctx->busy.push_back(p);
    }
  }
  cudaError_t e = cudaGraphLaunch(g->exec, stream);
  if (e != cudaSuccess) {
    release(ctx, g->parts);
    return cuda_fail(e, "cudaGraphLaunch");
  }
  if (ex->mode == TP_SYNC) {
    e = cudaStreamSynchronize(stream);
    release(ctx, g->parts);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return g->check_err ? read_device_error(ctx) : TP_OK;
  }
  e = cudaEventRecord(ex->event->ev, stream);
  if (e != cudaSuccess) {
    release(ctx, g->parts);
    return cuda_fail(e, "cudaEventRecord");
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  ex->event->recorded = true;
  ex->event->check_err |= g->check_err;
  for (auto* p : g->parts) ex->event->held.push_back(p);
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
  Op o;
  s = o.begin(ctx, ex, {out}, {x, y});
  if (s != TP_OK) return s;
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
  Op o;
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
  o.check_err = tc;
  s = simt ? launch_gemm_simt(ctx, c, a, b, cfg, ex, o.stream, q)
           : launch_gemm_tc(ctx, c, a, b, cfg, ex, o.stream, q);
  if (s != TP_OK) {
    o.abort();
    return s;
  }
  return o.end(cudaGetLastError());
}

}  // extern "C"
