// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <functional>
#include <mutex>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include "tp.h"

namespace tp {

// Device-side error codes written to the context's error word.
enum DeviceError : int {
  kDevOk = 0,
  kDevTimeout = 1,     // a bounded wait ran out of iterations
  kDevBounds = 2,      // debug bounds check failed
  kDevRace = 3,        // checked launch: a tile claimed twice or off the program's map
};

void set_detail(const std::string& s);
tp_status fail(tp_status s, const std::string& detail);
tp_status cuda_fail(cudaError_t e, const char* what);

size_t dtype_size(int32_t dtype);
bool is_contiguous(const tp_tensor& t);
int64_t numel(const tp_tensor& t);
// Byte range [lo, hi) reachable through the view (lo == hi for empty views).
void byte_range(const tp_tensor& t, uintptr_t* lo, uintptr_t* hi);

}  // namespace tp

namespace tp {
// `count` in-flight holds of one partition by work queued on one stream.
struct Hold {
  tp_partition* p;
  cudaStream_t stream;
  int64_t count;
};
using HoldKey = std::pair<tp_partition*, cudaStream_t>;
struct HoldKeyHash {
  size_t operator()(const HoldKey& k) const {
    return std::hash<const void*>()(k.first) * 31u ^ std::hash<const void*>()(k.second);
  }
};
}  // namespace tp

struct tp_ctx {
  int32_t device = 0;
  int32_t sm_count = 0;
  int32_t cc_major = 0, cc_minor = 0;
  size_t smem_optin = 0;
  std::mutex mu;
  // in-flight holds: (partition, stream) -> count; work chained on one
  // stream adds to the entry's count
  std::unordered_map<tp::HoldKey, int64_t, tp::HoldKeyHash> busy;
  tp_graph* capturing = nullptr;    // graph being captured, if any
  // Device workspace, allocated once at creation.
  int* d_err = nullptr;             // device error word (tp::DeviceError)
  unsigned* d_queue = nullptr;      // tile-queue counters (kQueueSlots)
  float* d_scratch = nullptr;       // small float scratch (kScratchFloats)
  float* d_partial = nullptr;       // matrix-vector partial sums (kPartialFloats)
  uint32_t* d_claims = nullptr;     // tile-claim bitmap of checked launches (kClaimBits), all clear
  unsigned* d_claim_done = nullptr; // CTAs of the running checked launch that finished
  int* h_err_slots = nullptr;       // pinned host copies of the error word (kErrSlots)
  std::atomic<uint32_t> err_slot{0};
  static constexpr int kErrSlots = 256;
  std::atomic<uint32_t> queue_slot{0};
  static constexpr int kQueueSlots = 256;
  static constexpr int kScratchFloats = 4096;
  static constexpr int64_t kPartialFloats = int64_t(1) << 20;
  static constexpr int64_t kClaimBits = int64_t(1) << 26;   // 8 MiB
};

struct tp_partition {
  tp_ctx* ctx = nullptr;
  tp_tensor t{};
  int32_t rank = 0;
  int64_t shape[3] = {1, 1, 1};
  int64_t tile[3] = {1, 1, 1};
  int64_t grid[3] = {1, 1, 1};
  int64_t num_tiles = 0;
  int64_t num_programs = 0;
  int32_t kind = TP_MAP_IDENTITY;
  uintptr_t lo = 0, hi = 0;  // output bytes
  std::atomic<int> busy{0};  // number of in-flight holds
};

struct tp_event {
  tp_ctx* ctx = nullptr;
  cudaEvent_t ev = nullptr;
  bool recorded = false;
  bool check_err = false;
  cudaStream_t stream = nullptr;  // stream of the last record
  int* h_err = nullptr;           // pinned copy of the error word, staged behind the work
  std::vector<tp::Hold> held;   // holds released when the event completes (appended per op)
};

struct tp_graph {
  tp_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool ended = false;
  bool check_err = false;
  std::vector<tp_partition*> parts;  // partitions written by recorded nodes
};

namespace tp {

// Makes the context's device current in the calling thread for one entry
// point: a thread that has not used CUDA yet gets the device's primary
// context bound (driver-API calls such as TMA descriptor encoding need a
// current context), and a caller whose current device differs gets it back
// when the guard goes out of scope.
struct DeviceGuard {
  int restore = -1;
  DeviceGuard() = default;
  explicit DeviceGuard(const tp_ctx* ctx) { bind(ctx); }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
  void bind(const tp_ctx* ctx) {
    static thread_local bool bound = false;
    if (!ctx) return;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) cur = -1;
    if (bound && cur == ctx->device) return;
    if (cudaSetDevice(ctx->device) == cudaSuccess) {
      if (bound && cur >= 0 && cur != ctx->device && restore < 0) restore = cur;
      bound = true;
    }
  }
  ~DeviceGuard() {
    if (restore >= 0) cudaSetDevice(restore);
  }
};

// Launch protocol shared by every operation (§3.2 / §3.3 semantics):
//   begin(): validate exec + aliasing + busy state, mark the output busy
//            (SYNC/ASYNC) or record it into the capturing graph (CAPTURE);
//   end():   after the kernel launches, synchronize + release (SYNC), record
//            the completion event (ASYNC), or nothing (CAPTURE).
struct Op {
  Op() = default;
  explicit Op(const char* op_name) : name(op_name) {}
  const char* name = "op";   // entry point, for the TP_LOG trace
  tp_ctx* ctx = nullptr;
  const tp_exec* ex = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<tp_partition*> outs;
  bool check_err = false;   // kernel may write the device error word
  bool marked = false;
  bool allow_checked = false;  // the op implements TP_EXEC_CHECKED (set before begin)
  bool allow_inject = false;   // the op implements TP_EXEC_INJECT_TIMEOUT (set before begin)
  bool allow_static_weights = false;  // the op implements TP_EXEC_STATIC_WEIGHTS (set before begin)
  DeviceGuard device;          // the context's device is current while the op launches

  tp_status begin(tp_ctx* c, const tp_exec* e, std::initializer_list<tp_partition*> outputs,
                  std::initializer_list<const tp_tensor*> inputs);
  tp_status begin_lists(tp_ctx* c, const tp_exec* e, const std::vector<tp_partition*>& outputs,
                        const std::vector<tp_tensor>& inputs);
  tp_status begin_impl(tp_ctx* c, const tp_exec* e, const std::vector<tp_partition*>& outputs,
                       const std::vector<const tp_tensor*>& inputs);
  tp_status end(cudaError_t launch_err);
  tp_status end_impl(cudaError_t launch_err);
  // Undo begin() after a failure that launched nothing (keeps the detail).
  void abort();
  bool capturing() const { return ex->mode == TP_CAPTURE; }
};

tp_status read_device_error(tp_ctx* ctx);
// Enqueue a copy of the device error word into pinned `slot` on `stream`
// (behind the work already queued there).
cudaError_t stage_device_error(tp_ctx* ctx, cudaStream_t stream, int* slot);
// Status for a staged error word `h` (read after the stream or event
// completed); clears the device word when it is set.
tp_status take_device_error(tp_ctx* ctx, int h);
// An ASYNC launch may record `ev` on `stream`: OK when the event tracks no
// unfinished work on another stream (completed work is released first).
tp_status event_claim(tp_event* ev, cudaStream_t stream);
// The context's tile-claim bitmap for one checked launch (TP_EXEC_CHECKED)
// that may set up to `bits` bits; the launch's last CTA clears them again.
tp_status claims_for(tp_ctx* ctx, int64_t bits, uint32_t** claims, unsigned** done);
// Reserve a tile-queue counter for one launch and zero it on `stream`.
tp_status queue_counter(tp_ctx* ctx, cudaStream_t stream, unsigned** out);

// Kernel launchers (defined in the kernel translation units).
enum MapOp : int { kMapAxpy = 0, kMapGeluMul = 1, kMapScale = 2, kMapAddAccum = 3 };
tp_status launch_map(tp_ctx* ctx, tp_partition* out, int op, float alpha, const tp_tensor* x,
                     const tp_tensor* y, const tp_exec* ex, cudaStream_t stream, unsigned* queue);
tp_status launch_gemm_simt(tp_ctx* ctx, tp_partition* c, const tp_tensor* a, const tp_tensor* b,
                           const tp_gemm_config* cfg, const tp_exec* ex, cudaStream_t stream,
                           unsigned* queue);
tp_status launch_gemm_tc(tp_ctx* ctx, tp_partition* c, const tp_tensor* a, const tp_tensor* b,
                         const tp_gemm_config* cfg, const tp_exec* ex, cudaStream_t stream,
                         unsigned* queue);

// Programs of the tensor-core GEMM (CTA pairs for 256-row tiles, CTAs
// otherwise) that can be resident at once for `cfg`.
tp_status gemm_tc_resident(tp_ctx* ctx, const tp_gemm_config* cfg, int32_t* programs);
// Whether the autotuner tries config c of its space on an M x N x K problem
// of `dtype` (a config it does not try is never proposed for it either).
bool autotune_config_runs(const tp_ctx* ctx, int64_t M, int64_t N, int64_t K, int32_t dtype,
                          const tp_gemm_config& c);

tp_status launch_gemm_tc_impl(tp_ctx* ctx, tp_partition* c, const tp_tensor* a, const tp_tensor* b,
                              const tp_gemm_config* cfg, const tp_exec* ex, cudaStream_t stream, int esize,
                              const float* scale_a, const float* scale_b);

}  // namespace tp
