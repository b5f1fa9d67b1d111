// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "tp.h"

namespace tp {

// Device-side error codes written to the context's error word.
enum DeviceError : int {
  kDevOk = 0,
  kDevTimeout = 1,     // a bounded wait ran out of iterations
  kDevBounds = 2,      // debug bounds check failed
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

struct tp_ctx {
  int32_t device = 0;
  int32_t sm_count = 0;
  int32_t cc_major = 0, cc_minor = 0;
  size_t smem_optin = 0;
  std::mutex mu;
  std::vector<tp_partition*> busy;  // partitions with work in flight
  tp_graph* capturing = nullptr;    // graph being captured, if any
  // Device workspace, allocated once at creation.
  int* d_err = nullptr;             // device error word (tp::DeviceError)
  unsigned* d_queue = nullptr;      // tile-queue counters (kQueueSlots)
  float* d_scratch = nullptr;       // small float scratch (kScratchFloats)
  float* d_partial = nullptr;       // matrix-vector partial sums (kPartialFloats)
  std::atomic<uint32_t> queue_slot{0};
  static constexpr int kQueueSlots = 256;
  static constexpr int kScratchFloats = 4096;
  static constexpr int64_t kPartialFloats = int64_t(1) << 20;
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
  std::atomic<int> busy{0};
};

struct tp_event {
  tp_ctx* ctx = nullptr;
  cudaEvent_t ev = nullptr;
  bool recorded = false;
  bool check_err = false;
  std::vector<tp_partition*> held;
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

// Launch protocol shared by every operation (§3.2 / §3.3 semantics):
//   begin(): validate exec + aliasing + busy state, mark the output busy
//            (SYNC/ASYNC) or record it into the capturing graph (CAPTURE);
//   end():   after the kernel launches, synchronize + release (SYNC), record
//            the completion event (ASYNC), or nothing (CAPTURE).
struct Op {
  tp_ctx* ctx;
  const tp_exec* ex;
  cudaStream_t stream;
  std::vector<tp_partition*> outs;
  bool check_err = false;   // kernel may write the device error word
  bool marked = false;

  tp_status begin(tp_ctx* c, const tp_exec* e, std::initializer_list<tp_partition*> outputs,
                  std::initializer_list<const tp_tensor*> inputs);
  tp_status begin_lists(tp_ctx* c, const tp_exec* e, const std::vector<tp_partition*>& outputs,
                        const std::vector<tp_tensor>& inputs);
  tp_status begin_impl(tp_ctx* c, const tp_exec* e, const std::vector<tp_partition*>& outputs,
                       const std::vector<const tp_tensor*>& inputs);
  tp_status end(cudaError_t launch_err);
  // Undo begin() after a failure that launched nothing (keeps the detail).
  void abort();
  bool capturing() const { return ex->mode == TP_CAPTURE; }
};

tp_status read_device_error(tp_ctx* ctx);
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

tp_status launch_gemm_tc_impl(tp_ctx* ctx, tp_partition* c, const tp_tensor* a, const tp_tensor* b,
                              const tp_gemm_config* cfg, const tp_exec* ex, cudaStream_t stream, int esize,
                              const float* scale_a, const float* scale_b);

}  // namespace tp
