// Diagnostic of the failure path shared by the pipelined kernels: a role
// that waits on an mbarrier gives up after a wall-time limit, records
// kDevTimeout in the context's error word and returns, so the launch ends and
// the host reports TP_ERR_TIMEOUT instead of the GPU hanging.
#include "sm100_ptx.cuh"
#include "tp_internal.h"

namespace tp {
namespace {

using namespace sm100;

__global__ void bounded_wait_kernel(int* err, uint64_t limit_ns, int arrive) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (arrive) mbar_arrive(smem_u32(&bar));
    mbar_wait(smem_u32(&bar), 0, &abort_flag, err, limit_ns);
  }
}

}  // namespace
}  // namespace tp

using namespace tp;

extern "C" tp_status tp_diag_bounded_wait(tp_ctx* ctx, int64_t limit_ns, int32_t arrive, const tp_exec* ex) {
  if (!ctx || !ex) return fail(TP_ERR_INVALID, "null argument");
  if (limit_ns < 1000 || limit_ns > 2000000000) return fail(TP_ERR_INVALID, "limit_ns must be in [1e3, 2e9]");
  Op o(__func__);
  tp_status s = o.begin(ctx, ex, {}, {});
  if (s != TP_OK) return s;
  o.check_err = true;
  bounded_wait_kernel<<<1, 32, 0, o.stream>>>(ctx->d_err, (uint64_t)limit_ns, arrive != 0);
  return o.end(cudaGetLastError());
}
