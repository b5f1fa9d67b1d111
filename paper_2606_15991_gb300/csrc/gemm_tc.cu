// BF16 tensor-core GEMM (tcgen05 / TMEM / TMA) - placeholder until the kernel lands.
#include "tp_internal.h"

namespace tp {
tp_status launch_gemm_tc(tp_ctx*, tp_partition*, const tp_tensor*, const tp_tensor*,
                         const tp_gemm_config*, const tp_exec*, cudaStream_t, unsigned*) {
  return fail(TP_ERR_UNSUPPORTED, "BF16 tensor-core GEMM not built yet");
}
}  // namespace tp
