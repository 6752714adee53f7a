// Mixed-precision block log-likelihood (placeholder until the kernel lands).
#include "sbv_internal.cuh"

namespace sbv {
struct LoglikArgs;
int launch_loglik_mixed(sbv_ctx* ctx, const LoglikArgs&, int, cudaStream_t) {
  return fail(ctx, SBV_EUNSUPPORTED, "mixed precision path not built");
}
}  // namespace sbv
