// surrogate.cu -- learned surrogate that seeds the search (placeholder until
// the MLP kernels land).
#include "runtime.h"

namespace opmm {

struct SurrogateState {};

void surrogate_release(opmm_ctx* ctx) {
  delete ctx->surrogate;
  ctx->surrogate = nullptr;
}

Status surrogate_prepare_plan(opmm_ctx* ctx, opmm_plan*, const opmm_saccade*, int32_t) {
  if (!ctx->surrogate) return Status(OPMM_EINVAL, "use_surrogate set but no surrogate is loaded");
  return Status(OPMM_EINVAL, "surrogate not available");
}

}  // namespace opmm
