// serve.cu -- continuous-batching request loop (placeholder).
#include "runtime.h"

namespace opmm {

struct ServeState {};

void serve_shutdown(opmm_ctx* ctx) {
  delete ctx->serve;
  ctx->serve = nullptr;
}

}  // namespace opmm
