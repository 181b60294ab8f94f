// C ABI of the batched projector, transpose and solver (batch.cu kernels).
#include "batch.cuh"
#include "host.h"

namespace tomo {
namespace host {

struct BatchPlan {
    int unused = 0;
};

void free_plan(tomo_ctx *ctx)
{
    if (ctx->plan) {
        delete ctx->plan;
        ctx->plan = nullptr;
    }
}

}  // namespace host
}  // namespace tomo
