// sched.cu -- plan choice for circuit runs without an explicit plan.
#include "common.cuh"

struct spdz_dag;

namespace spdz {

int scheduler_plan(spdz_ctx *ctx, spdz_dag *dag, spdz_plan *out) {
    (void)ctx; (void)dag; (void)out;
    return SPDZ_ERR_STATE;   // no tuned plan: the caller falls back to the fused default
}

}  // namespace spdz
