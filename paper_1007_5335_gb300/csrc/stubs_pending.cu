// Entry points whose implementation is still being written.
#include "mh_internal.cuh"

#define PENDING(ctx) return mh_fail((ctx), MH_ERR_INVALID_ARG, "%s: not implemented yet", __func__)

void volume_free(mh_tree*) {}
extern "C" mh_status mh_volume_potential(mh_ctx* ctx, mh_tree*, double, int, const double*, double*, mh_precision) { PENDING(ctx); }
extern "C" mh_status mh_problem_create(mh_ctx* ctx, mh_tree*, mh_boundary*, double, int, int, const double*, mh_problem**) { PENDING(ctx); }
extern "C" mh_status mh_problem_destroy(mh_problem*) { return MH_OK; }
extern "C" mh_status mh_problem_regions(mh_ctx* ctx, const mh_problem*, int32_t*) { PENDING(ctx); }
extern "C" mh_status heat_step(mh_ctx* ctx, mh_problem*, const double*, const double*, const double*, const double*, double*, double*, double, mh_precision, mh_step_info*) { PENDING(ctx); }
