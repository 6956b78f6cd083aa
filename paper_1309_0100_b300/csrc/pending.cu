// Entry points whose kernels are not built yet: they fail loudly.
#include "fredec_internal.cuh"

using namespace fredec;

extern "C" {
int fredec_periodogram_batch(const double *, const double *, const double *, const int64_t *, int64_t,
                             const double *, const int64_t *, const double *, const double *, const int64_t *,
                             const int64_t *, const fredec_opts *, double *, int64_t *) {
    return fail(FREDEC_EINVAL, "fredec_periodogram_batch: not available in this build");
}
int fredec_batch_plan_create(fredec_batch_plan **, const double *, const double *, const double *, const int64_t *,
                             int64_t, const double *, const int64_t *, const double *, const double *,
                             const int64_t *, const int64_t *, const fredec_opts *) {
    return fail(FREDEC_EINVAL, "fredec_batch_plan_create: not available in this build");
}
int fredec_batch_plan_run(fredec_batch_plan *, void *) { return fail(FREDEC_EINVAL, "no plan"); }
int fredec_batch_plan_outputs(fredec_batch_plan *, double **, int64_t **, int64_t *, int64_t *) {
    return fail(FREDEC_EINVAL, "no plan");
}
int fredec_batch_plan_download(fredec_batch_plan *, double *, int64_t *) { return fail(FREDEC_EINVAL, "no plan"); }
void fredec_batch_plan_destroy(fredec_batch_plan *) {}
}
