// Entry points whose kernels are not built yet: they fail loudly.
#include "fredec_internal.cuh"

using namespace fredec;

extern "C" {
int fredec_periodogram_vjp_dev(const double *, const double *, const double *, int64_t, const double *, int32_t,
                               double, double, int64_t, const double *, const double *, const double *, int32_t,
                               double *, void *) {
    return fail(FREDEC_EINVAL, "fredec_periodogram_vjp_dev: not available in this build");
}
int fredec_periodogram_vjp(const double *, const double *, const double *, int64_t, const double *, int32_t, double,
                           double, int64_t, const double *, int32_t, double *) {
    return fail(FREDEC_EINVAL, "fredec_periodogram_vjp: not available in this build");
}
int fredec_tuple_eval(const double *, const double *, const double *, int64_t, const double *, const int64_t *,
                      int64_t, double *, double *) {
    return fail(FREDEC_EINVAL, "fredec_tuple_eval: not available in this build");
}
int fredec_pool_subtuples_eval(const double *, const double *, const double *, int64_t, const double *, int32_t,
                               double *) {
    return fail(FREDEC_EINVAL, "fredec_pool_subtuples_eval: not available in this build");
}
int fredec_tuple_grad(const double *, const double *, const double *, int64_t, const double *, const int64_t *,
                      int64_t, int32_t, double *, double *) {
    return fail(FREDEC_EINVAL, "fredec_tuple_grad: not available in this build");
}
int fredec_tuple_refine(const double *, const double *, const double *, int64_t, double *, const int64_t *, int64_t,
                        int32_t, double, int32_t, double *, int32_t *) {
    return fail(FREDEC_EINVAL, "fredec_tuple_refine: not available in this build");
}
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
