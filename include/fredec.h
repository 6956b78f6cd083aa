/*
 * fredec.h -- C ABI of the B300 (sm_103a) FREDEC hot-path library, libfredec.so.
 *
 * What it computes (Baluev, "Detecting multiple periodicities ... II. Frequency
 * Decomposer", Sections 2-5):
 *
 *   Data: N observations (t_i, y_i) with uncertainties sigma_i; weights
 *   w_i = 1/sigma_i^2 (Section 2: the noise variance is kappa/w_i).
 *   Weighted sum <phi> = sum_i w_i phi(t_i)  (Section 2).
 *   Model H_n (Eq. Hn): mu(t) = c + sum_k a_k cos(2 pi f_k t) + b_k sin(2 pi f_k t).
 *   l(f) = min over (c, a, b) of <(y - mu)^2>  (Section 2).
 *
 *   Residual periodogram (Eq. zpowrel with the base tuple f' held fixed and the
 *   base amplitudes refitted jointly), in the known-noise difference form:
 *       z(f) = ( l(f') - l(f', f) ) / 2 ,
 *   evaluated on a trial-frequency grid.  The base model is the constant plus
 *   n_base fixed sinusoids.  f is in cycles per unit of t (omega = 2 pi f).
 *
 *   Tuples on a constant base (Section 2 and Phase 2 of Section 4):
 *       z_S = ( l_0 - l(S) ) / 2   for a frequency tuple S, l_0 = l of H_0.
 *   Local refinement (Section 3, Eq. lsqf): Gauss-Newton steps in the
 *   frequencies with the linear parameters refitted at each step.
 *
 * Conventions shared by all entry points
 *   - Return value: a fredec_status.  On any error nothing is written to the
 *     outputs of the host-pointer variants, and fredec_last_error() returns a
 *     message (thread-local, valid until the next call on the same thread).
 *     One exception: when z_out of fredec_periodogram / _ex is page-locked
 *     host memory (cudaHostAlloc, cudaHostRegister), the precision mixed, the
 *     grid uniform and the statistic the difference form, the kernels write
 *     z into it during the computation instead of copying it afterwards; an
 *     error found only after the launch (a non-finite grid entry,
 *     FREDEC_ETIMEOUT) can then leave z_out partly written.
 *   - Ownership: the caller owns every buffer.  The library keeps no pointer
 *     after a call returns (plans are the documented exception).
 *   - Host-pointer variants are synchronous and validate all values.
 *   - _dev variants take device pointers and a CUDA stream (cudaStream_t passed
 *     as void*; NULL = the legacy default stream).  They are stream-ordered:
 *     they return after enqueueing work, and the caller keeps the buffers alive
 *     until the stream has completed.  Sizes are validated on the host; values
 *     (sigma > 0, finite data) are not read back -- invalid values give
 *     non-finite outputs, not an error code.  Scratch memory is taken from the
 *     stream-ordered allocator (cudaMallocAsync) on the same stream.
 *   - Precision: FREDEC_FP64 computes everything in double precision.
 *     FREDEC_MIXED keeps phases (as exact 64-bit fixed-point turns), the
 *     re-seeding of the sin/cos recurrence, the base fit and every solve in
 *     FP64, and accumulates the trigonometric sums in FP32 with blocked
 *     summation; bins whose 2x2 system is ill-conditioned are re-evaluated
 *     with FP64-grade accuracy in float-float arithmetic (pairs of FP32
 *     numbers, compensated sums) on the FP32 pipe (see fredec_opts.flag_tau).
 *   - Degenerate trial columns (f = 0, f equal to a base frequency): a new
 *     column whose norm after projection on the previous columns is below
 *     1e-7 of its own norm is dropped (minimum-norm least squares); z is then
 *     the contribution of the remaining column, or 0.
 */
#ifndef FREDEC_H
#define FREDEC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FREDEC_MAX_NBASE 12   /* base sinusoids (p = 2*n_base + 1 <= 25)          */
#define FREDEC_MAX_TUPLE 20   /* frequencies per tuple for eval/grad/refine       */
#define FREDEC_MAX_TREND  3   /* degree of the base model's time polynomial */
#define FREDEC_Z_DIFF     0   /* statistic: difference form (l_base - l_new)/2 */
#define FREDEC_Z_LOG      1   /* statistic: log form of Eq. zpowrel */
#define FREDEC_MAX_POOL  24   /* pool size for the all-subtuple table (2^24 rows) */
#define FREDEC_MAX_TOPK  64

typedef enum {
    FREDEC_OK = 0,
    FREDEC_EINVAL = 1,     /* bad sizes or values                                */
    FREDEC_ENOMEM = 2,     /* device allocation failed                           */
    FREDEC_ECUDA = 3,      /* a CUDA call failed (message has the CUDA error)    */
    FREDEC_ESINGULAR = 4,  /* the base model's normal matrix is singular         */
    FREDEC_ETIMEOUT = 5    /* a bounded device wait gave up                      */
} fredec_status;

enum { FREDEC_FP64 = 0, FREDEC_MIXED = 1 };

typedef struct fredec_opts {
    int32_t precision;  /* FREDEC_FP64 (default) or FREDEC_MIXED                   */
    int32_t topk;       /* number of local maxima of z to report, 0..64 (default 0) */
    int32_t fpt;        /* frequencies per thread; 0 = tuned or built-in default    */
    int32_t warps;      /* warps per CTA (point splits); 0 = tuned or default       */
    double  flag_tau;   /* MIXED: a bin is recomputed with FP64-grade accuracy
                           (float-float sums on the FP32 pipe) when a pivot of its
                           2x2 system falls below flag_tau times its column norm.
                           0 = default (0.2); negative = never recompute.             */
    int32_t trend;      /* degree of the time polynomial that replaces the constant
                           of the base model (Section 2 allows H_0 to be a
                           polynomial); 0..FREDEC_MAX_TREND, default 0.  The base
                           has 1 + trend + 2 n_base columns, at most 25.         */
    int32_t statistic;  /* FREDEC_Z_DIFF (default): z = (l_base - l_new)/2;
                           FREDEC_Z_LOG: the log form of Eq. zpowrel,
                           z = (N_H/2) ln(l_base / l_new),
                           N_H = N - 3 (n_base + 1) - 1 - trend.                  */
} fredec_opts;

/* Fill *o with the defaults (FP64, no top-k, tuned launch shape). */
void fredec_opts_init(fredec_opts *o);

/* ------------------------------------------------------------------------ */
/* Residual periodogram                                                      */

/*
 * z_out[j] = z(f_grid[j]) for j < nf, FP64, host pointers.
 *   t, y, sigma : N observations (sigma > 0, all finite), any time order.
 *   base_freqs  : n_base fixed base frequencies (0 <= n_base <= FREDEC_MAX_NBASE;
 *                 may be NULL when n_base == 0).  N must be >= 2*n_base + 3.
 *   f_grid      : nf >= 0 finite trial frequencies.  Uniform grids
 *                 (f_j = f_0 + j*df to 8 ulps) use the rotation recurrence;
 *                 other grids use a per-term phase (slower).
 * Errors: EINVAL (sizes/values), ESINGULAR (base normal matrix singular, e.g.
 * duplicate base frequencies), ENOMEM, ECUDA.
 */
int fredec_periodogram(const double *t, const double *y, const double *sigma, int64_t N,
                       const double *base_freqs, int32_t n_base,
                       const double *f_grid, int64_t nf, double *z_out);

/*
 * As fredec_periodogram with options and extra outputs (each may be NULL):
 *   info_out[3]   : chi2_base = l(f'), W = sum of weights, t_c = the time origin
 *                   used for the coefficients below.
 *   topk_idx_out  : opts->topk grid indices of the largest local maxima of z
 *                   (z_j > z_{j-1} and z_j >= z_{j+1}; an end point counts when it
 *                   exceeds its one neighbour), by decreasing z, ties to the lower
 *                   index; -1 where fewer maxima exist.
 *   coef_out[2nf] : (a_j, b_j), the fitted amplitudes of cos and sin of
 *                   2 pi f_j (t - t_c) in the joint fit (needed by the VJP).
 */
int fredec_periodogram_ex(const double *t, const double *y, const double *sigma, int64_t N,
                          const double *base_freqs, int32_t n_base,
                          const double *f_grid, int64_t nf, const fredec_opts *opts,
                          double *z_out, double *info_out, int64_t *topk_idx_out,
                          double *coef_out);

/*
 * Device-pointer, stream-ordered variant on the uniform grid f_j = f0 + j*df,
 * j = 0..nf-1.  All array arguments are device pointers (base_freqs too);
 * outputs as in fredec_periodogram_ex (info_out, topk_idx_out, coef_out may be
 * NULL).
 */
int fredec_periodogram_dev(const double *t, const double *y, const double *sigma, int64_t N,
                           const double *base_freqs, int32_t n_base,
                           double f0, double df, int64_t nf, const fredec_opts *opts,
                           double *z_out, double *info_out, int64_t *topk_idx_out,
                           double *coef_out, void *stream);

/*
 * Top-k local maxima of a device array z[0..nf): the peak step of the
 * periodogram calls on its own (the candidate frequencies of Sect. 4, Phase 1,
 * are the highest peaks of the residual periodogram), e.g. for a statistic
 * computed elsewhere.  A local maximum is z_j > z_{j-1} and z_j >= z_{j+1}; an
 * end point counts when it exceeds its one neighbour, a single point counts;
 * a NaN is never a maximum and disqualifies its neighbours.  idx_out[0..k)
 * receives the indices by decreasing z, ties to the lower index, -1 where
 * fewer maxima exist (all -1 for nf = 0).  z and idx_out are device pointers;
 * stream-ordered on stream (cudaStream_t as void*; NULL: the legacy default
 * stream); nothing is retained after return.  Errors (nothing written):
 * FREDEC_EINVAL for k outside 1..FREDEC_MAX_TOPK, nf < 0 or a NULL pointer
 * (z may be NULL when nf = 0); FREDEC_ENOMEM / FREDEC_ECUDA from the
 * stream-ordered scratch allocation or the launch.
 */
int fredec_topk_dev(const double *z, int64_t nf, int32_t k, int64_t *idx_out, void *stream);

/*
 * Vector-Jacobian product of the periodogram with respect to the data y
 * (the adjoint of the map y -> z on a fixed uniform grid):
 *   dldy_out[i] = sum_j v_j dz_j/dy_i = w_i sum_j v_j ( mu_j(t_i) - mu_base(t_i) ),
 * where mu_j is the fit with trial frequency f_j (envelope theorem: the linear
 * parameters are optimal, so only the explicit y dependence of chi2 counts).
 * coef and info are the coef_out / info_out of the forward call on the same
 * inputs (precision of the forward call).  Device pointers, stream-ordered.
 */
int fredec_periodogram_vjp_dev(const double *t, const double *y, const double *sigma, int64_t N,
                               const double *base_freqs, int32_t n_base,
                               double f0, double df, int64_t nf,
                               const double *coef, const double *info, const double *v,
                               int32_t precision, double *dldy_out, void *stream);

/*
 * Frequency derivative of the residual periodogram on the uniform grid
 * f_j = f0 + j*df, j < nf (Section 3: the derivatives of the model of Eq. Hn,
 * built from the t-weighted averages of Eq. avrg1), for the local maxima of
 * Section 2 (the local test z*_loc) refined straight off the periodogram:
 *   z_out[j]    = z(f_j) as fredec_periodogram_dev computes it;
 *   dzdf_out[j] = dz/df at f_j = sum_i w_i r_i 2 pi t_i (b_j cos 2 pi f_j t_i
 *                 - a_j sin 2 pi f_j t_i), r the residual of the joint fit at
 *                 f_j and (a_j, b_j) its coefficients of cos and sin (the
 *                 envelope theorem: the linear parameters are optimal); f in
 *                 cycles per unit of t.  dz/df does not depend on the time
 *                 origin.  Where a trial column is dropped (the degenerate
 *                 columns above) the coefficient of that column is 0.
 *   info_out[3] (may be NULL) as in fredec_periodogram_ex.
 * opts: precision and trend as for fredec_periodogram_dev; topk must be 0,
 * statistic FREDEC_Z_DIFF, fpt 0 (or the one compiled value: mixed 4 for up to
 * 7 base columns (p <= 7, trend columns included), 2 above; FP64 1).
 * One pass over the observations gives both outputs (2 (2p + 4) sums per
 * trial frequency); in mixed precision the flagged bins are re-evaluated in
 * float-float, dz/df included.
 * All array arguments are device pointers (base_freqs too), stream-ordered on
 * stream as the other _dev calls; z_out and dzdf_out are NaN when the base
 * fit fails or a bounded device wait gives up (nothing is read back).
 * Errors (nothing enqueued): FREDEC_EINVAL for the checks of
 * fredec_periodogram_dev and the options above; FREDEC_ENOMEM, FREDEC_ECUDA.
 */
int fredec_periodogram_grad_dev(const double *t, const double *y, const double *sigma, int64_t N,
                                const double *base_freqs, int32_t n_base,
                                double f0, double df, int64_t nf, const fredec_opts *opts,
                                double *z_out, double *dzdf_out, double *info_out, void *stream);

/*
 * Host-pointer variant of fredec_periodogram_grad_dev (synchronous; values
 * validated as for fredec_periodogram; FREDEC_ESINGULAR for a singular base
 * model, FREDEC_ETIMEOUT when a bounded device wait gave up).
 */
int fredec_periodogram_grad(const double *t, const double *y, const double *sigma, int64_t N,
                            const double *base_freqs, int32_t n_base,
                            double f0, double df, int64_t nf, const fredec_opts *opts,
                            double *z_out, double *dzdf_out, double *info_out);

/*
 * No-allocation variant of fredec_periodogram_dev (z and info only; the paper
 * has no counterpart).  For callers that cannot allocate device memory when
 * they call -- applications whose device memory is reserved up front by their
 * own allocator, real-time loops that forbid allocation after start-up,
 * plug-in hosts that keep extension code away from the CUDA allocator -- it
 * calls no allocator: all of its scratch lives in one 16 MiB device array
 * compiled into the library, held on every GPU that loads the library until
 * the process exits.
 *   - Same arguments, checks and results as fredec_periodogram_dev without
 *     top-k (opts->topk must be 0) and without coefficients.  Every argument
 *     is checked before anything is enqueued.
 *   - z_out is all NaN when the base fit fails (singular base model) or when
 *     a bounded device wait gives up (the status the other entry points
 *     report as FREDEC_ETIMEOUT); the call itself still returns FREDEC_OK,
 *     since nothing is read back.
 *   - Scratch needed, in bytes, with p = 1 + trend + 2*n_base rounded up to
 *     an odd number, c = ceil(N/32) and R(x) = x rounded up to a multiple of
 *     256:  6912 + R(4c) + R(8c(p(p+1)/2 + p + 4)) + R(8pN) + R(rN), with
 *     r = 8(6 + 2 ceil(p/2)) for FREDEC_FP64 and r = 4(8 + 4 ceil((p + 2)/4))
 *     for FREDEC_MIXED; FREDEC_MIXED with re-evaluation (flag_tau >= 0) adds
 *     R(16 ceil((8 + 2p)/4) N) + R(8 nf + 8).  A problem that does not fit
 *     in 16 MiB is rejected with FREDEC_EINVAL and a message giving the
 *     required and available byte counts.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Every call reuses the same array and clears what must start at zero;
 *     calls whose work overlaps on the GPU (unordered streams or threads) race
 *     on it and must be serialised by the caller.
 */
int fredec_periodogram_noalloc_dev(const double *t, const double *y, const double *sigma, int64_t N,
                                   const double *base_freqs, int32_t n_base,
                                   double f0, double df, int64_t nf, const fredec_opts *opts,
                                   double *z_out, double *info_out, void *stream);

/* Host-pointer variant of the VJP on a uniform grid (recomputes the forward). */
int fredec_periodogram_vjp(const double *t, const double *y, const double *sigma, int64_t N,
                           const double *base_freqs, int32_t n_base,
                           double f0, double df, int64_t nf, const double *v,
                           int32_t precision, double *dldy_out);

/* ------------------------------------------------------------------------ */
/* Frequency tuples on a constant base                                       */

/*
 * z_out[k] = (l_0 - l(S_k))/2 for n_tuples tuples in CSR layout: tuple k holds
 * tuple_freqs[tuple_offsets[k] .. tuple_offsets[k+1]) (0..FREDEC_MAX_TUPLE
 * frequencies; offsets nondecreasing, offsets[0] = 0).  l0_out (may be NULL)
 * receives l_0.  FP64 sums and solves.  Host pointers.
 */
int fredec_tuple_eval(const double *t, const double *y, const double *sigma, int64_t N,
                      const double *tuple_freqs, const int64_t *tuple_offsets, int64_t n_tuples,
                      double *z_out, double *l0_out);

/*
 * All 2^n_pool subtuples of a candidate pool (Phase 2, Section 4):
 * l_table[mask] = l of the tuple {pool[k] : bit k of mask}; l_table[0] = l_0.
 * n_pool <= FREDEC_MAX_POOL.  One FP64 Gram of the pool's 2 n_pool + 1 columns,
 * then one Cholesky per mask.  Host pointers.
 */
int fredec_pool_subtuples_eval(const double *t, const double *y, const double *sigma, int64_t N,
                               const double *pool, int32_t n_pool, double *l_table);

/*
 * z and its gradient with respect to the tuple frequencies (CSR layout as in
 * fredec_tuple_eval; Section 3, Eq. lsqf):
 *     dz/df_k = sum_i w_i r_i 2 pi t_i (-a_k sin + b_k cos),
 * r the residual of the tuple's fit.  dz_df_out has the layout of tuple_freqs.
 * precision: FREDEC_FP64 sums, or FREDEC_MIXED: the sums in float-float
 * arithmetic on the FP32 pipe (pairs of FP32 numbers, compensated; FP64-grade),
 * since plain FP32 Gram sums leave the gradient near 1e-4 relative.  Solves
 * are always FP64.  Host pointers, synchronous; FREDEC_ESINGULAR when a
 * tuple's normal matrix is singular (a repeated frequency).
 */
int fredec_tuple_grad(const double *t, const double *y, const double *sigma, int64_t N,
                      const double *tuple_freqs, const int64_t *tuple_offsets, int64_t n_tuples,
                      int32_t precision, double *z_out, double *dz_df_out);

/*
 * Device-pointer, stream-ordered variant of fredec_tuple_grad (the route of
 * the differentiable tuple statistic): t, y, sigma, tuple_freqs, z_out and
 * dz_df_out are device pointers; tuple_offsets (n_tuples + 1 entries) is a
 * host array, since it sizes the launch.  Sizes are checked on the host,
 * values are not read back: a tuple whose normal matrix is singular gets NaN
 * in z_out and in its dz_df_out entries.  Scratch from the stream-ordered
 * allocator on stream (cudaStream_t as void*; NULL: the legacy default
 * stream).  Errors (nothing enqueued): FREDEC_EINVAL, FREDEC_ENOMEM,
 * FREDEC_ECUDA.
 */
int fredec_tuple_grad_dev(const double *t, const double *y, const double *sigma, int64_t N,
                          const double *tuple_freqs, const int64_t *tuple_offsets, int64_t n_tuples,
                          int32_t precision, double *z_out, double *dz_df_out, void *stream);

/*
 * Local refinement of every tuple (Section 3): up to max_iter Gauss-Newton
 * steps on the frequencies, each solving the extended system of Eq. lsqf by
 * extending the Cholesky factor of the linear normal matrix; a step that does
 * not lower l is halved.  Stops when max_k |df_k| * span(t) < tol.
 * tuple_freqs (CSR as above) is updated in place; l_out[k] = l at the final
 * frequencies; iters_out[k] (may be NULL) = iterations used.
 */
int fredec_tuple_refine(const double *t, const double *y, const double *sigma, int64_t N,
                        double *tuple_freqs, const int64_t *tuple_offsets, int64_t n_tuples,
                        int32_t max_iter, double tol, int32_t precision,
                        double *l_out, int32_t *iters_out);

/*
 * Local refinement of subtuples of a candidate pool (Phase 2 of Section 4 with
 * the local fits of Section 3): masks[k] selects the pool frequencies of tuple
 * k (bit j = pool[j]); each tuple is refined as in fredec_tuple_refine,
 * starting from its pool frequencies.  f_out[k * n_pool + j] receives the
 * refined frequency of pool member j in tuple k (0 where bit j is clear);
 * l_out[k] the final l; iters_out[k] (may be NULL) the iterations.  The exact
 * cos/sin at the pool frequencies are computed once for all tuples.
 * n_pool <= FREDEC_MAX_TUPLE.
 */
int fredec_pool_refine(const double *t, const double *y, const double *sigma, int64_t N,
                       const double *pool, int32_t n_pool, const uint32_t *masks, int64_t n_masks,
                       int32_t max_iter, double tol, int32_t precision,
                       double *f_out, double *l_out, int32_t *iters_out);

/* ------------------------------------------------------------------------ */
/* Batched residual periodograms (many series, one persistent launch)        */

/*
 * n_series independent series in CSR layout (host pointers):
 *   observations of series s: t/y/sigma[obs_offsets[s] .. obs_offsets[s+1])
 *   base frequencies:          base_freqs[base_offsets[s] .. base_offsets[s+1])
 *   uniform grid:              f0[s] + j*df[s], j < nf[s]
 *   output:                    z_out[z_offsets[s] .. z_offsets[s] + nf[s])
 *   topk_idx_out (may be NULL): n_series * opts->topk indices.
 * All series go through one batched prep and one persistent periodogram
 * kernel with a device work queue.
 */
int fredec_periodogram_batch(const double *t, const double *y, const double *sigma,
                             const int64_t *obs_offsets, int64_t n_series,
                             const double *base_freqs, const int64_t *base_offsets,
                             const double *f0, const double *df, const int64_t *nf,
                             const int64_t *z_offsets, const fredec_opts *opts,
                             double *z_out, int64_t *topk_idx_out);

/*
 * A batch plan: device-resident inputs plus the captured CUDA graph of
 * prep -> persistent periodogram -> FP64-grade re-evaluation -> top-k.  The plan
 * copies the host inputs once (same layout as fredec_periodogram_batch) and
 * keeps them; run replays the graph on a stream and leaves z and top-k in
 * device buffers owned by the plan.
 */
typedef struct fredec_batch_plan fredec_batch_plan;

int fredec_batch_plan_create(fredec_batch_plan **plan,
                             const double *t, const double *y, const double *sigma,
                             const int64_t *obs_offsets, int64_t n_series,
                             const double *base_freqs, const int64_t *base_offsets,
                             const double *f0, const double *df, const int64_t *nf,
                             const int64_t *z_offsets, const fredec_opts *opts);
int fredec_batch_plan_run(fredec_batch_plan *plan, void *stream);
/* Device pointers to the plan's outputs (valid until destroy). */
int fredec_batch_plan_outputs(fredec_batch_plan *plan, double **z_dev, int64_t **topk_dev,
                              int64_t *z_total, int64_t *terms);
/* Copy the outputs to host buffers (synchronous). Either may be NULL.
 * FREDEC_ESINGULAR when a series' base model is singular, FREDEC_ETIMEOUT
 * when a bounded device wait of the last replay gave up. */
int fredec_batch_plan_download(fredec_batch_plan *plan, double *z_out, int64_t *topk_idx_out);
void fredec_batch_plan_destroy(fredec_batch_plan *plan);

/* ------------------------------------------------------------------------ */
/* Phase 3 backward cascade, Phase 4 ordering, FAP levels (Section 4)        */

/*
 * FAP bound of Eq. zFAP for an n-frequency test statistic z:
 *     M_n(z) = A W^n exp(-z) z^(3n/2 - 1).
 * The paper does not give its coefficients A~_n: the caller supplies A.
 * W = f_max T_eff is the normalised bandwidth (fredec_effective_bandwidth).
 * Returns NaN for n < 1 or non-positive A, W or z.  Host computation.
 */
double fredec_fap_bound(int32_t n, double A, double W, double z);

/*
 * The z at which M_n(z) falls to fap, on the branch where M_n decreases
 * (z > 3n/2 - 1); 3n/2 - 1 itself when M_n never exceeds fap there.  NaN for
 * n < 1 or non-positive A, W or fap.  Host computation.
 */
double fredec_fap_threshold(int32_t n, double A, double W, double fap);

/*
 * W = f_max * sqrt(4 pi Var(t)), Var the variance of t weighted by 1/sigma^2
 * (Section 2).  Host pointers, synchronous; one FP64 reduction kernel.
 * FREDEC_EINVAL for N < 2, f_max <= 0, non-finite t or sigma <= 0.
 */
int fredec_effective_bandwidth(const double *t, const double *sigma, int64_t N, double f_max,
                               double *W_out);

/*
 * Phase 3 (backward cascade) on a table of subtuple minima, and the order of
 * Phase 4 (Section 4).
 *   l_table[mask] (2^n_pool entries, host): the minimised chi2 of the subtuple
 *     {pool[j] : bit j of mask}; l_table[0] = l_0.  Typically the l_out of
 *     fredec_pool_refine over all masks, or fredec_pool_subtuples_eval.
 *   N: number of observations (N_H = N - 3m - 1 for m frequencies).
 *   z_thr[c-1], c = 1..n_pool: the threshold on the log-form statistic for c
 *     added frequencies (e.g. fredec_fap_threshold(c, A_c, W, FAP_2)).
 * For every combination S (m members) and proper subset K (k members) the
 * relative test of Eq. zpowrel, z(S\K | K) = (N - 3m - 1)/2 ln(l_K / l_S),
 * must reach z_thr[m-k-1]; S passes when all its 2^m - 1 tests do.  A test
 * whose l_K is not positive, or whose l_S is negative, infinite or NaN, fails;
 * S fails when N - 3m - 1 <= 0.
 * Outputs:
 *   pass_bits (may be NULL): max(1, 2^n_pool/32) words, bit (S mod 32) of
 *     word S/32 set when S passes;
 *   the solutions: passing combinations contained in no other passing
 *     combination, ordered by m, then by l, then by mask; the first
 *     min(count, capacity) go to solutions[] (masks) and G_out[] (goodness of
 *     fit G = (l_S / l_0) (N - 1)/(N - 3m - 1)); *n_solutions = count.
 * n_pool <= FREDEC_MAX_POOL.  Host pointers, synchronous.
 */
int fredec_cascade(const double *l_table, int32_t n_pool, int64_t N, const double *z_thr,
                   uint32_t *pass_bits, uint32_t *solutions, double *G_out, int64_t capacity,
                   int64_t *n_solutions);

/* ------------------------------------------------------------------------ */
/* The decomposition: Phase 1 scan and Phases 1-4 (Section 4)                */

typedef struct {
    int32_t precision;    /* FREDEC_FP64 (default) or FREDEC_MIXED periodograms */
    int32_t max_pool;     /* pool cap; 0: N/10; never above FREDEC_MAX_TUPLE */
    int32_t max_base;     /* base frequencies (SLICK rounds); 0: FREDEC_MAX_NBASE;
                             never above (N-3)/2 */
    int32_t reserved;
    double z_thr0;        /* the top peak joins the base while its z reaches this
                             (FAP_0 for one frequency) */
    double z_thr1;        /* other peaks join the pool from this z (FAP_1) */
    double half;          /* ... and from this fraction of the top peak's z (0.5) */
    double merge_dist;    /* candidates closer than this are one; 0: 0.5/(t_max-t_min) */
} fredec_scan_opts;

void fredec_scan_opts_init(fredec_scan_opts *o);   /* FP64, half = 0.5, rest 0 */

/*
 * Phase 1 (Section 4, SLICK and QUICK) on the uniform grid f0 + j df, j < nf.
 * Each round computes the residual periodogram of the current base; its
 * statistic is the log form of Eq. zpowrel for one added frequency,
 *     z = (N - 3(m+1) - 1)/2 ln(l_base / (l_base - 2 z_diff)),
 * m the base size.  Of the 64 highest local maxima (ranked as in top-k), the
 * top one joins the base and the pool while its z reaches z_thr0, else the
 * scan stops; the others join the pool when their z reaches z_thr1 and
 * half * (top z).  A candidate within merge_dist of a pool member replaces it
 * when its z is larger and is dropped otherwise.  The scan stops after
 * max_base rounds.  The pool is returned in decreasing z (ties to the lower
 * frequency), cut to max_pool (*truncated_out = 1 when candidates were cut).
 * Outputs (host): pool_out / pool_z_out (FREDEC_MAX_TUPLE entries; pool_z_out
 * may be NULL), base_out (FREDEC_MAX_NBASE entries, may be NULL), counts.
 * Host pointers, synchronous.
 */
int fredec_scan(const double *t, const double *y, const double *sigma, int64_t N,
                double f0, double df, int64_t nf, const fredec_scan_opts *opts,
                double *pool_out, double *pool_z_out, int32_t *n_pool_out,
                double *base_out, int32_t *n_base_out, int32_t *truncated_out);

typedef struct {
    fredec_scan_opts scan;      /* Phase 1 */
    const double *z_thr;        /* Phase 3 thresholds, z_thr[c-1] for c = 1..FREDEC_MAX_TUPLE
                                   added frequencies (FAP_2); required */
    int32_t refine_precision;   /* Phase 2 sums: FREDEC_FP64 (default) or FREDEC_MIXED */
    int32_t refine_iter;        /* Gauss-Newton steps per subtuple; 0: 20 */
    double refine_tol;          /* stop when max |df| * span(t) < tol; 0: 1e-9 */
} fredec_decompose_opts;

void fredec_decompose_opts_init(fredec_decompose_opts *o);

/*
 * The whole decomposition (Section 4): Phase 1 (fredec_scan); Phase 2, the
 * local fit of every non-empty subtuple of the pool starting from its pool
 * frequencies (fredec_pool_refine); Phase 3 (fredec_cascade) on the table of
 * fitted minima; Phase 4 ordering.  Outputs (host):
 *   pool_out (FREDEC_MAX_TUPLE), *n_pool_out = n;
 *   l_table_out (may be NULL; 2^n entries): the Phase 2 minima, entry 0 = l_0;
 *   the first min(count, capacity) solutions in Phase 4 order: solutions[]
 *     (masks over the pool), G_out[], freqs_out (may be NULL;
 *     capacity x FREDEC_MAX_TUPLE, row i = the fitted frequencies of solution
 *     i in increasing order, zero-padded), resid_z_out (may be NULL): the
 *     log-form z of the highest peak left in the residual periodogram whose
 *     base is the solution, on the scan's grid (its single-frequency FAP is
 *     the last item Section 4 reports per solution; NaN for solutions of more
 *     than FREDEC_MAX_NBASE frequencies); *n_solutions = count.
 * Host pointers, synchronous.
 */
int fredec_decompose(const double *t, const double *y, const double *sigma, int64_t N,
                     double f0, double df, int64_t nf, const fredec_decompose_opts *opts,
                     double *pool_out, int32_t *n_pool_out, double *l_table_out,
                     uint32_t *solutions, double *G_out, double *freqs_out, double *resid_z_out,
                     int64_t capacity, int64_t *n_solutions);

/* ------------------------------------------------------------------------ */
/* Launch-shape autotuner                                                    */

/*
 * Time the compiled launch shapes (frequencies per thread, warps per CTA) for a
 * periodogram with this base size, N and nf on synthetic inputs, and remember
 * the fastest for later calls with the same (precision, n_base, N bucket,
 * nf bucket).  If the environment variable FREDEC_TUNE_CACHE names a file,
 * the table is loaded from it at first use and rewritten after each tuning.
 * best_fpt / best_warps (may be NULL) receive the winner.
 */
int fredec_tune(int32_t precision, int32_t n_base, int64_t N, int64_t nf,
                int32_t *best_fpt, int32_t *best_warps);

/* ------------------------------------------------------------------------ */
/* Measurement support (no counterpart in the paper)                        */

/*
 * When both are non-NULL CUDA events (cudaEvent_t as void*), every following
 * periodogram call on this host thread records ev_start immediately before and
 * ev_stop immediately after its main periodogram kernel, on the call's stream;
 * NULL, NULL switches this off.  The library does not own the events.
 */
int fredec_profile_events(void *ev_start, void *ev_stop);

/*
 * Measured whole-GPU pipe rates of the current device (lane operations per
 * second): out[0] FP32 FMA, out[1] FP64 FMA, out[2] MUFU sine.  Synchronous;
 * runs three short microbenchmark kernels.
 */
int fredec_pipe_peaks(double *out);

/*
 * Failure-detection self-test (no counterpart in the paper): runs one bounded
 * device wait that nothing completes and stores the status the library's
 * kernels report in that case (FREDEC_ETIMEOUT) in *status_out.  Synchronous;
 * nothing faults or hangs.  Setting the environment variable
 * FREDEC_FAIL_ALLOC=1 makes every scratch allocation of the library report
 * FREDEC_ENOMEM (allocation-failure injection for tests).
 */
int fredec_selftest_wait_timeout(int32_t *status_out);

/*
 * Self-test of the float-float sin/cos used where FP64-grade values are
 * computed with FP32 instructions (the re-evaluation of ill-conditioned bins
 * and tuples; no counterpart in the paper): for each 64-bit fixed-point phase
 * (turns * 2^64) it compares the float-float sin and cos -- from the fixed-point
 * phase and from the phase given as a float-float number of turns -- with the
 * FP64 path's and stores the largest absolute difference in *max_err_out.  Host pointers,
 * synchronous.
 */
int fredec_selftest_ff_sincos(const uint64_t *phases, int64_t n, double *max_err_out);

/* ------------------------------------------------------------------------ */
const char *fredec_last_error(void);
const char *fredec_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FREDEC_H */
