/*
 * FP64 CPU oracle for the FREDEC periodogram hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; only the tests, the package smoke check and the bench's
 * CPU-baseline leg do.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * Every quantity is computed from its plain definition: for each model the
 * design matrix is built explicitly and the weighted least-squares problem is
 * solved by Householder QR (no normal equations, no Cholesky, no reuse between
 * frequencies).  Single-threaded, double precision throughout.
 *
 * Definitions followed (Baluev, "FREDEC", Section 2 and Section 3):
 *   data x_i at times t_i with weights w_i = 1/sigma_i^2             (Sect. 2)
 *   <phi> = sum_i w_i phi(t_i)                                        (Sect. 2)
 *   chi2(theta, f) = <(x - mu)^2>                                     (Sect. 2)
 *   H_n : mu = c + sum_k a_k cos(2 pi f_k t) + b_k sin(2 pi f_k t)    (Eq. Hn)
 *   l_n(f) = min_theta chi2                                           (Sect. 2)
 *   relative statistic with base frequencies f' held fixed and joint linear
 *   refit (Eq. zpowrel): here in the known-noise difference form
 *       z(f) = ( l(f') - l(f', f) ) / 2
 *   local refinement of the frequencies (Sect. 3, Eq. lsqf): Gauss-Newton
 *   on f with the linear parameters refitted at every step.
 *
 * Column dropping: a column whose norm after the previous reflections is at
 * most ORACLE_DROPTOL times its own original norm is treated as linearly
 * dependent and left out (the residual is then the minimum-norm least-squares
 * residual).  The paper is silent on degenerate columns (f = 0, f equal to a
 * base frequency); this is the reading taken.
 *
 * Parity pins: every function is pinned by tests that use an independent
 * route (closed forms, library least squares, invariants, finite differences,
 * an independent nonlinear solver); see the "not gpu" tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_DROPTOL 1e-7

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0   /* 0 = correct oracle; >0 plants one known mistake (tests only) */
#endif

static const double TWO_PI = 6.283185307179586476925286766559;

/* sin and cos of 2*pi*f*t.  The product f*t is split into its rounded value and
 * its exact rounding error (fma), the nearest integer number of turns is removed
 * (exactly), and libm is called on the remaining angle in [-pi, pi]. */
static void trig(double f, double t, double *c, double *s)
{
    double x = f * t;
    double e = fma(f, t, -x);
    double r = (x - nearbyint(x)) + e;
#if ORACLE_MUTANT == 2
    r = -r;    /* planted: wrong sign of the phase of every column */
#endif
    double a = TWO_PI * r;
    *c = cos(a);
    *s = sin(a);
}

static double weight(double sigma)
{
#if ORACLE_MUTANT == 1
    (void)sigma;
    return 1.0;   /* planted: weights ignored */
#else
    return 1.0 / (sigma * sigma);
#endif
}

/*
 * Householder QR least squares (Golub & Van Loan, Sect. 5.1-5.3), no pivoting.
 *   A : N x m, column-major (leading dimension N); overwritten.
 *   b : N; overwritten by Q^T b.
 *   x : m coefficients (0 for dropped columns), may be NULL.
 *   ratio : m, remaining-norm / original-norm of each column when it was
 *           processed (1 = orthogonal to the previous ones), may be NULL.
 *   comp : m, the squared component of Q^T b along the orthonormal direction
 *          that column k adds (0 for a dropped column), may be NULL.  Adding
 *          column k to the model lowers the residual sum of squares by exactly
 *          comp[k], so a difference of two nested fits is a sum of comp[]
 *          entries; summing them avoids subtracting two large chi2 values.
 * Returns the residual sum of squares min_x ||b - A x||^2.
 */
static double hh_lsq(double *A, double *b, int64_t N, int m, double *x, double *ratio, double *comp)
{
    double orig[128];
    int rowof[128];
    int64_t r = 0;
    for (int k = 0; k < m; ++k) {
        double s = 0.0;
        const double *a = A + (size_t)k * N;
        for (int64_t i = 0; i < N; ++i) s += a[i] * a[i];
        orig[k] = sqrt(s);
    }
    for (int k = 0; k < m; ++k) {
        double *a = A + (size_t)k * N;
        double s = 0.0;
        for (int64_t i = r; i < N; ++i) s += a[i] * a[i];
        double sig = sqrt(s);
        double rat = orig[k] > 0.0 ? sig / orig[k] : 0.0;
        if (ratio) ratio[k] = rat;
        if (r >= N || orig[k] == 0.0 || rat <= ORACLE_DROPTOL) {
            rowof[k] = -1;
            if (comp) comp[k] = 0.0;
            continue;
        }
        double x0 = a[r];
        double alpha = x0 >= 0.0 ? -sig : sig;
        double v0 = x0 - alpha;
        double vtv = 2.0 * sig * (sig + fabs(x0));
        double beta = 2.0 / vtv;
        /* v = (v0, a[r+1..N-1]) ; apply H = I - beta v v^T to later columns and b */
        for (int j = k + 1; j <= m; ++j) {
            double *c = (j < m) ? A + (size_t)j * N : b;
            double d = v0 * c[r];
            for (int64_t i = r + 1; i < N; ++i) d += a[i] * c[i];
            d *= beta;
            c[r] -= d * v0;
            for (int64_t i = r + 1; i < N; ++i) c[i] -= d * a[i];
        }
        a[r] = alpha;
        /* keep v below the diagonal is not needed: only R and Q^T b are used */
        if (comp) comp[k] = b[r] * b[r];
        rowof[k] = (int)r;
        ++r;
    }
    double chi2 = 0.0;
    for (int64_t i = r; i < N; ++i) chi2 += b[i] * b[i];
    if (x) {
        for (int k = m - 1; k >= 0; --k) {
            if (rowof[k] < 0) { x[k] = 0.0; continue; }
            int64_t rk = rowof[k];
            double acc = b[rk];
            for (int j = k + 1; j < m; ++j)
                if (rowof[j] >= 0) acc -= A[(size_t)j * N + rk] * x[j];
            x[k] = acc / A[(size_t)k * N + rk];
        }
    }
    return chi2;
}

/* Fill the weighted design matrix of the model
 *   [1, cos 2pi g_0 t, sin 2pi g_0 t, ..., cos 2pi g_{n-1} t, sin 2pi g_{n-1} t]
 * (Eq. Hn) scaled row-wise by sqrt(w_i), and b = sqrt(w_i) x_i. */
static void design(const double *t, const double *y, const double *sigma, int64_t N,
                   const double *g, int n, double *A, double *b)
{
    for (int64_t i = 0; i < N; ++i) {
        double sw = sqrt(weight(sigma[i]));
#if ORACLE_MUTANT == 3
        A[i] = 0.0;   /* planted: the free constant c of Eq. H0 is missing */
#else
        A[i] = sw;
#endif
        for (int k = 0; k < n; ++k) {
            double c, s;
            trig(g[k], t[i], &c, &s);
            A[(size_t)(1 + 2 * k) * N + i] = sw * c;
            A[(size_t)(2 + 2 * k) * N + i] = sw * s;
        }
        if (b) b[i] = sw * y[i];
    }
}

/* l(g) = min over the linear parameters of chi2 for the model with the n
 * frequencies g (Sect. 2).  Optional: coefficients theta (2n+1, order
 * [c, a_0, b_0, a_1, b_1, ...]), the unweighted residual x_i - mu(t_i) and
 * the per-column chi2 reductions comp (see hh_lsq). */
static double model_fit(const double *t, const double *y, const double *sigma, int64_t N,
                        const double *g, int n, double *theta, double *ratio, double *resid, double *comp)
{
    int m = 2 * n + 1;
    double *A = (double *)malloc(sizeof(double) * (size_t)N * m);
    double *b = (double *)malloc(sizeof(double) * (size_t)N);
    double th[128];
    design(t, y, sigma, N, g, n, A, b);
    double chi2 = hh_lsq(A, b, N, m, th, ratio, comp);
    if (theta) memcpy(theta, th, sizeof(double) * m);
    if (resid) {
        for (int64_t i = 0; i < N; ++i) {
            double mu = th[0];
            for (int k = 0; k < n; ++k) {
                double c, s;
                trig(g[k], t[i], &c, &s);
                mu += th[1 + 2 * k] * c + th[2 + 2 * k] * s;
            }
            resid[i] = y[i] - mu;
        }
    }
    free(A);
    free(b);
    return chi2;
}

/* ------------------------------------------------------------------------- */
/* Residual periodogram (Eq. zpowrel, difference form).                       */

/*
 * For every trial frequency f_j the model [base model, cos 2pi f_j t,
 * sin 2pi f_j t] is fitted jointly (the base amplitudes are refitted; the base
 * frequencies stay fixed) and
 *     z_j = ( chi2_base - chi2_j ) / 2 .
 * The QR of [base | trial] starts with the base columns, so chi2_base - chi2_j
 * equals the sum of the two trial columns' comp[] terms; that sum is what is
 * returned (same quantity, without cancelling two large chi2 values).
 * Outputs: z (nf); chi2_base (1) may be NULL; coef (2*nf: a_j, b_j, the
 * coefficients of cos and sin of the trial frequency in raw time t) may be
 * NULL; ratio (nf: min over the two trial columns of remaining/original norm)
 * may be NULL.
 */
int oracle_periodogram(const double *t, const double *y, const double *sigma, int64_t N,
                       const double *base, int n_base, const double *fgrid, int64_t nf,
                       double *z, double *chi2_base, double *coef, double *ratio)
{
    if (N <= 0 || n_base < 0 || n_base > 40 || nf < 0) return 1;
    double *g = (double *)malloc(sizeof(double) * (n_base + 1));
    for (int k = 0; k < n_base; ++k) g[k] = base[k];
    double l0 = model_fit(t, y, sigma, N, g, n_base, NULL, NULL, NULL, NULL);
    if (chi2_base) *chi2_base = l0;
    double th[128], rat[128], comp[128];
    for (int64_t j = 0; j < nf; ++j) {
        g[n_base] = fgrid[j];
        model_fit(t, y, sigma, N, g, n_base + 1, th, rat, NULL, comp);
        z[j] = 0.5 * (comp[2 * n_base + 1] + comp[2 * n_base + 2]);
        if (coef) {
            coef[2 * j] = th[2 * n_base + 1];
            coef[2 * j + 1] = th[2 * n_base + 2];
        }
        if (ratio) {
            double a = rat[2 * n_base + 1], bb = rat[2 * n_base + 2];
            ratio[j] = a < bb ? a : bb;
        }
    }
    free(g);
    return 0;
}

/*
 * dz/df_j for the residual periodogram.  By the envelope theorem (the linear
 * parameters are at their optimum) only the explicit frequency dependence of
 * the model matters:
 *     dz/df = -1/2 d chi2/df = sum_i w_i r_i dmu/df(t_i),
 *     dmu/df = 2 pi t (-a sin 2pi f t + b cos 2pi f t),
 * with r the residual of the full fit and (a, b) its coefficients at f.
 */
int oracle_periodogram_grad(const double *t, const double *y, const double *sigma, int64_t N,
                            const double *base, int n_base, const double *fgrid, int64_t nf,
                            double *dzdf)
{
    if (N <= 0 || n_base < 0 || n_base > 40 || nf < 0) return 1;
    double *g = (double *)malloc(sizeof(double) * (n_base + 1));
    double *r = (double *)malloc(sizeof(double) * (size_t)N);
    double th[128];
    for (int k = 0; k < n_base; ++k) g[k] = base[k];
    for (int64_t j = 0; j < nf; ++j) {
        g[n_base] = fgrid[j];
        model_fit(t, y, sigma, N, g, n_base + 1, th, NULL, r, NULL);
        double a = th[2 * n_base + 1], b = th[2 * n_base + 2], acc = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            double c, s;
            trig(fgrid[j], t[i], &c, &s);
            acc += weight(sigma[i]) * r[i] * TWO_PI * t[i] * (-a * s + b * c);
        }
        dzdf[j] = acc;
    }
    free(g);
    free(r);
    return 0;
}

/*
 * Vector-Jacobian product of the periodogram with respect to the data:
 *     dL/dy_i = sum_j v_j dz_j/dy_i,   dz_j/dy_i = w_i ( mu_j(t_i) - mu_base(t_i) ),
 * (again the envelope theorem: d chi2/dy_i = 2 w_i r_i at the optimum), where
 * mu_j is the fitted model with trial frequency f_j and mu_base the base fit.
 */
int oracle_periodogram_vjp(const double *t, const double *y, const double *sigma, int64_t N,
                           const double *base, int n_base, const double *fgrid, int64_t nf,
                           const double *v, double *dldy)
{
    if (N <= 0 || n_base < 0 || n_base > 40 || nf < 0) return 1;
    double *g = (double *)malloc(sizeof(double) * (n_base + 1));
    double *rb = (double *)malloc(sizeof(double) * (size_t)N);
    double *r = (double *)malloc(sizeof(double) * (size_t)N);
    for (int k = 0; k < n_base; ++k) g[k] = base[k];
    model_fit(t, y, sigma, N, g, n_base, NULL, NULL, rb, NULL);
    for (int64_t i = 0; i < N; ++i) dldy[i] = 0.0;
    for (int64_t j = 0; j < nf; ++j) {
        if (v[j] == 0.0) continue;
        g[n_base] = fgrid[j];
        model_fit(t, y, sigma, N, g, n_base + 1, NULL, NULL, r, NULL);
        for (int64_t i = 0; i < N; ++i) dldy[i] += v[j] * (rb[i] - r[i]);   /* mu_j - mu_b */
    }
    for (int64_t i = 0; i < N; ++i) dldy[i] *= weight(sigma[i]);
    free(g);
    free(rb);
    free(r);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Frequency tuples on a constant base (Sect. 2, Phase 2 of Sect. 4).         */

/* l_0: chi2 of the constant-only model H_0 (Eq. H0). */
double oracle_l0(const double *t, const double *y, const double *sigma, int64_t N)
{
    return model_fit(t, y, sigma, N, NULL, 0, NULL, NULL, NULL, NULL);
}

/* l(S) for one tuple of m frequencies (model H_m, Eq. Hn). theta may be NULL. */
double oracle_tuple_l(const double *t, const double *y, const double *sigma, int64_t N,
                      const double *freqs, int m, double *theta)
{
    return model_fit(t, y, sigma, N, freqs, m, theta, NULL, NULL, NULL);
}

/* z(S) = (l_0 - l(S))/2 computed as half the sum of the comp[] terms of every
 * column after the constant (the QR starts with the constant column). */
static double tuple_z(const double *t, const double *y, const double *sigma, int64_t N,
                      const double *freqs, int m, double *theta, double *resid)
{
    double comp[128], z = 0.0;
    model_fit(t, y, sigma, N, freqs, m, theta, NULL, resid, comp);
    for (int k = 1; k < 2 * m + 1; ++k) z += comp[k];
    return 0.5 * z;
}

/*
 * Many tuples in CSR layout: tuple k holds freqs[off[k] .. off[k+1]).
 * z_k = (l_0 - l_k)/2.  l0_out may be NULL.
 */
int oracle_tuple_eval(const double *t, const double *y, const double *sigma, int64_t N,
                      const double *freqs, const int64_t *off, int64_t n_tuples,
                      double *z, double *l0_out)
{
    if (N <= 0 || n_tuples < 0) return 1;
    double l0 = oracle_l0(t, y, sigma, N);
    if (l0_out) *l0_out = l0;
    for (int64_t k = 0; k < n_tuples; ++k) {
        int m = (int)(off[k + 1] - off[k]);
        if (m < 0 || m > 60) return 1;
        z[k] = tuple_z(t, y, sigma, N, freqs + off[k], m, NULL, NULL);
    }
    return 0;
}

/*
 * All subtuples of a pool of n frequencies (Phase 2 forward cascade):
 * l_table[mask] = l of the tuple {pool[k] : bit k of mask set}, l_table[0] = l_0.
 */
int oracle_pool_table(const double *t, const double *y, const double *sigma, int64_t N,
                      const double *pool, int n, double *l_table)
{
    if (N <= 0 || n < 0 || n > 24) return 1;
    double g[64];
    for (uint64_t mask = 0; mask < (1ull << n); ++mask) {
        int m = 0;
        for (int k = 0; k < n; ++k)
            if (mask >> k & 1) g[m++] = pool[k];
        l_table[mask] = oracle_tuple_l(t, y, sigma, N, g, m, NULL);
    }
    return 0;
}

/*
 * z and its gradient for CSR tuples: dz/df_k = sum_i w_i r_i 2 pi t_i
 * (-a_k sin 2pi f_k t_i + b_k cos 2pi f_k t_i), r the residual of the tuple fit.
 */
int oracle_tuple_grad(const double *t, const double *y, const double *sigma, int64_t N,
                      const double *freqs, const int64_t *off, int64_t n_tuples,
                      double *z, double *dzdf)
{
    if (N <= 0 || n_tuples < 0) return 1;
    double *r = (double *)malloc(sizeof(double) * (size_t)N);
    double th[128];
    for (int64_t k = 0; k < n_tuples; ++k) {
        const double *g = freqs + off[k];
        int m = (int)(off[k + 1] - off[k]);
        z[k] = tuple_z(t, y, sigma, N, g, m, th, r);
        for (int q = 0; q < m; ++q) {
            double a = th[1 + 2 * q], b = th[2 + 2 * q], acc = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                double c, s;
                trig(g[q], t[i], &c, &s);
                acc += weight(sigma[i]) * r[i] * TWO_PI * t[i] * (-a * s + b * c);
            }
            dzdf[off[k] + q] = acc;
        }
    }
    free(r);
    return 0;
}

/*
 * Local refinement of one tuple (Sect. 3, Eq. lsqf): Gauss-Newton on the
 * frequencies.  Each iteration refits the linear parameters at the current f,
 * linearises the model in xi = (theta, f) with the frequency columns
 *     d mu / d f_k = 2 pi t (-a_k sin 2pi f_k t + b_k cos 2pi f_k t),
 * solves the linear least-squares step for (dtheta, df) by QR, and moves f by
 * df.  If the step does not lower chi2 it is halved (up to 40 times).
 * Stops when max_k |df_k| * span(t) < tol or after max_iter iterations; the
 * final l is the chi2 of the linear refit at the final f.
 * freqs is updated in place.  Returns the number of iterations (>= 0) or -1.
 */
int oracle_tuple_refine(const double *t, const double *y, const double *sigma, int64_t N,
                        double *freqs, int m, int max_iter, double tol, double *l_out)
{
    if (N <= 0 || m < 0 || m > 40) return -1;
    int p = 2 * m + 1, q = 3 * m + 1;
    double th[256], xi[256];
    double *r = (double *)malloc(sizeof(double) * (size_t)N);
    double *J = (double *)malloc(sizeof(double) * (size_t)N * q);
    double *rb = (double *)malloc(sizeof(double) * (size_t)N);
    double *trial = (double *)malloc(sizeof(double) * (m + 1));
    double tmin = t[0], tmax = t[0];
    for (int64_t i = 0; i < N; ++i) { if (t[i] < tmin) tmin = t[i]; if (t[i] > tmax) tmax = t[i]; }
    double span = tmax - tmin > 0 ? tmax - tmin : 1.0;
    double l = model_fit(t, y, sigma, N, freqs, m, th, NULL, r, NULL);
    int it = 0;
    for (; it < max_iter && m > 0; ++it) {
        design(t, y, sigma, N, freqs, m, J, NULL);
        for (int k = 0; k < m; ++k) {
            double a = th[1 + 2 * k], b = th[2 + 2 * k];
            for (int64_t i = 0; i < N; ++i) {
                double c, s;
                trig(freqs[k], t[i], &c, &s);
                J[(size_t)(p + k) * N + i] = sqrt(weight(sigma[i])) * TWO_PI * t[i] * (-a * s + b * c);
            }
        }
        for (int64_t i = 0; i < N; ++i) rb[i] = sqrt(weight(sigma[i])) * r[i];
        hh_lsq(J, rb, N, q, xi, NULL, NULL);
        double step = 1.0, dmax = 0.0, lnew = l;
        for (int k = 0; k < m; ++k) if (fabs(xi[p + k]) > dmax) dmax = fabs(xi[p + k]);
        int accepted = 0;
        for (int h = 0; h < 40; ++h, step *= 0.5) {
            for (int k = 0; k < m; ++k) trial[k] = freqs[k] + step * xi[p + k];
            lnew = model_fit(t, y, sigma, N, trial, m, NULL, NULL, NULL, NULL);
            if (lnew <= l) { accepted = 1; break; }
        }
        if (!accepted) break;
        for (int k = 0; k < m; ++k) freqs[k] = trial[k];
        l = model_fit(t, y, sigma, N, freqs, m, th, NULL, r, NULL);
        if (step * dmax * span < tol) { ++it; break; }
    }
    if (l_out) *l_out = l;
    free(r); free(J); free(rb); free(trial);
    return it;
}

/* ------------------------------------------------------------------------- */
/* Phase 3 backward cascade and the non-nested solutions (Sect. 4).          */

/*
 * FAP bound of Eq. zFAP for n frequencies: M_n(z) = A W^n exp(-z) z^(3n/2 - 1).
 * The coefficients A (the paper's A~_n) are not given in the paper; the caller
 * supplies them.  W = f_max T_eff is the normalised bandwidth (Sect. 2).
 */
double oracle_fap_bound(int n, double A, double W, double z)
{
    if (n < 1 || !(z > 0.0)) return NAN;
    return A * pow(W, n) * exp(-z) * pow(z, 1.5 * n - 1.0);
}

/*
 * The z at which M_n(z) falls to fap, on the branch where M_n decreases
 * (z above 3n/2 - 1, the maximum of the z-dependent factor).  Plain bisection
 * on log M_n(z) - log fap.  Returns the bracket's lower end when M_n never
 * exceeds fap there (every z passes).
 */
double oracle_fap_threshold(int n, double A, double W, double fap)
{
    if (n < 1 || !(A > 0.0) || !(W > 0.0) || !(fap > 0.0)) return NAN;
    double a = 1.5 * n - 1.0;
    double lo = a > 0.0 ? a : 1e-300;
    double target = log(fap);
#define LOGM(z) (log(A) + n * log(W) - (z) + a * log(z))
    if (LOGM(lo) <= target) return lo;
    double hi = lo + 1.0;
    while (LOGM(hi) > target) hi = 2.0 * hi + 1.0;
    for (int it = 0; it < 400 && hi - lo > 1e-15 * hi; ++it) {
        double mid = 0.5 * (lo + hi);
        if (LOGM(mid) > target) lo = mid; else hi = mid;
    }
#undef LOGM
    return 0.5 * (lo + hi);
}

static int popcount_u64(uint64_t x)
{
    int c = 0;
    for (; x; x &= x - 1) ++c;
    return c;
}

/*
 * Phase 3 (backward cascade).  l[mask] (2^n entries) holds the minimised chi2
 * of the subtuple {pool[j] : bit j of mask}; l[0] = l_0.  For a combination S
 * with m members and a proper subset K of S with k members (0 <= k < m), the
 * relative statistic of Eq. zpowrel in its log form, base K and alternative S,
 * is
 *     z(S\K | K) = (N - 3m - 1)/2 * ln( l[K] / l[S] ).
 * The tests of S are grouped in layers of equal k; a layer passes when its
 * smallest z reaches zthr[m-k-1], the threshold for m-k added frequencies
 * (FAP thresholds depend only on the number of added frequencies, Eq. zFAP).
 * S passes when all its layers pass.  A test with a negative or NaN l, or a
 * NaN ratio, fails; S fails when N - 3m - 1 <= 0.
 * Outputs: pass[S] (0/1), slack[S] = smallest (layer minimum - threshold)
 * over the layers of S (-INFINITY when a test fails outright; pass[S] is
 * slack[S] >= 0).  n_tests (may be NULL) receives the number of tests formed;
 * every K of every S is formed, so it is 3^n - 2^n when N is large enough.
 */
int oracle_cascade(const double *l, int n, int64_t N, const double *zthr,
                   unsigned char *pass, double *slack, int64_t *n_tests)
{
    if (n < 0 || n > 24 || N <= 0) return 1;
    uint64_t full = (1ull << n);
    int64_t tests = 0;
    double zmin[32];
    pass[0] = 0;
    slack[0] = -INFINITY;
    for (uint64_t S = 1; S < full; ++S) {
        int m = popcount_u64(S);
#if ORACLE_MUTANT == 4
        double NH = (double)(N - 3 * (int64_t)(m - 1) - 1);   /* planted: base model's N_H */
#else
        double NH = (double)(N - 3 * (int64_t)m - 1);
#endif
        for (int k = 0; k < m; ++k) zmin[k] = INFINITY;
        int bad = !(NH > 0.0) || !(l[S] >= 0.0);
        /* every proper subset K of S, visited once */
        for (uint64_t K = (S - 1) & S;; K = (K - 1) & S) {
            int k = popcount_u64(K);
            double z;
            ++tests;
            if (!(l[K] >= 0.0)) z = -INFINITY;
            else {
                z = 0.5 * NH * log(l[K] / l[S]);
                if (isnan(z)) z = -INFINITY;
            }
            if (z < zmin[k]) zmin[k] = z;
            if (K == 0) break;
        }
        double sl = INFINITY;
        for (int k = 0; k < m; ++k) {
            double d = zmin[k] - zthr[m - k - 1];
            if (isnan(d)) d = -INFINITY;
            if (d < sl) sl = d;
        }
        if (bad) sl = -INFINITY;
        slack[S] = sl;
        pass[S] = sl >= 0.0;
    }
    if (n_tests) *n_tests = tests;
    return 0;
}

/*
 * Non-nested solutions of Phase 3: the passing combinations that no other
 * passing combination contains (the output never holds nested tuples,
 * Sect. 4, Phase 4).  Writes up to cap masks in increasing mask order and
 * returns how many there are.
 */
int64_t oracle_cascade_solutions(const unsigned char *pass, int n, uint32_t *out, int64_t cap)
{
    if (n < 0 || n > 24) return -1;
    uint64_t full = (1ull << n) - 1;
    int64_t count = 0;
    for (uint64_t S = 1; S <= full; ++S) {
        if (!pass[S]) continue;
        uint64_t rest = full & ~S;
        int maximal = 1;
        for (uint64_t T = rest; T && maximal; T = (T - 1) & rest)
            if (pass[S | T]) maximal = 0;
        if (maximal) {
            if (count < cap) out[count] = (uint32_t)S;
            ++count;
        }
    }
    return count;
}

/* ------------------------------------------------------------------------- */
/* Polynomial-trend base model (Sect. 2: the constant of Eq. H0 extended to  */
/* a polynomial in time).                                                     */

/*
 * Residual periodogram with the base model
 *     mu_b(t) = sum_{d=0..ntrend} c_d tau^d + sum_k (a_k cos 2pi g_k t + b_k sin 2pi g_k t),
 * tau = (t - mean(t)) / half-span (any affine map of t spans the same
 * columns; this one keeps the powers of order one).  For every f_j the base
 * and the trial pair are fitted jointly by Householder QR and
 *     z_j = (chi2_base - chi2_j)/2
 * is the sum of the trial columns' comp[] terms, as in oracle_periodogram.
 * chi2_base and ratio (min over the trial columns of remaining/original
 * norm) may be NULL.
 */
int oracle_periodogram_trend(const double *t, const double *y, const double *sigma, int64_t N,
                             const double *base, int n_base, int ntrend, const double *fgrid, int64_t nf,
                             double *z, double *chi2_base, double *ratio)
{
    if (N <= 0 || n_base < 0 || n_base > 40 || ntrend < 0 || ntrend > 8 || nf < 0) return 1;
    int pb = 1 + ntrend + 2 * n_base, m = pb + 2;
    double tmin = t[0], tmax = t[0], tmean = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        if (t[i] < tmin) tmin = t[i];
        if (t[i] > tmax) tmax = t[i];
        tmean += t[i];
    }
    tmean /= (double)N;
    double half = 0.5 * (tmax - tmin) > 0 ? 0.5 * (tmax - tmin) : 1.0;
    double *A = (double *)malloc(sizeof(double) * (size_t)N * m);
    double *b = (double *)malloc(sizeof(double) * (size_t)N);
    double th[160], comp[160], rat[160];
    /* base columns (fixed for all trial frequencies) */
    for (int64_t i = 0; i < N; ++i) {
        double sw = sqrt(weight(sigma[i])), tau = (t[i] - tmean) / half, pw = 1.0;
        for (int d = 0; d <= ntrend; ++d) {
            A[(size_t)d * N + i] = sw * pw;
            pw *= tau;
        }
        for (int k = 0; k < n_base; ++k) {
            double c, s;
            trig(base[k], t[i], &c, &s);
            A[(size_t)(1 + ntrend + 2 * k) * N + i] = sw * c;
            A[(size_t)(2 + ntrend + 2 * k) * N + i] = sw * s;
        }
        b[i] = sw * y[i];
    }
    double *Ab = (double *)malloc(sizeof(double) * (size_t)N * m);
    double *bb = (double *)malloc(sizeof(double) * (size_t)N);
    memcpy(Ab, A, sizeof(double) * (size_t)N * pb);
    memcpy(bb, b, sizeof(double) * (size_t)N);
    double l0 = hh_lsq(Ab, bb, N, pb, th, NULL, NULL);
    if (chi2_base) *chi2_base = l0;
    for (int64_t j = 0; j < nf; ++j) {
        memcpy(Ab, A, sizeof(double) * (size_t)N * pb);
        memcpy(bb, b, sizeof(double) * (size_t)N);
        for (int64_t i = 0; i < N; ++i) {
            double sw = sqrt(weight(sigma[i])), c, s;
            trig(fgrid[j], t[i], &c, &s);
            Ab[(size_t)pb * N + i] = sw * c;
            Ab[(size_t)(pb + 1) * N + i] = sw * s;
        }
        hh_lsq(Ab, bb, N, m, th, rat, comp);
        z[j] = 0.5 * (comp[pb] + comp[pb + 1]);
        if (ratio) ratio[j] = rat[pb] < rat[pb + 1] ? rat[pb] : rat[pb + 1];
    }
    free(A); free(b); free(Ab); free(bb);
    return 0;
}
