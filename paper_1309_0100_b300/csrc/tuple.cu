// Frequency tuples on a constant base (Section 2; Phase 2 of Section 4):
//   l(S)   = min over (c, a, b) of <(y - mu_S)^2>,  mu_S = c + sum_k a_k cos + b_k sin,
//   z_S    = (l_0 - l(S))/2,
//   dz/df_k = sum_i w_i r_i 2 pi t'_i (-a_k sin 2 pi f_k t'_i + b_k cos 2 pi f_k t'_i),
//   local refinement (Section 3, Eq. lsqf): Gauss-Newton on f with the linear
//   parameters refitted at every step.
//
// Linear fit as in Section 3: Gram Q = <phi phi^T>, g = <phi y>, Q = L L^T,
// a = L^{-1} g, theta = L^{-T} a; the chi2 reduction of the frequency columns
// is sum_{k>=1} a_k^2 (y is centred by its weighted mean, so the constant
// column carries a_0 = 0 and l_0 = <y^2>).  Refinement: with the derivative
// columns d_k = d mu / d f_k the extended normal matrix is [[Q, C], [C^T, D]]
// and its Cholesky factor extends L incrementally (Section 3):
//   X = L^{-1} C,  S = D - X^T X = L2 L2^T,  df = S^{-1} <d r>
// (the theta part of the gradient vanishes at the linear optimum).
//
// Every tuple frequency is an index into a pool of base frequencies f0_k whose
// FP64-exact cos/sin at every point are computed once; a tuple frequency
// f = f0_k + delta (delta = 0 unless refined) is obtained with the small-angle
// rotation e^{i 2 pi delta t'} (|delta t'| well below one turn).
#include <algorithm>
#include <vector>

#include "device_util.cuh"
#include "fredec_internal.cuh"

namespace fredec {

namespace {

constexpr int TU_THREADS = 128;
constexpr int TU_TILE = 64;               // points per shared tile
constexpr int MAXM = FREDEC_MAX_POOL;     // frequencies per tuple (and per pool Gram)
constexpr int MAXC = 2 * MAXM + 1;        // linear columns
constexpr int MAXE = MAXC + MAXM + 1;     // + derivative columns + residual/data column

struct SeriesPrep {            // per-series constants (device)
    double W, ybar, tc, D;     // sum w, weighted mean of y, time origin, <(y - ybar)^2> = l_0
    double span;               // max t - min t
};

// Weighted mean of y and centred time origin; D = <(y-ybar)^2>.  One CTA.
__global__ void series_prep(const double *t, const double *y, const double *sigma, int64_t N, SeriesPrep *out) {
    __shared__ double sc[32], smin[32], smax[32];
    double W = 0, Wy = 0, Wt = 0, mn = 1e300, mx = -1e300;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double w = 1.0 / (sigma[i] * sigma[i]);
        W += w;
        Wy += w * y[i];
        Wt += w * t[i];
        mn = fmin(mn, t[i]);
        mx = fmax(mx, t[i]);
    }
    W = block_sum_d(W, sc);
    Wy = block_sum_d(Wy, sc);
    Wt = block_sum_d(Wt, sc);
    for (int o = 16; o > 0; o >>= 1) {
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        smin[threadIdx.x >> 5] = mn;
        smax[threadIdx.x >> 5] = mx;
    }
    const double ybar = Wy / W;
    double D = 0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double w = 1.0 / (sigma[i] * sigma[i]);
        D += w * (y[i] - ybar) * (y[i] - ybar);
    }
    D = block_sum_d(D, sc);   // (its barriers also publish smin/smax)
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            mn = fmin(mn, smin[w]);
            mx = fmax(mx, smax[w]);
        }
        mn = fmin(mn, smin[0]);
        mx = fmax(mx, smax[0]);
        out->W = W;
        out->ybar = ybar;
        out->tc = rint(Wt / W);
        out->D = D;
        out->span = mx - mn > 0 ? mx - mn : 1.0;
    }
}

// Exact cos/sin of every pool frequency at every point: cs[k*N + i] (FP64).
__global__ void pool_seeds(const double *t, int64_t N, const double *pool, int npool, const SeriesPrep *sp,
                           double2 *cs) {
    __shared__ SeedTable tab;
    fill_seed_table(tab);
    __syncthreads();
    const double tc = sp->tc;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)npool * N;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(q / N);
        const int64_t i = q - (int64_t)k * N;
        double s, c;
        seed_from_table(tab, frac_turns_u64(pool[k], t[i] - tc), &s, &c);
        cs[q] = make_double2(c, s);
    }
}

// Packed lower-triangular helpers for the FP64 solves.  chol_inplace also
// lowers *min_ratio to the smallest pivot / original diagonal seen (the
// squared fraction of a column's norm left after projecting out the earlier
// columns).
__device__ inline bool chol_inplace(double *A, int n, double *min_ratio = nullptr) {
    for (int j = 0; j < n; ++j) {
        double d = A[tri(j, j)];
        const double d0 = d;
        for (int k = 0; k < j; ++k) d -= A[tri(j, k)] * A[tri(j, k)];
        if (min_ratio && d0 > 0) *min_ratio = fmin(*min_ratio, d / d0);
        if (!(d > 1e-13 * d0) || !(d0 > 0)) return false;
        const double l = sqrt(d);
        A[tri(j, j)] = l;
        for (int i = j + 1; i < n; ++i) {
            double s = A[tri(i, j)];
            for (int k = 0; k < j; ++k) s -= A[tri(i, k)] * A[tri(j, k)];
            A[tri(i, j)] = s / l;
        }
    }
    return true;
}
__device__ inline void fwd(const double *L, double *x, int n) {
    for (int i = 0; i < n; ++i) {
        double s = x[i];
        for (int k = 0; k < i; ++k) s -= L[tri(i, k)] * x[k];
        x[i] = s / L[tri(i, i)];
    }
}
__device__ inline void bwd(const double *L, double *x, int n) {
    for (int i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int k = i + 1; k < n; ++k) s -= L[tri(k, i)] * x[k];
        x[i] = s / L[tri(i, i)];
    }
}

struct TupleArgs {
    const double *t, *y, *sigma;
    int64_t N;
    const SeriesPrep *sp;
    const double2 *seeds;      // [pool][N]
    const double *pool;        // pool frequencies
    const int32_t *idx;        // tuple -> pool indices (CSR)
    const int64_t *off;
    int64_t n_tuples;
    int mode;                  // 0 eval, 1 grad, 2 refine
    int max_iter;
    double tol;
    double *z, *dzdf, *f_out, *l_out;
    int32_t *iters;
    int32_t *status;           // per-tuple: 0 ok, 1 singular
    int32_t *next;             // work counter (persistent CTAs)
    double *gram_out;          // mode 3: packed Gram of [1, c_k, s_k, y - ybar]
};

// Shared state of one CTA working on one tuple.
template <class T>
struct TupleSmem {
    T X[MAXE][TU_TILE + 1];    // weighted columns of the tile (padded stride)
    double G[MAXE * (MAXE + 1) / 2];
    double Lq[MAXC * (MAXC + 1) / 2];
    double theta[MAXC], a[MAXC], delta[MAXM], step[MAXM], ftrial[MAXM], X2[MAXC * MAXM], S[MAXM * (MAXM + 1) / 2],
        gd[MAXM];
    int pidx[MAXM];
    int m, M;
    double l, red;             // chi2 of the fit and its reduction sum_{r>=1} a_r^2 (= l_0 - l)
    double min_ratio;          // smallest Cholesky pivot ratio met by this tuple
    int flag;
};

// FP32-accumulated Gram sums are trusted while every Cholesky pivot keeps at
// least this fraction of its column's squared norm; below it the tuple is
// recomputed with FP64 sums (same role as flag_tau for periodogram bins).
constexpr double TUPLE_TAU = 1e-2;

// Accumulate <x_r x_c> over all points for the packed entries of the first
// ncol columns, where the per-point column vector is produced by make(i, x).
// Entries are split over the threads; each sums a fixed subset in point order
// (deterministic), in T, then the totals are stored in G as FP64.
template <class T, class Make>
__device__ void gram_pass(TupleSmem<T> &sm, const TupleArgs &a, int ncol, Make make) {
    const int ne = ncol * (ncol + 1) / 2;
    constexpr int NQ = (MAXE * (MAXE + 1) / 2 + TU_THREADS - 1) / TU_THREADS;
    T acc[NQ];
    unsigned char rr[NQ], cc[NQ];
    const int per = (ne + TU_THREADS - 1) / TU_THREADS;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        acc[q] = T(0);
        const int e = threadIdx.x + q * TU_THREADS;
        int r = 0;
        while (tri(r + 1, 0) <= e) ++r;
        rr[q] = (unsigned char)r;
        cc[q] = (unsigned char)(e - tri(r, 0));
    }
    for (int64_t i0 = 0; i0 < a.N; i0 += TU_TILE) {
        const int n = (int)(a.N - i0 < TU_TILE ? a.N - i0 : TU_TILE);
        __syncthreads();
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            T x[MAXE];
            make(i0 + p, x);
            for (int c = 0; c < ncol; ++c) sm.X[c][p] = x[c];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            if (q >= per) break;
            const int e = threadIdx.x + q * TU_THREADS;
            if (e >= ne) break;
            const int r = rr[q], c = cc[q];
            T s = T(0);
            for (int p = 0; p < n; ++p) s = fma(sm.X[r][p], sm.X[c][p], s);
            acc[q] += s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int e = threadIdx.x + q * TU_THREADS;
        if (q < per && e < ne) sm.G[e] = (double)acc[q];
    }
    __syncthreads();
}

// cos/sin of tuple frequency k at point i: pool seed rotated by delta_k.
template <class T>
__device__ __forceinline__ void tuple_cs(const TupleArgs &a, const TupleSmem<T> &sm, const SeedTable &tab,
                                         const SeedTableF &tabf, int k, int64_t i, double tp, T *c, T *s) {
    const double2 cs0 = a.seeds[(int64_t)sm.pidx[k] * a.N + i];
    const double dl = sm.delta[k];
    if (dl == 0.0) {
        *c = (T)cs0.x;
        *s = (T)cs0.y;
        return;
    }
    if constexpr (sizeof(T) == 8) {
        double ds, dc;
        seed_from_table(tab, frac_turns_u64(dl, tp), &ds, &dc);
        *c = cs0.x * dc - cs0.y * ds;
        *s = cs0.y * dc + cs0.x * ds;
    } else {
        float ds, dc;
        const float turns = (float)dl * (float)tp;            // small: |delta t'| well below one turn
        const float r = turns - rintf(turns);
        const float sc = fminf(fmaxf(r * 4294967296.0f, -2147483648.0f), 2147483520.0f);
        seed_from_table_f(tabf, (uint32_t)__float2int_rn(sc), &ds, &dc);
        const float c0 = (float)cs0.x, s0 = (float)cs0.y;
        *c = c0 * dc - s0 * ds;
        *s = s0 * dc + c0 * ds;
    }
}

// Linear fit of the current tuple: Gram of [1, c_k, s_k, y], Cholesky, a,
// theta, l.  Returns false if the normal matrix is singular.
template <class T>
__device__ bool linear_fit(TupleSmem<T> &sm, const TupleArgs &a, const SeedTable &tab, const SeedTableF &tabf) {
    const int m = sm.m, M = sm.M;
    const double tc = a.sp->tc, ybar = a.sp->ybar;
    gram_pass<T>(sm, a, M + 1, [&](int64_t i, T *x) {
        const double sw = 1.0 / a.sigma[i];
        const double tp = a.t[i] - tc;
        x[0] = (T)sw;
        for (int k = 0; k < m; ++k) {
            T c, s;
            tuple_cs<T>(a, sm, tab, tabf, k, i, tp, &c, &s);
            x[1 + 2 * k] = (T)sw * c;
            x[2 + 2 * k] = (T)sw * s;
        }
        x[M] = (T)(sw * (a.y[i] - ybar));
    });
    if (threadIdx.x == 0) {
        for (int r = 0; r < M; ++r)
            for (int c = 0; c <= r; ++c) sm.Lq[tri(r, c)] = sm.G[tri(r, c)];
        sm.flag = chol_inplace(sm.Lq, M, &sm.min_ratio) ? 1 : 0;
        if (sm.flag) {
            for (int r = 0; r < M; ++r) sm.a[r] = sm.G[tri(M, r)];
            fwd(sm.Lq, sm.a, M);
            double red = 0.0;
            for (int r = 1; r < M; ++r) red += sm.a[r] * sm.a[r];
            sm.l = a.sp->D - red;
            sm.red = red;          // z = red/2 without cancelling against D
            for (int r = 0; r < M; ++r) sm.X2[r] = sm.a[r];
            bwd(sm.Lq, sm.X2, M);
        }
    }
    __syncthreads();
    return sm.flag != 0;
}

template <class T>
__device__ void tuple_work(TupleSmem<T> &sm, const TupleArgs &a, const SeedTable &tab, const SeedTableF &tabf,
                           int64_t k) {
    const int64_t o0 = a.off[k];
    if (threadIdx.x == 0) {
        sm.m = (int)(a.off[k + 1] - o0);
        sm.M = 2 * sm.m + 1;
        sm.min_ratio = 1.0;
        for (int q = 0; q < sm.m; ++q) {
            sm.pidx[q] = a.idx[o0 + q];
            sm.delta[q] = 0.0;
        }
    }
    __syncthreads();
    const int m = sm.m, M = sm.M;
    const double tc = a.sp->tc, ybar = a.sp->ybar;
    if (!linear_fit<T>(sm, a, tab, tabf)) {
        if (threadIdx.x == 0) {
            a.status[k] = 1;
            if (a.z) a.z[k] = NAN;
            if (a.l_out) a.l_out[k] = NAN;
        }
        return;
    }
    if (a.mode == 0) {
        if (threadIdx.x == 0) {
            a.z[k] = 0.5 * sm.red;
            a.status[k] = 0;
        }
        return;
    }
    if (a.mode == 3) {   // pool Gram for the subtuple table: [1, c_k, s_k, y]
        for (int e = threadIdx.x; e < (M + 1) * (M + 2) / 2; e += blockDim.x) a.gram_out[e] = sm.G[e];
        if (threadIdx.x == 0) a.status[k] = 0;
        return;
    }
    double zred = sm.red;
    // coefficients theta = L^{-T} a are in X2[0..M)
    int it = 0;
    double lcur = sm.l;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0)
            for (int r = 0; r < M; ++r) sm.theta[r] = sm.X2[r];
        __syncthreads();
        // derivative columns and residual: [phi (M), d (m), r (1)]
        const int ne = M + m + 1;
        gram_pass<T>(sm, a, ne, [&](int64_t i, T *x) {
            const double sw = 1.0 / a.sigma[i];
            const double tp = a.t[i] - tc;
            double mu = sm.theta[0];
            x[0] = (T)sw;
            for (int q = 0; q < m; ++q) {
                T c, s;
                tuple_cs<T>(a, sm, tab, tabf, q, i, tp, &c, &s);
                const double ta = sm.theta[1 + 2 * q], tb = sm.theta[2 + 2 * q];
                mu += ta * (double)c + tb * (double)s;
                x[1 + 2 * q] = (T)sw * c;
                x[2 + 2 * q] = (T)sw * s;
                x[M + q] = (T)(sw * TWO_PI_D * tp * (-ta * (double)s + tb * (double)c));
            }
            x[M + m] = (T)(sw * (a.y[i] - ybar - mu));
        });
        if (a.mode == 1) {
            if (threadIdx.x < m) a.dzdf[a.off[k] + threadIdx.x] = sm.G[tri(M + m, M + threadIdx.x)];
            if (threadIdx.x == 0) {
                a.z[k] = 0.5 * zred;
                a.status[k] = (sizeof(T) == 4 && sm.min_ratio < TUPLE_TAU) ? 2 : 0;
            }
            return;
        }
        // Gauss-Newton step through the Schur complement
        if (threadIdx.x == 0) {
            for (int q = 0; q < m; ++q) {
                for (int r = 0; r < M; ++r) sm.X2[q * MAXC + r] = sm.G[tri(M + q, r)];
                fwd(sm.Lq, &sm.X2[q * MAXC], M);
            }
            for (int q = 0; q < m; ++q)
                for (int p = 0; p <= q; ++p) {
                    double v = sm.G[tri(M + q, M + p)];
                    for (int r = 0; r < M; ++r) v -= sm.X2[q * MAXC + r] * sm.X2[p * MAXC + r];
                    sm.S[tri(q, p)] = v;
                }
            for (int q = 0; q < m; ++q) sm.gd[q] = sm.G[tri(M + m, M + q)];
            sm.flag = chol_inplace(sm.S, m, &sm.min_ratio) ? 1 : 0;
            if (sm.flag) {
                fwd(sm.S, sm.gd, m);
                bwd(sm.S, sm.gd, m);
            }
        }
        __syncthreads();
        if (!sm.flag || it >= a.max_iter) break;
        double dmax = 0.0;
        for (int q = 0; q < m; ++q) dmax = fmax(dmax, fabs(sm.gd[q]));
        // step with halving until l does not increase; with FP32-accumulated
        // Gram sums l is only known to a few 1e-6 of <y^2>, so a step is
        // accepted when it does not raise l by more than that
        const double margin = sizeof(T) == 4 ? 3e-6 * a.sp->D : 1e-15 * lcur;
        double fac = 1.0;
        bool accepted = false;
        for (int h = 0; h < 30; ++h, fac *= 0.5) {
            if (threadIdx.x == 0)
                for (int q = 0; q < m; ++q) {
                    sm.step[q] = sm.delta[q];
                    sm.delta[q] = sm.step[q] + fac * sm.gd[q];
                }
            __syncthreads();
            const bool ok = linear_fit<T>(sm, a, tab, tabf);
            if (ok && sm.l <= lcur + margin) {
                accepted = true;
                break;
            }
            if (threadIdx.x == 0)
                for (int q = 0; q < m; ++q) sm.delta[q] = sm.step[q];
            __syncthreads();
        }
        ++it;
        if (!accepted) {
            linear_fit<T>(sm, a, tab, tabf);   // restore the fit at the last accepted frequencies
            break;
        }
        lcur = sm.l;
        if (fac * dmax * a.sp->span < a.tol) break;
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < m; ++q) a.f_out[a.off[k] + q] = a.pool[sm.pidx[q]] + sm.delta[q];
        a.l_out[k] = lcur;
        if (a.iters) a.iters[k] = it;
        a.status[k] = (sizeof(T) == 4 && sm.min_ratio < TUPLE_TAU) ? 2 : 0;
    }
}

template <class T>
__global__ void __launch_bounds__(TU_THREADS) tuple_kernel(TupleArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    TupleSmem<T> &sm = *reinterpret_cast<TupleSmem<T> *>(smraw);
    SeedTable &tab = *reinterpret_cast<SeedTable *>(smraw + sizeof(TupleSmem<T>));
    SeedTableF &tabf = *reinterpret_cast<SeedTableF *>(smraw + sizeof(TupleSmem<T>) + sizeof(SeedTable));
    fill_seed_table(tab);
    fill_seed_table_f(tabf);
    __syncthreads();
    __shared__ int64_t cur;
    for (;;) {
        if (threadIdx.x == 0) cur = atomicAdd(a.next, 1);
        __syncthreads();
        const int64_t k = cur;
        if (k >= a.n_tuples) break;
        tuple_work<T>(sm, a, tab, tabf, k);
        __syncthreads();
    }
}

// One warp per mask: gather the mask's columns [1, c_k, s_k (k in mask)] and
// the data column from the pool Gram, Cholesky (right-looking, lanes over
// rows), forward substitution, l = l_0 - sum_{r>=1} a_r^2.
constexpr int PM_WARPS = 4;
constexpr int PM_MAXC = 2 * FREDEC_MAX_POOL + 1;

__global__ void __launch_bounds__(32 * PM_WARPS) pool_mask_kernel(const double *gram, int npool,
                                                                  const SeriesPrep *sp, int64_t nmask,
                                                                  double *l_table) {
    __shared__ double A[PM_WARPS][PM_MAXC * (PM_MAXC + 1) / 2];
    __shared__ double bb[PM_WARPS][PM_MAXC];
    __shared__ double d0[PM_WARPS][PM_MAXC];
    __shared__ int cols[PM_WARPS][PM_MAXC];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int Mf = 2 * npool + 1;     // index of the data column in the pool Gram
    const double D = sp->D;
    for (int64_t mask = (int64_t)blockIdx.x * PM_WARPS + w; mask < nmask; mask += (int64_t)gridDim.x * PM_WARPS) {
        int M = 0;
        if (lane == 0) {
            cols[w][M++] = 0;
            for (int k = 0; k < npool; ++k)
                if (mask >> k & 1) {
                    cols[w][M++] = 1 + 2 * k;
                    cols[w][M++] = 2 + 2 * k;
                }
        }
        M = __shfl_sync(0xffffffffu, M, 0);
        __syncwarp();
        for (int e = lane; e < M * (M + 1) / 2; e += 32) {
            int r = 0;
            while (tri(r + 1, 0) <= e) ++r;
            const int c = e - tri(r, 0);
            A[w][e] = gram[tri(cols[w][r], cols[w][c])];
        }
        for (int r = lane; r < M; r += 32) {
            bb[w][r] = gram[tri(Mf, cols[w][r])];
            d0[w][r] = gram[tri(cols[w][r], cols[w][r])];
        }
        __syncwarp();
        bool ok = true;
        for (int j = 0; j < M; ++j) {
            const double d = A[w][tri(j, j)];
            if (!(d > 1e-13 * d0[w][j])) {
                ok = false;
                break;
            }
            const double ljj = sqrt(d);
            __syncwarp();
            if (lane == 0) A[w][tri(j, j)] = ljj;
            for (int i = j + 1 + lane; i < M; i += 32) A[w][tri(i, j)] /= ljj;
            __syncwarp();
            for (int i = j + 1 + lane; i < M; i += 32) {
                const double lij = A[w][tri(i, j)];
                for (int k = j + 1; k <= i; ++k) A[w][tri(i, k)] -= lij * A[w][tri(k, j)];
            }
            __syncwarp();
        }
        if (lane == 0) {
            double red = 0.0;
            if (ok) {
                for (int i = 0; i < M; ++i) {
                    double s = bb[w][i];
                    for (int k = 0; k < i; ++k) s -= A[w][tri(i, k)] * bb[w][k];
                    bb[w][i] = s / A[w][tri(i, i)];
                    if (i >= 1) red += bb[w][i] * bb[w][i];
                }
            }
            l_table[mask] = ok ? D - red : NAN;
        }
        __syncwarp();
    }
}

}  // namespace

// Host side -------------------------------------------------------------------

static int tuple_run(const double *t, const double *y, const double *sigma, int64_t N, const double *pool_h,
                     int npool, const std::vector<int32_t> &idx_h, const std::vector<int64_t> &off_h, int mode,
                     int precision, int max_iter, double tol, double *z_h, double *dzdf_h, double *f_h, double *l_h,
                     int32_t *iters_h, double *l0_h, cudaStream_t st) {
    const int64_t nt = (int64_t)off_h.size() - 1;
    const int64_t nflat = off_h.back();
    size_t off = 0;
    auto take = [&](size_t n) { size_t at = off; off = (off + n + 255) / 256 * 256; return at; };
    const size_t o_in = take(3 * N * 8), o_sp = take(sizeof(SeriesPrep)), o_pool = take(npool * 8 + 8),
                 o_seed = take((size_t)npool * N * 16 + 16), o_idx = take(nflat * 4 + 4), o_off = take((nt + 1) * 8),
                 o_z = take(nt * 8 + 8), o_g = take(nflat * 8 + 8), o_f = take(nflat * 8 + 8), o_l = take(nt * 8 + 8),
                 o_it = take(nt * 4 + 4), o_st = take(nt * 4 + 4), o_next = take(8);
    DevBuf ws;
    if (int rc = ws.alloc(off, st)) return rc;
    unsigned char *b = ws.as<unsigned char>();
    double *dt = (double *)(b + o_in), *dy = dt + N, *ds = dy + N;
    FREDEC_CUDA_TRY(cudaMemcpyAsync(dt, t, N * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(dy, y, N * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(ds, sigma, N * 8, cudaMemcpyHostToDevice, st));
    if (npool) FREDEC_CUDA_TRY(cudaMemcpyAsync(b + o_pool, pool_h, npool * 8, cudaMemcpyHostToDevice, st));
    if (nflat) FREDEC_CUDA_TRY(cudaMemcpyAsync(b + o_idx, idx_h.data(), nflat * 4, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(b + o_off, off_h.data(), (nt + 1) * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemsetAsync(b + o_next, 0, 8, st));
    SeriesPrep *sp = (SeriesPrep *)(b + o_sp);
    series_prep<<<1, 256, 0, st>>>(dt, dy, ds, N, sp);
    if (npool)
        pool_seeds<<<(unsigned)std::min<int64_t>(4096, ((int64_t)npool * N + 255) / 256), 256, 0, st>>>(
            dt, N, (const double *)(b + o_pool), npool, sp, (double2 *)(b + o_seed));
    TupleArgs a{};
    a.t = dt;
    a.y = dy;
    a.sigma = ds;
    a.N = N;
    a.sp = sp;
    a.seeds = (const double2 *)(b + o_seed);
    a.pool = (const double *)(b + o_pool);
    a.idx = (const int32_t *)(b + o_idx);
    a.off = (const int64_t *)(b + o_off);
    a.n_tuples = nt;
    a.mode = mode;
    a.max_iter = max_iter;
    a.tol = tol;
    a.z = (double *)(b + o_z);
    a.dzdf = (double *)(b + o_g);
    a.f_out = (double *)(b + o_f);
    a.l_out = (double *)(b + o_l);
    a.iters = (int32_t *)(b + o_it);
    a.status = (int32_t *)(b + o_st);
    a.next = (int32_t *)(b + o_next);
    const int grid = (int)std::min<int64_t>(std::max<int64_t>(nt, 1), 8LL * sm_count());
    if (nt > 0) {
        if (precision == FREDEC_MIXED) {
            const size_t smem = sizeof(TupleSmem<float>) + sizeof(SeedTable) + sizeof(SeedTableF);
            FREDEC_CUDA_TRY(cudaFuncSetAttribute(tuple_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            tuple_kernel<float><<<grid, TU_THREADS, smem, st>>>(a);
        } else {
            const size_t smem = sizeof(TupleSmem<double>) + sizeof(SeedTable) + sizeof(SeedTableF);
            FREDEC_CUDA_TRY(cudaFuncSetAttribute(tuple_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            tuple_kernel<double><<<grid, TU_THREADS, smem, st>>>(a);
        }
    }
    FREDEC_CUDA_TRY(cudaGetLastError());
    FREDEC_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int32_t> status(std::max<int64_t>(nt, 1));
    if (nt) FREDEC_CUDA_TRY(cudaMemcpy(status.data(), b + o_st, nt * 4, cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < nt; ++k)
        if (status[k] == 1) return fail(FREDEC_ESINGULAR, "a tuple's normal matrix is singular (repeated frequency?)");
    // tuples whose FP32-accumulated systems were ill-conditioned: redo in FP64
    std::vector<int64_t> redo;
    for (int64_t k = 0; k < nt; ++k)
        if (status[k] == 2) redo.push_back(k);
    std::vector<double> z2, g2, f2, l2;
    std::vector<int32_t> it2;
    std::vector<int64_t> off2(1, 0);
    if (!redo.empty()) {
        std::vector<int32_t> idx2;
        for (int64_t k : redo) {
            for (int64_t q = off_h[k]; q < off_h[k + 1]; ++q) idx2.push_back(idx_h[q]);
            off2.push_back((int64_t)idx2.size());
        }
        const int64_t n2 = (int64_t)redo.size(), nf2 = off2.back();
        z2.resize(n2 + 1);
        l2.resize(n2 + 1);
        it2.resize(n2 + 1);
        g2.resize(nf2 + 1);
        f2.resize(nf2 + 1);
        if (int rc = tuple_run(t, y, sigma, N, pool_h, npool, idx2, off2, mode, FREDEC_FP64, max_iter, tol, z2.data(),
                               g2.data(), f2.data(), l2.data(), it2.data(), nullptr, st))
            return rc;
    }
    if (z_h && nt) FREDEC_CUDA_TRY(cudaMemcpy(z_h, b + o_z, nt * 8, cudaMemcpyDeviceToHost));
    if (dzdf_h && nflat) FREDEC_CUDA_TRY(cudaMemcpy(dzdf_h, b + o_g, nflat * 8, cudaMemcpyDeviceToHost));
    if (f_h && nflat) FREDEC_CUDA_TRY(cudaMemcpy(f_h, b + o_f, nflat * 8, cudaMemcpyDeviceToHost));
    if (l_h && nt) FREDEC_CUDA_TRY(cudaMemcpy(l_h, b + o_l, nt * 8, cudaMemcpyDeviceToHost));
    if (iters_h && nt) FREDEC_CUDA_TRY(cudaMemcpy(iters_h, b + o_it, nt * 4, cudaMemcpyDeviceToHost));
    for (size_t r = 0; r < redo.size(); ++r) {
        const int64_t k = redo[r];
        if (z_h) z_h[k] = z2[r];
        if (l_h) l_h[k] = l2[r];
        if (iters_h) iters_h[k] = it2[r];
        for (int64_t q = 0; q < off_h[k + 1] - off_h[k]; ++q) {
            if (dzdf_h) dzdf_h[off_h[k] + q] = g2[off2[r] + q];
            if (f_h) f_h[off_h[k] + q] = f2[off2[r] + q];
        }
    }
    if (l0_h) {
        SeriesPrep h;
        FREDEC_CUDA_TRY(cudaMemcpy(&h, sp, sizeof(h), cudaMemcpyDeviceToHost));
        *l0_h = h.D;
    }
    return FREDEC_OK;
}

static int pool_table_run(const double *t, const double *y, const double *sigma, int64_t N, const double *pool_h,
                          int npool, double *l_table_h, cudaStream_t st) {
    size_t off = 0;
    auto take = [&](size_t n) { size_t at = off; off = (off + n + 255) / 256 * 256; return at; };
    const int Mx = 2 * npool + 2;
    const int64_t nmask = 1LL << npool;
    const size_t o_in = take(3 * N * 8), o_sp = take(sizeof(SeriesPrep)), o_pool = take(npool * 8 + 8),
                 o_seed = take((size_t)npool * N * 16 + 16), o_idx = take(npool * 4 + 4), o_off = take(16),
                 o_gram = take((size_t)Mx * (Mx + 1) / 2 * 8), o_st = take(8), o_next = take(8),
                 o_tab = take(nmask * 8);
    DevBuf ws;
    if (int rc = ws.alloc(off, st)) return rc;
    unsigned char *b = ws.as<unsigned char>();
    double *dt = (double *)(b + o_in), *dy = dt + N, *ds = dy + N;
    FREDEC_CUDA_TRY(cudaMemcpyAsync(dt, t, N * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(dy, y, N * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(ds, sigma, N * 8, cudaMemcpyHostToDevice, st));
    if (npool) FREDEC_CUDA_TRY(cudaMemcpyAsync(b + o_pool, pool_h, npool * 8, cudaMemcpyHostToDevice, st));
    std::vector<int32_t> idx(std::max(npool, 1));
    for (int k = 0; k < npool; ++k) idx[k] = k;
    const int64_t off_h[2] = {0, npool};
    FREDEC_CUDA_TRY(cudaMemcpyAsync(b + o_idx, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(b + o_off, off_h, 16, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemsetAsync(b + o_next, 0, 8, st));
    SeriesPrep *sp = (SeriesPrep *)(b + o_sp);
    series_prep<<<1, 256, 0, st>>>(dt, dy, ds, N, sp);
    if (npool)
        pool_seeds<<<(unsigned)std::min<int64_t>(4096, ((int64_t)npool * N + 255) / 256), 256, 0, st>>>(
            dt, N, (const double *)(b + o_pool), npool, sp, (double2 *)(b + o_seed));
    TupleArgs a{};
    a.t = dt;
    a.y = dy;
    a.sigma = ds;
    a.N = N;
    a.sp = sp;
    a.seeds = (const double2 *)(b + o_seed);
    a.pool = (const double *)(b + o_pool);
    a.idx = (const int32_t *)(b + o_idx);
    a.off = (const int64_t *)(b + o_off);
    a.n_tuples = 1;
    a.mode = 3;
    a.status = (int32_t *)(b + o_st);
    a.next = (int32_t *)(b + o_next);
    a.gram_out = (double *)(b + o_gram);
    const size_t smem = sizeof(TupleSmem<double>) + sizeof(SeedTable) + sizeof(SeedTableF);
    FREDEC_CUDA_TRY(cudaFuncSetAttribute(tuple_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tuple_kernel<double><<<1, TU_THREADS, smem, st>>>(a);
    const int64_t blocks = std::min<int64_t>((nmask + PM_WARPS - 1) / PM_WARPS, 64LL * sm_count());
    pool_mask_kernel<<<(unsigned)blocks, 32 * PM_WARPS, 0, st>>>((const double *)(b + o_gram), npool, sp, nmask,
                                                                  (double *)(b + o_tab));
    FREDEC_CUDA_TRY(cudaGetLastError());
    FREDEC_CUDA_TRY(cudaStreamSynchronize(st));
    int32_t status = 0;
    FREDEC_CUDA_TRY(cudaMemcpy(&status, b + o_st, 4, cudaMemcpyDeviceToHost));
    if (status) return fail(FREDEC_ESINGULAR, "the pool's normal matrix is singular (repeated pool frequency?)");
    FREDEC_CUDA_TRY(cudaMemcpy(l_table_h, b + o_tab, nmask * 8, cudaMemcpyDeviceToHost));
    return FREDEC_OK;
}

static int check_tuple_inputs(const double *t, const double *y, const double *sigma, int64_t N, const double *freqs,
                              const int64_t *off, int64_t n) {
    if (!t || !y || !sigma || N < 1 || n < 0 || (n > 0 && !off)) return fail(FREDEC_EINVAL, "bad arguments");
    for (int64_t i = 0; i < N; ++i)
        if (!std::isfinite(t[i]) || !std::isfinite(y[i]) || !(sigma[i] > 0.0) || !std::isfinite(sigma[i]))
            return fail(FREDEC_EINVAL, "t, y must be finite and sigma finite and > 0");
    if (n > 0 && off[0] != 0) return fail(FREDEC_EINVAL, "tuple_offsets[0] must be 0");
    for (int64_t k = 0; k < n; ++k) {
        const int64_t m = off[k + 1] - off[k];
        if (m < 0 || m > FREDEC_MAX_POOL) return fail(FREDEC_EINVAL, "tuple sizes must be in 0..FREDEC_MAX_TUPLE");
        if (N < 2 * m + 2) return fail(FREDEC_EINVAL, "N must exceed 2m+1 for every tuple");
    }
    if (n > 0 && !freqs && off[n] > 0) return fail(FREDEC_EINVAL, "null frequencies");
    for (int64_t q = 0; n > 0 && q < off[n]; ++q)
        if (!std::isfinite(freqs[q])) return fail(FREDEC_EINVAL, "frequencies must be finite");
    return FREDEC_OK;
}

struct TStream {
    cudaStream_t s = nullptr;
    ~TStream() {
        if (s) cudaStreamDestroy(s);
    }
};

}  // namespace fredec

using namespace fredec;

extern "C" {

int fredec_tuple_eval(const double *t, const double *y, const double *sigma, int64_t N, const double *tuple_freqs,
                      const int64_t *tuple_offsets, int64_t n_tuples, double *z_out, double *l0_out) {
    if (int rc = check_tuple_inputs(t, y, sigma, N, tuple_freqs, tuple_offsets, n_tuples)) return rc;
    const int64_t nflat = n_tuples ? tuple_offsets[n_tuples] : 0;
    std::vector<int32_t> idx(nflat);
    for (int64_t q = 0; q < nflat; ++q) idx[q] = (int32_t)q;
    std::vector<int64_t> off(tuple_offsets, tuple_offsets + n_tuples + 1);
    if (!n_tuples) off.assign(1, 0);
    TStream ts;
    FREDEC_CUDA_TRY(cudaStreamCreateWithFlags(&ts.s, cudaStreamNonBlocking));
    return tuple_run(t, y, sigma, N, tuple_freqs, (int)nflat, idx, off, 0, FREDEC_FP64, 0, 0.0, z_out, nullptr,
                     nullptr, nullptr, nullptr, l0_out, ts.s);
}

int fredec_pool_subtuples_eval(const double *t, const double *y, const double *sigma, int64_t N, const double *pool,
                               int32_t n_pool, double *l_table) {
    if (n_pool < 0 || n_pool > FREDEC_MAX_POOL || !l_table || (n_pool > 0 && !pool))
        return fail(FREDEC_EINVAL, "n_pool must be in 0..FREDEC_MAX_POOL");
    const int64_t off[2] = {0, n_pool};
    if (int rc = check_tuple_inputs(t, y, sigma, N, pool, off, 1)) return rc;
    TStream ts;
    FREDEC_CUDA_TRY(cudaStreamCreateWithFlags(&ts.s, cudaStreamNonBlocking));
    return pool_table_run(t, y, sigma, N, pool, n_pool, l_table, ts.s);
}

int fredec_tuple_grad(const double *t, const double *y, const double *sigma, int64_t N, const double *tuple_freqs,
                      const int64_t *tuple_offsets, int64_t n_tuples, int32_t precision, double *z_out,
                      double *dz_df_out) {
    if (precision != FREDEC_FP64 && precision != FREDEC_MIXED) return fail(FREDEC_EINVAL, "bad precision");
    if (int rc = check_tuple_inputs(t, y, sigma, N, tuple_freqs, tuple_offsets, n_tuples)) return rc;
    const int64_t nflat = n_tuples ? tuple_offsets[n_tuples] : 0;
    std::vector<int32_t> idx(nflat);
    for (int64_t q = 0; q < nflat; ++q) idx[q] = (int32_t)q;
    std::vector<int64_t> off(tuple_offsets, tuple_offsets + n_tuples + 1);
    if (!n_tuples) off.assign(1, 0);
    std::vector<double> g(std::max<int64_t>(nflat, 1));
    TStream ts;
    FREDEC_CUDA_TRY(cudaStreamCreateWithFlags(&ts.s, cudaStreamNonBlocking));
    int rc = tuple_run(t, y, sigma, N, tuple_freqs, (int)nflat, idx, off, 1, precision, 0, 0.0, z_out, g.data(),
                       nullptr, nullptr, nullptr, nullptr, ts.s);
    if (rc) return rc;
    // the kernel returns <d r> with d = dmu/df; dz/df = -1/2 dchi2/df = <r dmu/df>
    for (int64_t q = 0; q < nflat; ++q) dz_df_out[q] = g[q];
    return FREDEC_OK;
}

int fredec_pool_refine(const double *t, const double *y, const double *sigma, int64_t N, const double *pool,
                       int32_t n_pool, const uint32_t *masks, int64_t n_masks, int32_t max_iter, double tol,
                       int32_t precision, double *f_out, double *l_out, int32_t *iters_out) {
    if (precision != FREDEC_FP64 && precision != FREDEC_MIXED) return fail(FREDEC_EINVAL, "bad precision");
    if (n_pool < 0 || n_pool > FREDEC_MAX_TUPLE || n_masks < 0 || (n_masks > 0 && (!masks || !f_out || !l_out)) ||
        (n_pool > 0 && !pool) || max_iter < 0 || !(tol >= 0.0))
        return fail(FREDEC_EINVAL, "bad pool refine arguments");
    const int64_t pool_off[2] = {0, n_pool};
    if (int rc = check_tuple_inputs(t, y, sigma, N, pool, pool_off, 1)) return rc;
    std::vector<int32_t> idx;
    std::vector<int64_t> off(1, 0);
    for (int64_t k = 0; k < n_masks; ++k) {
        if (n_pool < 32 && (masks[k] >> n_pool) != 0) return fail(FREDEC_EINVAL, "mask has bits beyond n_pool");
        for (int j = 0; j < n_pool; ++j)
            if (masks[k] >> j & 1) idx.push_back(j);
        off.push_back((int64_t)idx.size());
    }
    std::vector<double> f(std::max<size_t>(idx.size(), 1));
    TStream ts;
    FREDEC_CUDA_TRY(cudaStreamCreateWithFlags(&ts.s, cudaStreamNonBlocking));
    int rc = tuple_run(t, y, sigma, N, pool, n_pool, idx, off, 2, precision, max_iter, tol, nullptr, nullptr,
                       f.data(), l_out, iters_out, nullptr, ts.s);
    if (rc) return rc;
    for (int64_t k = 0; k < n_masks; ++k) {
        for (int j = 0; j < n_pool; ++j) f_out[k * n_pool + j] = 0.0;
        for (int64_t q = off[k]; q < off[k + 1]; ++q) f_out[k * n_pool + idx[q]] = f[q];
    }
    return FREDEC_OK;
}

int fredec_tuple_refine(const double *t, const double *y, const double *sigma, int64_t N, double *tuple_freqs,
                        const int64_t *tuple_offsets, int64_t n_tuples, int32_t max_iter, double tol,
                        int32_t precision, double *l_out, int32_t *iters_out) {
    if (precision != FREDEC_FP64 && precision != FREDEC_MIXED) return fail(FREDEC_EINVAL, "bad precision");
    if (max_iter < 0 || !(tol >= 0.0) || !l_out) return fail(FREDEC_EINVAL, "bad max_iter / tol / l_out");
    if (int rc = check_tuple_inputs(t, y, sigma, N, tuple_freqs, tuple_offsets, n_tuples)) return rc;
    const int64_t nflat = n_tuples ? tuple_offsets[n_tuples] : 0;
    std::vector<int32_t> idx(nflat);
    for (int64_t q = 0; q < nflat; ++q) idx[q] = (int32_t)q;
    std::vector<int64_t> off(tuple_offsets, tuple_offsets + n_tuples + 1);
    if (!n_tuples) off.assign(1, 0);
    std::vector<double> f(std::max<int64_t>(nflat, 1));
    TStream ts;
    FREDEC_CUDA_TRY(cudaStreamCreateWithFlags(&ts.s, cudaStreamNonBlocking));
    int rc = tuple_run(t, y, sigma, N, tuple_freqs, (int)nflat, idx, off, 2, precision, max_iter, tol, nullptr,
                       nullptr, f.data(), l_out, iters_out, nullptr, ts.s);
    if (rc) return rc;
    for (int64_t q = 0; q < nflat; ++q) tuple_freqs[q] = f[q];
    return FREDEC_OK;
}

}  // extern "C"
