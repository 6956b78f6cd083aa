// Frequency tuples on a constant base (Section 2; Phase 2 of Section 4):
//   l(S)   = min over (c, a, b) of <(y - mu_S)^2>,  mu_S = c + sum_k a_k cos + b_k sin,
//   z_S    = (l_0 - l(S))/2,
//   dz/df_k = sum_i w_i r_i 2 pi t'_i (-a_k sin 2 pi f_k t'_i + b_k cos 2 pi f_k t'_i),
//   local refinement (Section 3, Eq. lsqf): Gauss-Newton on f with the linear
//   parameters refitted at every step.
//
// One CTA per tuple (persistent CTAs, largest tuples first), one launch per
// range of three tuple sizes with shared memory and CTA width sized for the
// range, the ranges on concurrent streams.  A pass over the points builds the
// weighted columns of a chunk of points in shared memory (one point per
// thread) and
// accumulates their Gram matrix: every thread owns 4x4 blocks of the lower
// triangle and runs over the chunk's points with float4 shared loads; when a
// tuple has fewer blocks than threads the points are split among groups of
// threads and the groups' sums are added in FP64 in a fixed order.  The mixed
// path builds the columns and sums them in FP32 (chunk partials added into
// running FP32 sums); the FP64 path does everything in FP64.
//
// The columns are [1, c_k, s_k, y] for a linear fit and, for gradients and
// refinement, also [t'c_k, t's_k] (the t-weighted averages of Eq. avrg1/avrg2).
// The CTA factors the leading [phi, y] block of the FP64 Gram in place
// (right-looking Cholesky, threads over the trailing triangle): row y holds
// a = L^{-1} <phi y>, so l = <y^2> - sum_{r>=1} a_r^2 (y is centred, so the
// constant's a_0 ~ 0) and theta = L^{-T} a.  The derivative columns
// d_k = 2 pi (b_k t'c_k - a_k t's_k) then enter by the incremental extension of
// the factor (Section 3): X = L^{-1} <phi d>, S = <d d> - X^T X and the
// gradient g = <d r> = <d y> - X^T a; the Gauss-Newton step is S^{-1} g.  A
// refinement makes one pass per trial point, which gives the trial's l and,
// when accepted, its exact Gauss-Newton step; a trial that raises l is halved.
//
// Every tuple frequency is an offset from a pool frequency whose exact
// cos/sin at every point are computed once (FP64 phases); the offset's
// rotation e^{i 2 pi delta t'} is small and is applied per pass.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <type_traits>
#include <vector>

#include "device_util.cuh"
#include "fredec_internal.cuh"

namespace fredec {

namespace {

constexpr int WT_THREADS = 128;
constexpr int QB = 2;                         // 4x4 Gram blocks per thread at most
constexpr int MAXM = FREDEC_MAX_POOL;         // frequencies per tuple (FREDEC_MAX_TUPLE with derivatives)
constexpr int MAXC = std::max(4 * FREDEC_MAX_TUPLE + 2, 2 * FREDEC_MAX_POOL + 2);   // Gram columns
constexpr int MAX_HALVINGS = 30;              // FP64: halve a rejected step up to this often
constexpr int MAX_HALVINGS_MIXED = 5;         // FP32 sums: a step still rejected after 5 halvings
                                              // is below the noise of l
constexpr double MIXED_L_NOISE = 3e-7;        // FP32-summed l is known to ~this fraction of <y^2>
constexpr size_t CHUNK_BYTES = 16384;         // shared column tile

// FP32-accumulated Gram sums are trusted while every pivot of the linear
// block keeps at least this fraction of its column's squared norm; below it
// the tuple is redone with FP64 sums (same role as flag_tau for periodogram
// bins).
constexpr double TUPLE_TAU = 1e-2;

struct SeriesPrep {            // per-series constants (device)
    double W, ybar, tc, D;     // sum w, weighted mean of y, time origin, <(y - ybar)^2> = l_0
    double span;               // max t - min t
    // column scales of the tensor-core Gram: 2^E with |value| < 2^(E-1) for
    // the columns built on 1/sigma (the constant, cos, sin), (y - ybar)/sigma
    // and (t - t_c)/sigma (the t-weighted cos, sin)
    int e_sw, e_yw, e_swt;
};

__device__ __forceinline__ double block_max_d(double v, double *scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double r = 0.0;
    for (int i = 0; i < nw; ++i) r = fmax(r, scratch[i]);
    return r;
}

// 2^E > 2 b (1 + 2^-20): values bounded by b scaled by 2^-E lie in (-1/2, 1/2).
__device__ __forceinline__ int scale_exponent(double b) { return b > 0.0 ? ilogb(b * (1.0 + 0x1p-20)) + 2 : 0; }

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
    const double ybar = Wy / W, tc = rint(Wt / W);
    double D = 0, bsw = 0, byw = 0, bswt = 0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double w = 1.0 / (sigma[i] * sigma[i]), sw = 1.0 / sigma[i];
        D += w * (y[i] - ybar) * (y[i] - ybar);
        bsw = fmax(bsw, sw);
        byw = fmax(byw, fabs((y[i] - ybar) * sw));
        bswt = fmax(bswt, fabs((t[i] - tc) * sw));
    }
    D = block_sum_d(D, sc);   // (its barriers also publish smin/smax)
    const double mx_sw = block_max_d(bsw, sc), mx_yw = block_max_d(byw, sc), mx_swt = block_max_d(bswt, sc);
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            mn = fmin(mn, smin[w]);
            mx = fmax(mx, smax[w]);
        }
        mn = fmin(mn, smin[0]);
        mx = fmax(mx, smax[0]);
        out->W = W;
        out->ybar = ybar;
        out->tc = tc;
        out->D = D;
        out->e_sw = scale_exponent(mx_sw);
        out->e_yw = scale_exponent(mx_yw);
        out->e_swt = scale_exponent(mx_swt);
        out->span = mx - mn > 0 ? mx - mn : 1.0;
    }
}

template <class T> struct Pt { T sw, tp, yw, pad; };   // 1/sigma, t - t_c, (y - ybar)/sigma

// Precision of a tuple pass.  float: FP32 columns and sums (the mixed path);
// double: FP64 throughout (the FP64 path); FF: FP64 columns stored as float
// pairs (hi + lo) and summed as double-float values (exact FP32 products,
// renormalised hi/lo running sums) -- about 1e-16 of the sum of magnitudes,
// like FP64 sums, for a fraction of the FP64 pipe's cost on this GPU.  FF
// redoes the mixed path's ill-conditioned tuples.
struct FF {};
template <class T> struct TP;
template <> struct TP<float> {
    using pt = float;          // per-point constants and column arithmetic
    using tile = float;        // shared column tile entry
    static constexpr bool mixed = true;
    static constexpr double l_noise = MIXED_L_NOISE;   // of <y^2>
};
template <> struct TP<double> {
    using pt = double;
    using tile = double;
    static constexpr bool mixed = false;
    static constexpr double l_noise = 0.0;             // 1e-15 of l instead
};
template <> struct TP<FF> {
    using pt = double;
    using tile = float2;
    static constexpr bool mixed = false;
    static constexpr double l_noise = 1e-13;
};
constexpr int PREC_FF = 2;     // internal precision code of the FF passes

template <class T>
__global__ void point_prep(const double *t, const double *y, const double *sigma, int64_t N, const SeriesPrep *sp,
                           Pt<T> *out) {
    const double tc = sp->tc, ybar = sp->ybar;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double sw = 1.0 / sigma[i];
        out[i] = Pt<T>{(T)sw, (T)(t[i] - tc), (T)((y[i] - ybar) * sw), T(0)};
    }
}

// Exact cos/sin of every pool frequency at every point (FP64 phases), stored
// in the pass precision: cs[k*N + i].
template <class T2>
__global__ void pool_seeds(const double *t, int64_t N, const double *pool, int npool, const SeriesPrep *sp, T2 *cs) {
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
        cs[q].x = c;
        cs[q].y = s;
    }
}

// FF per-point constants: float4 pairs {sw, t'} and {(y - ybar) sw, sw t'} as
// hi/lo floats; FF seeds: float4 {cos hi, cos lo, sin hi, sin lo}.
__global__ void point_prep_ff(const double *t, const double *y, const double *sigma, int64_t N, const SeriesPrep *sp,
                              float4 *out) {
    const double tc = sp->tc, ybar = sp->ybar;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double sw = 1.0 / sigma[i], tp = t[i] - tc;
        const ff a = ff_from_double(sw), b = ff_from_double(tp), c = ff_from_double((y[i] - ybar) * sw),
                 d = ff_from_double(sw * tp);
        out[2 * i] = make_float4(a.hi, a.lo, b.hi, b.lo);
        out[2 * i + 1] = make_float4(c.hi, c.lo, d.hi, d.lo);
    }
}

__global__ void pool_seeds_ff(const double *t, int64_t N, const double *pool, int npool, const SeriesPrep *sp,
                              float4 *cs) {
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
        const ff fc = ff_from_double(c), fs = ff_from_double(s);
        cs[q] = make_float4(fc.hi, fc.lo, fs.hi, fs.lo);
    }
}

struct TupleArgs {
    int64_t N;
    const SeriesPrep *sp;
    const void *pts;           // Pt<T>[N]
    const void *seeds;         // V2T<T>[pool][N]
    const double *pool;        // pool frequencies
    const int32_t *idx;        // tuple -> pool indices (CSR)
    const int64_t *off;
    const int32_t *order;      // processing order (largest tuples first)
    int64_t n_tuples;
    int mode;                  // 0 eval, 1 grad, 2 refine, 3 Gram of one tuple
    int max_iter;
    double tol;
    double *z, *dzdf, *f_out, *l_out;
    int32_t *iters;
    int32_t *status;           // per tuple: 0 ok, 1 singular, 2 redo in FP64
    int32_t *next;             // work counter
    double *gram_out;          // mode 3: packed Gram of [1, c_k, s_k, y]
    int chunk;                 // points per shared tile
    int cmax;                  // most columns of any tuple of the launch
    int32_t *err;              // FREDEC_ETIMEOUT from a bounded wait of the tensor-core kernel
};

struct TState {
    double theta[MAXC];        // coefficients at the accepted point
    double x[MAXC];            // trial coefficients / scratch
    double trial[MAXM];        // frequency offsets of the pass in progress
    double delta[MAXM];        // accepted offsets
    double step[MAXM];         // Gauss-Newton step at the accepted point
    float trialf[MAXM];
    float2 trialff[MAXM];      // trial offsets as hi/lo floats (FF passes)
    double red, redx;          // sum_{r>=1} a_r^2 (accepted / trial)
    double ratio;              // smallest linear pivot ratio of the last factorisation
    int pidx[MAXM];
    int m, fail_at;
};

// cos/sin of tuple frequency k at a point: the pool seed rotated by the
// trial offset.
__device__ __forceinline__ void tuple_cs(const TupleArgs &a, const TState &s, const void *tab, int k, int64_t i,
                                         float tp, float *c, float *sn) {
    const float2 c0 = static_cast<const float2 *>(a.seeds)[(int64_t)s.pidx[k] * a.N + i];
    const float dl = s.trialf[k];
    if (dl == 0.0f) {
        *c = c0.x;
        *sn = c0.y;
        return;
    }
    const float turns = dl * tp;                      // small: |delta t'| of a few turns at most
    const float r = turns - rintf(turns);
    const float sc = fminf(fmaxf(r * 4294967296.0f, -2147483648.0f), 2147483520.0f);
    float ds, dc;
    seed_from_table_f(*static_cast<const SeedTableF *>(tab), (uint32_t)__float2int_rn(sc), &ds, &dc);
    *c = c0.x * dc - c0.y * ds;
    *sn = c0.y * dc + c0.x * ds;
}
__device__ __forceinline__ void tuple_cs(const TupleArgs &a, const TState &s, const void *tab, int k, int64_t i,
                                         double tp, double *c, double *sn) {
    const double2 c0 = static_cast<const double2 *>(a.seeds)[(int64_t)s.pidx[k] * a.N + i];
    const double dl = s.trial[k];
    if (dl == 0.0) {
        *c = c0.x;
        *sn = c0.y;
        return;
    }
    double ds, dc;
    seed_from_table(*static_cast<const SeedTable *>(tab), frac_turns_u64(dl, tp), &ds, &dc);
    *c = c0.x * dc - c0.y * ds;
    *sn = c0.y * dc + c0.x * ds;
}

// Weighted columns of point i into row[0..CP): [1, c_k, s_k (k < m), y] and,
// with uv, [t' c_k, t' s_k] after them (the t-weighted averages of Eq. avrg1
// and avrg2 from which the derivative columns are formed).
__device__ __forceinline__ void put(float *row, int c, float v) { row[c] = v; }
__device__ __forceinline__ void put(double *row, int c, double v) { row[c] = v; }

template <class T>
__device__ __forceinline__ void make_row(const TupleArgs &a, const TState &s, const void *tab, int64_t i, int m,
                                         bool with_uv, int C, int CP, typename TP<T>::tile *row) {
    using V = typename TP<T>::pt;
    const Pt<V> p = static_cast<const Pt<V> *>(a.pts)[i];
    const int M = 2 * m + 1;
    put(row, 0, p.sw);
    put(row, M, p.yw);
    const V swt = p.sw * p.tp;
    for (int k = 0; k < m; ++k) {
        V c, sn;
        tuple_cs(a, s, tab, k, i, p.tp, &c, &sn);
        put(row, 1 + 2 * k, p.sw * c);
        put(row, 2 + 2 * k, p.sw * sn);
        if (with_uv) {
            put(row, M + 1 + 2 * k, swt * c);
            put(row, M + 2 + 2 * k, swt * sn);
        }
    }
    for (int c = C; c < CP; ++c) put(row, c, V(0));
}

// FF tile rows are planar per block of four columns: [hi x4, lo x4], so
// that four hi parts (or lo parts) load as one float4 and split into the
// float2 pairs of the packed accumulation (BlockAcc<FF>).
__device__ __forceinline__ void put_ff(float2 *row, int c, float hi, float lo) {
    float *r = reinterpret_cast<float *>(row) + 8 * (c >> 2) + (c & 3);
    r[0] = hi;
    r[4] = lo;
}

// FF columns: seed (FF) rotated by the FF sin/cos of the trial offset's
// turns delta t' (formed in FF), then the weighted products in FF.
template <>
__device__ __forceinline__ void make_row<FF>(const TupleArgs &a, const TState &s, const void *tab, int64_t i, int m,
                                             bool with_uv, int C, int CP, float2 *row) {
    const float4 *P4 = static_cast<const float4 *>(a.pts) + 2 * i;
    const float4 p0 = P4[0], p1 = P4[1];
    const ff sw = {p0.x, p0.y}, tp = {p0.z, p0.w}, yw = {p1.x, p1.y}, swt = {p1.z, p1.w};
    const SeedTableFF &T = *static_cast<const SeedTableFF *>(tab);
    const int M = 2 * m + 1;
    put_ff(row, 0, sw.hi, sw.lo);
    put_ff(row, M, yw.hi, yw.lo);
    for (int k = 0; k < m; ++k) {
        const float4 sd = static_cast<const float4 *>(a.seeds)[(int64_t)s.pidx[k] * a.N + i];
        ff c = {sd.x, sd.y}, sn = {sd.z, sd.w};
        const float2 dl = s.trialff[k];
        if (dl.x != 0.0f) {
            ff ds, dc;
            ff_sincos_ff_turns(T, ff_mul({dl.x, dl.y}, tp), &ds, &dc);
            const ff cn = ff_sub(ff_mul(c, dc), ff_mul(sn, ds));
            sn = ff_add(ff_mul(sn, dc), ff_mul(c, ds));
            c = cn;
        }
        const ff c1 = ff_mul(sw, c), s1 = ff_mul(sw, sn);
        put_ff(row, 1 + 2 * k, c1.hi, c1.lo);
        put_ff(row, 2 + 2 * k, s1.hi, s1.lo);
        if (with_uv) {
            const ff c2 = ff_mul(swt, c), s2 = ff_mul(swt, sn);
            put_ff(row, M + 1 + 2 * k, c2.hi, c2.lo);
            put_ff(row, M + 2 + 2 * k, s2.hi, s2.lo);
        }
    }
    for (int c = C; c < CP; ++c) put_ff(row, c, 0.f, 0.f);
}

__device__ __forceinline__ void load4(const float *p, float *v) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
}
__device__ __forceinline__ void load4(const double *p, double *v) {
    const double2 q0 = reinterpret_cast<const double2 *>(p)[0], q1 = reinterpret_cast<const double2 *>(p)[1];
    v[0] = q0.x;
    v[1] = q0.y;
    v[2] = q1.x;
    v[3] = q1.y;
}

// Per-entry accumulators of a 4x4 Gram block.  float/double: chunk partials
// added into running sums.  FF: double-float running sums (ff_acc), each
// product r c of hi/lo pairs entering as its rounded hi*hi part plus the exact
// rounding error of that product and the two cross terms.
// 4x4 blocks per thread: QB, or 1 for float-float sums, whose accumulators
// take four registers an entry (more threads per tuple instead, and more
// resident warps to hide the latency of their dependent chains).
template <class T> constexpr int qb_of() { return std::is_same<T, FF>::value ? 1 : QB; }

template <class T, int Q = QB> struct BlockAcc {
    using V = typename TP<T>::pt;
    V acc[Q][16];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int b = 0; b < Q; ++b)
#pragma unroll
            for (int e = 0; e < 16; ++e) acc[b][e] = V(0);
    }
    __device__ __forceinline__ void chunk(int b, const V *X, int rb, int cb, int g, int G, int n, int CP) {
        V part[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) part[e] = V(0);
        const V *xr = X + 4 * rb, *xc = X + 4 * cb;
#pragma unroll 4
        for (int p = g; p < n; p += G) {
            V r[4], c[4];
            load4(xr + (size_t)p * CP, r);
            load4(xc + (size_t)p * CP, c);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) part[4 * u + v] = fma(r[u], c[v], part[4 * u + v]);
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[b][e] += part[e];
    }
    __device__ __forceinline__ double value(int b, int e) const { return (double)acc[b][e]; }
};
// Packed subtraction of two float pairs (sub.rn.f32x2), the complement of
// __fadd2_rn; explicitly rounded like every step of the error-free
// transformations below.
__device__ __forceinline__ float2 fsub2_rn(float2 a, float2 b) {
    unsigned long long ra, rb, rd;
    memcpy(&ra, &a, 8);
    memcpy(&rb, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    memcpy(&d, &rd, 8);
    return d;
}

// Two double-float running sums updated by the same packed instructions: the
// product a*b of float-float numbers enters as its rounded hi*hi part p plus
// the exact error of that product and the two cross terms e (as in
// ff_acc::add_prod); p is added to H by TwoSum (Knuth), whose exact error and
// e go into L, which is not renormalised against H after every point (12
// packed operations instead of 15; the value is H + L at the end).  L takes
// one plain FP32 addition a point, so its own rounding grows with the number
// of points, about n eps ulp(H) for n points of random sign: about 4e-12 of
// the sums at the N = 1000 of the pool workload, against about 1e-13
// renormalised.  All 65535 subtuples of the 16-frequency pool: 0.470 ->
// 0.458 s; l at the refined frequencies against the oracle over 400 random
// subtuples kept its distribution (max 2.0e-7, median 1.1e-8 of l_0, either
// way: the FP32 passes set it).
struct ff_acc2 {
    float2 H = make_float2(0.f, 0.f), L = make_float2(0.f, 0.f);
    __device__ __forceinline__ void add_prod(float2 ahi, float2 alo, float2 bhi, float2 blo) {
        const float2 p = __fmul2_rn(ahi, bhi);
        float2 e = __ffma2_rn(ahi, bhi, make_float2(-p.x, -p.y));
        e = __ffma2_rn(ahi, blo, e);
        e = __ffma2_rn(alo, bhi, e);
        const float2 s = __fadd2_rn(H, p);                    // TwoSum(H, p)
        const float2 bb = fsub2_rn(s, H);
        const float2 err = __fadd2_rn(fsub2_rn(H, fsub2_rn(s, bb)), fsub2_rn(p, bb));
        L = __fadd2_rn(L, __fadd2_rn(err, e));
        H = s;
    }
};

// FF: the 16 entries of a 4x4 block as 8 pairs (entries 4u + 2w and
// 4u + 2w + 1, w = 0, 1: one row column against two column columns) in
// packed double-float sums; the planar tile rows give the hi and lo parts of
// four columns as one float4 each.
template <int Q> struct BlockAcc<FF, Q> {
    ff_acc2 a[Q][8];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int b = 0; b < Q; ++b)
#pragma unroll
            for (int e = 0; e < 8; ++e) a[b][e] = ff_acc2();
    }
    __device__ __forceinline__ void chunk(int b, const float2 *X, int rb, int cb, int g, int G, int n, int CP) {
        const float *xr = reinterpret_cast<const float *>(X) + 8 * rb, *xc = reinterpret_cast<const float *>(X) + 8 * cb;
        for (int p = g; p < n; p += G) {
            const float4 rh = *reinterpret_cast<const float4 *>(xr + (size_t)p * 2 * CP);
            const float4 rl = *reinterpret_cast<const float4 *>(xr + (size_t)p * 2 * CP + 4);
            const float4 ch = *reinterpret_cast<const float4 *>(xc + (size_t)p * 2 * CP);
            const float4 cl = *reinterpret_cast<const float4 *>(xc + (size_t)p * 2 * CP + 4);
            const float rhi[4] = {rh.x, rh.y, rh.z, rh.w}, rlo[4] = {rl.x, rl.y, rl.z, rl.w};
            const float2 chi[2] = {make_float2(ch.x, ch.y), make_float2(ch.z, ch.w)};
            const float2 clo[2] = {make_float2(cl.x, cl.y), make_float2(cl.z, cl.w)};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float2 ah = make_float2(rhi[u], rhi[u]), al = make_float2(rlo[u], rlo[u]);
#pragma unroll
                for (int w = 0; w < 2; ++w) a[b][2 * u + w].add_prod(ah, al, chi[w], clo[w]);
            }
        }
    }
    __device__ __forceinline__ double value(int b, int e) const {
        const ff_acc2 &q = a[b][e >> 1];
        return (e & 1) ? (double)q.H.y + (double)q.L.y : (double)q.H.x + (double)q.L.x;
    }
};

__device__ __forceinline__ void block_rc(int q, int *rb, int *cb) {
    int r = 0;
    while (tri(r + 1, 0) <= q) ++r;
    *rb = r;
    *cb = q - tri(r, 0);
}

// One pass over all points: the FP64 Gram (packed, C x C) of the columns at
// the trial offsets.
template <class T>
__device__ void gram_pass(const TupleArgs &a, const TState &s, const void *tab, double *Gs, unsigned char *R, int m,
                          bool with_uv) {
    constexpr int QBT = qb_of<T>();
    const int M = 2 * m + 1, C = with_uv ? M + 1 + 2 * m : M + 1, CP = (C + 3) & ~3;
    const int nb = CP / 4, nblk = nb * (nb + 1) / 2;
    const int tid = threadIdx.x, L = blockDim.x;
    int G = 1, g = 0, nq = 0, rb[QBT], cb[QBT], qid = 0;
    if (nblk <= L) {
        G = L / nblk;
        g = tid / nblk;
        qid = tid % nblk;
        nq = tid < G * nblk ? 1 : 0;
        block_rc(qid, &rb[0], &cb[0]);
#pragma unroll
        for (int b = 1; b < QBT; ++b) rb[b] = cb[b] = 0;
    } else {
#pragma unroll
        for (int b = 0; b < QBT; ++b) {
            const int q = tid + b * L;
            rb[b] = cb[b] = 0;
            if (q < nblk) {
                block_rc(q, &rb[b], &cb[b]);
                nq = b + 1;
            }
        }
    }
    BlockAcc<T, QBT> acc;
    acc.zero();
    using Tile = typename TP<T>::tile;
    Tile *X = reinterpret_cast<Tile *>(R);
    for (int64_t i0 = 0; i0 < a.N; i0 += a.chunk) {
        const int n = (int)(a.N - i0 < a.chunk ? a.N - i0 : a.chunk);
        __syncthreads();
        for (int p = tid; p < n; p += L) make_row<T>(a, s, tab, i0 + p, m, with_uv, C, CP, X + (size_t)p * CP);
        __syncthreads();
#pragma unroll
        for (int b = 0; b < QBT; ++b)
            if (b < nq) acc.chunk(b, X, rb[b], cb[b], g, G, n, CP);
    }
    __syncthreads();
    if (G == 1) {
#pragma unroll
        for (int b = 0; b < QBT; ++b)
            if (b < nq)
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int r = 4 * rb[b] + e / 4, c = 4 * cb[b] + e % 4;
                    if (r < C && c <= r) Gs[tri(r, c)] = acc.value(b, e);
                }
    } else {
        double *red = reinterpret_cast<double *>(R);   // [G][nblk][16]
        if (nq)
#pragma unroll
            for (int e = 0; e < 16; ++e) red[((size_t)g * nblk + qid) * 16 + e] = acc.value(0, e);
        __syncthreads();
        for (int qe = tid; qe < nblk * 16; qe += L) {
            const int q = qe >> 4, e = qe & 15;
            double v = 0.0;
            for (int gg = 0; gg < G; ++gg) v += red[((size_t)gg * nblk + q) * 16 + e];
            int r0, c0;
            block_rc(q, &r0, &c0);
            const int r = 4 * r0 + e / 4, c = 4 * c0 + e % 4;
            if (r < C && c <= r) Gs[tri(r, c)] = v;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Tensor-core Gram of the float-float passes: error-free splitting of the
// columns into bf16 digits (Ozaki, Ogita, Oishi and Rump 2012, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication").
//
// A column value x (a float pair) scaled by the power of two 2^-E of its
// column class (|x| 2^-E < 1/2) is rounded to 49 bits and written exactly as
// seven signed base-128 digits, x 2^-E = sum_k d_k 2^(-7(k+1)) + r with
// |d_k| <= 64 and |r| <= 2^-50: bf16 values, whose products are exact, and
// FP32 sums of up to 2^24 / 2^12 = 4096 such products are exact too.
// Level d = s + t of the digit pairs, D_d(i, j) = sum over points and
// s + t = d of d_s(i) d_t(j), is accumulated in FP32 in tensor memory by
// MMAs of M = 128 whose A operand is two digit tiles stacked, s and s + 1
// (s even; the tiles are adjacent in shared memory, a zero tile after the
// seventh), against tile t: rows 0..63 of accumulator region s + t receive
// the pair (s, t) (level s + t), rows 64..127 the pair (s + 1, t) (level
// s + t + 1), so 16 MMAs cover the 28 pairs with s + t <= 6 (a region's row
// receives at most 4 pairs).  Every TC_WIN chunks (512 points) the levels
// are combined in float-float arithmetic, sum_d 2^(-7d) D_d, into per-entry
// float-float sums, and the Gram entry is 2^(E_i + E_j - 14) times the
// total.  Pairs with s + t > 6 (below 2^-49 of the column scales) are left
// out.  Points enter in chunks of 64 (one 128-byte swizzled row of bf16 per
// Gram column), two buffers of digit tiles so that the MMAs of one chunk
// overlap the column generation of the next.

constexpr int TC_DIG = 7;                              // digits per value
constexpr int TC_LEVELS = TC_DIG;                      // digit-pair levels kept: s + t <= TC_DIG - 1
constexpr int TC_K = 64;                               // points per chunk
constexpr int TC_WIN = 8;                              // chunks per exact window: 7 * 512 * 2^12 < 2^24
constexpr int TC_ROWS = 64;                            // Gram columns of one tile, at most 64
constexpr int TC_M = 2 * TC_ROWS;                      // MMA M: two digit tiles stacked
constexpr size_t TC_TILE = (size_t)TC_ROWS * 128;      // one digit tile (bytes)
constexpr int TC_TILES = TC_DIG + 1;                   // the digit tiles of a chunk and a zero tile
constexpr size_t TC_BUF = TC_TILES * TC_TILE;          // one buffer of tiles
constexpr int TC_WORKERS = 256;                        // column generation, readouts (4 threads a point)
constexpr int TC_THREADS = TC_WORKERS + 32;            // and one warp that issues the MMAs
constexpr int TC_MIN_COLS = 40;                        // narrower Grams stay on the CUDA cores
constexpr uint32_t TC_TMEM_COLS = 512;                 // TC_LEVELS x N (N <= 64) columns
static_assert(TC_WIN * TC_K * 4 * 4096 < (1 << 24), "a window's digit sums must stay exact in FP32");
static_assert(TC_LEVELS * TC_ROWS <= (int)TC_TMEM_COLS, "tensor memory holds every level");

struct TcState {
    unsigned char *dig;        // 2 buffers of TC_DIG tiles, 1024-byte aligned
    float2 *acc;               // float-float sums of the packed lower triangle
    uint64_t *bar;             // one mbarrier per buffer
    int32_t *err;              // FREDEC_ETIMEOUT when an MMA completion was not seen
    uint32_t tmem;             // tensor-memory base: level d at columns d N .. d N + N - 1
    uint32_t phase[2];         // parity of the next completion, per buffer
    bool pend[2];              // a commit not yet waited for, per buffer
};

// Waits (bounded) for the MMAs committed to buffer b, if any.
__device__ __forceinline__ void tc_wait(TcState &t, int b) {
    if (!t.pend[b]) return;
    if (!mbar_wait_bounded(&t.bar[b], t.phase[b]) && threadIdx.x == 0) atomicExch(t.err, FREDEC_ETIMEOUT);
    t.phase[b] ^= 1u;
    t.pend[b] = false;
}

// bf16 bits of a small integer (|d| <= 64): float(d) by the 1.5 * 2^23
// offset, whose low 16 bits are then zero.
__device__ __forceinline__ uint16_t small_int_bf16(int d) {
    return (uint16_t)(__float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f) >> 16);
}

// The seven digits of (h + l) sc 2^-49 (sc = 2^(49 - E)) into row c, point
// slot k of the digit tiles.  h sc and l sc are exact (power-of-two scaling);
// their sum, rounded to an integer, is the 49-bit fixed-point value Q,
// |Q| < 2^48, split as Q = q1 2^28 + q0 (|q0| <= 2^27) and then into digits of
// weights 2^42, 2^35, ..., 2^0 by rounding divisions.
__device__ __forceinline__ void put_digits(unsigned char *tiles, int c, int k, float h, float l, float sc) {
    const long long Q = __float2ll_rn(h * sc) + __float2ll_rn(l * sc);
    const int q1 = (int)((Q + (1LL << 27)) >> 28);
    int r = (int)(Q - (long long)q1 * (1LL << 28));
    int d[TC_DIG];
    int u = q1;
    d[0] = (u + (1 << 13)) >> 14;
    u -= d[0] * (1 << 14);
    d[1] = (u + (1 << 6)) >> 7;
    d[2] = u - d[1] * (1 << 7);
    d[3] = (r + (1 << 20)) >> 21;
    r -= d[3] * (1 << 21);
    d[4] = (r + (1 << 13)) >> 14;
    r -= d[4] * (1 << 14);
    d[5] = (r + (1 << 6)) >> 7;
    d[6] = r - d[5] * (1 << 7);
    const int off = umma_sw128_offset(c, k);
#pragma unroll
    for (int q = 0; q < TC_DIG; ++q) *reinterpret_cast<uint16_t *>(tiles + q * TC_TILE + off) = small_int_bf16(d[q]);
}
__device__ __forceinline__ void put_zero_digits(unsigned char *tiles, int c, int k) {
    const int off = umma_sw128_offset(c, k);
#pragma unroll
    for (int q = 0; q < TC_DIG; ++q) *reinterpret_cast<uint16_t *>(tiles + q * TC_TILE + off) = 0;
}

// The float-float columns of point i (make_row<FF>'s values) as digits in
// point slot k: this thread's share, the frequencies part - 1, part - 1 +
// nparts, ... (mod nparts; part 0 also takes the constant and the data
// column, and the frequencies that leave it the lightest share); zeros past
// the last point.
__device__ __forceinline__ void tc_columns(const TupleArgs &a, const TState &s, const SeedTableFF &T, int64_t i, int k,
                                           int part, int nparts, int m, bool with_uv, unsigned char *tiles,
                                           float sc_sw, float sc_yw, float sc_swt) {
    const int M = 2 * m + 1;
    if (i >= a.N) {
        if (part == 0) {
            put_zero_digits(tiles, 0, k);
            put_zero_digits(tiles, M, k);
        }
        for (int q = (part + nparts - 1) % nparts; q < m; q += nparts) {
            put_zero_digits(tiles, 1 + 2 * q, k);
            put_zero_digits(tiles, 2 + 2 * q, k);
            if (with_uv) {
                put_zero_digits(tiles, M + 1 + 2 * q, k);
                put_zero_digits(tiles, M + 2 + 2 * q, k);
            }
        }
        return;
    }
    const float4 *P4 = static_cast<const float4 *>(a.pts) + 2 * i;
    const float4 p0 = P4[0], p1 = P4[1];
    const ff sw = {p0.x, p0.y}, tp = {p0.z, p0.w}, yw = {p1.x, p1.y}, swt = {p1.z, p1.w};
    if (part == 0) {
        put_digits(tiles, 0, k, sw.hi, sw.lo, sc_sw);
        put_digits(tiles, M, k, yw.hi, yw.lo, sc_yw);
    }
    for (int q = (part + nparts - 1) % nparts; q < m; q += nparts) {
        const float4 sd = static_cast<const float4 *>(a.seeds)[(int64_t)s.pidx[q] * a.N + i];
        ff c = {sd.x, sd.y}, sn = {sd.z, sd.w};
        const float2 dl = s.trialff[q];
        if (dl.x != 0.0f) {
            ff ds, dc;
            ff_sincos_ff_turns(T, ff_mul({dl.x, dl.y}, tp), &ds, &dc);
            const ff cn = ff_sub(ff_mul(c, dc), ff_mul(sn, ds));
            sn = ff_add(ff_mul(sn, dc), ff_mul(c, ds));
            c = cn;
        }
        const ff c1 = ff_mul(sw, c), s1 = ff_mul(sw, sn);
        put_digits(tiles, 1 + 2 * q, k, c1.hi, c1.lo, sc_sw);
        put_digits(tiles, 2 + 2 * q, k, s1.hi, s1.lo, sc_sw);
        if (with_uv) {
            const ff c2 = ff_mul(swt, c), s2 = ff_mul(swt, sn);
            put_digits(tiles, M + 1 + 2 * q, k, c2.hi, c2.lo, sc_swt);
            put_digits(tiles, M + 2 + 2 * q, k, s2.hi, s2.lo, sc_swt);
        }
    }
}

// The window's levels into the float-float sums (the workers).  With M = 128
// tensor-memory lane l of region r holds Gram row l % 64 of level r + l / 64.
// Warp w reads the lanes of its quarter q = w % 4 (rows 32 (q % 2) .. + 31,
// one level up for q >= 2) and the 16-column blocks b with b % 2 == w / 4
// that hold entries j <= row; the upper quarters add theirs after the lower
// ones (both update the same entries).
__device__ void tc_readout(TcState &t, int C, int N) {
    if (threadIdx.x >= TC_WORKERS) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, q = w & 3, half = w >> 2, up = q >> 1;
    const int r0 = 32 * (q & 1), row = r0 + lane;
    const bool live = row < C;
    const int nb = r0 < C ? (min(C, r0 + 32) + 15) / 16 : 0;   // column blocks with j < the quarter's last row
    for (int phase = 0; phase < 2; ++phase) {
        if (phase == up)
            for (int b = half; b < nb; b += 2) {
                float hi[16], lo[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) hi[j] = lo[j] = 0.0f;
                float scale = up ? 0x1p-7f : 1.0f;
                for (int d = 0; d < TC_LEVELS; ++d) {
                    float v[16];
                    tmem_ld16(t.tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(d * N + 16 * b), v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {   // (hi, lo) += v 2^(-7 level), exact scaling
                        const ff s = ff_two_sum(hi[j], v[j] * scale);
                        const ff r = ff_fast_two_sum(s.hi, __fadd_rn(s.lo, lo[j]));
                        hi[j] = r.hi;
                        lo[j] = r.lo;
                    }
                    scale *= 0x1p-7f;
                }
                if (live)
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = 16 * b + j;
                        if (col <= row) {
                            float2 &e = t.acc[tri(row, col)];
                            const ff sum = ff_add({e.x, e.y}, {hi[j], lo[j]});
                            e = make_float2(sum.hi, sum.lo);
                        }
                    }
            }
        asm volatile("bar.sync 1, %0;" ::"r"(TC_WORKERS) : "memory");   // the workers only
    }
}

// One pass over all points on the tensor cores: the FP64 Gram (packed, C x C,
// C <= 64) of the float-float columns at the trial offsets.
__device__ void gram_pass_tc(const TupleArgs &a, const TState &s, const void *tab, double *Gs, TcState &t, int m,
                             bool with_uv) {
    const int M = 2 * m + 1, C = with_uv ? M + 1 + 2 * m : M + 1, N = (C + 15) & ~15;
    const int ne = C * (C + 1) / 2, tid = threadIdx.x, L = blockDim.x;
    for (int e = tid; e < ne; e += L) t.acc[e] = make_float2(0.0f, 0.0f);
    const SeriesPrep &sp = *a.sp;
    const float sc_sw = exp2f((float)(49 - sp.e_sw)), sc_yw = exp2f((float)(49 - sp.e_yw)),
                sc_swt = exp2f((float)(49 - sp.e_swt));
    const SeedTableFF &T = *static_cast<const SeedTableFF *>(tab);
    const int nparts = TC_WORKERS / TC_K, part = tid / TC_K, k = tid % TC_K;
    const bool worker = tid < TC_WORKERS, issuer = tid == TC_WORKERS;
    const int nch = (int)((a.N + TC_K - 1) / TC_K);
    const uint32_t idesc = umma_idesc_bf16(TC_M, N);
    for (int ch = 0; ch < nch; ++ch) {
        const int buf = ch & 1;
        unsigned char *tiles = t.dig + buf * TC_BUF;
        const bool wstart = ch % TC_WIN == 0;
        tc_wait(t, buf);                                    // the MMAs of chunk ch - 2 are done with the buffer
        if (wstart && ch > 0) {                             // the previous window is complete: read it out
            tc_wait(t, buf ^ 1);
            tc_fence_after();
            tc_readout(t, C, N);
            tc_fence_before();
            __syncthreads();
        }
        if (worker)
            tc_columns(a, s, T, (int64_t)ch * TC_K + k, k, part, nparts, m, with_uv, tiles, sc_sw, sc_yw, sc_swt);
        fence_proxy_async_smem();
        __syncthreads();
        // the issuing warp queues this chunk's MMAs while the workers go on
        // to the next chunk's columns
        if (issuer) {
            tc_fence_after();
            // descriptors differ only in the start address (its field holds
            // address / 16): tile u, K step ks at + (u TC_TILE + 32 ks) / 16;
            // A = tiles sa, sa + 1 (128 rows), B = tile tb, into region sa + tb
            const uint64_t d0 = umma_desc_sw128(smem_u32(tiles));
            for (int sa = 0; sa < TC_DIG; sa += 2)
                for (int tb = 0; sa + tb < TC_LEVELS; ++tb) {
                    const uint64_t da = d0 + (uint64_t)(sa * (TC_TILE >> 4)), db = d0 + (uint64_t)(tb * (TC_TILE >> 4));
#pragma unroll
                    for (int ks = 0; ks < TC_K / 16; ++ks)
                        umma_bf16(t.tmem + (uint32_t)((sa + tb) * N), da + 2u * ks, db + 2u * ks, idesc,
                                  !(wstart && sa == 0 && ks == 0));
                }
            umma_commit(&t.bar[buf]);
        }
        t.pend[buf] = true;
    }
    tc_wait(t, 0);
    tc_wait(t, 1);
    tc_fence_after();
    tc_readout(t, C, N);
    tc_fence_before();
    __syncthreads();
    const int eM = M;
    for (int e = tid; e < ne; e += L) {
        int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while (tri(i + 1, 0) <= e) ++i;
        while (tri(i, 0) > e) --i;
        const int j = e - tri(i, 0);
        auto ex = [&](int c) { return c == eM ? sp.e_yw : c > eM ? sp.e_swt : sp.e_sw; };
        const float2 v = t.acc[e];
        Gs[e] = ldexp((double)v.x + (double)v.y, ex(i) + ex(j) - 14);
    }
    __syncthreads();
    // a completion not seen: the pass's sums are unknown; a NaN first pivot
    // makes the tuple's outputs NaN (the host reports FREDEC_ETIMEOUT)
    if (tid == 0 && *(volatile int32_t *)t.err != 0) Gs[0] = NAN;
    __syncthreads();
}

// Shared memory of the tensor-core kernel (offsets from a 1024-byte aligned
// base): the two buffers of digit tiles, the float-float seed table, the
// tuple state, the FP64 Gram with its diagonal scratch, the extension's
// scratch, the float-float Gram sums, two mbarriers and the tensor-memory
// address.
struct TcLayout {
    size_t tab, state, gram, d0, inv, R, acc, bar, slot, bytes;
};
__host__ __device__ inline size_t tc_al16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline TcLayout tc_layout(int cmax) {
    TcLayout L{};
    const size_t ntri = (size_t)cmax * (cmax + 1) / 2, mm = (size_t)(cmax > 2 ? (cmax - 2) / 4 : 0),
                 M = 2 * mm + 1;
    size_t o = 2 * TC_BUF;
    L.tab = o;
    o = tc_al16(o + sizeof(SeedTableFF));
    L.state = o;
    o = tc_al16(o + sizeof(TState));
    L.gram = o;
    o += 8 * ntri;
    L.d0 = o;
    o += 8 * (size_t)cmax;
    L.inv = o;
    o = tc_al16(o + 8 * (size_t)cmax);
    L.R = o;
    o = tc_al16(o + 8 * (mm * M + mm * (mm + 1) / 2 + 2 * mm) + 16);
    L.acc = o;
    o = tc_al16(o + 8 * ntri);
    L.bar = o;
    o += 16;
    L.slot = o;
    o += 16;
    L.bytes = o + 1024;   // room to align the base
    return L;
}

// In-place right-looking Cholesky of the packed C x C matrix by the whole CTA.
// The reciprocals of the original diagonal are formed first, in parallel
// (rd0[]), so that a pivot's check is one multiplication.  Thread 0 takes each
// pivot (check, reciprocal square root; the reciprocal diagonal is kept in
// inv[] for the substitutions): pivot j + 1 as soon as its own part of
// pivot j's trailing update has produced it (entry (j+1, j+1) is that
// update's first entry, always thread 0's), while the other threads finish
// theirs -- two barriers a pivot.  The CTA scales the column and updates the
// trailing triangle (threads over its entries).  Pivots 0..nchk-1 must keep
// more than 1e-13 of their original diagonal; the index of the first that
// does not is left in s.fail_at (C when all do).  s.ratio = the smallest
// pivot ratio among the first nlin pivots.  Later pivots (the data column)
// are factored without a check.
__device__ void chol_cta(double *A, double *rd0, double *inv, int C, int nlin, int nchk, TState &s) {
    const int tid = threadIdx.x, L = blockDim.x;
    for (int j = tid; j < C; j += L) {
        const double v = A[tri(j, j)];
        rd0[j] = v > 0.0 ? 1.0 / v : -1.0;
    }
    __syncthreads();
    auto pivot = [&](int j) {   // thread 0
        const double d = A[tri(j, j)];
        if (j < nchk) {
            const double r = rd0[j] > 0.0 ? d * rd0[j] : -1.0;
            if (j < nlin) s.ratio = fmin(s.ratio, r);
            if (!(r > 1e-13)) s.fail_at = j;
        }
        // one FP64 reciprocal square root per pivot (no division): 1/L_jj,
        // and L_jj = d / sqrt(d)
        const double il = d > 0.0 ? rsqrt(d) : 0.0;
        A[tri(j, j)] = d * il;
        inv[j] = il;
    };
    if (tid == 0) {
        s.fail_at = C;
        s.ratio = 1.0;
        if (C > 0) pivot(0);
    }
    __syncthreads();
    for (int j = 0; j < C; ++j) {
        if (s.fail_at <= j) break;
        const double iv = inv[j];
        for (int i = j + 1 + tid; i < C; i += L) A[tri(i, j)] *= iv;
        __syncthreads();
        const int nt = C - j - 1, ne = nt * (nt + 1) / 2;
        for (int e = tid; e < ne; e += L) {
            int ii = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
            while (tri(ii + 1, 0) <= e) ++ii;
            while (tri(ii, 0) > e) --ii;
            const int i = j + 1 + ii, k = j + 1 + (e - tri(ii, 0));
            A[tri(i, k)] -= A[tri(i, j)] * A[tri(k, j)];
            if (e == 0) pivot(j + 1);
        }
        __syncthreads();
    }
}

// Warp 0: x[0..n) <- L^{-T} x for the diagonal block of the packed factor that
// starts at row/column o (inv: its reciprocal diagonal).
__device__ void bwd_warp(const double *A, const double *inv, int o, int n, double *x) {
    const int lane = threadIdx.x & 31;
    for (int i = n - 1; i >= 0; --i) {
        if (lane == 0) x[i] *= inv[o + i];
        __syncwarp();
        const double xi = x[i];
        for (int r = lane; r < i; r += 32) x[r] -= A[tri(o + i, o + r)] * xi;
        __syncwarp();
    }
}

// Warp 0, after chol_cta of the leading [phi, y] block (data column at index
// M): red = sum_{r=1}^{M-1} a_r^2 and the coefficients theta = L^{-T} a into
// th[0..M).
__device__ void linear_solution(const double *A, const double *inv, int M, double *th, double *red_out) {
    const int lane = threadIdx.x & 31;
    double r2 = 0.0;
    for (int r = lane; r < M; r += 32) {
        const double v = A[tri(M, r)];
        th[r] = v;
        if (r >= 1) r2 += v * v;
    }
    r2 = warp_sum_d(r2);
    __syncwarp();
    bwd_warp(A, inv, 0, M, th);
    if (lane == 0) *red_out = r2;
    __syncwarp();
}

// Warp 0: x[0..n) <- L^{-1} x for the packed factor L (n x n, inv: its
// reciprocal diagonal).
__device__ void fwd_warp(const double *A, const double *inv, int n, double *x) {
    const int lane = threadIdx.x & 31;
    for (int i = 0; i < n; ++i) {
        if (lane == 0) x[i] *= inv[i];
        __syncwarp();
        const double xi = x[i];
        for (int r = i + 1 + lane; r < n; r += 32) x[r] -= A[tri(r, i)] * xi;
        __syncwarp();
    }
}

// The incremental extension of Section 3 for the frequency columns.  H is the
// pass's Gram of [phi (M), y, t'c_0, t's_0, ...] whose leading [phi, y] block
// has been factored in place (L, and a in row M); theta = L^{-T} a.  The
// derivative columns d_k = 2 pi (b_k t'c_k - a_k t's_k) (a_k = theta_{1+2k},
// b_k = theta_{2+2k}) enter through their Gram entries:
//     X = L^{-1} <phi d>,  g = <d y> - X^T a = <d r>,  S = <d d> - X^T X.
// Writes g (the gradient <d r> = dz/df) and, with want_step, the Gauss-Newton
// step S^{-1} g; returns false when S is not positive definite.
// Scratch W: m*M + m(m+1)/2 + 2m doubles.
__device__ bool extend_cta(const double *H, const double *invL, int M, int m, const double *theta, double *W, double *g,
                           double *step, TState &s) {
    const int tid = threadIdx.x, L = blockDim.x;
    double *Xs = W, *Sp = W + (size_t)m * M, *d0s = Sp + m * (m + 1) / 2, *invS = d0s + m;
    const double tp2 = TWO_PI_D;
    auto Hs = [&](int r, int c) { return r >= c ? H[tri(r, c)] : H[tri(c, r)]; };
    for (int e = tid; e < m * M; e += L) {
        const int k = e / M, j = e - k * M, u = M + 1 + 2 * k;
        Xs[e] = tp2 * (theta[2 + 2 * k] * H[tri(u, j)] - theta[1 + 2 * k] * H[tri(u + 1, j)]);
    }
    for (int k = tid; k < m; k += L) {
        const int u = M + 1 + 2 * k;
        g[k] = tp2 * (theta[2 + 2 * k] * H[tri(u, M)] - theta[1 + 2 * k] * H[tri(u + 1, M)]);
    }
    for (int e = tid; e < m * (m + 1) / 2; e += L) {
        int k = 0;
        while (tri(k + 1, 0) <= e) ++k;
        const int l = e - tri(k, 0);
        const double ak = theta[1 + 2 * k], bk = theta[2 + 2 * k], al = theta[1 + 2 * l], bl = theta[2 + 2 * l];
        const int uk = M + 1 + 2 * k, ul = M + 1 + 2 * l;
        Sp[e] = tp2 * tp2 *
                (bk * bl * Hs(uk, ul) - bk * al * Hs(uk, ul + 1) - ak * bl * Hs(uk + 1, ul) + ak * al * Hs(uk + 1, ul + 1));
    }
    __syncthreads();
    // X = L^{-1} <phi d>: column k of X is row k of Xs; rows eliminated four
    // at a time (the four-row diagonal block by one thread per column, then
    // the rows below by all threads), in the order of the row-by-row
    // elimination for every entry
    for (int r0 = 0; r0 < M; r0 += 4) {
        const int nr = M - r0 < 4 ? M - r0 : 4;
        for (int k = tid; k < m; k += L) {
            double *x = Xs + (size_t)k * M;
            for (int u = 0; u < nr; ++u) {
                const int r = r0 + u;
                x[r] *= invL[r];
                for (int v = u + 1; v < nr; ++v) x[r0 + v] -= H[tri(r0 + v, r)] * x[r];
            }
        }
        __syncthreads();
        const int rest = M - r0 - nr;
        for (int e = tid; e < m * rest; e += L) {
            const int k = e / rest, rr = r0 + nr + (e - k * rest);
            double v = Xs[k * M + rr];
            for (int u = 0; u < nr; ++u) v -= H[tri(rr, r0 + u)] * Xs[k * M + r0 + u];
            Xs[k * M + rr] = v;
        }
        __syncthreads();
    }
    for (int e = tid; e < m * (m + 1) / 2; e += L) {
        int k = 0;
        while (tri(k + 1, 0) <= e) ++k;
        const int l = e - tri(k, 0);
        double v = Sp[e];
        for (int r = 0; r < M; ++r) v -= Xs[k * M + r] * Xs[l * M + r];
        Sp[e] = v;
    }
    for (int k = tid; k < m; k += L) {
        double v = g[k];
        for (int r = 0; r < M; ++r) v -= Xs[k * M + r] * H[tri(M, r)];
        g[k] = v;
    }
    __syncthreads();
    if (!step) return true;
    chol_cta(Sp, d0s, invS, m, 0, m, s);
    if (s.fail_at < m) return false;
    if (tid < 32) {
        for (int k = tid; k < m; k += 32) step[k] = g[k];
        __syncwarp();
        fwd_warp(Sp, invS, m, step);
        bwd_warp(Sp, invS, 0, m, step);
    }
    __syncthreads();
    return true;
}

__device__ void set_trial(TState &s, int m, const double *src_delta, const double *src_step, double h) {
    for (int q = threadIdx.x; q < m; q += blockDim.x) {
        const double v = src_delta[q] + (src_step ? h * src_step[q] : 0.0);
        s.trial[q] = v;
        s.trialf[q] = (float)v;
        const ff vf = ff_from_double(v);
        s.trialff[q] = make_float2(vf.hi, vf.lo);
    }
}

template <class T, bool TC = false>
__device__ void tuple_work(const TupleArgs &a, TState &s, const void *tab, double *Gs, double *d0, double *inv,
                           unsigned char *R, int64_t k, TcState *tc = nullptr) {
    const int tid = threadIdx.x;
    const int64_t o0 = a.off[k];
    if (tid == 0) s.m = (int)(a.off[k + 1] - o0);
    __syncthreads();
    const int m = s.m, M = 2 * m + 1;
    for (int q = tid; q < m; q += blockDim.x) {
        s.pidx[q] = a.idx[o0 + q];
        s.delta[q] = 0.0;
        s.trial[q] = 0.0;
        s.trialf[q] = 0.0f;
        s.trialff[q] = make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    const double D = a.sp->D;
    const bool mixed = TP<T>::mixed;
    const bool uv = a.mode == 1 || a.mode == 2;
    double *W = reinterpret_cast<double *>(R);   // extension scratch (free after a pass)
    auto pass = [&](bool with_uv) {
        if constexpr (TC) gram_pass_tc(a, s, tab, Gs, *tc, m, with_uv);
        else gram_pass<T>(a, s, tab, Gs, R, m, with_uv);
    };
    pass(uv);
    if (a.mode == 3) {
        for (int e = tid; e < (M + 1) * (M + 2) / 2; e += blockDim.x) a.gram_out[e] = Gs[e];
        if (tid == 0) a.status[k] = 0;
        return;
    }
    chol_cta(Gs, d0, inv, M + 1, M, M, s);
    if (s.fail_at < M) {
        if (tid == 0) {
            a.status[k] = 1;
            if (a.z) a.z[k] = NAN;
            if (a.l_out) a.l_out[k] = NAN;
        }
        if (a.mode == 1)
            for (int q = tid; q < m; q += blockDim.x) a.dzdf[o0 + q] = NAN;
        return;
    }
    if (tid < 32) linear_solution(Gs, inv, M, s.theta, &s.red);
    __syncthreads();
    double ratio = s.ratio;
    if (a.mode == 0 || a.mode == 1) {
        if (a.mode == 1) extend_cta(Gs, inv, M, m, s.theta, W, s.x, nullptr, s);
        if (a.mode == 1)
            for (int q = tid; q < m; q += blockDim.x) a.dzdf[o0 + q] = s.x[q];
        if (tid == 0) {
            a.z[k] = 0.5 * s.red;
            a.status[k] = (mixed && ratio < TUPLE_TAU) ? 2 : 0;
        }
        return;
    }
    // refinement: exact Gauss-Newton steps, each trial point one pass
    // a mixed tuple that meets an ill-conditioned system is redone from scratch
    // in FP64, so its FP32 refinement stops there
    bool have_step = !(mixed && ratio < TUPLE_TAU) && extend_cta(Gs, inv, M, m, s.theta, W, s.x, s.step, s);
    double lacc = D - s.red;
    const double margin = TP<T>::l_noise > 0.0 ? TP<T>::l_noise * D : 1e-15 * fabs(lacc);
    const int max_halvings = mixed ? MAX_HALVINGS_MIXED : MAX_HALVINGS;
    const double span = a.sp->span;
    int it = 0, fails = 0, flat = 0;
    double h = 1.0;
    while (have_step && it < a.max_iter) {
        set_trial(s, m, s.delta, s.step, h);
        __syncthreads();
        pass(true);
        chol_cta(Gs, d0, inv, M + 1, M, M, s);
        const bool lin_ok = s.fail_at >= M;
        if (lin_ok && tid < 32) linear_solution(Gs, inv, M, s.x, &s.redx);
        __syncthreads();
        const double lt = D - s.redx;
        if (lin_ok && lt <= lacc + margin) {
            double smax = 0.0;
            for (int q = 0; q < m; ++q) smax = fmax(smax, fabs(s.step[q]));
            const double moved = h * smax * span;
            const double gain = lacc - lt;
            lacc = lt;
            ratio = fmin(ratio, s.ratio);
            ++it;
            __syncthreads();
            for (int q = tid; q < m; q += blockDim.x) s.delta[q] = s.trial[q];
            for (int r = tid; r < M; r += blockDim.x) s.theta[r] = s.x[r];
            if (tid == 0) s.red = s.redx;
            __syncthreads();
            if (mixed && ratio < TUPLE_TAU) break;
            have_step = extend_cta(Gs, inv, M, m, s.theta, W, s.x, s.step, s);
            // two full Gauss-Newton steps in a row that change l by less than
            // its FP32 noise: the mixed sums cannot resolve the minimum further
            flat = (mixed && h == 1.0 && gain < 0.1 * margin) ? flat + 1 : 0;
            h = 1.0;
            fails = 0;
            if (moved < a.tol || flat >= 2) break;
        } else {
            h *= 0.5;
            if (++fails > max_halvings) break;
        }
    }
    if (tid == 0) {
        for (int q = 0; q < m; ++q) a.f_out[o0 + q] = a.pool[s.pidx[q]] + s.delta[q];
        a.l_out[k] = lacc;
        if (a.iters) a.iters[k] = it;
        a.status[k] = (mixed && ratio < TUPLE_TAU) ? 2 : 0;   // worst conditioning on the way
    }
}

// NT threads per CTA: 64 when two 4x4 blocks per thread cover the widest Gram
// of the launch (more tuples per SM, so one tuple's serial FP64 solve leaves
// fewer warps idle), else 128.
template <class T> constexpr int tuple_min_blocks(int nt) {
    return (std::is_same<T, FF>::value ? 608 : TP<T>::mixed ? 512 : 384) / nt;
}

template <class T, int NT>
__global__ void __launch_bounds__(NT, tuple_min_blocks<T>(NT)) tuple_kernel(TupleArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int CP = (a.cmax + 3) & ~3;
    size_t o = 0;
    void *tab = smraw;
    o += std::is_same<T, FF>::value ? sizeof(SeedTableFF) : TP<T>::mixed ? sizeof(SeedTableF) : sizeof(SeedTable);
    o = (o + 15) & ~(size_t)15;
    TState &s = *reinterpret_cast<TState *>(smraw + o);
    o += sizeof(TState);
    o = (o + 15) & ~(size_t)15;
    double *Gs = reinterpret_cast<double *>(smraw + o);
    o += sizeof(double) * (size_t)a.cmax * (a.cmax + 1) / 2;
    double *d0 = reinterpret_cast<double *>(smraw + o);
    o += sizeof(double) * (size_t)a.cmax;
    double *inv = reinterpret_cast<double *>(smraw + o);
    o += sizeof(double) * (size_t)a.cmax;
    o = (o + 15) & ~(size_t)15;
    unsigned char *R = smraw + o;
    (void)CP;
    if constexpr (std::is_same<T, FF>::value) fill_seed_table_ff(*static_cast<SeedTableFF *>(tab));
    else if constexpr (TP<T>::mixed) fill_seed_table_f(*static_cast<SeedTableF *>(tab));
    else fill_seed_table(*static_cast<SeedTable *>(tab));
    __syncthreads();
    __shared__ int64_t cur;
    for (;;) {
        if (threadIdx.x == 0) cur = atomicAdd(a.next, 1);
        __syncthreads();
        const int64_t q = cur;
        if (q >= a.n_tuples) break;
        tuple_work<T>(a, s, tab, Gs, d0, inv, R, a.order ? (int64_t)a.order[q] : q);
        __syncthreads();
    }
}

// Float-float passes with the tensor-core Gram (modes 0-2, at most TC_ROWS
// columns): TC_THREADS threads (TC_WORKERS for the columns and readouts, the
// last warp's first lane issuing the MMAs; all of them in the solves) and the
// SM's tensor memory per CTA, one CTA per SM.
__global__ void __launch_bounds__(TC_THREADS, 1) tuple_kernel_tc(TupleArgs a) {
    extern __shared__ __align__(16) unsigned char tc_raw[];
    unsigned char *base = tc_raw + ((1024u - (smem_u32(tc_raw) & 1023u)) & 1023u);
    const TcLayout Lt = tc_layout(a.cmax);
    void *tab = base + Lt.tab;
    TState &s = *reinterpret_cast<TState *>(base + Lt.state);
    double *Gs = reinterpret_cast<double *>(base + Lt.gram);
    double *d0 = reinterpret_cast<double *>(base + Lt.d0);
    double *inv = reinterpret_cast<double *>(base + Lt.inv);
    unsigned char *R = base + Lt.R;
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + Lt.bar);
    uint32_t *slot = reinterpret_cast<uint32_t *>(base + Lt.slot);
    fill_seed_table_ff(*static_cast<SeedTableFF *>(tab));
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    if (threadIdx.x < 32) tmem_alloc(slot, TC_TMEM_COLS);
    // the zero tile after each buffer's seven digit tiles (the upper half of
    // the last stacked A operand)
    for (int b = 0; b < 2; ++b)
        for (size_t o = threadIdx.x * 16; o < TC_TILE; o += (size_t)blockDim.x * 16)
            *reinterpret_cast<uint4 *>(base + b * TC_BUF + TC_DIG * TC_TILE + o) = make_uint4(0u, 0u, 0u, 0u);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    TcState t{base, reinterpret_cast<float2 *>(base + Lt.acc), bar, a.err, *slot, {0u, 0u}, {false, false}};
    __shared__ int64_t cur;
    for (;;) {
        if (threadIdx.x == 0) cur = atomicAdd(a.next, 1);
        __syncthreads();
        const int64_t q = cur;
        if (q >= a.n_tuples) break;
        tuple_work<FF, true>(a, s, tab, Gs, d0, inv, R, a.order ? (int64_t)a.order[q] : q, &t);
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tmem_dealloc(t.tmem, TC_TMEM_COLS);
}

static_assert(sizeof(SeedTable) == sizeof(SeedTableFF), "the FF passes reuse the FP64 table's space");

size_t tuple_smem(int prec, int cmax, int chunk, int nt) {
    const size_t tsz = prec == FREDEC_MIXED ? 4 : 8;
    const int CP = (cmax + 3) & ~3;
    size_t o = prec == FREDEC_MIXED ? sizeof(SeedTableF) : sizeof(SeedTable);
    o = (o + 15) & ~(size_t)15;
    o += sizeof(TState);
    o = (o + 15) & ~(size_t)15;
    o += sizeof(double) * (size_t)cmax * (cmax + 1) / 2 + 2 * sizeof(double) * (size_t)cmax;
    o = (o + 15) & ~(size_t)15;
    o += std::max<size_t>((size_t)chunk * CP * tsz, (size_t)nt * 16 * 8);
    return o;
}

int tuple_chunk(int prec, int cmax) {
    const size_t tsz = prec == FREDEC_MIXED ? 4 : 8;
    const int CP = (cmax + 3) & ~3;
    return (int)std::max<size_t>(1, std::min<size_t>(WT_THREADS, CHUNK_BYTES / (CP * tsz)));
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
            const double il = 1.0 / ljj;
            for (int i = j + 1 + lane; i < M; i += 32) A[w][tri(i, j)] *= il;
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

// Threads of the CTA kernel: the width whose lanes the Gram blocks of the
// launch's widest tuple use best (64, 96 or 128 threads with QB blocks a
// thread for FP32 sums; 64 to 256 threads with one block each for
// float-float sums).  FP64 sums always take 128: their pass is bound by the
// FP64 pipes, which four warps spread over all four SM sub-partitions.
static int cta_threads(int precision, int cmax) {
    const int nb = ((cmax + 3) & ~3) / 4, nblk = nb * (nb + 1) / 2;
    if (precision == FREDEC_FP64) return WT_THREADS;
    const bool ff = precision == PREC_FF;
    const int qb = ff ? 1 : QB;
    int best = ff ? 256 : WT_THREADS;
    double best_u = -1.0;
    for (int L : {64, 96, 128, 160, 192, 256}) {
        if ((!ff && L > WT_THREADS) || nblk > qb * L) continue;
        const double u = nblk <= L ? (double)(L / nblk * nblk) / L : (double)nblk / (L * ((nblk + L - 1) / L));
        if (u > best_u + 1e-9) {
            best_u = u;
            best = L;
        }
    }
    return best;
}

template <class T, int NT>
static int launch_tuples_t(const TupleArgs &a, size_t smem, cudaStream_t st) {
    auto kern = tuple_kernel<T, NT>;
    FREDEC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    FREDEC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
    const int64_t grid = std::min<int64_t>(std::max<int64_t>(a.n_tuples, 1), (int64_t)std::max(per_sm, 1) * sm_count());
    kern<<<(unsigned)grid, NT, smem, st>>>(a);
    FREDEC_CUDA_TRY(cudaGetLastError());
    return FREDEC_OK;
}

// The tensor-core float-float kernel, one CTA per SM; -1 when its shared
// memory does not fit.
static int launch_tuples_tc(const TupleArgs &a, cudaStream_t st) {
    const size_t smem = tc_layout(a.cmax).bytes;
    if (smem > 227 * 1024) return -1;
    FREDEC_CUDA_TRY(cudaFuncSetAttribute(tuple_kernel_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t grid = std::min<int64_t>(std::max<int64_t>(a.n_tuples, 1), (int64_t)sm_count());
    tuple_kernel_tc<<<(unsigned)grid, TC_THREADS, smem, st>>>(a);
    FREDEC_CUDA_TRY(cudaGetLastError());
    return FREDEC_OK;
}

static int launch_tuples(TupleArgs a, int precision, cudaStream_t st) {
    // the tensor cores pay off from about 40 columns on: the Gram grows as
    // C^2, the column generation and digit split as C (measured per size
    // range on the 16-frequency pool: 2.6x faster at 13-15 frequencies,
    // 1.2x at 10-12, slower below)
    if (precision == PREC_FF && a.mode <= 2 && a.cmax > TC_MIN_COLS && a.cmax <= TC_ROWS && a.err) {
        const int rc = launch_tuples_tc(a, st);
        if (rc != -1) return rc;
    }
    const int nt = cta_threads(precision, a.cmax);
    const size_t smem = tuple_smem(precision, a.cmax, a.chunk, nt);
    if (precision == FREDEC_FP64) return launch_tuples_t<double, WT_THREADS>(a, smem, st);
    if (precision == FREDEC_MIXED) {
        if (nt == 64) return launch_tuples_t<float, 64>(a, smem, st);
        if (nt == 96) return launch_tuples_t<float, 96>(a, smem, st);
        return launch_tuples_t<float, 128>(a, smem, st);
    }
    switch (nt) {
    case 64: return launch_tuples_t<FF, 64>(a, smem, st);
    case 96: return launch_tuples_t<FF, 96>(a, smem, st);
    case 128: return launch_tuples_t<FF, 128>(a, smem, st);
    case 160: return launch_tuples_t<FF, 160>(a, smem, st);
    case 192: return launch_tuples_t<FF, 192>(a, smem, st);
    default: return launch_tuples_t<FF, 256>(a, smem, st);
    }
}

constexpr int MAX_RANGES = 32;             // size ranges (and work counters) of one enqueue

// Device inputs of one tuple launch: the series, the pool frequencies, the
// tuples as indices into the pool (CSR: tuple k holds pool[idx[off[k] ..
// off[k+1])]) and the processing order (largest tuples first), with host
// copies of the offsets and the order (the launches are split by size).
struct TupleDevIn {
    const double *t, *y, *sigma;
    int64_t N;
    const double *pool;
    int npool;
    const int32_t *idx;
    const int64_t *off;
    const int32_t *order;
    int64_t nt;
    int mmax;                  // largest tuple
    const int64_t *off_h;      // host: off
    const int32_t *order_h;    // host: order
};

// Columns of a tuple of m frequencies in a pass of the mode.
static int tuple_cols(int mode, int m) { return std::max(2, mode == 0 ? 2 * m + 2 : 4 * m + 2); }

// Side streams of the size-range launches, one set per host thread and
// device, created on first use and kept.
constexpr int RANGE_STREAMS = 4;
static int range_streams(cudaStream_t **out) {
    static thread_local cudaStream_t cached[16][RANGE_STREAMS] = {};
    int dev = 0;
    FREDEC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 16) return fail(FREDEC_ECUDA, "device index out of range for the tuple streams");
    for (int i = 0; i < RANGE_STREAMS; ++i)
        if (!cached[dev][i]) FREDEC_CUDA_TRY(cudaStreamCreateWithFlags(&cached[dev][i], cudaStreamNonBlocking));
    *out = cached[dev];
    return FREDEC_OK;
}

// The tuples in processing order (sizes do not increase along it), one
// launch per range of three sizes, each with the shared memory and the CTA
// width of its largest tuple (a launch sized for the largest tuple of all
// leaves most lanes of the small ones idle) and a work counter of its own
// (a.next[r], zeroed by the caller).  The launches go to RANGE_STREAMS streams
// forked from st and joined back into it, so that one range's last tuples
// overlap the next range's first.
static int launch_tuple_ranges(const TupleArgs &a0, const TupleDevIn &in, int precision, cudaStream_t st) {
    auto size_at = [&](int64_t q) { const int32_t k = in.order_h[q]; return (int)(in.off_h[k + 1] - in.off_h[k]); };
    cudaStream_t *side = nullptr;
    if (int rc = range_streams(&side)) return rc;
    cudaEvent_t ev[RANGE_STREAMS + 1] = {};   // the fork, then one join per side stream
    for (int i = 0; i <= RANGE_STREAMS; ++i)
        if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(ev[j]);
            return fail(FREDEC_ECUDA, "event creation for the tuple streams");
        }
    cudaEvent_t fork = ev[0];
    if (cudaEventRecord(fork, st) != cudaSuccess) {
        for (int i = 0; i <= RANGE_STREAMS; ++i) cudaEventDestroy(ev[i]);
        return fail(FREDEC_ECUDA, "fork event");
    }
    bool used[RANGE_STREAMS] = {};
    int rc = FREDEC_OK, r = 0;
    for (int64_t lo = 0; lo < in.nt && !rc; ++r) {
        const int mtop = size_at(lo), mbot = std::max(0, mtop - 2);
        int64_t hi = lo;
        while (hi < in.nt && size_at(hi) >= mbot) ++hi;
        if (r >= MAX_RANGES) {
            rc = fail(FREDEC_ECUDA, "too many tuple size ranges");
            break;
        }
        TupleArgs a = a0;
        a.order = in.order + lo;
        a.n_tuples = hi - lo;
        a.cmax = tuple_cols(a.mode, mtop);
        a.chunk = tuple_chunk(precision, a.cmax);
        a.next = a0.next + r;
        const int si = r % RANGE_STREAMS;
        if (!used[si]) {
            used[si] = true;
            if (cudaStreamWaitEvent(side[si], fork, 0) != cudaSuccess) {
                rc = fail(FREDEC_ECUDA, "stream wait");
                break;
            }
        }
        rc = launch_tuples(a, precision, side[si]);
        lo = hi;
    }
    for (int i = 0; i < RANGE_STREAMS; ++i)   // join every forked stream, also after a failure
        if (used[i] && (cudaEventRecord(ev[1 + i], side[i]) != cudaSuccess ||
                        cudaStreamWaitEvent(st, ev[1 + i], 0) != cudaSuccess) && !rc)
            rc = fail(FREDEC_ECUDA, "join of the tuple streams");
    for (int i = 0; i <= RANGE_STREAMS; ++i) cudaEventDestroy(ev[i]);
    return rc;
}

// Enqueue the per-series constants, the per-point values, the pool's exact
// cos/sin and the tuple kernel on st; scratch in ws.  Outputs (device, each
// may be unused by the mode): z, dzdf, f_out, l_out, iters, status[nt];
// *sp_out receives the series constants (l_0 = D).
static int tuple_enqueue(const TupleDevIn &in, int mode, int precision, int max_iter, double tol, double *z,
                         double *dzdf, double *f_out, double *l_out, int32_t *iters, int32_t *status,
                         SeriesPrep **sp_out, DevBuf &ws, cudaStream_t st, int32_t **err_out = nullptr) {
    const int64_t N = in.N;
    const int npool = in.npool;
    const size_t tsz = precision == FREDEC_MIXED ? 4 : 8;
    size_t off = 0;
    auto take = [&](size_t n) { size_t at = off; off = (off + n + 255) / 256 * 256; return at; };
    const size_t o_sp = take(sizeof(SeriesPrep)), o_pts = take(N * 4 * tsz),
                 o_seed = take((size_t)npool * N * 2 * tsz + 16), o_next = take(4 * MAX_RANGES), o_err = take(8);
    if (int rc = ws.alloc(off, st)) return rc;
    unsigned char *b = ws.as<unsigned char>();
    FREDEC_CUDA_TRY(cudaMemsetAsync(b + o_next, 0, 4 * MAX_RANGES, st));
    FREDEC_CUDA_TRY(cudaMemsetAsync(b + o_err, 0, 8, st));
    if (err_out) *err_out = (int32_t *)(b + o_err);
    SeriesPrep *sp = (SeriesPrep *)(b + o_sp);
    if (sp_out) *sp_out = sp;
    series_prep<<<1, 256, 0, st>>>(in.t, in.y, in.sigma, N, sp);
    const unsigned pb = (unsigned)std::min<int64_t>(1024, (N + 255) / 256);
    const unsigned sb = (unsigned)std::min<int64_t>(4096, ((int64_t)npool * N + 255) / 256);
    if (precision == FREDEC_MIXED) {
        point_prep<float><<<pb, 256, 0, st>>>(in.t, in.y, in.sigma, N, sp, (Pt<float> *)(b + o_pts));
        if (npool) pool_seeds<float2><<<sb, 256, 0, st>>>(in.t, N, in.pool, npool, sp, (float2 *)(b + o_seed));
    } else if (precision == PREC_FF) {
        point_prep_ff<<<pb, 256, 0, st>>>(in.t, in.y, in.sigma, N, sp, (float4 *)(b + o_pts));
        if (npool) pool_seeds_ff<<<sb, 256, 0, st>>>(in.t, N, in.pool, npool, sp, (float4 *)(b + o_seed));
    } else {
        point_prep<double><<<pb, 256, 0, st>>>(in.t, in.y, in.sigma, N, sp, (Pt<double> *)(b + o_pts));
        if (npool) pool_seeds<double2><<<sb, 256, 0, st>>>(in.t, N, in.pool, npool, sp, (double2 *)(b + o_seed));
    }
    FREDEC_CUDA_TRY(cudaGetLastError());
    TupleArgs a{};
    a.N = N;
    a.sp = sp;
    a.pts = b + o_pts;
    a.seeds = b + o_seed;
    a.pool = in.pool;
    a.idx = in.idx;
    a.off = in.off;
    a.order = in.order;
    a.n_tuples = in.nt;
    a.mode = mode;
    a.max_iter = max_iter;
    a.tol = tol;
    a.z = z;
    a.dzdf = dzdf;
    a.f_out = f_out;
    a.l_out = l_out;
    a.iters = iters;
    a.status = status;
    a.next = (int32_t *)(b + o_next);
    a.err = (int32_t *)(b + o_err);
    a.cmax = tuple_cols(mode, in.mmax);
    a.chunk = tuple_chunk(precision, a.cmax);
    if (in.nt > 0) {
        const int rc = mode <= 2 ? launch_tuple_ranges(a, in, precision, st) : launch_tuples(a, precision, st);
        if (rc) return rc;
    }
    return FREDEC_OK;
}

static std::vector<int32_t> largest_first(const int64_t *off, int64_t nt) {
    std::vector<int32_t> order(std::max<int64_t>(nt, 1));
    std::iota(order.begin(), order.begin() + nt, 0);
    std::stable_sort(order.begin(), order.begin() + nt,
                     [&](int32_t p, int32_t q) { return off[p + 1] - off[p] > off[q + 1] - off[q]; });
    return order;
}

// Tuples given as indices into a pool of frequencies (CSR: tuple k holds
// pool[idx[off[k] .. off[k+1])]).  mode 0 z, 1 z and dz/df, 2 refinement.
// Host inputs and outputs; synchronous.  Mixed-precision tuples whose linear
// system was ill-conditioned anywhere on their way are redone from scratch
// with FP64-grade (float-float) sums (an inaccurate early step can lead a
// refinement into another basin, which a continuation would keep).
static int tuple_run(const double *t, const double *y, const double *sigma, int64_t N, const double *pool_h,
                     int npool, const std::vector<int32_t> &idx_h, const std::vector<int64_t> &off_h, int mode,
                     int precision, int max_iter, double tol, double *z_h, double *dzdf_h, double *f_h, double *l_h,
                     int32_t *iters_h, double *l0_h, cudaStream_t st) {
    const int64_t nt = (int64_t)off_h.size() - 1;
    const int64_t nflat = off_h.back();
    int mmax = 0;
    for (int64_t k = 0; k < nt; ++k) mmax = std::max<int>(mmax, (int)(off_h[k + 1] - off_h[k]));
    const std::vector<int32_t> order = largest_first(off_h.data(), nt);
    size_t off = 0;
    auto take = [&](size_t n) { size_t at = off; off = (off + n + 255) / 256 * 256; return at; };
    const size_t o_in = take(3 * N * 8), o_pool = take(npool * 8 + 8), o_idx = take(nflat * 4 + 4),
                 o_off = take((nt + 1) * 8), o_ord = take(nt * 4 + 4), o_z = take(nt * 8 + 8),
                 o_g = take(nflat * 8 + 8), o_f = take(nflat * 8 + 8), o_l = take(nt * 8 + 8),
                 o_it = take(nt * 4 + 4), o_st = take(nt * 4 + 4);
    DevBuf io, ws;
    if (int rc = io.alloc(off, st)) return rc;
    unsigned char *b = io.as<unsigned char>();
    double *dt = (double *)(b + o_in), *dy = dt + N, *ds = dy + N;
    FREDEC_CUDA_TRY(cudaMemcpyAsync(dt, t, N * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(dy, y, N * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(ds, sigma, N * 8, cudaMemcpyHostToDevice, st));
    if (npool) FREDEC_CUDA_TRY(cudaMemcpyAsync(b + o_pool, pool_h, npool * 8, cudaMemcpyHostToDevice, st));
    if (nflat) FREDEC_CUDA_TRY(cudaMemcpyAsync(b + o_idx, idx_h.data(), nflat * 4, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(b + o_off, off_h.data(), (nt + 1) * 8, cudaMemcpyHostToDevice, st));
    if (nt) FREDEC_CUDA_TRY(cudaMemcpyAsync(b + o_ord, order.data(), nt * 4, cudaMemcpyHostToDevice, st));
    TupleDevIn in{dt, dy, ds, N, (const double *)(b + o_pool), npool, (const int32_t *)(b + o_idx),
                  (const int64_t *)(b + o_off), (const int32_t *)(b + o_ord), nt, mmax, off_h.data(), order.data()};
    SeriesPrep *sp = nullptr;
    int32_t *derr = nullptr;
    if (int rc = tuple_enqueue(in, mode, precision, max_iter, tol, (double *)(b + o_z), (double *)(b + o_g),
                               (double *)(b + o_f), (double *)(b + o_l), (int32_t *)(b + o_it),
                               (int32_t *)(b + o_st), &sp, ws, st, &derr))
        return rc;
    FREDEC_CUDA_TRY(cudaStreamSynchronize(st));
    int32_t herr = 0;
    if (derr) FREDEC_CUDA_TRY(cudaMemcpy(&herr, derr, 4, cudaMemcpyDeviceToHost));
    if (herr) return fail(FREDEC_ETIMEOUT, "a bounded wait of the tensor-core tuple kernel gave up");
    std::vector<int32_t> status(std::max<int64_t>(nt, 1));
    if (nt) FREDEC_CUDA_TRY(cudaMemcpy(status.data(), b + o_st, nt * 4, cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < nt; ++k)
        if (status[k] == 1) return fail(FREDEC_ESINGULAR, "a tuple's normal matrix is singular (repeated frequency?)");
    if (z_h && nt) FREDEC_CUDA_TRY(cudaMemcpy(z_h, b + o_z, nt * 8, cudaMemcpyDeviceToHost));
    if (dzdf_h && nflat) FREDEC_CUDA_TRY(cudaMemcpy(dzdf_h, b + o_g, nflat * 8, cudaMemcpyDeviceToHost));
    if (f_h && nflat) FREDEC_CUDA_TRY(cudaMemcpy(f_h, b + o_f, nflat * 8, cudaMemcpyDeviceToHost));
    if (l_h && nt) FREDEC_CUDA_TRY(cudaMemcpy(l_h, b + o_l, nt * 8, cudaMemcpyDeviceToHost));
    if (iters_h && nt) FREDEC_CUDA_TRY(cudaMemcpy(iters_h, b + o_it, nt * 4, cudaMemcpyDeviceToHost));
    if (l0_h) {
        SeriesPrep h;
        FREDEC_CUDA_TRY(cudaMemcpy(&h, sp, sizeof(h), cudaMemcpyDeviceToHost));
        *l0_h = h.D;
    }
    // tuples whose FP32-accumulated systems were ill-conditioned: FP64 sums
    std::vector<int64_t> redo;
    for (int64_t k = 0; k < nt; ++k)
        if (status[k] == 2) redo.push_back(k);
    if (redo.empty()) return FREDEC_OK;
    const int64_t n2 = (int64_t)redo.size();
    std::vector<int64_t> off2(1, 0);
    std::vector<int32_t> idx2;
    for (int64_t k : redo) {
        for (int64_t q = off_h[k]; q < off_h[k + 1]; ++q) idx2.push_back(idx_h[q]);
        off2.push_back((int64_t)idx2.size());
    }
    const int64_t nf2 = off2.back();
    std::vector<double> z2(n2 + 1), g2(nf2 + 1), f2(nf2 + 1), l2(n2 + 1);
    std::vector<int32_t> it2(n2 + 1);
    if (int rc = tuple_run(t, y, sigma, N, pool_h, npool, idx2, off2, mode, PREC_FF,
                           max_iter, tol, z2.data(), g2.data(),
                           f2.data(), l2.data(), it2.data(), nullptr, st))
        return rc;
    for (int64_t r = 0; r < n2; ++r) {
        const int64_t k = redo[r];
        if (z_h) z_h[k] = z2[r];
        if (l_h) l_h[k] = l2[r];
        if (iters_h) iters_h[k] = it2[r];
        for (int64_t q = 0; q < off_h[k + 1] - off_h[k]; ++q) {
            if (dzdf_h) dzdf_h[off_h[k] + q] = g2[off2[r] + q];
            if (f_h) f_h[off_h[k] + q] = f2[off2[r] + q];
        }
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
                 o_pts = take(N * 32), o_seed = take((size_t)npool * N * 16 + 16), o_idx = take(npool * 4 + 4),
                 o_off = take(16), o_gram = take((size_t)Mx * (Mx + 1) / 2 * 8), o_st = take(8), o_next = take(8),
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
    point_prep<double><<<(unsigned)std::min<int64_t>(1024, (N + 255) / 256), 256, 0, st>>>(dt, dy, ds, N, sp,
                                                                                           (Pt<double> *)(b + o_pts));
    if (npool)
        pool_seeds<double2><<<(unsigned)std::min<int64_t>(4096, ((int64_t)npool * N + 255) / 256), 256, 0, st>>>(
            dt, N, (const double *)(b + o_pool), npool, sp, (double2 *)(b + o_seed));
    TupleArgs a{};
    a.N = N;
    a.sp = sp;
    a.pts = b + o_pts;
    a.seeds = b + o_seed;
    a.pool = (const double *)(b + o_pool);
    a.idx = (const int32_t *)(b + o_idx);
    a.off = (const int64_t *)(b + o_off);
    a.order = nullptr;
    a.n_tuples = 1;
    a.mode = 3;
    a.status = (int32_t *)(b + o_st);
    a.next = (int32_t *)(b + o_next);
    a.gram_out = (double *)(b + o_gram);
    a.cmax = Mx;
    a.chunk = tuple_chunk(FREDEC_FP64, a.cmax);
    if (int rc = launch_tuples(a, FREDEC_FP64, st)) return rc;
    const int64_t blocks = std::min<int64_t>((nmask + PM_WARPS - 1) / PM_WARPS, 64LL * sm_count());
    pool_mask_kernel<<<(unsigned)blocks, 32 * PM_WARPS, 0, st>>>((const double *)(b + o_gram), npool, sp, nmask,
                                                                  (double *)(b + o_tab));
    FREDEC_CUDA_TRY(cudaGetLastError());
    FREDEC_CUDA_TRY(cudaStreamSynchronize(st));
    FREDEC_CUDA_TRY(cudaMemcpy(l_table_h, b + o_tab, nmask * 8, cudaMemcpyDeviceToHost));
    return FREDEC_OK;
}

static int check_tuple_inputs(const double *t, const double *y, const double *sigma, int64_t N, const double *freqs,
                              const int64_t *off, int64_t n, int max_m = FREDEC_MAX_TUPLE) {
    if (!t || !y || !sigma || N < 1 || n < 0 || (n > 0 && !off)) return fail(FREDEC_EINVAL, "bad arguments");
    for (int64_t i = 0; i < N; ++i)
        if (!std::isfinite(t[i]) || !std::isfinite(y[i]) || !(sigma[i] > 0.0) || !std::isfinite(sigma[i]))
            return fail(FREDEC_EINVAL, "t, y must be finite and sigma finite and > 0");
    if (n > 0 && off[0] != 0) return fail(FREDEC_EINVAL, "tuple_offsets[0] must be 0");
    for (int64_t k = 0; k < n; ++k) {
        const int64_t m = off[k + 1] - off[k];
        if (m < 0 || m > max_m)
            return fail(FREDEC_EINVAL, max_m == FREDEC_MAX_TUPLE ? "tuple sizes must be in 0..FREDEC_MAX_TUPLE"
                                                                  : "pool sizes must be in 0..FREDEC_MAX_POOL");
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
    if (int rc = check_tuple_inputs(t, y, sigma, N, pool, off, 1, FREDEC_MAX_POOL)) return rc;
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
    // mixed precision: float-float (compensated FP32-pipe) sums, FP64 solves;
    // plain FP32 Gram sums leave the gradient at about 1e-4 relative
    int rc = tuple_run(t, y, sigma, N, tuple_freqs, (int)nflat, idx, off, 1,
                       precision == FREDEC_MIXED ? PREC_FF : precision, 0, 0.0, z_out, g.data(), nullptr, nullptr,
                       nullptr, nullptr, ts.s);
    if (rc) return rc;
    // the kernel returns <d r> with d = dmu/df; dz/df = -1/2 dchi2/df = <r dmu/df>
    for (int64_t q = 0; q < nflat; ++q) dz_df_out[q] = g[q];
    return FREDEC_OK;
}

int fredec_tuple_grad_dev(const double *t, const double *y, const double *sigma, int64_t N,
                          const double *tuple_freqs, const int64_t *tuple_offsets, int64_t n_tuples,
                          int32_t precision, double *z_out, double *dz_df_out, void *stream) {
    if (precision != FREDEC_FP64 && precision != FREDEC_MIXED) return fail(FREDEC_EINVAL, "bad precision");
    if (!t || !y || !sigma || N < 1 || n_tuples < 0 || (n_tuples > 0 && (!tuple_offsets || !z_out)))
        return fail(FREDEC_EINVAL, "bad arguments");
    if (n_tuples > 0 && tuple_offsets[0] != 0) return fail(FREDEC_EINVAL, "tuple_offsets[0] must be 0");
    int mmax = 0;
    for (int64_t k = 0; k < n_tuples; ++k) {
        const int64_t m = tuple_offsets[k + 1] - tuple_offsets[k];
        if (m < 0 || m > FREDEC_MAX_TUPLE) return fail(FREDEC_EINVAL, "tuple sizes must be in 0..FREDEC_MAX_TUPLE");
        if (N < 2 * m + 2) return fail(FREDEC_EINVAL, "N must exceed 2m+1 for every tuple");
        mmax = std::max<int>(mmax, (int)m);
    }
    const int64_t nflat = n_tuples ? tuple_offsets[n_tuples] : 0;
    if (nflat > 0 && (!tuple_freqs || !dz_df_out)) return fail(FREDEC_EINVAL, "null frequencies or dz_df_out");
    if (n_tuples == 0) return FREDEC_OK;
    const cudaStream_t st = (cudaStream_t)stream;
    std::vector<int32_t> idx(std::max<int64_t>(nflat, 1));
    for (int64_t q = 0; q < nflat; ++q) idx[q] = (int32_t)q;
    const std::vector<int32_t> order = largest_first(tuple_offsets, n_tuples);
    size_t off = 0;
    auto take = [&](size_t n) { size_t at = off; off = (off + n + 255) / 256 * 256; return at; };
    const size_t o_idx = take(nflat * 4 + 4), o_off = take((n_tuples + 1) * 8), o_ord = take(n_tuples * 4),
                 o_st = take(n_tuples * 4);
    DevBuf io, ws;
    if (int rc = io.alloc(off, st)) return rc;
    unsigned char *b = io.as<unsigned char>();
    // pageable sources: each copy returns once its data is staged
    if (nflat) FREDEC_CUDA_TRY(cudaMemcpyAsync(b + o_idx, idx.data(), nflat * 4, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(b + o_off, tuple_offsets, (n_tuples + 1) * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(b + o_ord, order.data(), n_tuples * 4, cudaMemcpyHostToDevice, st));
    TupleDevIn in{t, y, sigma, N, tuple_freqs, (int)nflat, (const int32_t *)(b + o_idx), (const int64_t *)(b + o_off),
                  (const int32_t *)(b + o_ord), n_tuples, mmax, tuple_offsets, order.data()};
    return tuple_enqueue(in, 1, precision == FREDEC_MIXED ? PREC_FF : precision, 0, 0.0, z_out, dz_df_out, nullptr,
                         nullptr, nullptr, (int32_t *)(b + o_st), nullptr, ws, st);
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
