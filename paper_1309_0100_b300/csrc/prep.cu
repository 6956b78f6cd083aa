// Prep of one or many series (FP64): weights w = 1/sigma^2, time origin t_c,
// the base model's columns orthonormalised in the weighted inner product
// <phi> = sum w phi (two rounds of Cholesky-QR), the base fit l(f') and the
// per-point records that the periodogram kernels stream.
//
// Paper: the base model is H_m with fixed frequencies f' (Eq. Hn); its linear
// fit is the Cholesky solve of Section 3 (Q = L L^T, a = L^{-1} g).  Here the
// factor is applied to the columns themselves (psi = L^{-1} phi), so that the
// per-frequency solve becomes the incremental two-row extension of L described
// for Q_f in Section 3.  The normalisations of Section 4.1 (Eq. idn) are used
// in the form that matters for the kernels: centred time, and
// <sin^2> = <1> - <cos^2>.
//
// Every kernel works on chunks of PREP_THREADS points of one series (one point
// per thread).  Each chunk writes partial sums; the last chunk of a series to
// finish (atomic counter) reduces them in chunk order, so results do not
// depend on scheduling.
#include <atomic>
#include <mutex>

#include <cooperative_groups.h>

#include "device_util.cuh"
#include "fredec_internal.cuh"

namespace fredec {

int prep_npart(int pmax) { return pmax * (pmax + 1) / 2 + pmax + 4; }

namespace {

struct PrepArgs {
    const SeriesDesc *desc;
    SeriesState *state;
    const int32_t *chunk_series;
    double *partials;
    int npart;
    double *psi;
    unsigned char *rec;
    unsigned char *rec64;   // optional float-float records (mixed runs with re-evaluation of flagged bins)
    const double *t, *y, *sigma, *base;
    int precision;
    int nset;               // 2: records also carry the t'-weighted values (frequency derivative)
};

constexpr int PREP_NV = NTRI + PMAX + 4;    // values summed per point, at most
constexpr int TR_WORDS = 32 * 33;           // a warp's transpose scratch (doubles)

// Dynamic shared memory of the chunk kernels: per warp a transpose scratch and
// its nv sums.
constexpr size_t prep_chunk_smem() { return sizeof(double) * (PREP_THREADS / 32) * (TR_WORDS + PREP_NV); }

// Reduce nv per-thread values over the CTA and store them as this chunk's
// partials.  vals may live in local memory.  Within a warp the values go
// through shared memory transposed, 32 at a time, and lane q adds the 32
// lanes' value q in lane order: nv FP64 additions per warp instead of the
// 5 nv of a butterfly (FP64 runs at 1/64 of the FP32 rate on this GPU).
__device__ void store_partials(const PrepArgs &a, int64_t chunk, const double *vals, int nv, double *sm) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    double *tr = sm + wid * TR_WORDS, *ws = sm + nw * TR_WORDS;
    for (int q0 = 0; q0 < nv; q0 += 32) {
        const int m = min(32, nv - q0);
        for (int q = 0; q < m; ++q) tr[lane * 33 + q] = vals[q0 + q];
        __syncwarp();
        if (lane < m) {
            double s = 0.0;
            for (int l = 0; l < 32; ++l) s += tr[l * 33 + lane];
            ws[wid * PREP_NV + q0 + lane] = s;
        }
        __syncwarp();
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nv; q += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += ws[w * PREP_NV + q];
        a.partials[chunk * a.npart + q] = s;
    }
}

// Last-block-done: returns true in exactly one CTA of the series (the last to
// arrive), after all partials of the series are visible.
__device__ bool arrive_last(SeriesState &st, int which, int nchunks) {
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(&st.counter[which], 1u);
        last = (prev == (unsigned)nchunks - 1);
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Sums of partials 0..nv-1 over the series' chunks into out[] (shared), by the
// whole CTA: lanes take values, every value is summed over the chunks in chunk
// order (deterministic); a chunk's values are contiguous, so the loads are
// coalesced and independent across chunks.  (Measured: four chunks in flight
// are faster here than sixteen.)
__device__ void sum_partials(const PrepArgs &a, const SeriesDesc &d, int nv, double *out) {
    for (int q = threadIdx.x; q < nv; q += blockDim.x) {
        const double *col = a.partials + d.chunk_off * a.npart + q;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int c = 0;
        for (; c + 4 <= d.nchunks; c += 4) {   // four chunks in flight, combined in a fixed order
            s0 += __ldcg(col + (int64_t)c * a.npart);
            s1 += __ldcg(col + (int64_t)(c + 1) * a.npart);
            s2 += __ldcg(col + (int64_t)(c + 2) * a.npart);
            s3 += __ldcg(col + (int64_t)(c + 3) * a.npart);
        }
        for (; c < d.nchunks; ++c) s0 += __ldcg(col + (int64_t)c * a.npart);
        out[q] = (s0 + s1) + (s2 + s3);
    }
    __syncthreads();
}
extern __shared__ double prep_sm[];
__device__ double *fin_buf() { return prep_sm; }

// Base columns at t' = t - t_c: [1, tau, ..., tau^npoly, cos, sin of every
// base frequency], tau = t' / tscale (the polynomial extension of Eq. H0).
// PT > 0: a base of PT = 1 + 2 nb columns without polynomial terms, known at
// compile time; PT = 0: the widths of the series descriptor.
template <int PT = 0>
__device__ __forceinline__ void base_basis(const PrepArgs &a, const SeriesDesc &d, double tscale, double tp,
                                           double *phi) {
    const int npoly = PT > 0 ? 0 : d.npoly, nb = PT > 0 ? (PT - 1) / 2 : d.nb;
    phi[0] = 1.0;
    const double tau = tp / tscale;
    for (int q = 1; q <= npoly; ++q) phi[q] = phi[q - 1] * tau;
    const int o = 1 + npoly;
    for (int k = 0; k < nb; ++k) {
        const double g = a.base[d.base_off + k];
        const uint64_t ph = frac_turns_u64(g, tp);
        double s, c;
        sincos_turns_d(ph, &s, &c);
        phi[o + 2 * k] = c;
        phi[o + 1 + 2 * k] = s;
    }
}

// Time scale of the polynomial columns from sum w, sum w u, sum w u^2 with
// u = t - t_first (shift-safe): twice the weighted standard deviation of t.
__device__ __forceinline__ double time_scale(double W, double Su, double Suu) {
    const double mu = Su / W, var = Suu / W - mu * mu;
    return var > 0.0 ? 2.0 * sqrt(var) : 1.0;
}

// K1: sum w, sum w t  ->  W, t_c.
__global__ void __launch_bounds__(PREP_THREADS) prep_k1(PrepArgs a) {
    const int64_t chunk = blockIdx.x;
    const int s = a.chunk_series[chunk];
    const SeriesDesc d = a.desc[s];
    SeriesState &st = a.state[s];
    const int64_t i = (chunk - d.chunk_off) * PREP_THREADS + threadIdx.x;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < d.N) {
        const double sg = a.sigma[d.obs_off + i];
        const double w = 1.0 / (sg * sg);
        const double ti = a.t[d.obs_off + i], u = ti - a.t[d.obs_off];
        v[0] = w;
        v[1] = w * ti;
        v[2] = w * u;
        v[3] = w * u * u;
    }
    store_partials(a, chunk, v, 4, prep_sm);
    if (arrive_last(st, 0, d.nchunks)) {
        double *f = fin_buf();
        sum_partials(a, d, 4, f);
        const double W = f[0], Swt = f[1];
        if (threadIdx.x == 0) {
            st.W = W;
            st.Swt = Swt;
            st.tscale = time_scale(W, f[2], f[3]);
            st.tc = rint(Swt / W);
            st.status = FREDEC_OK;
            st.counter[0] = 0;
        }
    }
}

// K2: raw base columns phi(t'), Gram Q1 = <phi phi^T>  ->  L1 = chol(Q1).
__global__ void __launch_bounds__(PREP_THREADS) prep_k2(PrepArgs a) {
    const int64_t chunk = blockIdx.x;
    const int s = a.chunk_series[chunk];
    const SeriesDesc d = a.desc[s];
    SeriesState &st = a.state[s];
    const int p = d.pb;
    const int64_t i = (chunk - d.chunk_off) * PREP_THREADS + threadIdx.x;
    double phi[PMAX], v[NTRI];
    for (int q = 0; q < p * (p + 1) / 2; ++q) v[q] = 0.0;
    if (i < d.N) {
        const double sg = a.sigma[d.obs_off + i];
        const double w = 1.0 / (sg * sg);
        const double tp = a.t[d.obs_off + i] - st.tc;
        base_basis(a, d, st.tscale, tp, phi);
        for (int q = 0; q < p; ++q) a.psi[d.psi_off + (int64_t)q * d.N + i] = phi[q];
        for (int r = 0; r < p; ++r)
            for (int c = 0; c <= r; ++c) v[tri(r, c)] = w * phi[r] * phi[c];
    }
    store_partials(a, chunk, v, p * (p + 1) / 2, prep_sm);
    if (arrive_last(st, 1, d.nchunks)) {
        double *f = fin_buf();
        sum_partials(a, d, p * (p + 1) / 2, f);
        for (int q = threadIdx.x; q < p * (p + 1) / 2; q += blockDim.x) st.L1[q] = f[q];
        __syncthreads();
        if (threadIdx.x == 0) {
            if (!chol_packed(st.L1, p, 1e-12, st.R1)) st.status = FREDEC_ESINGULAR;
            st.counter[1] = 0;
        }
    }
}

// K3: psi1 = L1^{-1} phi, Gram Q2 = <psi1 psi1^T>, <psi1 y>  ->  L2, a = L2^{-1}<psi1 y>.
__global__ void __launch_bounds__(PREP_THREADS) prep_k3(PrepArgs a) {
    const int64_t chunk = blockIdx.x;
    const int s = a.chunk_series[chunk];
    const SeriesDesc d = a.desc[s];
    SeriesState &st = a.state[s];
    const int p = d.pb, nt = p * (p + 1) / 2;
    const int64_t i = (chunk - d.chunk_off) * PREP_THREADS + threadIdx.x;
    double x[PMAX], v[NTRI + PMAX];
    for (int q = 0; q < nt + p; ++q) v[q] = 0.0;
    if (i < d.N && st.status == FREDEC_OK) {
        const double sg = a.sigma[d.obs_off + i];
        const double w = 1.0 / (sg * sg);
        const double yi = a.y[d.obs_off + i];
        for (int q = 0; q < p; ++q) x[q] = a.psi[d.psi_off + (int64_t)q * d.N + i];
        forward_packed(st.L1, st.R1, x, p);
        for (int q = 0; q < p; ++q) a.psi[d.psi_off + (int64_t)q * d.N + i] = x[q];
        for (int r = 0; r < p; ++r)
            for (int c = 0; c <= r; ++c) v[tri(r, c)] = w * x[r] * x[c];
        for (int q = 0; q < p; ++q) v[nt + q] = w * x[q] * yi;
    }
    store_partials(a, chunk, v, nt + p, prep_sm);
    if (arrive_last(st, 2, d.nchunks)) {
        double *f = fin_buf();
        sum_partials(a, d, nt + p, f);
        for (int q = threadIdx.x; q < nt + p; q += blockDim.x) {
            if (q < nt) st.L2[q] = f[q]; else st.a[q - nt] = f[q];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (st.status == FREDEC_OK) {
                if (!chol_packed(st.L2, p, 1e-12, st.R2)) st.status = FREDEC_ESINGULAR;
                else forward_packed(st.L2, st.R2, st.a, p);
            }
            st.counter[2] = 0;
        }
    }
}

// K4: psi = L2^{-1} psi1 (final orthonormal columns), r = y - a^T psi,
// <psi r>  ->  a2 (second-pass coefficients; tiny).
__global__ void __launch_bounds__(PREP_THREADS) prep_k4(PrepArgs a) {
    const int64_t chunk = blockIdx.x;
    const int s = a.chunk_series[chunk];
    const SeriesDesc d = a.desc[s];
    SeriesState &st = a.state[s];
    const int p = d.pb;
    const int64_t i = (chunk - d.chunk_off) * PREP_THREADS + threadIdx.x;
    double x[PMAX], v[PMAX];
    for (int q = 0; q < p; ++q) v[q] = 0.0;
    if (i < d.N && st.status == FREDEC_OK) {
        const double sg = a.sigma[d.obs_off + i];
        const double w = 1.0 / (sg * sg);
        double r = a.y[d.obs_off + i];
        for (int q = 0; q < p; ++q) x[q] = a.psi[d.psi_off + (int64_t)q * d.N + i];
        forward_packed(st.L2, st.R2, x, p);
        for (int q = 0; q < p; ++q) {
            a.psi[d.psi_off + (int64_t)q * d.N + i] = x[q];
            r -= st.a[q] * x[q];
        }
        for (int q = p; q < d.p; ++q) a.psi[d.psi_off + (int64_t)q * d.N + i] = 0.0;   // odd-width padding
        for (int q = 0; q < p; ++q) v[q] = w * x[q] * r;
    }
    store_partials(a, chunk, v, p, prep_sm);
    if (arrive_last(st, 3, d.nchunks)) {
        double *f = fin_buf();
        sum_partials(a, d, p, f);
        for (int q = threadIdx.x; q < p; q += blockDim.x) st.a2[q] = f[q];
        __syncthreads();
        if (threadIdx.x == 0) st.counter[3] = 0;
    }
}

// Slot of point i in the mixed-precision records: i K mod N, K the first
// integer >= 0.618 N coprime with N (a bijection of 0..N-1).  The weighted
// sums do not depend on the order of the points; in time order, the running
// FP32 sums of a low-frequency bin (sum w c psi_k, sum w r c) drift over long
// coherent stretches before they cancel, and their rounding grows with them
// (measured: z error 1.05e-5 at N = 70000 in time order).  Points spread over
// the whole span make them random walks.  The FP64 records stay in time order
// (the adjoint reads them per point).
// record_multiplier: K, computed once per thread; record_slot: i K mod N.
__device__ inline int64_t record_multiplier(int64_t N) {
    if (N <= 2) return 1;
    int64_t K = (int64_t)(0.6180339887498949 * (double)N);
    for (;; ++K) {   // ends at K = N - 1 at the latest (gcd(N - 1, N) = 1); in practice within a few steps
        int64_t x = K, y = N;
        while (y) {
            const int64_t r = x % y;
            x = y;
            y = r;
        }
        if (x == 1) return K;
    }
}
__device__ __forceinline__ int64_t record_slot(int64_t i, int64_t K, int64_t N) {
    return (int64_t)(((unsigned long long)i * (unsigned long long)K) % (unsigned long long)N);
}

// Writes the records of point i of series d (residual r, w, u = w psi; with
// a.nset == 2 also their products with t' = tp, the t-weighted averages of
// Eq. avrg1 that the frequency derivative needs; mixed records carry them
// divided by sqrt(w), the scale of the kernel's cos/sin); K = record_multiplier(d.N);
// PT as for base_basis (d.p = PT when PT > 0).
template <int PT = 0>
__device__ __forceinline__ void write_records(const PrepArgs &a, const SeriesDesc &d, int64_t i, int64_t K, double tp,
                                              double w, double r, const double *u) {
    const int p = PT > 0 ? PT : d.p;
    const int ns = a.nset;
    const int64_t slot = a.precision == FREDEC_MIXED ? record_slot(i, K, d.N) : i;
    const uint64_t A = frac_turns_u64(d.f0, tp);
    const uint64_t B = frac_turns_u64(d.df, tp);
    double sr, cr;
    sincos_turns_d(B, &sr, &cr);
    if (a.precision == FREDEC_MIXED) {
        const double sw = sqrt(w), isw = sw > 0.0 ? 1.0 / sw : 0.0;
        uint32_t *R = (uint32_t *)(a.rec + d.rec_off) + slot * rec32_words(p, ns);
        R[0] = (uint32_t)A;
        R[1] = (uint32_t)(A >> 32);
        R[2] = (uint32_t)B;
        R[3] = (uint32_t)(B >> 32);
        float *Rf = (float *)R;
        double s2, c2;   // the two-step rotation from the doubled exact phase
        sincos_turns_d(2 * B, &s2, &c2);
        Rf[4] = (float)cr;
        Rf[5] = (float)sr;
        Rf[6] = (float)c2;
        Rf[7] = (float)s2;
        Rf[8] = (float)rec_sqrt_w(w);
        Rf[9] = (float)(sw * r);
        for (int q = 0; q < p; ++q) Rf[10 + q] = (float)(u[q] * isw);
        for (int q = 10 + p; q < rec32_words(p); ++q) Rf[q] = 0.f;
        if (ns == 2) {
            float *R2 = Rf + rec32_words(p);
            R2[0] = (float)tp;
            R2[1] = (float)(sw * r * tp);
            for (int q = 0; q < p; ++q) R2[2 + q] = (float)(u[q] * isw * tp);
            for (int q = 2 + p; q < rec32_set_words(p); ++q) R2[q] = 0.f;
        }
    }
    if (a.precision == FREDEC_MIXED && a.rec64) {   // float-float records for the re-evaluation
        uint32_t *R = (uint32_t *)(a.rec64 + d.rec64_off) + slot * recff_words(p, ns);
        R[0] = (uint32_t)A;
        R[1] = (uint32_t)(A >> 32);
        R[2] = (uint32_t)B;
        R[3] = (uint32_t)(B >> 32);
        float *Rf = (float *)R;
        auto put = [&](float *at, double v) {
            const float hi = (float)v;
            at[0] = hi;
            at[1] = (float)(v - (double)hi);
        };
        put(Rf + 4, w);
        put(Rf + 6, w * r);
        for (int q = 0; q < p; ++q) put(Rf + 8 + 2 * q, u[q]);
        for (int q = 8 + 2 * p; q < recff_words(p); ++q) Rf[q] = 0.f;
        if (ns == 2) {
            float *R2 = Rf + recff_words(p);
            put(R2, w * tp);
            put(R2 + 2, w * r * tp);
            for (int q = 0; q < p; ++q) put(R2 + 4 + 2 * q, u[q] * tp);
            for (int q = 4 + 2 * p; q < recff_set_words(p); ++q) R2[q] = 0.f;
        }
    }
    unsigned char *r64 = a.precision == FREDEC_FP64 ? a.rec : nullptr;
    if (r64) {
        const int64_t off64 = d.rec_off;
        uint64_t *R = (uint64_t *)(r64 + off64) + i * rec64_words(p, ns);
        R[0] = A;
        R[1] = B;
        double *Rd = (double *)R;
        Rd[2] = cr;
        Rd[3] = sr;
        Rd[4] = w;
        Rd[5] = w * r;
        for (int q = 0; q < p; ++q) Rd[6 + q] = u[q];
        for (int q = 6 + p; q < rec64_words(p); ++q) Rd[q] = 0.0;
        if (ns == 2) {
            double *R2 = Rd + rec64_words(p);
            R2[0] = w * tp;
            R2[1] = w * r * tp;
            for (int q = 0; q < p; ++q) R2[2 + q] = u[q] * tp;
            for (int q = 2 + p; q < 2 + rec64_set_words(p); ++q) R2[q] = 0.0;
        }
    }
}

// K5: final residual r2 = y - (a + a2)^T psi, records for the grid, chi2 and
// the sum of the weights as the mixed kernel sees them.
__global__ void __launch_bounds__(PREP_THREADS) prep_k5(PrepArgs a) {
    const int64_t chunk = blockIdx.x;
    const int s = a.chunk_series[chunk];
    const SeriesDesc d = a.desc[s];
    SeriesState &st = a.state[s];
    const int p = d.pb;
    const int64_t i = (chunk - d.chunk_off) * PREP_THREADS + threadIdx.x;
    double v[2] = {0.0, 0.0};
    if (i < d.N && st.status == FREDEC_OK) {
        const double sg = a.sigma[d.obs_off + i];
        const double w = 1.0 / (sg * sg);
        const double tp = a.t[d.obs_off + i] - st.tc;
        double r = a.y[d.obs_off + i];
        double u[PMAX];
        for (int q = 0; q < p; ++q) {
            const double ps = a.psi[d.psi_off + (int64_t)q * d.N + i];
            r -= (st.a[q] + st.a2[q]) * ps;
            u[q] = w * ps;
        }
        for (int q = p; q < d.p; ++q) u[q] = 0.0;
        write_records(a, d, i, record_multiplier(d.N), tp, w, r, u);
        v[0] = w * r * r;
        v[1] = rec_weight(w);
    }
    store_partials(a, chunk, v, 2, prep_sm);
    if (arrive_last(st, 4, d.nchunks)) {
        double *f = fin_buf();
        sum_partials(a, d, 2, f);
        const double c2 = f[0], wf = f[1];
        if (threadIdx.x == 0) {
            st.chi2 = c2;
            st.Wf = wf;
            st.counter[4] = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// One CTA per series (series up to SERIES_PREP_MAX_N points): the same five
// phases as prep_k1..k5, separated by block barriers instead of kernel
// boundaries.  Per-thread partial sums over a strided set of points are
// combined by a fixed-order block reduction (deterministic).

constexpr int SP_THREADS = 256;
constexpr int SP_NV = PREP_NV;

// Block sum of vals[0..nv) (per-thread, may be local memory) into out[0..nv)
// (shared); all threads see out after return.  NV > 0: nv = NV at compile
// time (the loop unrolls and vals stays in registers).
template <int NV = 0>
__device__ __forceinline__ void block_reduce_vals(const double *vals, int nv_rt, double *red, double *out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nv = NV > 0 ? NV : nv_rt;
#pragma unroll
    for (int q = 0; q < nv; ++q) {
        const double v = warp_sum_d(vals[q]);
        if (lane == 0) red[wid * SP_NV + q] = v;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nv; q += blockDim.x) {
        double sm = 0.0;
        for (int w = 0; w < nw; ++w) sm += red[w * SP_NV + q];
        out[q] = sm;
    }
    __syncthreads();
}

// PT as for prep_cluster: the series' base of PT sinusoidal columns known at
// compile time, or 0 for any base.
template <int PT>
__device__ __forceinline__ void prep_series_body(const PrepArgs &a, const SeriesDesc &d, double *red, double *out,
                                                 int &ok) {
    const int s = blockIdx.x;
    SeriesState &st = a.state[s];
    const int p = PT > 0 ? PT : d.pb, nt = p * (p + 1) / 2, pw = PT > 0 ? PT : d.p;
    constexpr int NT = PT * (PT + 1) / 2;
    constexpr int PA = PT > 0 ? PT : PMAX;
    const int64_t N = d.N;
    double v[PT > 0 ? NT + PT + 4 : SP_NV];
    // 1: W, <t>  ->  t_c and the polynomial time scale
    v[0] = v[1] = v[2] = v[3] = 0.0;
    const double t_first = a.t[d.obs_off];
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double sg = a.sigma[d.obs_off + i], w = 1.0 / (sg * sg);
        const double ti = a.t[d.obs_off + i], u = ti - t_first;
        v[0] += w;
        v[1] += w * ti;
        v[2] += w * u;
        v[3] += w * u * u;
    }
    block_reduce_vals<4>(v, 4, red, out);
    const double W = out[0], tc = rint(out[1] / W), tscale = time_scale(W, out[2], out[3]);
    // 2: raw base columns, Gram Q1 -> L1
    for (int q = 0; q < nt; ++q) v[q] = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double sg = a.sigma[d.obs_off + i], w = 1.0 / (sg * sg);
        double phi[PA];
        base_basis<PT>(a, d, tscale, a.t[d.obs_off + i] - tc, phi);
        for (int q = 0; q < p; ++q) a.psi[d.psi_off + (int64_t)q * N + i] = phi[q];
        for (int r = 0; r < p; ++r)
            for (int c = 0; c <= r; ++c) v[tri(r, c)] += w * phi[r] * phi[c];
    }
    block_reduce_vals<NT>(v, nt, red, out);
    if (threadIdx.x == 0) {
        st.W = W;
        st.tc = tc;
        st.tscale = tscale;
        for (int q = 0; q < nt; ++q) st.L1[q] = out[q];
        ok = chol_packed(st.L1, p, 1e-12, st.R1);
        st.status = ok ? FREDEC_OK : FREDEC_ESINGULAR;
    }
    __syncthreads();
    if (!ok) return;
    // 3: psi1 = L1^{-1} phi, Gram Q2 and <psi1 y>  ->  L2, a
    for (int q = 0; q < nt + p; ++q) v[q] = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double sg = a.sigma[d.obs_off + i], w = 1.0 / (sg * sg), yi = a.y[d.obs_off + i];
        double x[PA];
        for (int q = 0; q < p; ++q) x[q] = a.psi[d.psi_off + (int64_t)q * N + i];
        forward_packed(st.L1, st.R1, x, p);
        for (int q = 0; q < p; ++q) a.psi[d.psi_off + (int64_t)q * N + i] = x[q];
        for (int r = 0; r < p; ++r)
            for (int c = 0; c <= r; ++c) v[tri(r, c)] += w * x[r] * x[c];
        for (int q = 0; q < p; ++q) v[nt + q] += w * x[q] * yi;
    }
    block_reduce_vals<NT + PT>(v, nt + p, red, out);
    if (threadIdx.x == 0) {
        for (int q = 0; q < nt; ++q) st.L2[q] = out[q];
        for (int q = 0; q < p; ++q) st.a[q] = out[nt + q];
        ok = chol_packed(st.L2, p, 1e-12, st.R2);
        if (ok) forward_packed(st.L2, st.R2, st.a, p);
        else st.status = FREDEC_ESINGULAR;
    }
    __syncthreads();
    if (!ok) return;
    // 4: psi = L2^{-1} psi1, r = y - a^T psi, <psi r>  ->  a2
    for (int q = 0; q < p; ++q) v[q] = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double sg = a.sigma[d.obs_off + i], w = 1.0 / (sg * sg);
        double x[PA], r = a.y[d.obs_off + i];
        for (int q = 0; q < p; ++q) x[q] = a.psi[d.psi_off + (int64_t)q * N + i];
        forward_packed(st.L2, st.R2, x, p);
        for (int q = 0; q < p; ++q) {
            a.psi[d.psi_off + (int64_t)q * N + i] = x[q];
            r -= st.a[q] * x[q];
        }
        for (int q = p; q < pw; ++q) a.psi[d.psi_off + (int64_t)q * N + i] = 0.0;   // odd-width padding
        for (int q = 0; q < p; ++q) v[q] += w * x[q] * r;
    }
    block_reduce_vals<PT>(v, p, red, out);
    if (threadIdx.x == 0)
        for (int q = 0; q < p; ++q) st.a2[q] = out[q];
    __syncthreads();
    // 5: final residual, records, chi2, sum of FP32 weights
    v[0] = v[1] = 0.0;
    const int64_t K = record_multiplier(N);
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double sg = a.sigma[d.obs_off + i], w = 1.0 / (sg * sg);
        const double tp = a.t[d.obs_off + i] - tc;
        double r = a.y[d.obs_off + i], u[PA];
        for (int q = 0; q < p; ++q) {
            const double ps = a.psi[d.psi_off + (int64_t)q * N + i];
            r -= (st.a[q] + st.a2[q]) * ps;
            u[q] = w * ps;
        }
        for (int q = p; q < pw; ++q) u[q] = 0.0;
        write_records<PT>(a, d, i, K, tp, w, r, u);
        v[0] += w * r * r;
        v[1] += rec_weight(w);
    }
    block_reduce_vals<2>(v, 2, red, out);
    if (threadIdx.x == 0) {
        st.chi2 = out[0];
        st.Wf = out[1];
    }
}

// One CTA per series; each series takes the body specialised for its base
// width when it has no polynomial terms.
__global__ void __launch_bounds__(SP_THREADS) prep_series(PrepArgs a) {
    extern __shared__ double sp_sm[];
    double *red = sp_sm, *out = sp_sm + (SP_THREADS / 32) * SP_NV;
    __shared__ int ok;
    const SeriesDesc d = a.desc[blockIdx.x];
    switch (d.npoly == 0 ? d.pb : 0) {
    case 1: prep_series_body<1>(a, d, red, out, ok); break;
    case 3: prep_series_body<3>(a, d, red, out, ok); break;
    case 5: prep_series_body<5>(a, d, red, out, ok); break;
    case 7: prep_series_body<7>(a, d, red, out, ok); break;
    default: prep_series_body<0>(a, d, red, out, ok); break;
    }
}

// ---------------------------------------------------------------------------
// One thread-block cluster per series (up to CL_MAX CTAs of CL_THREADS
// threads; series up to CLUSTER_PREP_MAX_N points): the five phases of
// prep_k1..k5 in one launch.  The phases are separated by cluster barriers
// instead of kernel boundaries, and the per-phase sums are exchanged through
// distributed shared memory: each CTA reduces its points (transposed warp
// sums, then its warps in order), publishes the CTA sums, and after the
// barrier every CTA adds the published sums of all CTAs in rank order, so all
// CTAs hold bitwise the same totals.  Each CTA then factors the Gram matrix
// itself: the factors, and every branch taken on them, are identical in all
// CTAs of the cluster, so every CTA reaches every barrier.

constexpr int CL_THREADS = 128;
constexpr int CL_MAX = 16;
constexpr int CL_WARPS = CL_THREADS / 32;

struct ClusterSmem {
    double tr[CL_WARPS][TR_WORDS];   // per-warp transpose scratch
    double ws[CL_WARPS][PREP_NV];    // per-warp sums
    double x[2][PREP_NV];            // published CTA sums (alternating)
    double out[PREP_NV];             // cluster totals
    double L1[NTRI], L2[NTRI], R1[PMAX], R2[PMAX], av[PMAX], a2[PMAX];
    int64_t K;                       // record multiplier (one-point-per-thread kernel)
    int ok;
};

// Cluster totals of nv per-thread values into sm.out (all threads of all CTAs).
// Buffer x[ph] is written before the barrier and read remotely after it; the
// next use of the same buffer comes after the next reduction's barrier, by
// which time every CTA has finished reading it.  NV > 0: nv = NV, known at
// compile time (the loops unroll and vals stays in registers).
template <int NV>
__device__ __forceinline__ void cluster_reduce(const double *vals, int nv_rt, ClusterSmem &sm, int &ph) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nv = NV > 0 ? NV : nv_rt;
#pragma unroll
    for (int q0 = 0; q0 < nv; q0 += 32) {
        const int m = min(32, nv - q0);
#pragma unroll
        for (int q = 0; q < m; ++q) sm.tr[wid][lane * 33 + q] = vals[q0 + q];
        __syncwarp();
        if (lane < m) {   // the 32 lanes' values in eight interleaved chains, combined as a fixed tree
            double c[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) c[k] = sm.tr[wid][k * 33 + lane];
#pragma unroll
            for (int l = 8; l < 32; l += 8)
#pragma unroll
                for (int k = 0; k < 8; ++k) c[k] += sm.tr[wid][(l + k) * 33 + lane];
            sm.ws[wid][q0 + lane] = ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
        }
        __syncwarp();
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nv; q += CL_THREADS) {
        static_assert(CL_WARPS == 4, "CTA sum tree");
        sm.x[ph][q] = (sm.ws[0][q] + sm.ws[1][q]) + (sm.ws[2][q] + sm.ws[3][q]);
    }
    cl.sync();
    const int nr = (int)cl.num_blocks();
    for (int q = threadIdx.x; q < nv; q += CL_THREADS) {
        double x[CL_MAX];   // all remote loads in flight, then added in rank order
#pragma unroll
        for (int r = 0; r < CL_MAX; ++r) x[r] = r < nr ? cl.map_shared_rank(&sm.x[ph][0], r)[q] : 0.0;
#pragma unroll
        for (int h = CL_MAX / 2; h >= 1; h /= 2)   // pairwise tree in rank order (absent ranks add 0)
#pragma unroll
            for (int r = 0; r < h; ++r) x[r] = x[2 * r] + x[2 * r + 1];
        sm.out[q] = x[0];
    }
    __syncthreads();
    ph ^= 1;
}

// PT > 0: every series has the PT = 1 + 2 nb columns of a sinusoidal base
// (no polynomial terms), so that the per-point sums and columns are
// compile-time sized and stay in registers; PT = 0: any base.
template <int PT>
__global__ void __launch_bounds__(CL_THREADS) prep_cluster(PrepArgs a) {
    allow_dependents();   // the periodogram kernel's CTAs may launch on the other SMs and wait there
    grid_dependency_wait();   // the series descriptor and state initialised by the previous kernel
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char cl_raw[];
    ClusterSmem &sm = *reinterpret_cast<ClusterSmem *>(cl_raw);
    const int nr = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int s = blockIdx.x / nr;
    const SeriesDesc d = a.desc[s];
    SeriesState &st = a.state[s];
    const int p = PT > 0 ? PT : d.pb, nt = p * (p + 1) / 2, pw = PT > 0 ? PT : d.p;
    constexpr int NT = PT * (PT + 1) / 2;                 // compile-time counts (0 when PT = 0)
    constexpr int PA = PT > 0 ? PT : PMAX;                // extent of the per-point column arrays
    const int64_t N = d.N, i0 = (int64_t)rank * CL_THREADS + threadIdx.x, di = (int64_t)nr * CL_THREADS;
    const bool lead = rank == 0 && threadIdx.x == 0;
    double v[PT > 0 ? NT + PT + 4 : PREP_NV];
    int ph = 0;
    // 1: W, <t>  ->  t_c and the polynomial time scale
    v[0] = v[1] = v[2] = v[3] = 0.0;
    const double t_first = a.t[d.obs_off];
    for (int64_t i = i0; i < N; i += di) {
        const double sg = a.sigma[d.obs_off + i], w = 1.0 / (sg * sg);
        const double ti = a.t[d.obs_off + i], u = ti - t_first;
        v[0] += w;
        v[1] += w * ti;
        v[2] += w * u;
        v[3] += w * u * u;
    }
    cluster_reduce<4>(v, 4, sm, ph);
    const double W = sm.out[0], tc = rint(sm.out[1] / W), tscale = time_scale(W, sm.out[2], sm.out[3]);
    // 2: raw base columns, Gram Q1 -> L1
    for (int q = 0; q < nt; ++q) v[q] = 0.0;
    for (int64_t i = i0; i < N; i += di) {
        const double sg = a.sigma[d.obs_off + i], w = 1.0 / (sg * sg);
        double phi[PA];
        base_basis<PT>(a, d, tscale, a.t[d.obs_off + i] - tc, phi);
        for (int q = 0; q < p; ++q) a.psi[d.psi_off + (int64_t)q * N + i] = phi[q];
        for (int r = 0; r < p; ++r)
            for (int c = 0; c <= r; ++c) v[tri(r, c)] += w * phi[r] * phi[c];
    }
    cluster_reduce<NT>(v, nt, sm, ph);
    if (threadIdx.x < 32) {   // warp 0 factors
        for (int q = threadIdx.x; q < nt; q += 32) sm.L1[q] = sm.out[q];
        __syncwarp();
        const bool ok = chol_packed_warp(sm.L1, p, 1e-12, sm.R1);
        if (threadIdx.x == 0) sm.ok = ok;
    }
    __syncthreads();
    if (lead) {
        st.W = W;
        st.tc = tc;
        st.tscale = tscale;
        st.status = sm.ok ? FREDEC_OK : FREDEC_ESINGULAR;
    }
    if (sm.ok) {
        // 3: psi1 = L1^{-1} phi, Gram Q2 and <psi1 y>  ->  L2, a
        for (int q = 0; q < nt + p; ++q) v[q] = 0.0;
        for (int64_t i = i0; i < N; i += di) {
            const double sg = a.sigma[d.obs_off + i], w = 1.0 / (sg * sg), yi = a.y[d.obs_off + i];
            double x[PA];
            for (int q = 0; q < p; ++q) x[q] = a.psi[d.psi_off + (int64_t)q * N + i];
            forward_packed(sm.L1, sm.R1, x, p);
            for (int q = 0; q < p; ++q) a.psi[d.psi_off + (int64_t)q * N + i] = x[q];
            for (int r = 0; r < p; ++r)
                for (int c = 0; c <= r; ++c) v[tri(r, c)] += w * x[r] * x[c];
            for (int q = 0; q < p; ++q) v[nt + q] += w * x[q] * yi;
        }
        cluster_reduce<NT + PT>(v, nt + p, sm, ph);
        if (threadIdx.x < 32) {   // warp 0 factors
            for (int q = threadIdx.x; q < nt; q += 32) sm.L2[q] = sm.out[q];
            for (int q = threadIdx.x; q < p; q += 32) sm.av[q] = sm.out[nt + q];
            __syncwarp();
            const bool ok = chol_packed_warp(sm.L2, p, 1e-12, sm.R2);
            if (threadIdx.x == 0) {
                sm.ok = ok;
                if (ok) forward_packed(sm.L2, sm.R2, sm.av, p);
            }
        }
        __syncthreads();
        if (lead && !sm.ok) st.status = FREDEC_ESINGULAR;
    }
    if (sm.ok) {
        // 4: psi = L2^{-1} psi1, r = y - a^T psi, <psi r>  ->  a2
        for (int q = 0; q < p; ++q) v[q] = 0.0;
        for (int64_t i = i0; i < N; i += di) {
            const double sg = a.sigma[d.obs_off + i], w = 1.0 / (sg * sg);
            double x[PA], r = a.y[d.obs_off + i];
            for (int q = 0; q < p; ++q) x[q] = a.psi[d.psi_off + (int64_t)q * N + i];
            forward_packed(sm.L2, sm.R2, x, p);
            for (int q = 0; q < p; ++q) {
                a.psi[d.psi_off + (int64_t)q * N + i] = x[q];
                r -= sm.av[q] * x[q];
            }
            for (int q = p; q < pw; ++q) a.psi[d.psi_off + (int64_t)q * N + i] = 0.0;   // odd-width padding
            for (int q = 0; q < p; ++q) v[q] += w * x[q] * r;
        }
        cluster_reduce<PT>(v, p, sm, ph);
        if (threadIdx.x < p) sm.a2[threadIdx.x] = sm.out[threadIdx.x];
        __syncthreads();
        // 5: final residual, records, chi2, sum of FP32 weights
        v[0] = v[1] = 0.0;
        const int64_t K = record_multiplier(N);
        for (int64_t i = i0; i < N; i += di) {
            const double sg = a.sigma[d.obs_off + i], w = 1.0 / (sg * sg);
            const double tp = a.t[d.obs_off + i] - tc;
            double r = a.y[d.obs_off + i], u[PA];
            for (int q = 0; q < p; ++q) {
                const double ps = a.psi[d.psi_off + (int64_t)q * N + i];
                r -= (sm.av[q] + sm.a2[q]) * ps;
                u[q] = w * ps;
            }
            for (int q = p; q < pw; ++q) u[q] = 0.0;
            write_records<PT>(a, d, i, K, tp, w, r, u);
            v[0] += w * r * r;
            v[1] += rec_weight(w);
        }
        cluster_reduce<2>(v, 2, sm, ph);
        if (lead) {
            for (int q = 0; q < nt; ++q) {
                st.L1[q] = sm.L1[q];
                st.L2[q] = sm.L2[q];
            }
            for (int q = 0; q < p; ++q) {
                st.R1[q] = sm.R1[q];
                st.R2[q] = sm.R2[q];
                st.a[q] = sm.av[q];
                st.a2[q] = sm.a2[q];
            }
            st.chi2 = sm.out[0];
            st.Wf = sm.out[1];
        }
    }
    cl.sync();   // no CTA leaves while another may still read its published sums
}

// The same for series of at most one point per thread (N <= CTAs x
// CL_THREADS) with a sinusoidal base of PT columns, kept in registers: each
// thread loads its point once, its weight is computed once, and its base
// columns stay in registers from phase to phase (only the final orthonormal
// columns are stored, for the adjoint).  The time origin's sums are added
// with the first Gram matrix, so the raw base columns take the series' first
// time as their origin (an origin shift rotates each cos/sin pair, so the
// columns' span, its orthonormal basis up to that rotation, and every result
// are unchanged); the records use t_c as before.  Warp 1 computes the record
// multiplier while warp 0 factors the first Gram matrix.
template <int PT>
__global__ void __launch_bounds__(CL_THREADS) prep_cluster_one(PrepArgs a) {
    allow_dependents();   // the periodogram kernel's CTAs may launch on the other SMs and wait there
    grid_dependency_wait();   // the series descriptor and state initialised by the previous kernel
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char cl_raw[];
    ClusterSmem &sm = *reinterpret_cast<ClusterSmem *>(cl_raw);
    const int nr = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int s = blockIdx.x / nr;
    const SeriesDesc d = a.desc[s];
    SeriesState &st = a.state[s];
    constexpr int NT = PT * (PT + 1) / 2;
    constexpr int NV = NT + PT > NT + 4 ? NT + PT : NT + 4;
    const int64_t N = d.N, i = (int64_t)rank * CL_THREADS + threadIdx.x;
    const bool has = i < N, lead = rank == 0 && threadIdx.x == 0;
    int ph = 0;
    const double t_first = a.t[d.obs_off];
    double w = 0.0, ti = t_first, yi = 0.0;
    if (has) {
        const double sg = a.sigma[d.obs_off + i];
        w = 1.0 / (sg * sg);
        ti = a.t[d.obs_off + i];
        yi = a.y[d.obs_off + i];
    }
    double x[PT], v[NV];
    // 1-2: W, <t>, the time scale's sums and the Gram Q1 of the raw columns -> t_c, L1
    const double u = ti - t_first;
    base_basis<PT>(a, d, 1.0, u, x);
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = 0.0;
    if (has) {
        v[0] = w;
        v[1] = w * ti;
        v[2] = w * u;
        v[3] = w * u * u;
#pragma unroll
        for (int r = 0; r < PT; ++r)
#pragma unroll
            for (int c = 0; c <= r; ++c) v[4 + tri(r, c)] += w * x[r] * x[c];
    }
    cluster_reduce<NT + 4>(v, NT + 4, sm, ph);
    const double W = sm.out[0], tc = rint(sm.out[1] / W), tscale = time_scale(W, sm.out[2], sm.out[3]);
    if (threadIdx.x < 32) {   // warp 0 factors
        for (int q = threadIdx.x; q < NT; q += 32) sm.L1[q] = sm.out[4 + q];
        __syncwarp();
        const bool ok = chol_packed_warp(sm.L1, PT, 1e-12, sm.R1);
        if (threadIdx.x == 0) sm.ok = ok;
    } else if (threadIdx.x == 32) {
        sm.K = record_multiplier(N);
    }
    __syncthreads();
    if (lead) {
        st.W = W;
        st.tc = tc;
        st.tscale = tscale;
        st.status = sm.ok ? FREDEC_OK : FREDEC_ESINGULAR;
    }
    if (sm.ok) {
        // 3: psi1 = L1^{-1} phi, Gram Q2 and <psi1 y>  ->  L2, a
        forward_packed(sm.L1, sm.R1, x, PT);
#pragma unroll
        for (int q = 0; q < NT + PT; ++q) v[q] = 0.0;
        if (has) {
#pragma unroll
            for (int r = 0; r < PT; ++r)
#pragma unroll
                for (int c = 0; c <= r; ++c) v[tri(r, c)] += w * x[r] * x[c];
#pragma unroll
            for (int q = 0; q < PT; ++q) v[NT + q] += w * x[q] * yi;
        }
        cluster_reduce<NT + PT>(v, NT + PT, sm, ph);
        if (threadIdx.x < 32) {   // warp 0 factors
            for (int q = threadIdx.x; q < NT; q += 32) sm.L2[q] = sm.out[q];
            for (int q = threadIdx.x; q < PT; q += 32) sm.av[q] = sm.out[NT + q];
            __syncwarp();
            const bool ok = chol_packed_warp(sm.L2, PT, 1e-12, sm.R2);
            if (threadIdx.x == 0) {
                sm.ok = ok;
                if (ok) forward_packed(sm.L2, sm.R2, sm.av, PT);
            }
        }
        __syncthreads();
        if (lead && !sm.ok) st.status = FREDEC_ESINGULAR;
    }
    if (sm.ok) {
        // 4: psi = L2^{-1} psi1, r = y - a^T psi, <psi r>  ->  a2
        forward_packed(sm.L2, sm.R2, x, PT);
        double r = yi;
#pragma unroll
        for (int q = 0; q < PT; ++q) r -= sm.av[q] * x[q];
#pragma unroll
        for (int q = 0; q < PT; ++q) v[q] = 0.0;
        if (has) {
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                a.psi[d.psi_off + (int64_t)q * N + i] = x[q];
                v[q] += w * x[q] * r;
            }
        }
        cluster_reduce<PT>(v, PT, sm, ph);
        if (threadIdx.x < PT) sm.a2[threadIdx.x] = sm.out[threadIdx.x];
        __syncthreads();
        // 5: final residual, records, chi2, sum of FP32 weights
        v[0] = v[1] = 0.0;
        if (has) {
            double r2 = yi, uu[PT];
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                r2 -= (sm.av[q] + sm.a2[q]) * x[q];
                uu[q] = w * x[q];
            }
            write_records<PT>(a, d, i, sm.K, ti - tc, w, r2, uu);
            v[0] += w * r2 * r2;
            v[1] += rec_weight(w);
        }
        cluster_reduce<2>(v, 2, sm, ph);
        if (lead) {
            for (int q = 0; q < NT; ++q) {
                st.L1[q] = sm.L1[q];
                st.L2[q] = sm.L2[q];
            }
            for (int q = 0; q < PT; ++q) {
                st.R1[q] = sm.R1[q];
                st.R2[q] = sm.R2[q];
                st.a[q] = sm.av[q];
                st.a2[q] = sm.a2[q];
            }
            st.chi2 = sm.out[0];
            st.Wf = sm.out[1];
        }
    }
    cl.sync();   // no CTA leaves while another may still read its published sums
}

}  // namespace

int launch_prep(const PrepPlan &pp, const double *t, const double *y, const double *sigma,
                const double *base, int precision, cudaStream_t st) {
    return run_prep_records(pp, t, y, sigma, base, precision, nullptr, st);
}

using PrepKernel = void (*)(PrepArgs);

// The cluster prep for a base width: specialised for the sinusoidal bases of
// up to five base frequencies, generic otherwise.
// Slots 1-6: prep_cluster for base widths 1, 3, ..., 11; 7-12: prep_cluster_one
// for the same widths; 0: the generic prep_cluster.
constexpr int CLUSTER_SLOTS = 13;
static int cluster_slot(int base_p) { return base_p >= 1 && base_p <= 11 && (base_p & 1) ? (base_p + 1) / 2 : 0; }
static PrepKernel cluster_kernel(int slot) {
    switch (slot) {
    case 1: return prep_cluster<1>;
    case 2: return prep_cluster<3>;
    case 3: return prep_cluster<5>;
    case 4: return prep_cluster<7>;
    case 5: return prep_cluster<9>;
    case 6: return prep_cluster<11>;
    case 7: return prep_cluster_one<1>;
    case 8: return prep_cluster_one<3>;
    case 9: return prep_cluster_one<5>;
    case 10: return prep_cluster_one<7>;
    case 11: return prep_cluster_one<9>;
    case 12: return prep_cluster_one<11>;
    default: return prep_cluster<0>;
    }
}

// CTAs per cluster for series of up to max_n points: enough for about one
// point per thread, at most 16 (8 where the device refuses 16); 0 when cluster
// launches cannot be used.  The attributes are set once per kernel and device
// (kernel attributes belong to the current device).
constexpr int CLUSTER_DEVICES = 64;
static int cluster_size_for(int64_t max_n, int slot) {
    static std::atomic<int> caps[CLUSTER_DEVICES][CLUSTER_SLOTS];
    static std::once_flag once;
    std::call_once(once, [] {
        for (auto &row : caps)
            for (auto &c : row) c.store(-1);
    });
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= CLUSTER_DEVICES) {
        cudaGetLastError();
        return 0;   // the chunked prep needs no attributes
    }
    int cap = caps[dev][slot].load();
    if (cap < 0) {
        const PrepKernel k = cluster_kernel(slot);
        cap = 0;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ClusterSmem)) ==
            cudaSuccess) {
            cap = 8;
            if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(CL_MAX);
                cfg.blockDim = dim3(CL_THREADS);
                cfg.dynamicSmemBytes = sizeof(ClusterSmem);
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeClusterDimension;
                at[0].val.clusterDim.x = CL_MAX;
                at[0].val.clusterDim.y = 1;
                at[0].val.clusterDim.z = 1;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                int nclusters = 0;
                if (cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg) == cudaSuccess && nclusters > 0)
                    cap = CL_MAX;
            }
        }
        cudaGetLastError();   // clear a refused attribute
        caps[dev][slot].store(cap);
    }
    if (cap == 0) return 0;
    const int64_t want = (max_n + CL_THREADS - 1) / CL_THREADS;
    int cs = 1;
    while (cs < cap && cs < want) cs *= 2;
    return cs;
}

// As launch_prep; rec64 (optional, mixed runs) also receives float-float
// records at each series' rec64_off.
int run_prep_records(const PrepPlan &pp, const double *t, const double *y, const double *sigma,
                     const double *base, int precision, void *rec64, cudaStream_t st, int nset) {
    PrepArgs a;
    a.nset = nset;
    a.rec64 = (unsigned char *)rec64;
    a.desc = pp.desc;
    a.state = pp.state;
    a.chunk_series = pp.chunk_series;
    a.partials = pp.partials;
    a.npart = prep_npart(pp.pmax);
    a.psi = pp.psi;
    a.rec = (unsigned char *)pp.rec;
    a.t = t;
    a.y = y;
    a.sigma = sigma;
    a.base = base;
    a.precision = precision;
    if (pp.nchunks <= 0) return FREDEC_OK;
    // One CTA per series when there are many series (the FP64 work of a single
    // series on one SM is slower than spreading it over many one-warp chunks).
    if (pp.S >= 256 && pp.max_n > 0 && pp.max_n <= SERIES_PREP_MAX_N) {
        const size_t smem = sizeof(double) * (SP_THREADS / 32 + 1) * SP_NV;
        prep_series<<<(unsigned)pp.S, SP_THREADS, smem, st>>>(a);
        FREDEC_CUDA_TRY(cudaGetLastError());
        return FREDEC_OK;
    }
    // A few series of moderate length: one cluster of up to 16 CTAs per series.
    if (pp.max_n > 0 && pp.max_n <= CLUSTER_PREP_MAX_N) {
        int slot = cluster_slot(pp.base_p);
        int cs = cluster_size_for(pp.max_n, slot);
        if (slot > 0 && cs > 0 && pp.max_n <= (int64_t)cs * CL_THREADS) {   // at most one point per thread
            const int one = cluster_size_for(pp.max_n, slot + 6);
            if (one == cs) slot += 6;
        }
        if (cs > 0) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)(pp.S * cs));
            cfg.blockDim = dim3(CL_THREADS);
            cfg.dynamicSmemBytes = sizeof(ClusterSmem);
            cfg.stream = st;
            cudaLaunchAttribute at[2];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = (unsigned)cs;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // see grid_dependency_wait
            at[1].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = at;
            cfg.numAttrs = 2;
            FREDEC_CUDA_TRY(cudaLaunchKernelEx(&cfg, cluster_kernel(slot), a));
            return FREDEC_OK;
        }
    }
    const size_t smem = prep_chunk_smem();
    const dim3 grid((unsigned)pp.nchunks);
    prep_k1<<<grid, PREP_THREADS, smem, st>>>(a);
    prep_k2<<<grid, PREP_THREADS, smem, st>>>(a);
    prep_k3<<<grid, PREP_THREADS, smem, st>>>(a);
    prep_k4<<<grid, PREP_THREADS, smem, st>>>(a);
    prep_k5<<<grid, PREP_THREADS, smem, st>>>(a);
    FREDEC_CUDA_TRY(cudaGetLastError());
    return FREDEC_OK;
}

}  // namespace fredec
