// Vector-Jacobian product of the residual periodogram with respect to y.
//
// Envelope theorem (the linear parameters are at their least-squares optimum):
//     dz_j/dy_i = w_i ( mu_j(t_i) - mu_base(t_i) ),
// and mu_j - mu_base is the projection of the base residual on the trial
// columns with the base part removed:
//     mu_j - mu_base = a_j c~_j + b_j s~_j,  c~ = c - P_base c,  s~ likewise,
// (a_j, b_j) the joint-fit amplitudes of cos/sin of 2 pi f_j (t - t_c).  So
//     dL/dy_i = sum_j v_j dz_j/dy_i = w_i ( g_i - sum_k psi_k(t_i) gamma_k ),
//     g_i = sum_j v_j ( a_j cos 2 pi f_j t'_i + b_j sin 2 pi f_j t'_i ),
//     gamma_k = <psi_k g>   (psi = orthonormal base columns).
// The hot part is g: the transpose of the forward trigonometric sums, one
// point per thread-lane and all grid frequencies along the loop, with the same
// exact fixed-point seeds and rotation recurrence as the forward kernels.
#include <algorithm>

#include "device_util.cuh"
#include "fredec_internal.cuh"

namespace fredec {


namespace {

constexpr int VJ_THREADS = 128;
constexpr int VJ_PT = 8;            // points per thread (measured: 5% faster than 4 on 1e5 points x 1e7 bins)
constexpr int VJ_TILE = 2048;       // frequencies staged per shared-memory tile
constexpr int VJ_SEG = 32;          // re-seed every 32 frequencies

__global__ void vjp_init(SeriesDesc *desc, SeriesDesc v, SeriesState *state, int32_t *cs, int64_t nchunks) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        *desc = v;
        for (int k = 0; k < 6; ++k) state->counter[k] = 0;
        state->status = FREDEC_OK;
    }
    for (int64_t q = i; q < nchunks; q += (int64_t)gridDim.x * blockDim.x) cs[q] = 0;
}

// (v_j a_j, v_j b_j) per frequency, in the accumulation precision.
template <class T>
__global__ void vjp_coef(const double *coef, const double *v, int64_t nf, T *ab) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nf; j += (int64_t)gridDim.x * blockDim.x) {
        ab[2 * j] = (T)(v[j] * coef[2 * j]);
        ab[2 * j + 1] = (T)(v[j] * coef[2 * j + 1]);
    }
}

// g partials: block (x: points, y: frequency chunk).  Records are the FP64
// records of the prep (phases A, B).  gpart[chunk * N + i].
template <class T>
__global__ void __launch_bounds__(VJ_THREADS) vjp_trig(const SeriesDesc *desc, const unsigned char *rec64,
                                                       const T *ab, int64_t chunk_len, double *gpart) {
    __shared__ __align__(16) T sab[2 * VJ_TILE];
    __shared__ SeedTable tab;
    __shared__ SeedTableF tabf;
    if constexpr (sizeof(T) == 8) fill_seed_table(tab); else fill_seed_table_f(tabf);
    const SeriesDesc d = *desc;
    const int p = d.p;
    const int rw = rec64_words(p);
    const int64_t j_begin = (int64_t)blockIdx.y * chunk_len;
    const int64_t j_end = std::min<int64_t>(d.nf, j_begin + chunk_len);
    uint64_t A[VJ_PT], B[VJ_PT];
    T cr[VJ_PT], sr[VJ_PT];
    double g[VJ_PT];            // FP64 path: running sum
    float ghi[VJ_PT], glo[VJ_PT];   // FP32 path: float-float running sum (no FP64-pipe conversions)
    int64_t idx[VJ_PT];
#pragma unroll
    for (int q = 0; q < VJ_PT; ++q) {
        const int64_t i = ((int64_t)blockIdx.x * VJ_PT + q) * VJ_THREADS + threadIdx.x;
        idx[q] = i;
        const int64_t ic = i < d.N ? i : d.N - 1;
        const uint64_t *R = reinterpret_cast<const uint64_t *>(rec64) + ic * rw;
        A[q] = R[0];
        B[q] = R[1];
        cr[q] = (T)reinterpret_cast<const double *>(R)[2];
        sr[q] = (T)reinterpret_cast<const double *>(R)[3];
        g[q] = 0.0;
        ghi[q] = 0.f;
        glo[q] = 0.f;
    }
    for (int64_t j0 = j_begin; j0 < j_end; j0 += VJ_TILE) {
        const int nt = (int)std::min<int64_t>(VJ_TILE, j_end - j0);
        __syncthreads();
        for (int k = threadIdx.x; k < 2 * nt; k += blockDim.x) sab[k] = ab[2 * j0 + k];
        __syncthreads();
        for (int seg = 0; seg < nt; seg += VJ_SEG) {
            const int ns = min(VJ_SEG, nt - seg);
            T c[VJ_PT], s[VJ_PT], acc[VJ_PT];
#pragma unroll
            for (int q = 0; q < VJ_PT; ++q) {
                const uint64_t ph = A[q] + (uint64_t)(j0 + seg) * B[q];
                if constexpr (sizeof(T) == 8) {
                    double ss, cc;
                    seed_from_table(tab, ph, &ss, &cc);
                    c[q] = cc;
                    s[q] = ss;
                } else {
                    float ss, cc;
                    seed_from_table_f(tabf, (uint32_t)(ph >> 32), &ss, &cc);
                    c[q] = cc;
                    s[q] = ss;
                }
                acc[q] = T(0);
            }
            auto step = [&](int k) {
                const T a = sab[2 * (seg + k)], b = sab[2 * (seg + k) + 1];
#pragma unroll
                for (int q = 0; q < VJ_PT; ++q) {
                    acc[q] = fma(a, c[q], fma(b, s[q], acc[q]));
                    const T cn = fma(c[q], cr[q], -s[q] * sr[q]);
                    s[q] = fma(s[q], cr[q], c[q] * sr[q]);
                    c[q] = cn;
                }
            };
            if (ns == VJ_SEG) {   // full segments: no loop bookkeeping
#pragma unroll
                for (int k = 0; k < VJ_SEG; ++k) step(k);
            } else {
                for (int k = 0; k < ns; ++k) step(k);
            }
#pragma unroll
            for (int q = 0; q < VJ_PT; ++q) {
                if constexpr (sizeof(T) == 8) {
                    g[q] += acc[q];
                } else {   // float-float running sum of the FP32 segment sums (TwoSum)
                    const float h = ghi[q], sum = h + acc[q], bp = sum - h;
                    glo[q] += (h - (sum - bp)) + (acc[q] - bp);
                    ghi[q] = sum;
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < VJ_PT; ++q) {
        if constexpr (sizeof(T) == 4) g[q] = (double)ghi[q] + (double)glo[q];
        if (idx[q] < d.N) gpart[(int64_t)blockIdx.y * d.N + idx[q]] = g[q];
    }
}

// Sum the frequency-chunk partials of g (in chunk order) and form the base
// projections gamma_k = <psi_k g> (per-CTA partials, last CTA combines).
__global__ void vjp_gamma(const SeriesDesc *desc, const double *psi, const double *t, const double *sigma,
                          double *gpart, int nchunk, double *gamma_part, double *gamma, uint32_t *counter) {
    const SeriesDesc d = *desc;
    const int p = d.p;
    __shared__ double red[32][PMAX];
    __shared__ int last;
    double loc[PMAX];
    for (int k = 0; k < p; ++k) loc[k] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += (int64_t)gridDim.x * blockDim.x) {
        double g = 0.0;
        for (int c = 0; c < nchunk; ++c) g += gpart[(int64_t)c * d.N + i];
        gpart[i] = g;                                   // chunk 0 now holds the total
        const double sg = sigma[i];
        const double w = 1.0 / (sg * sg);
        for (int k = 0; k < p; ++k) loc[k] += w * psi[(int64_t)k * d.N + i] * g;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < p; ++k) {
        const double v = warp_sum_d(loc[k]);
        if (lane == 0) red[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < p) {
        double v = 0.0;
        for (int w = 0; w < nw; ++w) v += red[w][threadIdx.x];
        gamma_part[(int64_t)blockIdx.x * PMAX + threadIdx.x] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (last) {
        __threadfence();
        if (threadIdx.x < p) {
            double v = 0.0;
            for (int b = 0; b < (int)gridDim.x; ++b) v += __ldcg(&gamma_part[(int64_t)b * PMAX + threadIdx.x]);
            gamma[threadIdx.x] = v;
        }
        if (threadIdx.x == 0) *counter = 0;
    }
}

__global__ void vjp_final(const SeriesDesc *desc, const double *psi, const double *sigma, const double *g,
                          const double *gamma, const SeriesState *state, double *out) {
    const SeriesDesc d = *desc;
    const bool ok = state->status == FREDEC_OK;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += (int64_t)gridDim.x * blockDim.x) {
        double s = g[i];
        for (int k = 0; k < d.p; ++k) s -= gamma[k] * psi[(int64_t)k * d.N + i];
        const double sg = sigma[i];
        out[i] = ok ? s / (sg * sg) : NAN;
    }
}

}  // namespace

int launch_vjp_pipeline(const double *t, const double *y, const double *sigma, int64_t N, const double *base, int nb,
                        double f0, double df, int64_t nf, const double *coef, const double *v, int precision,
                        double *dldy, cudaStream_t st) {
    const int p = 2 * nb + 1;
    const int64_t nchunks = (N + PREP_THREADS - 1) / PREP_THREADS;
    const int64_t npt = (int64_t)VJ_THREADS * VJ_PT;
    const int64_t gx = (N + npt - 1) / npt;
    // frequency chunks: enough CTAs to fill the GPU at least twice
    int64_t gy = std::max<int64_t>(1, (4LL * sm_count() + gx - 1) / gx);
    gy = std::min<int64_t>(gy, std::max<int64_t>(1, (nf + VJ_TILE - 1) / VJ_TILE));
    const int64_t chunk_len = (nf + gy - 1) / gy;
    const int gamma_blocks = (int)std::min<int64_t>(256, (N + 255) / 256);
    const size_t abw = precision == FREDEC_MIXED ? 4 : 8;
    size_t off = 0;
    auto take = [&](size_t n) { size_t at = off; off = (off + n + 255) / 256 * 256; return at; };
    const size_t o_desc = take(sizeof(SeriesDesc)), o_state = take(sizeof(SeriesState));
    const size_t o_cs = take(nchunks * 4), o_part = take(nchunks * prep_npart(p) * 8);
    const size_t o_psi = take((size_t)p * N * 8), o_rec = take(N * (size_t)rec_bytes(p, FREDEC_FP64));
    const size_t o_ab = take(2 * nf * abw + 16), o_g = take(gy * N * 8);
    const size_t o_gp = take(gamma_blocks * PMAX * 8), o_gm = take(PMAX * 8), o_cnt = take(4);
    DevBuf ws;
    if (int rc = ws.alloc(off, st)) return rc;
    unsigned char *b = ws.as<unsigned char>();
    SeriesDesc *desc = (SeriesDesc *)(b + o_desc);
    SeriesState *state = (SeriesState *)(b + o_state);
    SeriesDesc d{};
    d.f0 = f0;
    d.df = df;
    d.nf = nf;
    d.N = (int32_t)N;
    d.nb = nb;
    d.p = p;
    d.pb = p;
    d.npoly = 0;
    d.nchunks = (int32_t)nchunks;
    vjp_init<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(1024, (nchunks + 255) / 256)), 256, 0, st>>>(
        desc, d, state, (int32_t *)(b + o_cs), nchunks);
    FREDEC_CUDA_TRY(cudaMemsetAsync(b + o_cnt, 0, 4, st));
    PrepPlan pp;
    pp.S = 1;
    pp.max_n = N;
    pp.nchunks = nchunks;
    pp.pmax = p;
    pp.base_p = p;
    pp.desc = desc;
    pp.state = state;
    pp.chunk_series = (int32_t *)(b + o_cs);
    pp.partials = (double *)(b + o_part);
    pp.psi = (double *)(b + o_psi);
    pp.rec = b + o_rec;
    if (int rc = run_prep_records(pp, t, y, sigma, base, FREDEC_FP64, nullptr, st)) return rc;
    const dim3 grid((unsigned)gx, (unsigned)gy);
    if (precision == FREDEC_MIXED) {
        vjp_coef<float><<<256, 256, 0, st>>>(coef, v, nf, (float *)(b + o_ab));
        vjp_trig<float><<<grid, VJ_THREADS, 0, st>>>(desc, b + o_rec, (const float *)(b + o_ab), chunk_len,
                                                     (double *)(b + o_g));
    } else {
        vjp_coef<double><<<256, 256, 0, st>>>(coef, v, nf, (double *)(b + o_ab));
        vjp_trig<double><<<grid, VJ_THREADS, 0, st>>>(desc, b + o_rec, (const double *)(b + o_ab), chunk_len,
                                                      (double *)(b + o_g));
    }
    vjp_gamma<<<gamma_blocks, 256, 0, st>>>(desc, (const double *)(b + o_psi), t, sigma, (double *)(b + o_g), (int)gy,
                                            (double *)(b + o_gp), (double *)(b + o_gm), (uint32_t *)(b + o_cnt));
    vjp_final<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(1024, (N + 255) / 256)), 256, 0, st>>>(
        desc, (const double *)(b + o_psi), sigma, (const double *)(b + o_g), (const double *)(b + o_gm), state, dldy);
    FREDEC_CUDA_TRY(cudaGetLastError());
    return FREDEC_OK;
}

}  // namespace fredec
