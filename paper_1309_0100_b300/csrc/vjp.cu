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
static_assert(VJ_PT % 2 == 0, "the mixed kernel takes the points in pairs");

__global__ void vjp_init(SeriesDesc *desc, SeriesDesc v, SeriesState *state, int32_t *cs, int64_t nchunks) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        *desc = v;
        for (int k = 0; k < 6; ++k) state->counter[k] = 0;
        state->status = FREDEC_OK;
    }
    for (int64_t q = i; q < nchunks; q += (int64_t)gridDim.x * blockDim.x) cs[q] = 0;
}

// (v_j a_j, v_j b_j) per frequency (FP64 path).
__global__ void vjp_coef(const double *coef, const double *v, int64_t nf, double *ab) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nf; j += (int64_t)gridDim.x * blockDim.x) {
        ab[2 * j] = v[j] * coef[2 * j];
        ab[2 * j + 1] = v[j] * coef[2 * j + 1];
    }
}

// Mixed path: (v_j a_j, v_j a_j, v_j b_j, v_j b_j) per frequency, the
// duplicated pairs that the packed instructions of vjp_trig_mixed take.
__global__ void vjp_coef_pairs(const double *coef, const double *v, int64_t nf, float4 *ab) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nf; j += (int64_t)gridDim.x * blockDim.x) {
        const float a = (float)(v[j] * coef[2 * j]), b = (float)(v[j] * coef[2 * j + 1]);
        ab[j] = make_float4(a, a, b, b);
    }
}

// g partials of the mixed path: as vjp_trig with FP32 values, the thread's
// VJ_PT points in pairs held in float2 registers and updated by packed FP32
// instructions: per frequency and pair, acc += a c + b s (two FFMA2) and the
// rotation of (c, s) (two FMUL2, two FFMA2) -- half the warp instructions of
// the scalar loop, the same arithmetic per component.
__global__ void __launch_bounds__(VJ_THREADS) vjp_trig_mixed(const SeriesDesc *desc, const unsigned char *rec64,
                                                             const float4 *ab, int64_t chunk_len, double *gpart) {
    constexpr int NP = VJ_PT / 2;
    __shared__ __align__(16) float4 sab[VJ_TILE];
    __shared__ SeedTableF tabf;
    fill_seed_table_f(tabf);
    const SeriesDesc d = *desc;
    const int rw = rec64_words(d.p);
    const int64_t j_begin = (int64_t)blockIdx.y * chunk_len;
    const int64_t j_end = std::min<int64_t>(d.nf, j_begin + chunk_len);
    uint64_t A[VJ_PT], B[VJ_PT];
    float2 cr[NP], sr[NP], nsr[NP];
    float ghi[VJ_PT], glo[VJ_PT];   // float-float running sums (no FP64-pipe conversions)
    int64_t idx[VJ_PT];
#pragma unroll
    for (int q = 0; q < VJ_PT; ++q) {
        const int64_t i = ((int64_t)blockIdx.x * VJ_PT + q) * VJ_THREADS + threadIdx.x;
        idx[q] = i;
        const int64_t ic = i < d.N ? i : d.N - 1;
        const uint64_t *R = reinterpret_cast<const uint64_t *>(rec64) + ic * rw;
        A[q] = R[0];
        B[q] = R[1];
        const float c1 = (float)reinterpret_cast<const double *>(R)[2], s1 = (float)reinterpret_cast<const double *>(R)[3];
        if (q & 1) {
            cr[q / 2].y = c1;
            sr[q / 2].y = s1;
            nsr[q / 2].y = -s1;
        } else {
            cr[q / 2].x = c1;
            sr[q / 2].x = s1;
            nsr[q / 2].x = -s1;
        }
        ghi[q] = 0.f;
        glo[q] = 0.f;
    }
    for (int64_t j0 = j_begin; j0 < j_end; j0 += VJ_TILE) {
        const int nt = (int)std::min<int64_t>(VJ_TILE, j_end - j0);
        __syncthreads();
        for (int k = threadIdx.x; k < nt; k += blockDim.x) sab[k] = ab[j0 + k];
        __syncthreads();
        for (int seg = 0; seg < nt; seg += VJ_SEG) {
            const int ns = min(VJ_SEG, nt - seg);
            float2 c[NP], s[NP], acc[NP];
#pragma unroll
            for (int q = 0; q < VJ_PT; ++q) {
                const uint64_t ph = A[q] + (uint64_t)(j0 + seg) * B[q];
                float ss, cc;
                seed_from_table_f(tabf, (uint32_t)(ph >> 32), &ss, &cc);
                if (q & 1) {
                    c[q / 2].y = cc;
                    s[q / 2].y = ss;
                } else {
                    c[q / 2].x = cc;
                    s[q / 2].x = ss;
                }
            }
#pragma unroll
            for (int q = 0; q < NP; ++q) acc[q] = make_float2(0.f, 0.f);
            auto step = [&](int k) {
                const float4 w = sab[seg + k];
                const float2 a = make_float2(w.x, w.y), b = make_float2(w.z, w.w);
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    acc[q] = __ffma2_rn(a, c[q], __ffma2_rn(b, s[q], acc[q]));
                    const float2 cn = __ffma2_rn(c[q], cr[q], __fmul2_rn(s[q], nsr[q]));
                    s[q] = __ffma2_rn(s[q], cr[q], __fmul2_rn(c[q], sr[q]));
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
            for (int q = 0; q < VJ_PT; ++q) {   // float-float running sum of the segment sums (TwoSum)
                const float a = (q & 1) ? acc[q / 2].y : acc[q / 2].x;
                const float h = ghi[q], sum = h + a, bp = sum - h;
                glo[q] += (h - (sum - bp)) + (a - bp);
                ghi[q] = sum;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < VJ_PT; ++q)
        if (idx[q] < d.N) gpart[(int64_t)blockIdx.y * d.N + idx[q]] = (double)ghi[q] + (double)glo[q];
}

// g partials of the FP64 path: block (x: points, y: frequency chunk).  Records
// are the FP64 records of the prep (phases A, B).  gpart[chunk * N + i].
__global__ void __launch_bounds__(VJ_THREADS) vjp_trig(const SeriesDesc *desc, const unsigned char *rec64,
                                                       const double *ab, int64_t chunk_len, double *gpart) {
    __shared__ __align__(16) double sab[2 * VJ_TILE];
    __shared__ SeedTable tab;
    fill_seed_table(tab);
    const SeriesDesc d = *desc;
    const int rw = rec64_words(d.p);
    const int64_t j_begin = (int64_t)blockIdx.y * chunk_len;
    const int64_t j_end = std::min<int64_t>(d.nf, j_begin + chunk_len);
    uint64_t A[VJ_PT], B[VJ_PT];
    double cr[VJ_PT], sr[VJ_PT], g[VJ_PT];
    int64_t idx[VJ_PT];
#pragma unroll
    for (int q = 0; q < VJ_PT; ++q) {
        const int64_t i = ((int64_t)blockIdx.x * VJ_PT + q) * VJ_THREADS + threadIdx.x;
        idx[q] = i;
        const int64_t ic = i < d.N ? i : d.N - 1;
        const uint64_t *R = reinterpret_cast<const uint64_t *>(rec64) + ic * rw;
        A[q] = R[0];
        B[q] = R[1];
        cr[q] = reinterpret_cast<const double *>(R)[2];
        sr[q] = reinterpret_cast<const double *>(R)[3];
        g[q] = 0.0;
    }
    for (int64_t j0 = j_begin; j0 < j_end; j0 += VJ_TILE) {
        const int nt = (int)std::min<int64_t>(VJ_TILE, j_end - j0);
        __syncthreads();
        for (int k = threadIdx.x; k < 2 * nt; k += blockDim.x) sab[k] = ab[2 * j0 + k];
        __syncthreads();
        for (int seg = 0; seg < nt; seg += VJ_SEG) {
            const int ns = min(VJ_SEG, nt - seg);
            double c[VJ_PT], s[VJ_PT], acc[VJ_PT];
#pragma unroll
            for (int q = 0; q < VJ_PT; ++q) {
                seed_from_table(tab, A[q] + (uint64_t)(j0 + seg) * B[q], &s[q], &c[q]);
                acc[q] = 0.0;
            }
            auto step = [&](int k) {
                const double a = sab[2 * (seg + k)], b = sab[2 * (seg + k) + 1];
#pragma unroll
                for (int q = 0; q < VJ_PT; ++q) {
                    acc[q] = fma(a, c[q], fma(b, s[q], acc[q]));
                    const double cn = fma(c[q], cr[q], -s[q] * sr[q]);
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
            for (int q = 0; q < VJ_PT; ++q) g[q] += acc[q];
        }
    }
#pragma unroll
    for (int q = 0; q < VJ_PT; ++q)
        if (idx[q] < d.N) gpart[(int64_t)blockIdx.y * d.N + idx[q]] = g[q];
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
    size_t off = 0;
    auto take = [&](size_t n) { size_t at = off; off = (off + n + 255) / 256 * 256; return at; };
    const size_t o_desc = take(sizeof(SeriesDesc)), o_state = take(sizeof(SeriesState));
    const size_t o_cs = take(nchunks * 4), o_part = take(nchunks * prep_npart(p) * 8);
    const size_t o_psi = take((size_t)p * N * 8), o_rec = take(N * (size_t)rec_bytes(p, FREDEC_FP64));
    // 16 bytes per frequency: (a, b) doubles, or (a, a, b, b) floats (mixed)
    const size_t o_ab = take(16 * nf + 16), o_g = take(gy * N * 8);
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
        vjp_coef_pairs<<<256, 256, 0, st>>>(coef, v, nf, (float4 *)(b + o_ab));
        vjp_trig_mixed<<<grid, VJ_THREADS, 0, st>>>(desc, b + o_rec, (const float4 *)(b + o_ab), chunk_len,
                                                    (double *)(b + o_g));
    } else {
        vjp_coef<<<256, 256, 0, st>>>(coef, v, nf, (double *)(b + o_ab));
        vjp_trig<<<grid, VJ_THREADS, 0, st>>>(desc, b + o_rec, (const double *)(b + o_ab), chunk_len,
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
