// The FREDEC decomposition (Section 4) on the GPU: Phase 1 scan of iterated
// residual periodograms, Phase 2 local fits of every subtuple of the pool,
// Phase 3 backward cascade, Phase 4 ordering.
//
// Phase 1 (SLICK/QUICK): each round computes the residual periodogram of the
// current base on the device (fredec_periodogram_dev, top-k local maxima on
// the device) and reads back only the 64 highest peaks and chi2 of the base.
// The statistic is the log form of Eq. zpowrel for one added frequency,
//     z = (N - 3(m+1) - 1)/2 ln(l_base / (l_base - 2 z_diff)),
// m = current base size.  The top peak joins the base and the pool while its z
// reaches z_thr0 (FAP_0); the other peaks join the pool when their z reaches
// z_thr1 (FAP_1) and half of the top peak's z.  Candidates closer than
// merge_dist (default 0.5/T) are one candidate, keeping the larger z.  At the
// end the pool is ordered by decreasing z and cut to max_pool (default N/10).
// Phases 2-4 reuse the pool-refinement and cascade kernels.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fredec_internal.cuh"

namespace fredec {

int cascade_run(const double *l_dev, int n, int64_t N, const double *zthr, double l0, uint32_t *pass_words_host,
                std::vector<uint32_t> *masks_host, std::vector<double> *G_host, cudaStream_t st);

namespace {

constexpr int SCAN_PEAKS = FREDEC_MAX_TOPK;

__global__ void gather_peaks(const double *z, const int64_t *idx, int k, double *out) {
    const int q = threadIdx.x;
    if (q < k) out[q] = idx[q] >= 0 ? z[idx[q]] : NAN;
}

struct Stream {
    cudaStream_t s = nullptr;
    ~Stream() {
        if (s) cudaStreamDestroy(s);
    }
};

struct Cand {
    double f, z;
};



int check_scan_opts(const fredec_scan_opts *in, int64_t N, fredec_scan_opts *o) {
    fredec_scan_opts_init(o);
    if (in) *o = *in;
    if (o->precision != FREDEC_FP64 && o->precision != FREDEC_MIXED)
        return fail(FREDEC_EINVAL, "scan precision must be FREDEC_FP64 or FREDEC_MIXED");
    if (o->max_pool < 0 || o->max_base < 0 || o->max_base > FREDEC_MAX_NBASE)
        return fail(FREDEC_EINVAL, "bad max_pool / max_base");
    if (std::isnan(o->z_thr0) || std::isnan(o->z_thr1) || !(o->half >= 0.0) || !(o->merge_dist >= 0.0))
        return fail(FREDEC_EINVAL, "bad scan thresholds");
    if (o->max_pool == 0) o->max_pool = (int32_t)std::min<int64_t>(N / 10, FREDEC_MAX_TUPLE);
    o->max_pool = std::min(o->max_pool, FREDEC_MAX_TUPLE);
    if (o->max_base == 0) o->max_base = FREDEC_MAX_NBASE;
    // the residual periodogram needs N >= 2 n_base + 3 for the largest base
    o->max_base = (int32_t)std::min<int64_t>(o->max_base, std::max<int64_t>(0, (N - 3) / 2));
    return FREDEC_OK;
}

int check_series(const double *t, const double *y, const double *sigma, int64_t N) {
    if (!t || !y || !sigma || N < 3) return fail(FREDEC_EINVAL, "null series or N < 3");
    for (int64_t i = 0; i < N; ++i) {
        if (!std::isfinite(t[i]) || !std::isfinite(y[i])) return fail(FREDEC_EINVAL, "t and y must be finite");
        if (!(sigma[i] > 0.0) || !std::isfinite(sigma[i])) return fail(FREDEC_EINVAL, "sigma must be finite and > 0");
    }
    return FREDEC_OK;
}

// Phase 1 on device-resident series.  l0_out receives chi2 of the constant
// model (the first round's base chi2).
int scan_run(const double *t_d, const double *y_d, const double *s_d, int64_t N, double span, double f0, double df,
             int64_t nf, const fredec_scan_opts &o, std::vector<Cand> *pool_out, std::vector<double> *base_out,
             bool *truncated, double *l0_out, cudaStream_t st) {
    const double md = o.merge_dist > 0.0 ? o.merge_dist : (span > 0.0 ? 0.5 / span : 0.0);
    const double half = o.half == 0.0 ? 0.5 : o.half;
    size_t off = 0;
    auto take = [&](size_t b) { size_t at = off; off = (off + b + 255) / 256 * 256; return at; };
    const size_t o_z = take((size_t)std::max<int64_t>(nf, 1) * 8), o_b = take(FREDEC_MAX_NBASE * 8);
    // top indices, their z and info are contiguous: one copy back per round
    const size_t o_k = take(SCAN_PEAKS * 8), o_zk = take(SCAN_PEAKS * 8), o_i = take(4 * 8);
    const size_t back = o_i + 4 * 8 - o_k;
    DevBuf buf;
    if (int rc = buf.alloc(off, st)) return rc;
    void *pin = pinned_scratch(PIN_SCAN, FREDEC_MAX_NBASE * 8 + back);   // [base frequencies | the copied-back block]
    if (!pin) return fail(FREDEC_ECUDA, "cudaMallocHost of the scan's transfer buffer failed");
    double *base_h = static_cast<double *>(pin);
    char *back_h = static_cast<char *>(pin) + FREDEC_MAX_NBASE * 8;
    char *b = buf.as<char>();
    double *z_d = (double *)(b + o_z), *base_d = (double *)(b + o_b), *zk_d = (double *)(b + o_zk);
    double *info_d = (double *)(b + o_i);
    int64_t *top_d = (int64_t *)(b + o_k);
    std::vector<double> base;
    std::vector<Cand> pool;
    auto add = [&](double f, double z) {
        int best = -1;
        for (int k = 0; k < (int)pool.size(); ++k)
            if (std::fabs(pool[k].f - f) < md && (best < 0 || std::fabs(pool[k].f - f) < std::fabs(pool[best].f - f)))
                best = k;
        if (best < 0) pool.push_back({f, z});
        else if (z > pool[best].z) pool[best] = {f, z};
    };
    *l0_out = NAN;
    fredec_opts po;
    fredec_opts_init(&po);
    po.precision = o.precision;
    po.topk = SCAN_PEAKS;
    while ((int)base.size() < o.max_base || (base.empty() && !std::isfinite(*l0_out))) {
        const int m = (int)base.size();
        if (m) {
            std::copy(base.begin(), base.end(), base_h);
            FREDEC_CUDA_TRY(cudaMemcpyAsync(base_d, base_h, m * 8, cudaMemcpyHostToDevice, st));
        }
        if (int rc = fredec_periodogram_dev(t_d, y_d, s_d, N, base_d, m, f0, df, nf, &po, z_d, info_d, top_d,
                                            nullptr, st))
            return rc;
        gather_peaks<<<1, SCAN_PEAKS, 0, st>>>(z_d, top_d, SCAN_PEAKS, zk_d);
        FREDEC_CUDA_TRY(cudaGetLastError());
        FREDEC_CUDA_TRY(cudaMemcpyAsync(back_h, b + o_k, back, cudaMemcpyDeviceToHost, st));
        FREDEC_CUDA_TRY(cudaStreamSynchronize(st));
        const int64_t *top = reinterpret_cast<const int64_t *>(back_h);
        const double *zk = reinterpret_cast<const double *>(back_h + (o_zk - o_k));
        const double *info = reinterpret_cast<const double *>(back_h + (o_i - o_k));
        if (m == 0) *l0_out = info[0];
        if (o.max_base == 0 || top[0] < 0) break;
        const double lb = info[0], NH = (double)(N - 3 * (int64_t)(m + 1) - 1);
        auto logz = [&](double zd) {
            const double lnew = lb - 2.0 * zd;
            return lnew > 0.0 ? 0.5 * NH * std::log(lb / lnew) : INFINITY;
        };
        const double ztop = logz(zk[0]);
        if (!(ztop >= o.z_thr0)) break;
        const double ftop = f0 + (double)top[0] * df;
        base.push_back(ftop);
        add(ftop, ztop);
        for (int q = 1; q < SCAN_PEAKS && top[q] >= 0; ++q) {
            const double zq = logz(zk[q]);
            if (zq >= o.z_thr1 && zq >= half * ztop) add(f0 + (double)top[q] * df, zq);
        }
    }
    std::stable_sort(pool.begin(), pool.end(),
                     [](const Cand &a, const Cand &c) { return a.z > c.z || (a.z == c.z && a.f < c.f); });
    *truncated = (int)pool.size() > o.max_pool;
    if (*truncated) pool.resize(o.max_pool);
    *pool_out = pool;
    *base_out = base;
    return FREDEC_OK;
}

int upload_series(const double *t, const double *y, const double *sigma, int64_t N, DevBuf &buf, cudaStream_t st,
                  double **t_d, double **y_d, double **s_d) {
    if (int rc = buf.alloc((size_t)3 * N * 8, st)) return rc;
    *t_d = buf.as<double>();
    *y_d = *t_d + N;
    *s_d = *y_d + N;
    FREDEC_CUDA_TRY(cudaMemcpyAsync(*t_d, t, N * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(*y_d, y, N * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(*s_d, sigma, N * 8, cudaMemcpyHostToDevice, st));
    return FREDEC_OK;
}

double span_of(const double *t, int64_t N) {
    double lo = t[0], hi = t[0];
    for (int64_t i = 1; i < N; ++i) {
        lo = std::min(lo, t[i]);
        hi = std::max(hi, t[i]);
    }
    return hi - lo;
}

}  // namespace
}  // namespace fredec

using namespace fredec;

extern "C" void fredec_scan_opts_init(fredec_scan_opts *o) {
    if (!o) return;
    *o = fredec_scan_opts{};
    o->precision = FREDEC_FP64;
    o->half = 0.5;
}

extern "C" void fredec_decompose_opts_init(fredec_decompose_opts *o) {
    if (!o) return;
    *o = fredec_decompose_opts{};
    fredec_scan_opts_init(&o->scan);
    o->refine_precision = FREDEC_FP64;
    o->refine_iter = 20;
    o->refine_tol = 1e-9;
}

extern "C" int fredec_scan(const double *t, const double *y, const double *sigma, int64_t N, double f0, double df,
                           int64_t nf, const fredec_scan_opts *opts, double *pool_out, double *pool_z_out,
                           int32_t *n_pool_out, double *base_out, int32_t *n_base_out, int32_t *truncated_out) {
    if (int rc = check_series(t, y, sigma, N)) return rc;
    if (!std::isfinite(f0) || !std::isfinite(df) || nf < 1 || nf > (1LL << 31) - 1)
        return fail(FREDEC_EINVAL, "bad frequency grid");
    if (!pool_out || !n_pool_out) return fail(FREDEC_EINVAL, "null pool output");
    fredec_scan_opts o;
    if (int rc = check_scan_opts(opts, N, &o)) return rc;
    Stream s;
    FREDEC_CUDA_TRY(cudaStreamCreateWithFlags(&s.s, cudaStreamNonBlocking));
    DevBuf sb;
    double *t_d, *y_d, *s_d;
    if (int rc = upload_series(t, y, sigma, N, sb, s.s, &t_d, &y_d, &s_d)) return rc;
    std::vector<Cand> pool;
    std::vector<double> base;
    bool trunc = false;
    double l0 = 0.0;
    if (int rc = scan_run(t_d, y_d, s_d, N, span_of(t, N), f0, df, nf, o, &pool, &base, &trunc, &l0, s.s)) return rc;
    *n_pool_out = (int32_t)pool.size();
    for (size_t k = 0; k < pool.size(); ++k) {
        pool_out[k] = pool[k].f;
        if (pool_z_out) pool_z_out[k] = pool[k].z;
    }
    if (n_base_out) *n_base_out = (int32_t)base.size();
    if (base_out) std::copy(base.begin(), base.end(), base_out);
    if (truncated_out) *truncated_out = trunc;
    return FREDEC_OK;
}

extern "C" int fredec_decompose(const double *t, const double *y, const double *sigma, int64_t N, double f0,
                                double df, int64_t nf, const fredec_decompose_opts *opts, double *pool_out,
                                int32_t *n_pool_out, double *l_table_out, uint32_t *solutions, double *G_out,
                                double *freqs_out, double *resid_z_out, int64_t capacity, int64_t *n_solutions) {
    if (int rc = check_series(t, y, sigma, N)) return rc;
    if (!std::isfinite(f0) || !std::isfinite(df) || nf < 1 || nf > (1LL << 31) - 1)
        return fail(FREDEC_EINVAL, "bad frequency grid");
    if (!opts || !opts->z_thr) return fail(FREDEC_EINVAL, "opts with z_thr are required");
    if (!n_solutions || capacity < 0 || (capacity > 0 && (!solutions || !G_out)))
        return fail(FREDEC_EINVAL, "bad solution outputs");
    fredec_decompose_opts o = *opts;
    if (o.refine_precision != FREDEC_FP64 && o.refine_precision != FREDEC_MIXED)
        return fail(FREDEC_EINVAL, "bad refine precision");
    if (o.refine_iter < 0 || !(o.refine_tol >= 0.0)) return fail(FREDEC_EINVAL, "bad refine iteration limits");
    fredec_scan_opts so;
    if (int rc = check_scan_opts(&o.scan, N, &so)) return rc;
    Stream s;
    FREDEC_CUDA_TRY(cudaStreamCreateWithFlags(&s.s, cudaStreamNonBlocking));
    DevBuf sb;
    double *t_d, *y_d, *s_d;
    if (int rc = upload_series(t, y, sigma, N, sb, s.s, &t_d, &y_d, &s_d)) return rc;
    // Phase 1
    std::vector<Cand> pool;
    std::vector<double> base;
    bool trunc = false;
    double l0 = 0.0;
    if (int rc = scan_run(t_d, y_d, s_d, N, span_of(t, N), f0, df, nf, so, &pool, &base, &trunc, &l0, s.s))
        return rc;
    const int n = (int)pool.size();
    std::vector<double> pf(n);
    for (int k = 0; k < n; ++k) pf[k] = pool[k].f;
    if (n_pool_out) *n_pool_out = n;
    if (pool_out) std::copy(pf.begin(), pf.end(), pool_out);
    // Phase 2: local fit of every non-empty subtuple
    const int64_t nmask = (int64_t)1 << n;
    std::vector<uint32_t> masks(std::max<int64_t>(nmask - 1, 1));
    for (int64_t S = 1; S < nmask; ++S) masks[S - 1] = (uint32_t)S;
    std::vector<double> fref((size_t)std::max<int64_t>(nmask - 1, 1) * std::max(n, 1));
    std::vector<double> l(nmask);
    l[0] = l0;
    if (n > 0) {
        const int iters = o.refine_iter == 0 ? 20 : o.refine_iter;
        const double tol = o.refine_tol == 0.0 ? 1e-9 : o.refine_tol;
        if (int rc = fredec_pool_refine(t, y, sigma, N, pf.data(), n, masks.data(), nmask - 1, iters, tol,
                                        o.refine_precision, fref.data(), l.data() + 1, nullptr))
            return rc;
    }
    if (l_table_out) std::copy(l.begin(), l.end(), l_table_out);
    // Phase 3 and the Phase 4 order
    DevBuf lb;
    if (int rc = lb.alloc((size_t)nmask * 8, s.s)) return rc;
    FREDEC_CUDA_TRY(cudaMemcpyAsync(lb.ptr, l.data(), nmask * 8, cudaMemcpyHostToDevice, s.s));
    std::vector<uint32_t> sol;
    std::vector<double> G;
    std::vector<double> zt(std::max(n, 1), 0.0);
    for (int c = 0; c < n; ++c) zt[c] = o.z_thr[c];
    if (int rc = cascade_run(lb.as<double>(), n, N, zt.data(), l0, nullptr, &sol, &G, s.s)) return rc;
    *n_solutions = (int64_t)sol.size();
    const int64_t nout = std::min<int64_t>(capacity, (int64_t)sol.size());
    DevBuf rb;   // Phase 4 residual periodograms: z, base frequencies, top index
    if (resid_z_out && nout > 0) {
        if (int rc = rb.alloc((size_t)(nf + FREDEC_MAX_NBASE + 4) * 8, s.s)) return rc;
    }
    for (int64_t i = 0; i < nout; ++i) {
        solutions[i] = sol[i];
        G_out[i] = G[i];
        std::vector<double> f;
        for (int j = 0; j < n; ++j)
            if (sol[i] >> j & 1) f.push_back(fref[(size_t)(sol[i] - 1) * n + j]);
        std::sort(f.begin(), f.end());
        if (freqs_out)
            for (int j = 0; j < FREDEC_MAX_TUPLE; ++j)
                freqs_out[i * FREDEC_MAX_TUPLE + j] = j < (int)f.size() ? f[j] : 0.0;
        if (resid_z_out) {
            // Phase 4: the highest peak left in the residual periodogram whose
            // base is this solution (log form, N_H = N - 3(m+1) - 1)
            resid_z_out[i] = NAN;
            const int m = (int)f.size();
            if (m > FREDEC_MAX_NBASE || N - 3LL * (m + 1) - 1 <= 0 || N < 2LL * m + 3) continue;
            double *zr = rb.as<double>(), *bd = zr + nf;
            int64_t *top = reinterpret_cast<int64_t *>(bd + FREDEC_MAX_NBASE);
            if (m) FREDEC_CUDA_TRY(cudaMemcpyAsync(bd, f.data(), m * 8, cudaMemcpyHostToDevice, s.s));
            fredec_opts po;
            fredec_opts_init(&po);
            po.precision = so.precision;
            po.topk = 1;
            po.statistic = FREDEC_Z_LOG;
            if (int rc = fredec_periodogram_dev(t_d, y_d, s_d, N, bd, m, f0, df, nf, &po, zr, nullptr, top, nullptr,
                                                s.s))
                return rc;
            gather_peaks<<<1, 32, 0, s.s>>>(zr, top, 1, bd + FREDEC_MAX_NBASE - 1);
            FREDEC_CUDA_TRY(cudaGetLastError());
            FREDEC_CUDA_TRY(cudaMemcpyAsync(&resid_z_out[i], bd + FREDEC_MAX_NBASE - 1, 8, cudaMemcpyDeviceToHost,
                                            s.s));
            FREDEC_CUDA_TRY(cudaStreamSynchronize(s.s));
        }
    }
    return FREDEC_OK;
}
