// Frequency derivative of the residual periodogram on a uniform grid:
// z(f_j) and dz/df(f_j) in one pass over the observations.
//
// By the envelope theorem (the linear parameters are at their optimum),
//     dz/df = -1/2 dchi2/df = <r_f dmu/df>,  dmu/df = 2 pi t (-a sin + b cos),
// with r_f the residual of the joint fit at f and (a, b) its coefficients of
// cos and sin (Section 3: the derivatives of the model of Eq. Hn; the sums
// involved are the t-weighted averages of Eq. avrg1).  Every record carries
// the weighted values (w, w r, w psi_k) and their products with t' (the
// second set), so one pass gives the 2P+4 sums of z and the 2P+4 t'-weighted
// sums; the epilogue combines them with (a, b) and the projections on the
// orthonormal base (dz_df in pgram_impl.cuh).  The derivative does not depend
// on the time origin, so t' = t - t_c serves as well as t.
//
// Pipeline: initialisation -> prep (two-set records) -> <t'> over the records
// -> two-set periodogram kernel -> (mixed) float-float re-evaluation of
// flagged bins, z and dz/df -> NaN fill of a failed call, info.
#include <algorithm>
#include <cmath>
#include <string>

#include "pgram_impl.cuh"

namespace fredec {

int launch_pgram_grad_a(int prec, int p, const PgramParams &prm, int64_t nblocks, int warps, cudaStream_t st,
                        const TailParams *tail);
int launch_pgram_grad_b(int prec, int p, const PgramParams &prm, int64_t nblocks, int warps, cudaStream_t st,
                        const TailParams *tail);

namespace {

__global__ void grad_init(SeriesDesc *desc, SeriesDesc v, SeriesState *state, int32_t *chunk_series, int64_t nchunks,
                          int32_t *flag_count, int32_t *err, int32_t *tail_cnt, int n_tail) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        *desc = v;
        for (int k = 0; k < 6; ++k) state->counter[k] = 0;
        state->status = FREDEC_OK;
        *flag_count = 0;
        *err = FREDEC_OK;
    }
    for (int64_t q = i; q < nchunks; q += (int64_t)gridDim.x * blockDim.x) chunk_series[q] = 0;
    for (int64_t q = i; q < n_tail; q += (int64_t)gridDim.x * blockDim.x) tail_cnt[q] = 0;
}

// <t'> = sum of the records' w t' values (FP64 records: the first word of
// the second set; mixed records: that word, t', times the square of the
// first word of the first set, s = sqrt(w)), exactly the values the
// periodogram kernel integrates; the order of the points does not matter.  One CTA, fixed-order
// reduction (deterministic).
__global__ void wt_sum_kernel(const unsigned char *rec, int64_t N, int p, int prec, double *out) {
    __shared__ double sc[32];
    double v = 0.0;
    if (prec == FREDEC_MIXED) {
        const int rw = rec32_words(p, 2), at = rec32_words(p);
        const float *R = reinterpret_cast<const float *>(rec);
        for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
            const double s = (double)R[i * rw + 8];
            v += (double)R[i * rw + at] * s * s;
        }
    } else {
        const int rw = rec64_words(p, 2), at = rec64_words(p);
        const double *R = reinterpret_cast<const double *>(rec);
        for (int64_t i = threadIdx.x; i < N; i += blockDim.x) v += R[i * rw + at];
    }
    v = block_sum_d(v, sc);
    if (threadIdx.x == 0) *out = v;
}

// NaN in z and dz/df when the base fit failed or a bounded wait gave up; info.
__global__ void grad_finish(const SeriesState *state, const int32_t *err, double *z, double *dzdf, int64_t nf,
                            double *info) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (info && i == 0) {
        info[0] = state->chi2;
        info[1] = state->W;
        info[2] = state->tc;
    }
    if (state->status != FREDEC_OK || *err != FREDEC_OK)
        for (int64_t j = i; j < nf; j += (int64_t)gridDim.x * blockDim.x) {
            z[j] = NAN;
            dzdf[j] = NAN;
        }
}

int launch_pgram_grad(int prec, int p, const PgramParams &prm, int64_t nblocks, int warps, cudaStream_t st,
                      const TailParams *tail) {
    int rc = launch_pgram_grad_a(prec, p, prm, nblocks, warps, st, tail);
    if (rc == -2) rc = launch_pgram_grad_b(prec, p, prm, nblocks, warps, st, tail);
    return rc == -2 ? fail(FREDEC_EINVAL, "no two-set kernel for this base size") : rc;
}

struct GradWork {
    SeriesState *state = nullptr;
    int32_t *err = nullptr;
};

// The device pipeline; every pointer a device pointer.
int grad_core(const double *t, const double *y, const double *sigma, int64_t N, const double *base, int nb, double f0,
              double df, int64_t nf, const fredec_opts &o, double *z, double *dzdf, double *info, cudaStream_t st,
              DevBuf &ws, GradWork &gw) {
    const int pb = base_cols(nb, o.trend), p = padded_cols(pb);
    const int prec = o.precision;
    const double tau = o.flag_tau == 0.0 ? 0.2 : o.flag_tau;
    const bool fix = prec == FREDEC_MIXED && tau >= 0.0;
    const int fpt = prec == FREDEC_MIXED ? grad_fpt_mixed(p) : GRAD_FPT_FP64;
    const int warps = o.warps > 0 ? o.warps : (N < 256 ? 2 : 4);
    const int64_t nchunks = (N + PREP_THREADS - 1) / PREP_THREADS;
    size_t off = 0;
    auto take = [&](size_t n) { size_t at = off; off = (off + n + 255) / 256 * 256; return at; };
    const size_t o_desc = take(sizeof(SeriesDesc)), o_state = take(sizeof(SeriesState));
    const size_t o_cs = take(nchunks * 4), o_part = take(nchunks * prep_npart(p) * 8);
    const size_t o_psi = take((size_t)p * N * 8), o_rec = take(N * (size_t)rec_bytes(p, prec, 2));
    const size_t o_rec64 = fix ? take(N * (size_t)recff_bytes(p, 2)) : 0;
    const size_t o_fl = fix ? take(nf * 8 + 8) : 0;
    const size_t o_fc = take(4), o_err = take(4), o_wt = take(8);
    int tail_gcap = 0;
    const size_t tail_bytes = nf > 0 ? pgram_tail_bytes(prec, p, fpt, &tail_gcap, 2) : 0;
    const size_t o_tp = tail_bytes ? take(tail_bytes) : 0, o_tc = tail_bytes ? take((size_t)tail_gcap * 4) : 0;
    if (int rc = ws.alloc(off, st)) return rc;
    unsigned char *b = ws.as<unsigned char>();
    SeriesDesc *desc = (SeriesDesc *)(b + o_desc);
    SeriesState *state = (SeriesState *)(b + o_state);
    int32_t *cs = (int32_t *)(b + o_cs);
    int64_t *flag_list = fix ? (int64_t *)(b + o_fl) : nullptr;
    int32_t *flag_count = (int32_t *)(b + o_fc);
    int32_t *err = (int32_t *)(b + o_err);
    double *wt = (double *)(b + o_wt);
    void *rec = b + o_rec;
    void *rec64 = fix ? (void *)(b + o_rec64) : nullptr;
    gw.state = state;
    gw.err = err;

    SeriesDesc d{};
    d.f0 = f0;
    d.df = df;
    d.nf = nf;
    d.N = (int32_t)N;
    d.nb = nb;
    d.p = p;
    d.pb = pb;
    d.npoly = o.trend;
    d.nchunks = (int32_t)nchunks;
    grad_init<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(1024, (nchunks + 255) / 256)), 256, 0, st>>>(
        desc, d, state, cs, nchunks, flag_count, err, tail_bytes ? (int32_t *)(b + o_tc) : nullptr,
        tail_bytes ? tail_gcap : 0);
    FREDEC_CUDA_TRY(cudaGetLastError());
    PrepPlan pp;
    pp.S = 1;
    pp.max_n = N;
    pp.nchunks = nchunks;
    pp.pmax = p;
    pp.base_p = o.trend == 0 ? pb : 0;
    pp.desc = desc;
    pp.state = state;
    pp.chunk_series = cs;
    pp.partials = (double *)(b + o_part);
    pp.psi = (double *)(b + o_psi);
    pp.rec = rec;
    if (int rc = run_prep_records(pp, t, y, sigma, base, prec, rec64, st, 2))
        return fail(rc, std::string("prep: ") + fredec_last_error());
    wt_sum_kernel<<<1, 256, 0, st>>>((const unsigned char *)rec, N, p, prec, wt);
    if (cudaError_t e = cudaGetLastError()) return fail(FREDEC_ECUDA, std::string("<t'> sum: ") + cudaGetErrorString(e));
    if (nf > 0) {
        PgramParams prm{};
        prm.desc = desc;
        prm.state = state;
        prm.rec = (const unsigned char *)rec;
        prm.z = z;
        prm.flag_tau = fix ? tau : -1.0;
        prm.flag_list = flag_list;
        prm.flag_cap = flag_list ? nf : 0;
        prm.flag_count = flag_count;
        prm.err = err;
        prm.seed_mode = seed_mode();
        prm.comp = pgram_comp(N, warps);
        prm.dzdf = dzdf;
        prm.wt_sum = wt;
        const int64_t nblocks = (nf + 32LL * fpt - 1) / (32LL * fpt);
        cudaEvent_t e0, e1;
        profile_events(&e0, &e1);
        if (e0) cudaEventRecord(e0, st);
        TailParams tail{};   // the tail split of the last part-filled wave (mixed)
        if (tail_bytes) {
            tail.part = (float2 *)(b + o_tp);
            tail.cnt = (int32_t *)(b + o_tc);
            tail.gcap = tail_gcap;
            tail.n_points = (int)N;
        }
        if (int rc = launch_pgram_grad(prec, p, prm, nblocks, warps, st, tail_bytes ? &tail : nullptr))
            return fail(rc, std::string("two-set periodogram kernel: ") + fredec_last_error());
        if (e1) cudaEventRecord(e1, st);
        if (fix)
            if (int rc = launch_fixup_bins(desc, state, 1, rec64, p, flag_list, flag_count, nf, z, nullptr, st,
                                           nullptr, 0, dzdf, err))
                return fail(rc, std::string("re-evaluation of flagged bins: ") + fredec_last_error());
    }
    grad_finish<<<64, 256, 0, st>>>(state, err, z, dzdf, nf, info);
    if (cudaError_t e = cudaGetLastError()) return fail(FREDEC_ECUDA, std::string("finish: ") + cudaGetErrorString(e));
    return FREDEC_OK;
}

int check_grad_args(const fredec_opts *opts, fredec_opts *o, int64_t N, int32_t n_base, int64_t nf, double f0,
                    double df) {
    if (int rc = check_opts(opts, o)) return rc;
    if (o->topk != 0) return fail(FREDEC_EINVAL, "the derivative entry points do not compute top-k (opts.topk must be 0)");
    if (o->statistic != FREDEC_Z_DIFF)
        return fail(FREDEC_EINVAL, "the derivative entry points compute the difference form (opts.statistic)");
    const int p = padded_cols(base_cols(n_base, o->trend));
    const int fpt = o->precision == FREDEC_MIXED ? grad_fpt_mixed(p) : GRAD_FPT_FP64;
    if (o->fpt != 0 && o->fpt != fpt)
        return fail(FREDEC_EINVAL, "opts.fpt must be 0 or " + std::to_string(fpt) + " for the derivative kernels");
    if (int rc = check_sizes(N, n_base, nf, *o)) return rc;
    if (!std::isfinite(f0) || !std::isfinite(df)) return fail(FREDEC_EINVAL, "f0 and df must be finite");
    return FREDEC_OK;
}

}  // namespace

}  // namespace fredec

using namespace fredec;

extern "C" {

int fredec_periodogram_grad_dev(const double *t, const double *y, const double *sigma, int64_t N,
                                const double *base_freqs, int32_t n_base, double f0, double df, int64_t nf,
                                const fredec_opts *opts, double *z_out, double *dzdf_out, double *info_out,
                                void *stream) {
    fredec_opts o;
    if (int rc = check_grad_args(opts, &o, N, n_base, nf, f0, df)) return rc;
    if (!t || !y || !sigma || (n_base > 0 && !base_freqs) || (nf > 0 && (!z_out || !dzdf_out)))
        return fail(FREDEC_EINVAL, "null pointer argument");
    DevBuf ws;
    GradWork gw;
    return grad_core(t, y, sigma, N, base_freqs, n_base, f0, df, nf, o, z_out, dzdf_out, info_out,
                     (cudaStream_t)stream, ws, gw);
}

int fredec_periodogram_grad(const double *t, const double *y, const double *sigma, int64_t N,
                            const double *base_freqs, int32_t n_base, double f0, double df, int64_t nf,
                            const fredec_opts *opts, double *z_out, double *dzdf_out, double *info_out) {
    fredec_opts o;
    if (int rc = check_grad_args(opts, &o, N, n_base, nf, f0, df)) return rc;
    if (!t || !y || !sigma || (n_base > 0 && !base_freqs) || (nf > 0 && (!z_out || !dzdf_out)))
        return fail(FREDEC_EINVAL, "null pointer argument");
    for (int64_t i = 0; i < N; ++i)
        if (!std::isfinite(t[i]) || !std::isfinite(y[i]) || !(sigma[i] > 0.0) || !std::isfinite(sigma[i]))
            return fail(FREDEC_EINVAL, "t, y must be finite and sigma finite and > 0");
    for (int32_t k = 0; k < n_base; ++k)
        if (!std::isfinite(base_freqs[k])) return fail(FREDEC_EINVAL, "base frequencies must be finite");
    cudaStream_t st;
    FREDEC_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    int rc = FREDEC_OK;
    {
        DevBuf io;
        const int64_t nz = std::max<int64_t>(nf, 1);
        if ((rc = io.alloc((3 * N + n_base + 2 * nz + 3) * 8 + 16, st))) {
            cudaStreamDestroy(st);
            return rc;
        }
        double *d = io.as<double>();
        double *dt = d, *dy = d + N, *ds = d + 2 * N, *db = d + 3 * N, *dz = db + n_base, *dg = dz + nz,
               *dinfo = dg + nz;
        int32_t words[2] = {FREDEC_OK, FREDEC_OK};
        do {
            if (cudaMemcpyAsync(dt, t, N * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaMemcpyAsync(dy, y, N * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaMemcpyAsync(ds, sigma, N * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                (n_base && cudaMemcpyAsync(db, base_freqs, n_base * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)) {
                rc = fail(FREDEC_ECUDA, "input copies failed");
                break;
            }
            DevBuf ws;
            GradWork gw;
            if ((rc = grad_core(dt, dy, ds, N, db, n_base, f0, df, nf, o, dz, dg, dinfo, st, ws, gw))) break;
            if (cudaMemcpyAsync(&words[0], &gw.state->status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaMemcpyAsync(&words[1], gw.err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                rc = fail(FREDEC_ECUDA, std::string("derivative pipeline: ") + cudaGetErrorString(cudaGetLastError()));
                break;
            }
        } while (0);
        if (!rc && words[0] == FREDEC_ESINGULAR)
            rc = fail(FREDEC_ESINGULAR, "the base model's normal matrix is singular (duplicate base frequencies?)");
        if (!rc && words[1] == FREDEC_ETIMEOUT) rc = fail(FREDEC_ETIMEOUT, "a bounded device wait gave up");
        if (!rc && words[1] != FREDEC_OK)
            rc = fail(FREDEC_ECUDA, "a device-side index check failed (the access was skipped)");
        if (!rc && nf > 0 &&
            (cudaMemcpyAsync(z_out, dz, nf * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
             cudaMemcpyAsync(dzdf_out, dg, nf * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess))
            rc = fail(FREDEC_ECUDA, "output copies failed");
        if (!rc && info_out && cudaMemcpyAsync(info_out, dinfo, 3 * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            rc = fail(FREDEC_ECUDA, "output copies failed");
        if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = fail(FREDEC_ECUDA, "stream synchronisation failed");
    }
    cudaStreamDestroy(st);
    return rc;
}

}  // extern "C"
