// Periodogram on an arbitrary (non-uniform) frequency grid.  Without a constant
// grid step there is no rotation recurrence, so every (frequency, point) term
// computes its own exact phase frac(f t') and FP64 sin/cos; the sums and the
// solve are FP64.  One thread per trial frequency; the records are read
// through the cache (all lanes of a warp read the same point).
#include "device_util.cuh"
#include "fredec_internal.cuh"
#include "pgram_impl.cuh"

namespace fredec {


namespace {

__global__ void generic_init(SeriesDesc *desc, SeriesDesc v, SeriesState *state, int32_t *cs, int64_t nchunks) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        *desc = v;
        for (int k = 0; k < 6; ++k) state->counter[k] = 0;
        state->status = FREDEC_OK;
    }
    for (int64_t q = i; q < nchunks; q += (int64_t)gridDim.x * blockDim.x) cs[q] = 0;
}

__global__ void __launch_bounds__(128) generic_kernel(const SeriesDesc *desc, const SeriesState *state,
                                                      const unsigned char *rec, const double *t, const double *fgrid,
                                                      double *z, double *coef, double *info) {
    __shared__ SeedTable tab;
    fill_seed_table(tab);
    __syncthreads();
    const SeriesDesc d = *desc;
    const SeriesState &st = *state;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (info && j == 0) {
        info[0] = st.chi2;
        info[1] = st.W;
        info[2] = st.tc;
    }
    if (j >= d.nf) return;
    if (st.status != FREDEC_OK) {
        z[j] = NAN;
        return;
    }
    const int p = d.p;
    const double f = fgrid[j];
    double acc[2 * PMAX + 4];
    for (int q = 0; q < 2 * p + 4; ++q) acc[q] = 0.0;
    const int rw = rec64_words(p);
    for (int i = 0; i < d.N; ++i) {
        const double *R = reinterpret_cast<const double *>(rec) + (int64_t)i * rw;
        const double tp = t[d.obs_off + i] - st.tc;
        double s, c;
        seed_from_table(tab, frac_turns_u64(f, tp), &s, &c);
        const double w = R[4], wr = R[5], wc = w * c;
        for (int q = 0; q < p; ++q) {
            acc[q] = fma(R[6 + q], c, acc[q]);
            acc[p + q] = fma(R[6 + q], s, acc[p + q]);
        }
        acc[2 * p] = fma(wr, c, acc[2 * p]);
        acc[2 * p + 1] = fma(wr, s, acc[2 * p + 1]);
        acc[2 * p + 2] = fma(wc, c, acc[2 * p + 2]);
        acc[2 * p + 3] = fma(wc, s, acc[2 * p + 3]);
    }
    double vcc = 0.0, vcs = 0.0, vss = 0.0;
    for (int q = 0; q < p; ++q) {
        vcc = fma(acc[q], acc[q], vcc);
        vcs = fma(acc[q], acc[p + q], vcs);
        vss = fma(acc[p + q], acc[p + q], vss);
    }
    const double CC = acc[2 * p + 2];
    double a, b, ratio;
    z[j] = solve2(CC, acc[2 * p + 3], st.W - CC, vcc, vcs, vss, acc[2 * p], acc[2 * p + 1], &a, &b, &ratio);
    if (coef) {
        coef[2 * j] = a;
        coef[2 * j + 1] = b;
    }
}

}  // namespace

int generic_grid_periodogram(const double *t, const double *y, const double *sigma, int64_t N, const double *base,
                             int nb, const double *f_grid_dev, int64_t nf, const fredec_opts &o, double *z, double *coef,
                             double *info, cudaStream_t st, SeriesState **state_out, DevBuf &ws) {
    const int pb = base_cols(nb, o.trend), p = padded_cols(pb);
    const int64_t nchunks = (N + PREP_THREADS - 1) / PREP_THREADS;
    size_t off = 0;
    auto take = [&](size_t n) { size_t at = off; off = (off + n + 255) / 256 * 256; return at; };
    const size_t o_desc = take(sizeof(SeriesDesc)), o_state = take(sizeof(SeriesState));
    const size_t o_cs = take(nchunks * 4), o_part = take(nchunks * prep_npart(p) * 8);
    const size_t o_psi = take((size_t)p * N * 8), o_rec = take(N * (size_t)rec_bytes(p, FREDEC_FP64));
    if (int rc = ws.alloc(off, st)) return rc;
    unsigned char *b = ws.as<unsigned char>();
    SeriesDesc d{};
    d.nf = nf;
    d.N = (int32_t)N;
    d.nb = nb;
    d.p = p;
    d.pb = pb;
    d.npoly = o.trend;
    d.nchunks = (int32_t)nchunks;
    SeriesDesc *dd = (SeriesDesc *)(b + o_desc);
    SeriesState *ss = (SeriesState *)(b + o_state);
    generic_init<<<std::max<int64_t>(1, std::min<int64_t>(1024, (nchunks + 255) / 256)), 256, 0, st>>>(
        dd, d, ss, (int32_t *)(b + o_cs), nchunks);
    PrepPlan pp;
    pp.S = 1;
    pp.max_n = N;
    pp.nchunks = nchunks;
    pp.pmax = p;
    pp.base_p = o.trend == 0 ? pb : 0;
    pp.desc = dd;
    pp.state = ss;
    pp.chunk_series = (int32_t *)(b + o_cs);
    pp.partials = (double *)(b + o_part);
    pp.psi = (double *)(b + o_psi);
    pp.rec = b + o_rec;
    if (int rc = run_prep_records(pp, t, y, sigma, base, FREDEC_FP64, nullptr, st)) return rc;
    generic_kernel<<<(unsigned)std::max<int64_t>(1, (nf + 127) / 128), 128, 0, st>>>(dd, ss, b + o_rec, t, f_grid_dev, z,
                                                                                     coef, info);
    FREDEC_CUDA_TRY(cudaGetLastError());
    if (o.statistic == FREDEC_Z_LOG)
        if (int rc = launch_log_form(dd, ss, 1, nf, z, st)) return rc;
    *state_out = ss;
    return FREDEC_OK;
}

}  // namespace fredec
