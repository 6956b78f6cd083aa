// Batched residual periodograms: many series of uneven length and base size
// in one plan.  The plan keeps the inputs on the device, builds the work list
// of (series, frequency block) items (longest series first), and captures
//   reset counters -> prep (all series) -> persistent periodogram kernel ->
//   FP64-grade (float-float) re-evaluation of flagged bins -> segmented top-k
// into one CUDA graph that fredec_batch_plan_run replays.  The number of warps
// per CTA is picked at plan creation by timing the captured graph (autotuner).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>
#include <vector>

#include "batch_impl.cuh"

namespace fredec {

int launch_batch_p5(int prec, const BatchParams &bp, int warps, int grid, bool comp, cudaStream_t st);
int launch_batch_p15(int prec, const BatchParams &bp, int warps, int grid, bool comp, cudaStream_t st);
int launch_batch_p25(int prec, const BatchParams &bp, int warps, int grid, bool comp, cudaStream_t st);
int batch_occupancy_p5(int prec, int warps, bool comp);
int batch_occupancy_p15(int prec, int warps, bool comp);
int batch_occupancy_p25(int prec, int warps, bool comp);
size_t topk_plan_size(int S, int64_t nch, int k);
int topk_plan_bytes(const int64_t *nf_h, int S, int k, int64_t *nchunks_out);
int topk_plan_make(const int64_t *z_off_h, const int64_t *nf_h, int S, int k, int64_t *idx_out, const double *z,
                   unsigned char *dev, void *args_out);
int topk_plan_launch(const void *args, int64_t nch, int S, cudaStream_t st);

}  // namespace fredec

using namespace fredec;

struct fredec_batch_plan {
    int S = 0, precision = 0, topk = 0, pmax = 1, warps = 4, statistic = 0;
    int64_t nf_max = 0;
    double tau = 0.2;
    bool fix = false;
    int64_t ntot = 0, nbase = 0, z_total = 0, nchunks = 0, n_items = 0, terms = 0, tk_chunks = 0, max_n = 0;
    std::vector<int> p_present;
    void *mem = nullptr;   // one device allocation holding everything
    double *t = nullptr, *y = nullptr, *sigma = nullptr, *base = nullptr, *z = nullptr, *partials = nullptr,
           *psi = nullptr;
    SeriesDesc *desc = nullptr;
    SeriesState *state = nullptr;
    int32_t *chunk_series = nullptr, *flag_count = nullptr, *err = nullptr;
    int64_t *flag_list = nullptr, *topk_out = nullptr;
    unsigned char *rec = nullptr, *rec64 = nullptr, *tk_meta = nullptr;
    int2 *items = nullptr;
    unsigned long long *counter = nullptr;
    unsigned char tk_args[256];
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;

    int enqueue(cudaStream_t st, int w) {
        FREDEC_CUDA_TRY(cudaMemsetAsync(counter, 0, 8, st));
        FREDEC_CUDA_TRY(cudaMemsetAsync(flag_count, 0, 4, st));
        FREDEC_CUDA_TRY(cudaMemsetAsync(err, 0, 4, st));   // status of this replay
        PrepPlan pp;
        pp.S = S;
        pp.max_n = max_n;
        pp.nchunks = nchunks;
        pp.pmax = pmax;
        pp.desc = desc;
        pp.state = state;
        pp.chunk_series = chunk_series;
        pp.partials = partials;
        pp.psi = psi;
        pp.rec = rec;
        if (int rc = run_prep_records(pp, t, y, sigma, base, precision, fix ? rec64 : nullptr, st)) return rc;
        BatchParams bp{};
        bp.prm.desc = desc;
        bp.prm.state = state;
        bp.prm.rec = rec;
        bp.prm.z = z;
        bp.prm.coef = nullptr;
        bp.prm.flag_tau = fix ? tau : -1.0;
        bp.prm.flag_list = fix ? flag_list : nullptr;
        bp.prm.flag_count = flag_count;
        bp.prm.flag_cap = fix ? z_total : 0;
        bp.prm.err = err;
        bp.prm.seed_mode = seed_mode();
        bp.items = items;
        bp.n_items = n_items;
        bp.counter = counter;
        // the smallest compiled class of base sizes that covers the batch;
        // compensated residual totals when its longest series needs them
        const bool comp = batch_comp(max_n, w);
        const int occ = pmax <= 5    ? batch_occupancy_p5(precision, w, comp)
                        : pmax <= 15 ? batch_occupancy_p15(precision, w, comp)
                                     : batch_occupancy_p25(precision, w, comp);
        const int grid = std::max(1, occ * sm_count());
        const int rc = pmax <= 5    ? launch_batch_p5(precision, bp, w, grid, comp, st)
                       : pmax <= 15 ? launch_batch_p15(precision, bp, w, grid, comp, st)
                                    : launch_batch_p25(precision, bp, w, grid, comp, st);
        if (rc) return rc;
        if (fix)
            for (int p : p_present)
                if (int rc = launch_fixup_bins(desc, state, S, rec64, p, flag_list, flag_count, z_total, z, nullptr, st,
                                               nullptr, 0, nullptr, err))
                    return rc;
        if (statistic == FREDEC_Z_LOG)
            if (int rc = launch_log_form(desc, state, S, nf_max, z, st)) return rc;
        if (topk > 0)
            if (int rc = topk_plan_launch(tk_args, tk_chunks, S, st)) return rc;
        return FREDEC_OK;
    }

    int capture(int w) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        FREDEC_CUDA_TRY(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        const int rc = enqueue(stream, w);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return fail(FREDEC_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        graph = g;
        FREDEC_CUDA_TRY(cudaGraphInstantiate(&exec, graph, 0));
        warps = w;
        return FREDEC_OK;
    }

    ~fredec_batch_plan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (mem) cudaFree(mem);
        if (stream) cudaStreamDestroy(stream);
    }
};

namespace {

int validate_batch(const double *t, const double *y, const double *sigma, const int64_t *obs, int64_t S,
                   const double *base, const int64_t *bo, const double *f0, const double *df, const int64_t *nf,
                   const int64_t *zo, const fredec_opts &o) {
    if (S < 1 || S > (1LL << 30)) return fail(FREDEC_EINVAL, "n_series must be >= 1");
    if (!t || !y || !sigma || !obs || !bo || !f0 || !df || !nf || !zo) return fail(FREDEC_EINVAL, "null pointer");
    if (obs[0] != 0 || bo[0] != 0) return fail(FREDEC_EINVAL, "offset arrays must start at 0");
    for (int64_t s = 0; s < S; ++s) {
        const int64_t N = obs[s + 1] - obs[s], nb = bo[s + 1] - bo[s];
        const int pb = base_cols((int)nb, o.trend);
        if (nb < 0 || nb > FREDEC_MAX_NBASE || padded_cols(pb) > PMAX || N < pb + 2 || N > (1LL << 31) - 1 ||
            (o.statistic == FREDEC_Z_LOG && N - 3 * (nb + 1) - 1 - o.trend <= 0))
            return fail(FREDEC_EINVAL, "series " + std::to_string(s) + ": bad N or base size");
        if (nf[s] < 0 || nf[s] > (1LL << 31) - 1 || !std::isfinite(f0[s]) || !std::isfinite(df[s]) || zo[s] < 0)
            return fail(FREDEC_EINVAL, "series " + std::to_string(s) + ": bad grid");
    }
    for (int64_t s = 0; s + 1 < S; ++s)
        if (zo[s] + nf[s] > zo[s + 1])
            return fail(FREDEC_EINVAL, "z_offsets must be increasing with z_offsets[s] + nf[s] <= z_offsets[s+1]");
    for (int64_t i = 0; i < obs[S]; ++i)
        if (!std::isfinite(t[i]) || !std::isfinite(y[i]) || !(sigma[i] > 0.0) || !std::isfinite(sigma[i]))
            return fail(FREDEC_EINVAL, "t, y must be finite and sigma finite and > 0");
    for (int64_t q = 0; q < bo[S]; ++q)
        if (!base || !std::isfinite(base[q])) return fail(FREDEC_EINVAL, "base frequencies must be finite");
    if (o.precision != FREDEC_FP64 && o.precision != FREDEC_MIXED) return fail(FREDEC_EINVAL, "bad precision");
    if (o.topk < 0 || o.topk > FREDEC_MAX_TOPK) return fail(FREDEC_EINVAL, "bad topk");
    if (o.trend < 0 || o.trend > FREDEC_MAX_TREND) return fail(FREDEC_EINVAL, "opts.trend must be in 0..3");
    if (o.statistic != FREDEC_Z_DIFF && o.statistic != FREDEC_Z_LOG) return fail(FREDEC_EINVAL, "bad opts.statistic");
    return FREDEC_OK;
}

}  // namespace

extern "C" {

int fredec_batch_plan_create(fredec_batch_plan **plan_out, const double *t, const double *y, const double *sigma,
                             const int64_t *obs, int64_t S, const double *base, const int64_t *bo, const double *f0,
                             const double *df, const int64_t *nf, const int64_t *zo, const fredec_opts *opts) {
    if (!plan_out) return fail(FREDEC_EINVAL, "null plan pointer");
    *plan_out = nullptr;
    fredec_opts o;
    fredec_opts_init(&o);
    if (opts) o = *opts;
    if (int rc = validate_batch(t, y, sigma, obs, S, base, bo, f0, df, nf, zo, o)) return rc;
    auto P = std::make_unique<fredec_batch_plan>();
    fredec_batch_plan &pl = *P;
    pl.S = (int)S;
    pl.precision = o.precision;
    pl.topk = o.topk;
    pl.statistic = o.statistic;
    pl.tau = o.flag_tau == 0.0 ? 0.2 : o.flag_tau;
    pl.fix = o.precision == FREDEC_MIXED && pl.tau >= 0.0;
    pl.ntot = obs[S];
    pl.nbase = bo[S];
    // per-series layout
    std::vector<SeriesDesc> desc(S);
    std::vector<int32_t> chunk_series;
    int64_t rec_off = 0, rec64_off = 0, psi_off = 0, chunk_off = 0, z_total = 0;
    std::vector<int> present(2 * FREDEC_MAX_NBASE + 2, 0);
    for (int64_t s = 0; s < S; ++s) {
        SeriesDesc &d = desc[s];
        d.N = (int32_t)(obs[s + 1] - obs[s]);
        d.nb = (int32_t)(bo[s + 1] - bo[s]);
        d.pb = base_cols(d.nb, o.trend);
        d.p = padded_cols(d.pb);
        d.npoly = o.trend;
        d.obs_off = obs[s];
        d.base_off = bo[s];
        d.f0 = f0[s];
        d.df = df[s];
        d.nf = nf[s];
        d.z_off = zo[s];
        d.rec_off = rec_off;
        d.rec64_off = rec64_off;
        d.psi_off = psi_off;
        d.chunk_off = chunk_off;
        d.nchunks = (d.N + PREP_THREADS - 1) / PREP_THREADS;
        rec_off += (int64_t)d.N * rec_bytes(d.p, o.precision);
        rec64_off += pl.fix ? (int64_t)d.N * recff_bytes(d.p) : 0;
        psi_off += (int64_t)d.p * d.N;
        chunk_off += d.nchunks;
        for (int c = 0; c < d.nchunks; ++c) chunk_series.push_back((int32_t)s);
        z_total = std::max(z_total, zo[s] + nf[s]);
        pl.pmax = std::max(pl.pmax, d.p);
        present[d.p] = 1;
        pl.terms += (int64_t)d.N * nf[s];
        pl.max_n = std::max<int64_t>(pl.max_n, d.N);
        pl.nf_max = std::max<int64_t>(pl.nf_max, d.nf);
    }
    for (int p = 1; p < (int)present.size(); ++p)
        if (present[p]) pl.p_present.push_back(p);
    pl.z_total = z_total;
    pl.nchunks = chunk_off;
    // work items: blocks of 32*F frequencies, longest series first
    std::vector<int64_t> order(S);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return desc[a].N > desc[b].N; });
    std::vector<int2> items;
    for (int64_t s : order) {
        const int64_t bw = 32LL * batch_fpt(o.precision, desc[s].p);
        const int64_t nb = (desc[s].nf + bw - 1) / bw;
        for (int64_t b = 0; b < nb; ++b) items.push_back(make_int2((int)s, (int)b));
    }
    pl.n_items = (int64_t)items.size();
    if (pl.topk > 0) topk_plan_bytes(nf, (int)S, pl.topk, &pl.tk_chunks);
    // one allocation
    size_t off = 0;
    auto take = [&](size_t n) { size_t at = off; off = (off + n + 255) / 256 * 256; return at; };
    const size_t o_t = take(pl.ntot * 8), o_y = take(pl.ntot * 8), o_s = take(pl.ntot * 8),
                 o_b = take(pl.nbase * 8 + 8), o_z = take(z_total * 8 + 8), o_desc = take(S * sizeof(SeriesDesc)),
                 o_state = take(S * sizeof(SeriesState)), o_cs = take(pl.nchunks * 4 + 4),
                 o_part = take(pl.nchunks * prep_npart(pl.pmax) * 8), o_psi = take(psi_off * 8 + 8),
                 o_rec = take(rec_off + 16), o_rec64 = take(rec64_off + 16),
                 o_fl = take(pl.fix ? z_total * 8 + 8 : 8), o_fc = take(4), o_err = take(4),
                 o_items = take(pl.n_items * sizeof(int2) + 8), o_cnt = take(8),
                 o_top = take((size_t)S * std::max(pl.topk, 1) * 8),
                 o_tk = take(pl.topk > 0 ? topk_plan_size((int)S, pl.tk_chunks, pl.topk) : 8);
    cudaError_t e = cudaMalloc(&pl.mem, off);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        pl.mem = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? FREDEC_ENOMEM : FREDEC_ECUDA,
                    std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    unsigned char *b = (unsigned char *)pl.mem;
    pl.t = (double *)(b + o_t);
    pl.y = (double *)(b + o_y);
    pl.sigma = (double *)(b + o_s);
    pl.base = (double *)(b + o_b);
    pl.z = (double *)(b + o_z);
    pl.desc = (SeriesDesc *)(b + o_desc);
    pl.state = (SeriesState *)(b + o_state);
    pl.chunk_series = (int32_t *)(b + o_cs);
    pl.partials = (double *)(b + o_part);
    pl.psi = (double *)(b + o_psi);
    pl.rec = b + o_rec;
    pl.rec64 = b + o_rec64;
    pl.flag_list = (int64_t *)(b + o_fl);
    pl.flag_count = (int32_t *)(b + o_fc);
    pl.err = (int32_t *)(b + o_err);
    pl.items = (int2 *)(b + o_items);
    pl.counter = (unsigned long long *)(b + o_cnt);
    pl.topk_out = (int64_t *)(b + o_top);
    pl.tk_meta = b + o_tk;
    FREDEC_CUDA_TRY(cudaMemcpy(pl.t, t, pl.ntot * 8, cudaMemcpyHostToDevice));
    FREDEC_CUDA_TRY(cudaMemcpy(pl.y, y, pl.ntot * 8, cudaMemcpyHostToDevice));
    FREDEC_CUDA_TRY(cudaMemcpy(pl.sigma, sigma, pl.ntot * 8, cudaMemcpyHostToDevice));
    if (pl.nbase) FREDEC_CUDA_TRY(cudaMemcpy(pl.base, base, pl.nbase * 8, cudaMemcpyHostToDevice));
    FREDEC_CUDA_TRY(cudaMemcpy(pl.desc, desc.data(), S * sizeof(SeriesDesc), cudaMemcpyHostToDevice));
    FREDEC_CUDA_TRY(cudaMemset(pl.state, 0, S * sizeof(SeriesState)));
    FREDEC_CUDA_TRY(cudaMemset(pl.z, 0, z_total * 8 + 8));
    FREDEC_CUDA_TRY(cudaMemcpy(pl.chunk_series, chunk_series.data(), pl.nchunks * 4, cudaMemcpyHostToDevice));
    FREDEC_CUDA_TRY(cudaMemcpy(pl.items, items.data(), pl.n_items * sizeof(int2), cudaMemcpyHostToDevice));
    FREDEC_CUDA_TRY(cudaMemset(pl.err, 0, 4));
    if (pl.topk > 0)
        if (int rc = topk_plan_make(zo, nf, (int)S, pl.topk, pl.topk_out, pl.z, pl.tk_meta, pl.tk_args)) return rc;
    FREDEC_CUDA_TRY(cudaStreamCreateWithFlags(&pl.stream, cudaStreamNonBlocking));
    // autotune warps per CTA on the real batch: capture each candidate, replay, keep the fastest
    const int cand[2] = {2, 4};
    int best_w = opts && opts->warps > 0 ? opts->warps : 0;
    if (!best_w) {
        float best_ms = 1e30f;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int w : cand) {
            if (int rc = pl.capture(w)) return rc;
            float ms_min = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, pl.stream);
                FREDEC_CUDA_TRY(cudaGraphLaunch(pl.exec, pl.stream));
                cudaEventRecord(e1, pl.stream);
                FREDEC_CUDA_TRY(cudaEventSynchronize(e1));
                float ms;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep) ms_min = std::min(ms_min, ms);
            }
            if (ms_min < best_ms) {
                best_ms = ms_min;
                best_w = w;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    if (int rc = pl.capture(best_w)) return rc;
    *plan_out = P.release();
    return FREDEC_OK;
}

int fredec_batch_plan_run(fredec_batch_plan *plan, void *stream) {
    if (!plan || !plan->exec) return fail(FREDEC_EINVAL, "null plan");
    FREDEC_CUDA_TRY(cudaGraphLaunch(plan->exec, (cudaStream_t)stream));
    return FREDEC_OK;
}

int fredec_batch_plan_outputs(fredec_batch_plan *plan, double **z_dev, int64_t **topk_dev, int64_t *z_total,
                              int64_t *terms) {
    if (!plan) return fail(FREDEC_EINVAL, "null plan");
    if (z_dev) *z_dev = plan->z;
    if (topk_dev) *topk_dev = plan->topk > 0 ? plan->topk_out : nullptr;
    if (z_total) *z_total = plan->z_total;
    if (terms) *terms = plan->terms;
    return FREDEC_OK;
}

int fredec_batch_plan_download(fredec_batch_plan *plan, double *z_out, int64_t *topk_idx_out) {
    if (!plan) return fail(FREDEC_EINVAL, "null plan");
    FREDEC_CUDA_TRY(cudaDeviceSynchronize());
    std::vector<int32_t> status(plan->S);
    for (int s = 0; s < plan->S; ++s)
        FREDEC_CUDA_TRY(cudaMemcpy(&status[s], &plan->state[s].status, 4, cudaMemcpyDeviceToHost));
    for (int s = 0; s < plan->S; ++s)
        if (status[s] != FREDEC_OK)
            return fail(FREDEC_ESINGULAR, "series " + std::to_string(s) + ": base normal matrix is singular");
    int32_t e = FREDEC_OK;   // the last replay's bounded waits and index checks
    FREDEC_CUDA_TRY(cudaMemcpy(&e, plan->err, 4, cudaMemcpyDeviceToHost));
    if (e == FREDEC_ETIMEOUT) return fail(FREDEC_ETIMEOUT, "a bounded device wait gave up");
    if (e != FREDEC_OK) return fail(FREDEC_ECUDA, "a device-side index check failed (the access was skipped)");
    if (z_out) FREDEC_CUDA_TRY(cudaMemcpy(z_out, plan->z, plan->z_total * 8, cudaMemcpyDeviceToHost));
    if (topk_idx_out && plan->topk > 0)
        FREDEC_CUDA_TRY(cudaMemcpy(topk_idx_out, plan->topk_out, (size_t)plan->S * plan->topk * 8,
                                   cudaMemcpyDeviceToHost));
    return FREDEC_OK;
}

void fredec_batch_plan_destroy(fredec_batch_plan *plan) { delete plan; }

int fredec_periodogram_batch(const double *t, const double *y, const double *sigma, const int64_t *obs, int64_t S,
                             const double *base, const int64_t *bo, const double *f0, const double *df,
                             const int64_t *nf, const int64_t *zo, const fredec_opts *opts, double *z_out,
                             int64_t *topk_idx_out) {
    fredec_opts o;
    fredec_opts_init(&o);
    if (opts) o = *opts;
    if (o.warps == 0) o.warps = 4;   // one-shot call: no tuning replays
    fredec_batch_plan *plan = nullptr;
    if (int rc = fredec_batch_plan_create(&plan, t, y, sigma, obs, S, base, bo, f0, df, nf, zo, &o)) return rc;
    int rc = fredec_batch_plan_run(plan, plan->stream);
    if (!rc) rc = fredec_batch_plan_download(plan, z_out, topk_idx_out);
    fredec_batch_plan_destroy(plan);
    return rc;
}

}  // extern "C"
