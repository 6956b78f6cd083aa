// Public C ABI (include/fredec.h): validation, workspace and the single-series
// periodogram pipeline  prep -> periodogram -> FP64-grade (float-float) re-evaluation -> top-k.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "fredec_internal.cuh"

namespace fredec {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

// Keep freed blocks cached in the device's default stream-ordered pool so that
// repeated calls do not return memory to the driver (once per device).
static void keep_pool_cached() {
    static thread_local int done_dev = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev == done_dev) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    (void)cudaGetLastError();
    done_dev = dev;
}

int DevBuf::alloc(size_t n, cudaStream_t s) {
    stream = s;
    bytes = n;
    if (n == 0) return FREDEC_OK;
    const char *inj = std::getenv("FREDEC_FAIL_ALLOC");
    if (inj && inj[0] == '1') return fail(FREDEC_ENOMEM, "allocation failure injected (FREDEC_FAIL_ALLOC=1)");
    keep_pool_cached();
    cudaError_t e = cudaMallocAsync(&ptr, n, s);
    if (e != cudaSuccess) {
        ptr = nullptr;
        (void)cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? FREDEC_ENOMEM : FREDEC_ECUDA,
                    std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    }
    return FREDEC_OK;
}
DevBuf::~DevBuf() {
    if (ptr) cudaFreeAsync(ptr, stream);
}

// SM count of the device current at the first call (thread-safe static
// initialisation; every device of this build is a B300).
int sm_count() {
    static const int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
        return v;
    }();
    return n;
}

size_t pgram_smem(int p, int prec, int F, int warps);

// ---------------------------------------------------------------------------
// Small device helpers for the pipeline

namespace {

__global__ void init_series_kernel(SeriesDesc *desc, SeriesDesc v, SeriesState *state, int32_t *chunk_series,
                                   int64_t nchunks, int32_t *flag_count, int32_t *err, int32_t *tail_cnt = nullptr,
                                   int n_tail = 0) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        *desc = v;
        for (int k = 0; k < 6; ++k) state->counter[k] = 0;
        state->status = FREDEC_OK;
        if (flag_count) *flag_count = 0;
        if (err) *err = FREDEC_OK;
    }
    for (int64_t q = i; q < nchunks; q += (int64_t)gridDim.x * blockDim.x) chunk_series[q] = 0;
    for (int64_t q = i; q < n_tail; q += (int64_t)gridDim.x * blockDim.x) tail_cnt[q] = 0;
}

__global__ void info_kernel(const SeriesState *state, double *info) {
    info[0] = state->chi2;
    info[1] = state->W;
    info[2] = state->tc;
}

__global__ void nan_fill_if_failed(const SeriesState *state, double *z, int64_t nf) {
    if (state->status == FREDEC_OK) return;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nf; j += (int64_t)gridDim.x * blockDim.x)
        z[j] = NAN;
}

bool finite_all(const double *a, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

}  // namespace

// Workspace of one single-series periodogram call.
struct SingleWork {
    SeriesDesc *desc;
    SeriesState *state;
    int32_t *chunk_series;
    double *partials;
    double *psi;
    void *rec;       // records of the main precision
    void *rec64;     // float-float records for the re-evaluation (mixed) or == rec (FP64)
    int64_t *flag_list;
    int32_t *flag_count;
    int32_t *err;
    int64_t nchunks;
    float2 *tail_part;   // tail split of the periodogram launch (mixed)
    int32_t *tail_cnt;
    int tail_gcap;
};


// The device pipeline for one series on a uniform grid.  All pointers device
// (z_mirror: optional second destination of z, e.g. page-locked host memory).
static int periodogram_core(const double *t, const double *y, const double *sigma, int64_t N, const double *base,
                            int nb, double f0, double df, int64_t nf, const fredec_opts &o, double *z,
                            double *info, int64_t *topk, double *coef, cudaStream_t st, DevBuf &ws,
                            SingleWork &w, double *z_mirror = nullptr, unsigned char *host_block = nullptr) {
    const int pb = base_cols(nb, o.trend), p = padded_cols(pb);
    const int prec = o.precision;
    const double tau = o.flag_tau == 0.0 ? 0.2 : o.flag_tau;
    const bool fix = prec == FREDEC_MIXED && tau >= 0.0;
    const int64_t nchunks = (N + PREP_THREADS - 1) / PREP_THREADS;
    const int64_t nflag = fix ? nf : 0;   // worst case: every bin flagged
    const size_t rb = (size_t)rec_bytes(p, prec);
    const size_t rbff = (size_t)recff_bytes(p);
    // carve one allocation
    size_t off = 0;
    auto take = [&](size_t n) { size_t at = off; off = (off + n + 255) / 256 * 256; return at; };
    const size_t o_desc = take(sizeof(SeriesDesc)), o_state = take(sizeof(SeriesState));
    const size_t o_cs = take(nchunks * 4), o_part = take(nchunks * prep_npart(p) * 8);
    const size_t o_psi = take((size_t)p * N * 8), o_rec = take(N * rb);
    const size_t o_rec64 = fix ? take(N * rbff) : 0;
    PgramShape shape;
    if (o.fpt > 0 || o.warps > 0) {
        shape = default_shape(prec, p, N, nf);
        if (o.fpt > 0) shape.fpt = o.fpt;
        if (o.warps > 0) shape.warps = o.warps;
    } else if (!tuned_shape(prec, p, N, nf, &shape)) {
        shape = default_shape(prec, p, N, nf);
    }
    int tail_gcap = 0;
    const size_t tail_bytes = nf > 0 ? pgram_tail_bytes(prec, p, shape.fpt, &tail_gcap) : 0;
    const size_t o_fl = take(nflag * 8 + 8), o_fc = take(4), o_err = take(4);
    const size_t o_tp = tail_bytes ? take(tail_bytes) : 0, o_tc = tail_bytes ? take((size_t)tail_gcap * 4) : 0;
    if (int rc = ws.alloc(off, st)) return rc;
    unsigned char *b = ws.as<unsigned char>();
    w.desc = (SeriesDesc *)(b + o_desc);
    w.state = (SeriesState *)(b + o_state);
    w.chunk_series = (int32_t *)(b + o_cs);
    w.partials = (double *)(b + o_part);
    w.psi = (double *)(b + o_psi);
    w.rec = b + o_rec;
    w.rec64 = fix ? (void *)(b + o_rec64) : (prec == FREDEC_FP64 ? w.rec : nullptr);
    w.flag_list = fix ? (int64_t *)(b + o_fl) : nullptr;
    w.flag_count = (int32_t *)(b + o_fc);
    w.err = (int32_t *)(b + o_err);
    w.nchunks = nchunks;
    w.tail_part = tail_bytes ? (float2 *)(b + o_tp) : nullptr;
    w.tail_cnt = tail_bytes ? (int32_t *)(b + o_tc) : nullptr;
    w.tail_gcap = tail_bytes ? tail_gcap : 0;

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
    init_series_kernel<<<std::max<int64_t>(1, std::min<int64_t>(1024, (nchunks + 255) / 256)), 256, 0, st>>>(
        w.desc, d, w.state, w.chunk_series, nchunks, w.flag_count, w.err, w.tail_cnt, w.tail_gcap);
    FREDEC_CUDA_TRY(cudaGetLastError());

    PrepPlan pp;
    pp.S = 1;
    pp.max_n = N;
    pp.nchunks = nchunks;
    pp.pmax = p;
    pp.base_p = o.trend == 0 ? pb : 0;
    pp.desc = w.desc;
    pp.state = w.state;
    pp.chunk_series = w.chunk_series;
    pp.partials = w.partials;
    pp.psi = w.psi;
    pp.rec = w.rec;
    if (int rc = run_prep_records(pp, t, y, sigma, base, prec, fix ? w.rec64 : nullptr, st)) return rc;

    if (nf > 0) {
        if (int rc = launch_pgram(prec, w.desc, w.state, w.rec, p, (int)N, nf, shape, tau, z, coef, w.flag_list,
                                  w.flag_count, w.err, st, z_mirror, w.tail_part, w.tail_cnt, w.tail_gcap))
            return rc;
        // the NaN fill of a failed prep rides on the re-evaluation launch when there is one
        if (fix) {
            if (int rc = launch_fixup_bins(w.desc, w.state, 1, w.rec64, p, w.flag_list, w.flag_count, nf, z, coef,
                                           st, z_mirror, nf, nullptr, w.err))
                return rc;
        } else {
            nan_fill_if_failed<<<64, 256, 0, st>>>(w.state, z, nf);
        }
        if (o.statistic == FREDEC_Z_LOG)
            if (int rc = launch_log_form(w.desc, w.state, 1, nf, z, st)) return rc;
        if (topk && o.topk > 0) {   // its last kernel also copies info
            if (int rc = launch_topk_single(z, nf, o.topk, topk, st, w.state, info, w.err, host_block)) return rc;
            info = nullptr;
        }
    }
    if (info) info_kernel<<<1, 1, 0, st>>>(w.state, info);
    FREDEC_CUDA_TRY(cudaGetLastError());
    return FREDEC_OK;
}

// Host-side checks shared by the entry points (declared in fredec_internal.cuh).
int check_opts(const fredec_opts *o, fredec_opts *out) {
    fredec_opts_init(out);
    if (o) *out = *o;
    if (out->precision != FREDEC_FP64 && out->precision != FREDEC_MIXED)
        return fail(FREDEC_EINVAL, "opts.precision must be FREDEC_FP64 or FREDEC_MIXED");
    if (out->topk < 0 || out->topk > FREDEC_MAX_TOPK) return fail(FREDEC_EINVAL, "opts.topk must be in 0..64");
    if (out->fpt < 0 || out->warps < 0 || out->warps > 8) return fail(FREDEC_EINVAL, "bad opts.fpt / opts.warps");
    if (!std::isfinite(out->flag_tau)) return fail(FREDEC_EINVAL, "opts.flag_tau must be finite");
    if (out->trend < 0 || out->trend > FREDEC_MAX_TREND) return fail(FREDEC_EINVAL, "opts.trend must be in 0..3");
    if (out->statistic != FREDEC_Z_DIFF && out->statistic != FREDEC_Z_LOG)
        return fail(FREDEC_EINVAL, "opts.statistic must be FREDEC_Z_DIFF or FREDEC_Z_LOG");
    return FREDEC_OK;
}

int check_sizes(int64_t N, int32_t n_base, int64_t nf, const fredec_opts &o) {
    if (n_base < 0 || n_base > FREDEC_MAX_NBASE) return fail(FREDEC_EINVAL, "n_base must be in 0..FREDEC_MAX_NBASE");
    const int pb = base_cols(n_base, o.trend);
    if (padded_cols(pb) > PMAX) return fail(FREDEC_EINVAL, "1 + trend + 2*n_base must not exceed 25");
    if (N < pb + 2) return fail(FREDEC_EINVAL, "N must be at least 1 + trend + 2*n_base + 2");
    if (o.statistic == FREDEC_Z_LOG && N - 3LL * (n_base + 1) - 1 - o.trend <= 0)
        return fail(FREDEC_EINVAL, "the log-form statistic needs N > 3 (n_base + 1) + 1 + trend");
    if (N > (1LL << 31) - 1) return fail(FREDEC_EINVAL, "N too large");
    if (nf < 0 || nf > (1LL << 31) - 1) return fail(FREDEC_EINVAL, "nf must be in 0..2^31-1");
    return FREDEC_OK;
}

static int check_series_host(const double *t, const double *y, const double *sigma, int64_t N,
                             const double *base, int32_t nb) {
    if (!t || !y || !sigma || (nb > 0 && !base)) return fail(FREDEC_EINVAL, "null input pointer");
    if (!finite_all(t, N) || !finite_all(y, N)) return fail(FREDEC_EINVAL, "t and y must be finite");
    for (int64_t i = 0; i < N; ++i)
        if (!(sigma[i] > 0.0) || !std::isfinite(sigma[i])) return fail(FREDEC_EINVAL, "sigma must be finite and > 0");
    if (nb > 0 && !finite_all(base, nb)) return fail(FREDEC_EINVAL, "base frequencies must be finite");
    return FREDEC_OK;
}

// Uniform-grid detection: f_j = f0 + j*df within 8 ulps of max |f| (a uniform
// grid is monotone, so max |f| is at an end point).  f0 and df come from the
// end points; a NaN or infinite entry fails the test.  grid_uniform_sampled
// tests 65 evenly spaced entries (the cheap check that decides whether to
// start the uniform-grid pipeline before the full test); grid_uniform tests
// every entry, in blocks of 4096 without early exit inside a block.
static bool grid_params(const double *f, int64_t nf, double *f0, double *df, double *tol) {
    *f0 = f[0];
    *df = nf > 1 ? (f[nf - 1] - f[0]) / (double)(nf - 1) : 0.0;
    const double fmax = std::max(std::fabs(f[0]), std::fabs(f[nf - 1]));
    if (!std::isfinite(fmax) || !std::isfinite(*df)) return false;
    *tol = 8.0 * std::ldexp(1.0, std::ilogb(fmax > 0 ? fmax : 1.0) - 52);
    return true;
}

static bool grid_uniform_sampled(const double *f, int64_t nf, double *f0, double *df) {
    double tol;
    if (nf <= 0) { *f0 = 0.0; *df = 0.0; return true; }
    if (!grid_params(f, nf, f0, df, &tol)) return false;
    for (int s = 0; s <= 64; ++s) {
        const int64_t j = (int64_t)((double)(nf - 1) * s / 64.0);
        if (!(std::fabs(f[j] - (*f0 + (double)j * *df)) <= tol)) return false;
    }
    return true;
}

static bool grid_uniform(const double *f, int64_t nf, double *f0, double *df) {
    double tol;
    if (nf <= 0) { *f0 = 0.0; *df = 0.0; return true; }
    if (!grid_params(f, nf, f0, df, &tol)) return false;
    const double a = *f0, d = *df;
    for (int64_t j0 = 0; j0 < nf; j0 += 4096) {
        const int64_t j1 = std::min<int64_t>(nf, j0 + 4096);
        int bad = 0;
        for (int64_t j = j0; j < j1; ++j) bad |= !(std::fabs(f[j] - (a + (double)j * d)) <= tol);
        if (bad) return false;
    }
    return true;
}

// Host-pointer calls run on one non-blocking stream per host thread and
// device, created on first use and kept.
struct HostStream {
    cudaStream_t s = nullptr;
    int make() {
        static thread_local cudaStream_t cached[64] = {};
        int dev = 0;
        FREDEC_CUDA_TRY(cudaGetDevice(&dev));
        if (dev < 0 || dev >= 64) {
            FREDEC_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
            owned = true;
            return FREDEC_OK;
        }
        if (!cached[dev]) FREDEC_CUDA_TRY(cudaStreamCreateWithFlags(&cached[dev], cudaStreamNonBlocking));
        s = cached[dev];
        return FREDEC_OK;
    }
    bool owned = false;
    ~HostStream() {
        if (owned && s) cudaStreamDestroy(s);
    }
};

void *pinned_scratch(int slot, size_t bytes) {
    static thread_local void *p[PIN_SLOTS] = {};
    static thread_local size_t have[PIN_SLOTS] = {};
    if (slot < 0 || slot >= PIN_SLOTS) return nullptr;
    if (have[slot] < bytes) {
        if (p[slot]) cudaFreeHost(p[slot]);
        p[slot] = nullptr;
        have[slot] = 0;
        if (cudaMallocHost(&p[slot], bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        have[slot] = bytes;
    }
    return p[slot];
}

// Read back status words after a synchronous host call.
static int finish_host(cudaStream_t st, const SeriesState *state, const int32_t *err) {
    FREDEC_CUDA_TRY(cudaStreamSynchronize(st));
    int32_t status = FREDEC_OK, e = FREDEC_OK;
    if (state) FREDEC_CUDA_TRY(cudaMemcpy(&status, &state->status, 4, cudaMemcpyDeviceToHost));
    if (err) FREDEC_CUDA_TRY(cudaMemcpy(&e, err, 4, cudaMemcpyDeviceToHost));
    if (status == FREDEC_ESINGULAR)
        return fail(FREDEC_ESINGULAR, "the base model's normal matrix is singular (duplicate base frequencies?)");
    if (e == FREDEC_ETIMEOUT) return fail(FREDEC_ETIMEOUT, "a bounded device wait gave up");
    if (e != FREDEC_OK) return fail(FREDEC_ECUDA, "a device-side index check failed (the access was skipped)");
    return FREDEC_OK;
}

int generic_grid_periodogram(const double *t, const double *y, const double *sigma, int64_t N, const double *base,
                             int nb, const double *f_grid_dev, int64_t nf, const fredec_opts &o, double *z, double *coef,
                             double *info, cudaStream_t st, SeriesState **state_out, DevBuf &ws);

}  // namespace fredec

using namespace fredec;

extern "C" {

void fredec_opts_init(fredec_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = FREDEC_FP64;
}

const char *fredec_last_error(void) { return g_last_error.c_str(); }
const char *fredec_version(void) { return "fredec-b300 0.1 (sm_103a)"; }

int fredec_periodogram_dev(const double *t, const double *y, const double *sigma, int64_t N, const double *base_freqs,
                           int32_t n_base, double f0, double df, int64_t nf, const fredec_opts *opts, double *z_out,
                           double *info_out, int64_t *topk_idx_out, double *coef_out, void *stream) {
    fredec_opts o;
    if (int rc = check_opts(opts, &o)) return rc;
    if (int rc = check_sizes(N, n_base, nf, o)) return rc;
    if (!t || !y || !sigma || (n_base > 0 && !base_freqs) || (nf > 0 && !z_out))
        return fail(FREDEC_EINVAL, "null pointer argument");
    if (!std::isfinite(f0) || !std::isfinite(df)) return fail(FREDEC_EINVAL, "f0 and df must be finite");
    DevBuf ws;
    SingleWork w;
    return periodogram_core(t, y, sigma, N, base_freqs, n_base, f0, df, nf, o, z_out, info_out, topk_idx_out,
                            coef_out, (cudaStream_t)stream, ws, w);
}

int fredec_topk_dev(const double *z, int64_t nf, int32_t k, int64_t *idx_out, void *stream) {
    if (k < 1 || k > FREDEC_MAX_TOPK) return fail(FREDEC_EINVAL, "k must be in 1..64");
    if (nf < 0) return fail(FREDEC_EINVAL, "nf must be >= 0");
    if (!idx_out || (nf > 0 && !z)) return fail(FREDEC_EINVAL, "null pointer argument");
    return launch_topk_single(z, nf, k, idx_out, (cudaStream_t)stream);
}

int fredec_periodogram_ex(const double *t, const double *y, const double *sigma, int64_t N, const double *base_freqs,
                          int32_t n_base, const double *f_grid, int64_t nf, const fredec_opts *opts, double *z_out,
                          double *info_out, int64_t *topk_idx_out, double *coef_out) {
    fredec_opts o;
    if (int rc = check_opts(opts, &o)) return rc;
    if (int rc = check_sizes(N, n_base, nf, o)) return rc;
    if (int rc = check_series_host(t, y, sigma, N, base_freqs, n_base)) return rc;
    if (nf > 0 && (!f_grid || !z_out)) return fail(FREDEC_EINVAL, "null f_grid or z_out");
    // A grid that looks uniform on a sample starts the uniform-grid pipeline
    // at once; the full test of every entry runs on the host meanwhile, and a
    // grid that fails it is redone by the generic-grid kernel.
    double f0, df;
    const bool spec = grid_uniform_sampled(f_grid, nf, &f0, &df);
    // A page-locked z_out is written by the kernels themselves, during the
    // computation, instead of by a copy after it (mixed precision, uniform
    // grid, difference statistic: the only passes that write z are then the
    // periodogram and the re-evaluation of flagged bins).
    double *z_mirror = nullptr;
    if (spec && nf > 0 && o.statistic == FREDEC_Z_DIFF && o.precision == FREDEC_MIXED) {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, z_out) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer)
            z_mirror = static_cast<double *>(pa.devicePointer);
        cudaGetLastError();
    }
    // a CUDA failure before the full grid check: a non-finite grid entry is
    // still reported as the validation error it is
    auto early = [&](int code) {
        return nf > 0 && !finite_all(f_grid, nf) ? fail(FREDEC_EINVAL, "trial frequencies must be finite") : code;
    };
    HostStream hs;
    if (int rc = hs.make()) return early(rc);
    cudaStream_t st = hs.s;
    const int nb = n_base;
    const int k = o.topk;
    int rc = FREDEC_OK;
    {
        DevBuf io;
        const size_t nin = 3 * N + nb + nf;
        const size_t bytes = nin * 8 + (size_t)nf * 8 + 3 * 8 + (size_t)k * 8 + (coef_out ? 16 * nf : 0) + 64;
        if ((rc = io.alloc(bytes, st))) return early(rc);
        double *d = io.as<double>();
        double *dt = d, *dy = d + N, *ds = d + 2 * N, *db = d + 3 * N, *dfg = db + nb;
        double *dz = dfg + nf, *dinfo = dz + nf, *dcoef = dinfo + 3;
        int64_t *dtop = (int64_t *)(dcoef + (coef_out ? 2 * nf : 0));
        FREDEC_CUDA_TRY(cudaMemcpyAsync(dt, t, N * 8, cudaMemcpyHostToDevice, st));
        FREDEC_CUDA_TRY(cudaMemcpyAsync(dy, y, N * 8, cudaMemcpyHostToDevice, st));
        FREDEC_CUDA_TRY(cudaMemcpyAsync(ds, sigma, N * 8, cudaMemcpyHostToDevice, st));
        if (nb) FREDEC_CUDA_TRY(cudaMemcpyAsync(db, base_freqs, nb * 8, cudaMemcpyHostToDevice, st));
        DevBuf ws, ws_generic;
        const SeriesState *state = nullptr;
        const int32_t *err = nullptr;
        bool uniform = false;
        // the status words and the small outputs in one page-locked block: written
        // by the last top-k kernel itself when there is one, else copied behind
        // the device work; one synchronisation either way
        char *pin = static_cast<char *>(pinned_scratch(PIN_HOST_CALL, 32 + (size_t)FREDEC_MAX_TOPK * 8));
        unsigned char *pin_dev = nullptr;
        if (pin && spec && k && topk_idx_out && nf > 0) {
            void *dp = nullptr;
            if (cudaHostGetDevicePointer(&dp, pin, 0) == cudaSuccess) pin_dev = static_cast<unsigned char *>(dp);
            cudaGetLastError();
        }
        if (spec) {
            SingleWork w;
            rc = periodogram_core(dt, dy, ds, N, db, nb, f0, df, nf, o, dz, dinfo, k ? dtop : nullptr,
                                  coef_out ? dcoef : nullptr, st, ws, w, z_mirror, pin_dev);
            state = w.state;
            err = w.err;
            uniform = grid_uniform(f_grid, nf, &f0, &df);   // overlaps the device work
            if (!uniform && !rc) rc = cudaStreamSynchronize(st) == cudaSuccess ? FREDEC_OK : FREDEC_ECUDA;
        }
        if (!rc && !uniform) {
            if (!finite_all(f_grid, nf)) return fail(FREDEC_EINVAL, "trial frequencies must be finite");
            FREDEC_CUDA_TRY(cudaMemcpyAsync(dfg, f_grid, nf * 8, cudaMemcpyHostToDevice, st));
            SeriesState *sp = nullptr;
            rc = generic_grid_periodogram(dt, dy, ds, N, db, nb, dfg, nf, o, dz, coef_out ? dcoef : nullptr,
                                          dinfo, st, &sp, ws_generic);
            state = sp;
            err = nullptr;
            if (!rc && k) rc = launch_topk_single(dz, nf, k, dtop, st);
        }
        if (rc) {
            cudaStreamSynchronize(st);
            return rc;
        }
        if (!pin) {
            if ((rc = finish_host(st, state, err))) return rc;
        } else {
            int32_t *words = reinterpret_cast<int32_t *>(pin);
            if (!(pin_dev && uniform)) {   // no kernel of this call writes the block any more
                words[0] = FREDEC_OK;
                words[1] = FREDEC_OK;
                if (state) FREDEC_CUDA_TRY(cudaMemcpyAsync(&words[0], &state->status, 4, cudaMemcpyDeviceToHost, st));
                if (err) FREDEC_CUDA_TRY(cudaMemcpyAsync(&words[1], err, 4, cudaMemcpyDeviceToHost, st));
                if (info_out) FREDEC_CUDA_TRY(cudaMemcpyAsync(pin + 8, dinfo, 3 * 8, cudaMemcpyDeviceToHost, st));
                if (k && topk_idx_out)
                    FREDEC_CUDA_TRY(cudaMemcpyAsync(pin + 32, dtop, k * 8, cudaMemcpyDeviceToHost, st));
            }
            FREDEC_CUDA_TRY(cudaStreamSynchronize(st));
            if (words[0] == FREDEC_ESINGULAR)
                return fail(FREDEC_ESINGULAR, "the base model's normal matrix is singular (duplicate base frequencies?)");
            if (words[1] == FREDEC_ETIMEOUT) return fail(FREDEC_ETIMEOUT, "a bounded device wait gave up");
            if (words[1] != FREDEC_OK)
                return fail(FREDEC_ECUDA, "a device-side index check failed (the access was skipped)");
        }
        const bool copies = (nf && !(uniform && z_mirror)) || (coef_out && nf);
        if (nf && !(uniform && z_mirror)) FREDEC_CUDA_TRY(cudaMemcpyAsync(z_out, dz, nf * 8, cudaMemcpyDeviceToHost, st));
        if (coef_out && nf) FREDEC_CUDA_TRY(cudaMemcpyAsync(coef_out, dcoef, 16 * nf, cudaMemcpyDeviceToHost, st));
        if (pin) {
            if (info_out) std::memcpy(info_out, pin + 8, 3 * 8);
            if (k && topk_idx_out) std::memcpy(topk_idx_out, pin + 32, (size_t)k * 8);
        } else {
            if (info_out) FREDEC_CUDA_TRY(cudaMemcpyAsync(info_out, dinfo, 3 * 8, cudaMemcpyDeviceToHost, st));
            if (k && topk_idx_out)
                FREDEC_CUDA_TRY(cudaMemcpyAsync(topk_idx_out, dtop, k * 8, cudaMemcpyDeviceToHost, st));
        }
        if (copies || !pin) FREDEC_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return FREDEC_OK;
}

int fredec_periodogram_vjp_dev(const double *t, const double *y, const double *sigma, int64_t N,
                               const double *base_freqs, int32_t n_base, double f0, double df, int64_t nf,
                               const double *coef, const double *info, const double *v, int32_t precision,
                               double *dldy_out, void *stream) {
    (void)info;   // the time origin is recomputed identically from the same inputs
    if (precision != FREDEC_FP64 && precision != FREDEC_MIXED) return fail(FREDEC_EINVAL, "bad precision");
    fredec_opts o;   // the adjoint is built for the constant-plus-sinusoids base
    fredec_opts_init(&o);
    if (int rc = check_sizes(N, n_base, nf, o)) return rc;
    if (!t || !y || !sigma || (n_base > 0 && !base_freqs) || !dldy_out || (nf > 0 && (!coef || !v)))
        return fail(FREDEC_EINVAL, "null pointer argument");
    if (!std::isfinite(f0) || !std::isfinite(df)) return fail(FREDEC_EINVAL, "f0 and df must be finite");
    return launch_vjp_pipeline(t, y, sigma, N, base_freqs, n_base, f0, df, nf, coef, v, precision, dldy_out,
                               (cudaStream_t)stream);
}

int fredec_periodogram_vjp(const double *t, const double *y, const double *sigma, int64_t N, const double *base_freqs,
                           int32_t n_base, double f0, double df, int64_t nf, const double *v, int32_t precision,
                           double *dldy_out) {
    if (precision != FREDEC_FP64 && precision != FREDEC_MIXED) return fail(FREDEC_EINVAL, "bad precision");
    fredec_opts o;   // the adjoint is built for the constant-plus-sinusoids base
    fredec_opts_init(&o);
    if (int rc = check_sizes(N, n_base, nf, o)) return rc;
    if (int rc = check_series_host(t, y, sigma, N, base_freqs, n_base)) return rc;
    if (!dldy_out || (nf > 0 && !v)) return fail(FREDEC_EINVAL, "null pointer argument");
    if (!std::isfinite(f0) || !std::isfinite(df) || (nf > 0 && !finite_all(v, nf)))
        return fail(FREDEC_EINVAL, "f0, df and v must be finite");
    HostStream hs;
    if (int rc = hs.make()) return rc;
    cudaStream_t st = hs.s;
    int rc = FREDEC_OK;
    {
        DevBuf io;
        if ((rc = io.alloc((3 * N + n_base + nf + 2 * nf + N + 8) * 8, st))) return rc;
        double *d = io.as<double>();
        double *dt = d, *dy = d + N, *ds = d + 2 * N, *db = d + 3 * N, *dv = db + n_base, *dcoef = dv + nf,
               *dout = dcoef + 2 * nf, *dinfo = dout + N;
        FREDEC_CUDA_TRY(cudaMemcpyAsync(dt, t, N * 8, cudaMemcpyHostToDevice, st));
        FREDEC_CUDA_TRY(cudaMemcpyAsync(dy, y, N * 8, cudaMemcpyHostToDevice, st));
        FREDEC_CUDA_TRY(cudaMemcpyAsync(ds, sigma, N * 8, cudaMemcpyHostToDevice, st));
        if (n_base) FREDEC_CUDA_TRY(cudaMemcpyAsync(db, base_freqs, n_base * 8, cudaMemcpyHostToDevice, st));
        if (nf) FREDEC_CUDA_TRY(cudaMemcpyAsync(dv, v, nf * 8, cudaMemcpyHostToDevice, st));
        fredec_opts o;
        fredec_opts_init(&o);
        o.precision = precision;
        const SeriesState *state = nullptr;
        {
            DevBuf ws;
            SingleWork w;
            DevBuf zbuf;
            if ((rc = zbuf.alloc(std::max<int64_t>(nf, 1) * 8, st))) return rc;
            if ((rc = periodogram_core(dt, dy, ds, N, db, n_base, f0, df, nf, o, zbuf.as<double>(), dinfo, nullptr,
                                       dcoef, st, ws, w)))
                return rc;
            state = w.state;
            if ((rc = finish_host(st, state, w.err))) return rc;
        }
        if ((rc = launch_vjp_pipeline(dt, dy, ds, N, db, n_base, f0, df, nf, dcoef, dv, precision, dout, st)))
            return rc;
        FREDEC_CUDA_TRY(cudaStreamSynchronize(st));
        FREDEC_CUDA_TRY(cudaMemcpy(dldy_out, dout, N * 8, cudaMemcpyDeviceToHost));
    }
    FREDEC_CUDA_TRY(cudaStreamSynchronize(st));
    return FREDEC_OK;
}

int fredec_periodogram(const double *t, const double *y, const double *sigma, int64_t N, const double *base_freqs,
                       int32_t n_base, const double *f_grid, int64_t nf, double *z_out) {
    return fredec_periodogram_ex(t, y, sigma, N, base_freqs, n_base, f_grid, nf, nullptr, z_out, nullptr, nullptr,
                                 nullptr);
}

}  // extern "C"
