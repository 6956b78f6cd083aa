// fredec_periodogram_noalloc_dev: the single-series periodogram pipeline
// (prep -> periodogram -> FP64-grade re-evaluation) with all of its scratch memory in
// one file-scope device array instead of the stream-ordered allocator.
//
// It exists for callers that cannot allocate device memory when they call:
// applications whose device memory is entirely reserved up front by their own
// allocator, real-time loops that forbid allocation after start-up, or
// plug-in hosts that do not let extension code call the CUDA allocator.  The
// paper has no counterpart.
//
// The array (NOALLOC_SCRATCH_BYTES) is loaded with the library and held on
// every GPU that loads it until the process exits.  All calls share it and it
// keeps the last call's contents; every field that must start at zero is
// cleared by the call itself.  Calls whose work overlaps on the GPU (different
// streams, or different host threads, without ordering) race on the array.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "fredec_internal.cuh"

namespace fredec {


namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 16u << 20;   // 16 MiB

// The fixed part of the scratch layout (descriptor, state, two status words,
// each in its own 256-byte block), as stated in the header's size formula.
constexpr size_t round256(size_t x) { return (x + 255) / 256 * 256; }
static_assert(round256(sizeof(SeriesDesc)) + round256(sizeof(SeriesState)) + 2 * 256 == 6912,
              "the header's scratch-size formula must follow the layout");

// Host code must not use this name as a device address: it is a host-side
// stand-in.  The device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device does this set-up).
int scratch_address(void **out) {
    int dev = 0;
    FREDEC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) return fail(FREDEC_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(FREDEC_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return FREDEC_OK;
}

__global__ void noalloc_init(SeriesDesc *desc, SeriesDesc v, SeriesState *state, int32_t *chunk_series,
                             int64_t nchunks, int32_t *flag_count, int32_t *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        *desc = v;
        for (int k = 0; k < 6; ++k) state->counter[k] = 0;
        state->status = FREDEC_OK;
        *flag_count = 0;
        *err = FREDEC_OK;
    }
    for (int64_t q = i; q < nchunks; q += (int64_t)gridDim.x * blockDim.x) chunk_series[q] = 0;
}

// info, and NaN in z when the base fit failed (singular base) or a bounded
// device wait gave up (FREDEC_ETIMEOUT): a z computed from a half-staged tile
// is never returned as if it were valid.
__global__ void noalloc_finish(const SeriesState *state, const int32_t *err, double *z, int64_t nf, double *info) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (info && i == 0) {
        info[0] = state->chi2;
        info[1] = state->W;
        info[2] = state->tc;
    }
    if (state->status != FREDEC_OK || *err != FREDEC_OK)
        for (int64_t j = i; j < nf; j += (int64_t)gridDim.x * blockDim.x) z[j] = NAN;
}

}  // namespace

}  // namespace fredec

using namespace fredec;

extern "C" int fredec_periodogram_noalloc_dev(const double *t, const double *y, const double *sigma, int64_t N,
                                              const double *base_freqs, int32_t n_base, double f0, double df,
                                              int64_t nf, const fredec_opts *opts, double *z_out, double *info_out,
                                              void *stream) {
    // every argument is checked before anything is enqueued
    fredec_opts o;
    if (int rc = check_opts(opts, &o)) return rc;
    if (o.topk != 0) return fail(FREDEC_EINVAL, "the no-allocation entry point does not compute top-k (opts.topk must be 0)");
    if (int rc = check_sizes(N, n_base, nf, o)) return rc;
    if (!t || !y || !sigma || (n_base > 0 && !base_freqs) || (nf > 0 && !z_out))
        return fail(FREDEC_EINVAL, "null pointer argument");
    if (!std::isfinite(f0) || !std::isfinite(df)) return fail(FREDEC_EINVAL, "f0 and df must be finite");
    const cudaStream_t st = (cudaStream_t)stream;
    const int pb = base_cols(n_base, o.trend), p = padded_cols(pb);
    const int prec = o.precision;
    const double tau = o.flag_tau == 0.0 ? 0.2 : o.flag_tau;
    const bool fix = prec == FREDEC_MIXED && tau >= 0.0;
    const int64_t nchunks = (N + PREP_THREADS - 1) / PREP_THREADS;
    size_t off = 0;
    auto take = [&](size_t n) { size_t at = off; off = (off + n + 255) / 256 * 256; return at; };
    const size_t o_desc = take(sizeof(SeriesDesc)), o_state = take(sizeof(SeriesState));
    const size_t o_cs = take(nchunks * 4), o_part = take(nchunks * prep_npart(p) * 8);
    const size_t o_psi = take((size_t)p * N * 8), o_rec = take(N * (size_t)rec_bytes(p, prec));
    const size_t o_rec64 = fix ? take(N * (size_t)recff_bytes(p)) : 0;
    const size_t o_fl = fix ? take(nf * 8 + 8) : 0;
    const size_t o_fc = take(4), o_err = take(4);
    PgramShape shape;
    if (o.fpt > 0 || o.warps > 0) {
        shape = default_shape(prec, p, N, nf);
        if (o.fpt > 0) shape.fpt = o.fpt;
        if (o.warps > 0) shape.warps = o.warps;
    } else if (!tuned_shape(prec, p, N, nf, &shape)) {
        shape = default_shape(prec, p, N, nf);
    }
    if (!shape_supported(prec, p, shape.fpt) || shape.warps < 1 || shape.warps > 8)
        return fail(FREDEC_EINVAL, "no compiled kernel for this (precision, p, opts.fpt, opts.warps)");
    if (off > NOALLOC_SCRATCH_BYTES)
        return fail(FREDEC_EINVAL, "fredec_periodogram_noalloc_dev: this problem needs " + std::to_string(off) +
                                       " bytes of scratch, more than the fixed " +
                                       std::to_string(NOALLOC_SCRATCH_BYTES) + " bytes");
    void *base_ptr = nullptr;
    if (int rc = scratch_address(&base_ptr)) return rc;
    unsigned char *b = static_cast<unsigned char *>(base_ptr);
    SeriesDesc *desc = (SeriesDesc *)(b + o_desc);
    SeriesState *state = (SeriesState *)(b + o_state);
    int32_t *cs = (int32_t *)(b + o_cs);
    int64_t *flag_list = fix ? (int64_t *)(b + o_fl) : nullptr;
    int32_t *flag_count = (int32_t *)(b + o_fc);
    int32_t *err = (int32_t *)(b + o_err);
    void *rec = b + o_rec;
    void *rec64 = fix ? (void *)(b + o_rec64) : nullptr;

    SeriesDesc d{};
    d.f0 = f0;
    d.df = df;
    d.nf = nf;
    d.N = (int32_t)N;
    d.nb = n_base;
    d.p = p;
    d.pb = pb;
    d.npoly = o.trend;
    d.nchunks = (int32_t)nchunks;
    noalloc_init<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(1024, (nchunks + 255) / 256)), 256, 0, st>>>(
        desc, d, state, cs, nchunks, flag_count, err);
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
    if (int rc = run_prep_records(pp, t, y, sigma, base_freqs, prec, rec64, st)) return rc;
    if (nf > 0) {
        if (int rc = launch_pgram(prec, desc, state, rec, p, (int)N, nf, shape, tau, z_out, nullptr, flag_list,
                                  flag_count, err, st))
            return rc;
        if (fix)
            if (int rc = launch_fixup_bins(desc, state, 1, rec64, p, flag_list, flag_count, nf, z_out, nullptr, st,
                                           nullptr, 0, nullptr, err))
                return rc;
        if (o.statistic == FREDEC_Z_LOG)
            if (int rc = launch_log_form(desc, state, 1, nf, z_out, st)) return rc;
    }
    noalloc_finish<<<64, 256, 0, st>>>(state, err, z_out, nf, info_out);
    FREDEC_CUDA_TRY(cudaGetLastError());
    return FREDEC_OK;
}
