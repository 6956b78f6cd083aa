// Internal declarations shared by the CUDA translation units of libfredec.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/fredec.h"

namespace fredec {

// ---------------------------------------------------------------------------
// Limits and layout constants

constexpr int PMAX = 2 * FREDEC_MAX_NBASE + 1;      // base columns (constant + cos/sin pairs)
constexpr int NTRI = PMAX * (PMAX + 1) / 2;         // packed lower triangle
constexpr int PREP_THREADS = 32;                     // one point per thread, one warp per prep chunk
constexpr int TILE_POINTS = 128;                     // observation records per smem tile (at most)
constexpr double DROP2 = 1e-14;                      // squared column-drop ratio (1e-7)^2

// Record widths.  Mixed records (32-bit words):
//   [0..1] phase A = frac(f0 t') as u64 turns, [2..3] phase B = frac(df t'),
//   [4] cos(2 pi df t'), [5] sin(2 pi df t'), [6] cos(4 pi df t'),
//   [7] sin(4 pi df t') (the two-step rotation, rounded once from FP64),
//   then the set [s, s r, s psi_k (p)] padded to a multiple of 4 words, with
//   s = sqrt(w) rounded to FP32: the mixed kernels scale each point's cos/sin
//   by s, so that s psi_k (s c) = w psi_k c and (s c)^2 = s^2 c^2; the weight
//   they integrate is s^2 (rec_weight).
// FP64 records (64-bit words): [0] A, [1] B, [2] cos, [3] sin, [4] w, [5] w r,
//   [6..6+p) w psi_k.  Both are padded to a multiple of 16 bytes.
// Records with a second set (nset = 2, the periodogram's frequency derivative)
// append the t'-weighted values of the weighted ones, padded the same way:
//   mixed [t', s r t', s psi_k t' (p)] (t' multiplies the scaled (s c)^2 and
//   (s c)(s s) sums); FP64 [w t', w r t', w psi_k t' (p)].
__host__ __device__ constexpr int rec32_set_words(int p) { return 4 * ((p + 2 + 3) / 4); }
#ifdef __CUDACC__
// s = sqrt(w) as the mixed records carry it, and the weight s^2 that the
// mixed kernels integrate in place of w.
__device__ __forceinline__ double rec_sqrt_w(double w) { return (double)__double2float_rn(sqrt(w)); }
__device__ __forceinline__ double rec_weight(double w) {
    const double s = rec_sqrt_w(w);
    return s * s;
}
#endif
__host__ __device__ constexpr int rec64_set_words(int p) { return 2 * ((p + 1) / 2); }
__host__ __device__ constexpr int rec32_words(int p, int nset = 1) { return 8 + nset * rec32_set_words(p); }
__host__ __device__ constexpr int rec64_words(int p, int nset = 1) {
    return 6 + rec64_set_words(p) + (nset == 2 ? 2 + rec64_set_words(p) : 0);
}
__host__ __device__ constexpr int rec_bytes(int p, int prec, int nset = 1) {
    return prec == FREDEC_MIXED ? 4 * rec32_words(p, nset) : 8 * rec64_words(p, nset);
}
// Float-float records for the re-evaluation of flagged mixed bins (32-bit
// words): [0..1] phase A, [2..3] phase B (u64), then hi/lo pairs of w, w r and
// w psi_k; padded to 16 bytes.  With nset = 2 hi/lo pairs of w t', w r t' and
// w psi_k t' follow, padded the same way.
__host__ __device__ constexpr int recff_set_words(int p) { return 4 * ((4 + 2 * p + 3) / 4); }
__host__ __device__ constexpr int recff_words(int p, int nset = 1) {
    return 4 * ((8 + 2 * p + 3) / 4) + (nset == 2 ? recff_set_words(p) : 0);
}
__host__ __device__ constexpr int recff_bytes(int p, int nset = 1) { return 4 * recff_words(p, nset); }

// Per-series description (host-built, device-resident).
struct SeriesDesc {
    int64_t obs_off;     // into t, y, sigma
    int64_t base_off;    // into base frequencies
    int64_t rec_off;     // into the record buffer, bytes
    int64_t rec64_off;   // into the extra FP64 record buffer (mixed with re-evaluation), bytes
    int64_t psi_off;     // into the psi scratch, doubles (p*N per series)
    int64_t z_off;       // into z (and 2*z_off into coef)
    int64_t chunk_off;   // first prep chunk of this series
    double f0, df;       // uniform grid f_j = f0 + j df
    int64_t nf;
    int32_t N, nb, nchunks, p;
    int32_t pb;          // base columns: 1 + npoly + 2 nb (p = pb rounded up to odd; column pb, if any, is zero)
    int32_t npoly;       // degree of the time polynomial of the base model
};

// Per-series results of the prep kernels.
struct SeriesState {
    double W;            // sum of weights (FP64)
    double Wf;           // sum of s^2, s = sqrt(w) rounded to FP32 (the weight the mixed kernels integrate)
    double tc;           // time origin
    double chi2;         // l(f') of the base model
    double Swt;          // sum w t (scratch)
    double tscale;       // time scale of the polynomial columns: tau = (t - tc) / tscale
    double L1[NTRI];     // Cholesky factor of the raw base Gram
    double L2[NTRI];     // Cholesky factor of the second (re-orthogonalisation) Gram
    double R1[PMAX];     // 1 / diagonal of L1
    double R2[PMAX];     // 1 / diagonal of L2
    double a[PMAX];      // coefficients of y on the orthonormal base columns
    double a2[PMAX];     // second-pass correction
    int32_t status;      // FREDEC_OK or FREDEC_ESINGULAR
    uint32_t counter[6]; // last-block-done counters (reset by the finishing block)
};

// ---------------------------------------------------------------------------
// Host-side error plumbing

void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
#define FREDEC_CUDA_TRY(expr)                                                        \
    do {                                                                             \
        cudaError_t e_ = (expr);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return ::fredec::fail(FREDEC_ECUDA, std::string(#expr) + ": " +         \
                                                     cudaGetErrorString(e_));        \
    } while (0)

// Workspace from the stream-ordered allocator; freed on destruction.
struct DevBuf {
    void *ptr = nullptr;
    cudaStream_t stream = nullptr;
    size_t bytes = 0;
    int alloc(size_t n, cudaStream_t s);
    template <class T> T *as() const { return static_cast<T *>(ptr); }
    ~DevBuf();
};

// ---------------------------------------------------------------------------
// Prep (prep.cu)

constexpr int64_t SERIES_PREP_MAX_N = 16384;   // one prep CTA per series up to this N
constexpr int64_t CLUSTER_PREP_MAX_N = 65536;  // one prep cluster per series up to this N (fewer than 256 series)

struct PrepPlan {
    int S = 0;                 // series
    int64_t max_n = 0;         // largest series (chooses the one-CTA-per-series prep)
    int64_t nchunks = 0;       // total prep chunks
    int pmax = 1;
    int base_p = 0;            // base columns of every series when none has polynomial terms, else 0
    SeriesDesc *desc = nullptr;      // device [S]
    SeriesState *state = nullptr;    // device [S]
    int32_t *chunk_series = nullptr; // device [nchunks]
    double *partials = nullptr;      // device [nchunks * NPART(pmax)]
    double *psi = nullptr;           // device scratch
    void *rec = nullptr;             // device records
};
int prep_npart(int pmax);
// The prep kernels and the per-point records (rec, and float-float records in
// rec64 when given); nset = 2 adds the t'-weighted values to every record.
int run_prep_records(const PrepPlan &pp, const double *t, const double *y, const double *sigma,
                     const double *base, int precision, void *rec64, cudaStream_t st, int nset = 1);
// Enqueue the prep kernels (uniform grids).  Writes state[] and records.
int launch_prep(const PrepPlan &pp, const double *t, const double *y, const double *sigma,
                const double *base, int precision, cudaStream_t st);

// ---------------------------------------------------------------------------
// Periodogram kernels (pgram.cu)

struct PgramShape { int fpt; int warps; };
PgramShape default_shape(int precision, int p, int64_t N, int64_t nf);
bool shape_supported(int precision, int p, int fpt);
// sin/cos seed of the mixed periodogram kernels (1 = MUFU, 0 = table)
int seed_mode();
// Page-locked host scratch for small asynchronous transfers, per host thread
// and slot (one slot per user, so that one user's pointer stays valid while
// another runs), allocated once (page-locking is an operating-system call)
// and kept for the life of the process; nullptr if cudaMallocHost fails.
enum PinnedSlot { PIN_HOST_CALL = 0, PIN_SCAN = 1, PIN_SLOTS = 2 };
void *pinned_scratch(int slot, size_t bytes);
// Single-series launch: z (and optional coef) for all nf grid points; the
// mixed path appends ill-conditioned bins (global z indices) to flag_list.
// z_mirror (optional): a second destination of every z value, e.g. the
// device address of the caller's page-locked host output.
int launch_pgram(int precision, const SeriesDesc *desc_dev, const SeriesState *state_dev,
                 const void *rec, int p, int N, int64_t nf, PgramShape shape, double flag_tau,
                 double *z, double *coef, int64_t *flag_list, int32_t *flag_count, int32_t *err,
                 cudaStream_t st, double *z_mirror = nullptr, float2 *tail_part = nullptr,
                 int32_t *tail_cnt = nullptr, int tail_gcap = 0);
// Bytes of the tail-split arrays of a mixed single-series launch of shape fpt
// with nset sets of sums (partial sums; 0 for FP64) and the tail CTAs they
// hold (*gcap); the tiles counters take 4 bytes per tail CTA more and must be
// zero at launch.
size_t pgram_tail_bytes(int precision, int p, int fpt, int *gcap, int nset = 1);
// FP64-grade re-evaluation of the listed bins (fixup.cu); z_mirror as above.
// nan_nf > 0 (one series): if the series' prep failed, the launch sets
// z[0..nan_nf) to NaN instead (the NaN fill of a failed call).
// dzdf (optional, single series): the records carry the t'-weighted set
// (nset = 2) and dz/df of each re-evaluated bin is written there too.
// max_items: entries of list and of z; err (optional) receives FREDEC_EINVAL
// when a listed index lies outside them (the bin is skipped).
int launch_fixup_bins(const SeriesDesc *desc, const SeriesState *state, int nseries, const void *rec64, int p,
                      const int64_t *list, const int32_t *count, int64_t max_items, double *z, double *coef,
                      cudaStream_t st, double *z_mirror = nullptr, int64_t nan_nf = 0, double *dzdf = nullptr,
                      int32_t *err = nullptr);

// Log form of the statistic (Eq. zpowrel) in place, per series (fixup.cu).
int launch_log_form(const SeriesDesc *desc, const SeriesState *state, int nseries, int64_t nf_max, double *z,
                    cudaStream_t st);

// Host-side validation shared by the single-series entry points (abi.cu):
// options (defaults when o is NULL) and sizes; FREDEC_EINVAL with a message.
int check_opts(const fredec_opts *o, fredec_opts *out);
int check_sizes(int64_t N, int32_t n_base, int64_t nf, const fredec_opts &o);

// Base column counts for n_base sinusoids and a time polynomial of degree npoly:
// pb real columns, padded to the odd count the periodogram kernels are built for.
inline int base_cols(int nb, int npoly) { return 1 + npoly + 2 * nb; }
inline int padded_cols(int pb) { return pb | 1; }

// Top-k local maxima (topk.cu); segmented over series.
int launch_topk(const double *z, const int64_t *z_off, const int64_t *nf, int S, int k,
                int64_t *idx_out, cudaStream_t st);
// info (optional): (chi2, W, t_c) of *state, written by the last top-k kernel.
// host (optional, with state): device address of a page-locked block that the
// same kernel fills with [state->status, *err] (int32), (chi2, W, t_c) at +8
// and the k indices at +32, so that a host caller needs no copies.
int launch_topk_single(const double *z, int64_t nf, int k, int64_t *idx_out, cudaStream_t st,
                       const SeriesState *state = nullptr, double *info = nullptr, const int32_t *err = nullptr,
                       unsigned char *host = nullptr);

// VJP (vjp.cu): dL/dy for one series on a uniform grid, all pointers device.
int launch_vjp_pipeline(const double *t, const double *y, const double *sigma, int64_t N, const double *base, int nb,
                        double f0, double df, int64_t nf, const double *coef, const double *v, int precision,
                        double *dldy, cudaStream_t st);

// Tuples (tuple.cu)
int tuple_eval_dev(const double *t, const double *y, const double *sigma, int64_t N,
                   const double *freqs, const int64_t *off, int64_t n_tuples, int max_m,
                   double *z, double *l0, cudaStream_t st);
int pool_table_dev(const double *t, const double *y, const double *sigma, int64_t N,
                   const double *pool, int n_pool, double *l_table, cudaStream_t st);
int tuple_grad_dev(const double *t, const double *y, const double *sigma, int64_t N,
                   const double *freqs, const int64_t *off, int64_t n_tuples, int max_m,
                   int precision, double *z, double *dzdf, cudaStream_t st);
int tuple_refine_dev(const double *t, const double *y, const double *sigma, int64_t N,
                     double *freqs, const int64_t *off, int64_t n_tuples, int max_m,
                     int max_iter, double tol, int precision, double *l_out, int32_t *iters,
                     cudaStream_t st);

// Tuning table (tune.cu)
bool tuned_shape(int precision, int p, int64_t N, int64_t nf, PgramShape *out);

int sm_count();

// Launch with the programmatic stream serialization attribute (the kernel
// calls grid_dependency_wait() before reading its predecessor's results).
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}
// Events recorded around the main periodogram kernel (fredec_profile_events).
void set_profile_events(cudaEvent_t a, cudaEvent_t b);
void profile_events(cudaEvent_t *a, cudaEvent_t *b);

}  // namespace fredec
