// Phase 3 backward cascade and the Phase 4 ordering (Section 4), FAP helpers of
// Eq. zFAP, and the normalised bandwidth W of Section 2.
//
// Input: a table l[mask] over all 2^n subtuples of a candidate pool (the
// minimised chi2 of each subtuple, l[0] = l_0).  For every combination S
// (m members) and every proper subset K of S (k members), the relative test of
// Eq. zpowrel in its log form, base K and alternative S,
//     z(S\K | K) = (N - 3m - 1)/2 * ln(l[K] / l[S]),
// must reach the threshold for m - k added frequencies.  The comparison is
// done without a logarithm: z >= zthr  <=>  l[K] >= l[S] * exp(2 zthr / N_H),
// with the factors exp(2 zthr[m-k-1] / (N - 3m - 1)) computed once on the host.
//
// GPU layout:
//   cascade_pass_kernel   one thread per mask; layers in the order
//                         k = 0, m-1, 1, m-2, ... (the large middle layers
//                         last, as Section 4 suggests), every layer's subsets
//                         enumerated in colex order inside S, exit at the first
//                         failed test; pass flags packed 32 masks to a word by
//                         a warp ballot.
//   sup_*                 superset-OR transform of the packed flags: bit S of
//                         sup = some passing combination contains S.
//   maximal_kernel        passing S with no passing strict superset (the
//                         solutions never nest, Section 4), appended to a list.
//   bitonic sort          by (m, chi2, mask): the order of Phase 4.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fredec_internal.cuh"

namespace fredec {
namespace {

constexpr int QROW = FREDEC_MAX_POOL + 1;   // q table row: k = 0..m-1 for m <= FREDEC_MAX_POOL

struct Sol {
    double l;
    uint32_t mask;
    uint32_t m;
};

__device__ __forceinline__ uint32_t lowest_members(uint32_t S, int r) {
    uint32_t out = 0;
    for (int i = 0; i < r; ++i) {
        const uint32_t b = S & (0u - S);
        out |= b;
        S ^= b;
    }
    return out;
}

// Tests compare the bit patterns of the doubles as signed 64-bit integers:
// for non-negative values (and +inf) the order of the patterns is the numeric
// order, so a test is integer work (the FP64 pipe of this GPU is narrow).  A
// table entry passes as l_K when 0 < l_K <= +inf (NaN and negative patterns
// fall outside); the threshold l_S * q >= 0 is formed once per layer.
__global__ void cascade_pass_kernel(const double *__restrict__ l, int n, const double *__restrict__ qtab,
                                    uint32_t valid_m, uint32_t *__restrict__ pass_words) {
    constexpr long long INF_BITS = 0x7FF0000000000000LL;
    const long long *lb = reinterpret_cast<const long long *>(l);
    const uint32_t S = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nmask = 1u << n;
    bool ok = false;
    if (S < nmask && S != 0) {
        const int m = __popc(S);
        const double lS = l[S];
        ok = ((valid_m >> m) & 1u) && lS >= 0.0 && lS < INFINITY;
        for (int i = 0; ok && i < m; ++i) {
            const int k = (i & 1) ? m - 1 - (i >> 1) : (i >> 1);
            // l_S = 0: every l_K > 0 passes (its z is +inf), whatever q is
            const long long thr = lS == 0.0 ? 0LL : __double_as_longlong(lS * qtab[m * QROW + k]);
            uint32_t K = lowest_members(S, k);
            for (;;) {
                const long long lK = __ldg(lb + K);
                if (!(lK > 0 && lK <= INF_BITS && lK >= thr)) {
                    ok = false;
                    break;
                }
                if (k == 0) break;
                // next k-subset of S in colex order: clear the lowest run of K
                // (run = consecutive members of S), set the next member of S
                // above it, refill the lowest run-1 members of S.
                const uint64_t x = (uint64_t)K | ~(uint64_t)S;
                const uint64_t u = (uint64_t)(K & (0u - K));
                const uint64_t sum = x + u;
                if (sum < x) break;   // the run reached the top member: last subset
                const uint32_t v = (uint32_t)(sum & S);
                K = v | lowest_members(S, k - __popc(v));
            }
        }
    }
    const uint32_t bits = __ballot_sync(0xffffffffu, ok);
    if ((threadIdx.x & 31) == 0 && S < (nmask < 32 ? 32u : nmask)) pass_words[S >> 5] = bits;
}

// positions whose in-word index has bit j clear
__device__ __forceinline__ uint32_t nobit_mask(int j) {
    switch (j) {
        case 0: return 0x55555555u;
        case 1: return 0x33333333u;
        case 2: return 0x0F0F0F0Fu;
        case 3: return 0x00FF00FFu;
        default: return 0x0000FFFFu;
    }
}

__global__ void sup_init_kernel(const uint32_t *__restrict__ pass, uint32_t *__restrict__ sup, int64_t nwords,
                                int nlow) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nwords) return;
    uint32_t w = pass[i];
    for (int j = 0; j < nlow; ++j) w |= (w >> (1 << j)) & nobit_mask(j);
    sup[i] = w;
}

__global__ void sup_word_kernel(uint32_t *__restrict__ sup, int64_t nwords, int b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nwords || (i >> b & 1)) return;
    sup[i] |= sup[i | ((int64_t)1 << b)];
}

__global__ void maximal_kernel(const uint32_t *__restrict__ pass, const uint32_t *__restrict__ sup,
                               const double *__restrict__ l, int64_t nwords, int n, Sol *__restrict__ out,
                               int64_t cap, unsigned long long *__restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nwords) return;
    const int nlow = n < 5 ? n : 5;
    const uint32_t s = sup[i];
    uint32_t acc = 0;
    for (int j = 0; j < nlow; ++j) acc |= (s >> (1 << j)) & nobit_mask(j);
    for (int b = 0; b < n - 5; ++b)
        if (!(i >> b & 1)) acc |= sup[i | ((int64_t)1 << b)];
    uint32_t mw = pass[i] & ~acc;
    if (!mw) return;
    unsigned long long slot = atomicAdd(count, (unsigned long long)__popc(mw));
    while (mw) {
        const int pos = __ffs(mw) - 1;
        mw &= mw - 1;
        const uint32_t S = (uint32_t)(i * 32 + pos);
        if ((int64_t)slot < cap) out[slot] = Sol{l[S], S, (uint32_t)__popc(S)};
        ++slot;
    }
}

__device__ __forceinline__ bool sol_less(const Sol &a, const Sol &b) {
    if (a.m != b.m) return a.m < b.m;
    if (a.l != b.l) return a.l < b.l;
    return a.mask < b.mask;
}

__device__ __forceinline__ void cmp_swap(Sol *v, int64_t a, int64_t b, bool asc) {
    Sol x = v[a], y = v[b];
    if (sol_less(y, x) == asc) {
        v[a] = y;
        v[b] = x;
    }
}

constexpr int SMEM_SORT = 2048;

__global__ void __launch_bounds__(1024) sort_small_kernel(Sol *data, int64_t count, int P) {
    __shared__ Sol v[SMEM_SORT];
    for (int i = threadIdx.x; i < P; i += blockDim.x)
        v[i] = i < count ? data[i] : Sol{0.0, 0xffffffffu, 0xffffffffu};
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
                const int a = (i / j) * 2 * j + (i % j);
                cmp_swap(v, a, a + j, (a & k) == 0);
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < count; i += blockDim.x) data[i] = v[i];
}

__global__ void pad_kernel(Sol *data, int64_t count, int64_t P) {
    const int64_t i = count + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P) data[i] = Sol{0.0, 0xffffffffu, 0xffffffffu};
}

__global__ void bitonic_step_kernel(Sol *v, int64_t P, int64_t k, int64_t j) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P / 2) return;
    const int64_t a = (i / j) * 2 * j + (i % j);
    cmp_swap(v, a, a + j, (a & k) == 0);
}

__global__ void emit_kernel(const Sol *sorted, int64_t n_out, double l0, int64_t N, uint32_t *masks, double *G) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_out) return;
    const Sol s = sorted[i];
    masks[i] = s.mask;
    G[i] = (s.l / l0) * (double)(N - 1) / (double)(N - 3 * (int64_t)s.m - 1);
}

// W = f_max sqrt(4 pi Var_w(t)), weights 1/sigma^2; two passes in one CTA.
__global__ void __launch_bounds__(1024) bandwidth_kernel(const double *t, const double *sigma, int64_t N,
                                                         double f_max, double *W_out) {
    __shared__ double red[2][32];
    __shared__ double mean_s;
    double sw = 0.0, swt = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double w = 1.0 / (sigma[i] * sigma[i]);
        sw += w;
        swt = fma(w, t[i], swt);
    }
    for (int o = 16; o; o >>= 1) {
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
        swt += __shfl_xor_sync(0xffffffffu, swt, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) {
        red[0][warp] = sw;
        red[1][warp] = swt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < nw; ++q) {
            a += red[0][q];
            b += red[1][q];
        }
        red[0][0] = a;
        mean_s = b / a;
    }
    __syncthreads();
    const double W = red[0][0], mean = mean_s;
    __syncthreads();
    double sv = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double d = t[i] - mean;
        sv = fma(d * d, 1.0 / (sigma[i] * sigma[i]), sv);
    }
    for (int o = 16; o; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
    if (lane == 0) red[1][warp] = sv;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int q = 0; q < nw; ++q) v += red[1][q];
        *W_out = f_max * sqrt(4.0 * 3.14159265358979323846 * (v / W));
    }
}

int64_t binom(int n, int k) {
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

struct Stream {
    cudaStream_t s = nullptr;
    ~Stream() {
        if (s) cudaStreamDestroy(s);
    }
};

}  // namespace

// Device cascade on a device table; results copied to host vectors in the
// Phase 4 order.  pass_words_host (may be NULL) receives the packed flags.
int cascade_run(const double *l_dev, int n, int64_t N, const double *zthr, double l0, uint32_t *pass_words_host,
                std::vector<uint32_t> *masks_host, std::vector<double> *G_host, cudaStream_t st) {
    std::vector<double> q((size_t)QROW * QROW, 0.0);
    uint32_t valid = 0;
    for (int m = 1; m <= n; ++m) {
        const int64_t NH = N - 3 * (int64_t)m - 1;
        if (NH <= 0) continue;
        valid |= 1u << m;
        for (int k = 0; k < m; ++k) q[(size_t)m * QROW + k] = std::exp(2.0 * zthr[m - k - 1] / (double)NH);
    }
    const int64_t nmask = (int64_t)1 << n;
    const int64_t nwords = std::max<int64_t>(1, nmask / 32);
    const int64_t cap = std::max<int64_t>(1, std::min<int64_t>(nmask, binom(n, n / 2)));
    int64_t P = 2;
    while (P < cap) P <<= 1;
    size_t off = 0;
    auto take = [&](size_t b) { size_t at = off; off = (off + b + 255) / 256 * 256; return at; };
    const size_t o_q = take(q.size() * 8), o_pass = take(nwords * 4), o_sup = take(nwords * 4);
    const size_t o_sol = take((size_t)P * sizeof(Sol)), o_cnt = take(8);
    const size_t o_masks = take((size_t)cap * 4), o_G = take((size_t)cap * 8);
    DevBuf buf;
    if (int rc = buf.alloc(off, st)) return rc;
    char *b = buf.as<char>();
    double *q_d = (double *)(b + o_q);
    uint32_t *pass = (uint32_t *)(b + o_pass), *sup = (uint32_t *)(b + o_sup);
    Sol *sol = (Sol *)(b + o_sol);
    unsigned long long *cnt = (unsigned long long *)(b + o_cnt);
    uint32_t *masks_d = (uint32_t *)(b + o_masks);
    double *G_d = (double *)(b + o_G);
    FREDEC_CUDA_TRY(cudaMemcpyAsync(q_d, q.data(), q.size() * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemsetAsync(cnt, 0, 8, st));
    const int64_t threads = std::max<int64_t>(32, nmask);
    cascade_pass_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(l_dev, n, q_d, valid, pass);
    FREDEC_CUDA_TRY(cudaGetLastError());
    const unsigned wb = (unsigned)((nwords + 255) / 256);
    sup_init_kernel<<<wb, 256, 0, st>>>(pass, sup, nwords, n < 5 ? n : 5);
    for (int bit = 0; bit < n - 5; ++bit) sup_word_kernel<<<wb, 256, 0, st>>>(sup, nwords, bit);
    maximal_kernel<<<wb, 256, 0, st>>>(pass, sup, l_dev, nwords, n, sol, cap, cnt);
    FREDEC_CUDA_TRY(cudaGetLastError());
    unsigned long long count = 0;
    FREDEC_CUDA_TRY(cudaMemcpyAsync(&count, cnt, 8, cudaMemcpyDeviceToHost, st));
    if (pass_words_host)
        FREDEC_CUDA_TRY(cudaMemcpyAsync(pass_words_host, pass, nwords * 4, cudaMemcpyDeviceToHost, st));
    FREDEC_CUDA_TRY(cudaStreamSynchronize(st));
    if ((int64_t)count > cap) return fail(FREDEC_ECUDA, "cascade: more solutions than the antichain bound");
    masks_host->assign(count, 0);
    G_host->assign(count, 0.0);
    if (count == 0) return FREDEC_OK;
    int64_t Pc = 2;
    while (Pc < (int64_t)count) Pc <<= 1;
    if (Pc <= SMEM_SORT) {
        sort_small_kernel<<<1, 1024, 0, st>>>(sol, (int64_t)count, (int)Pc);
    } else {
        if (Pc > (int64_t)count)
            pad_kernel<<<(unsigned)((Pc - count + 255) / 256), 256, 0, st>>>(sol, (int64_t)count, Pc);
        for (int64_t k = 2; k <= Pc; k <<= 1)
            for (int64_t j = k >> 1; j > 0; j >>= 1)
                bitonic_step_kernel<<<(unsigned)((Pc / 2 + 255) / 256), 256, 0, st>>>(sol, Pc, k, j);
    }
    emit_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(sol, (int64_t)count, l0, N, masks_d, G_d);
    FREDEC_CUDA_TRY(cudaGetLastError());
    FREDEC_CUDA_TRY(cudaMemcpyAsync(masks_host->data(), masks_d, count * 4, cudaMemcpyDeviceToHost, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(G_host->data(), G_d, count * 8, cudaMemcpyDeviceToHost, st));
    FREDEC_CUDA_TRY(cudaStreamSynchronize(st));
    return FREDEC_OK;
}

int bandwidth_dev(const double *t, const double *sigma, int64_t N, double f_max, double *W_dev, cudaStream_t st) {
    bandwidth_kernel<<<1, 1024, 0, st>>>(t, sigma, N, f_max, W_dev);
    FREDEC_CUDA_TRY(cudaGetLastError());
    return FREDEC_OK;
}

}  // namespace fredec

using namespace fredec;

extern "C" double fredec_fap_bound(int32_t n, double A, double W, double z) {
    if (n < 1 || !(z > 0.0) || !(A > 0.0) || !(W > 0.0)) return NAN;
    return std::exp(std::log(A) + n * std::log(W) - z + (1.5 * n - 1.0) * std::log(z));
}

extern "C" double fredec_fap_threshold(int32_t n, double A, double W, double fap) {
    if (n < 1 || !(A > 0.0) || !(W > 0.0) || !(fap > 0.0)) return NAN;
    // g(z) = log M_n(z) - log fap, decreasing for z > a = 3n/2 - 1.
    const double a = 1.5 * n - 1.0, c = std::log(A) + n * std::log(W) - std::log(fap);
    auto g = [&](double z) { return c - z + a * std::log(z); };
    double lo = a > 0.0 ? a : 1e-300;
    if (g(lo) <= 0.0) return lo;
    double hi = std::max(2.0 * lo, 1.0);
    while (g(hi) > 0.0) hi *= 2.0;
    // Newton from the upper end (g is convex there), kept inside the bracket
    double z = hi;
    for (int it = 0; it < 100; ++it) {
        const double gz = g(z);
        if (gz > 0.0) lo = z; else hi = z;
        double zn = z - gz / (a / z - 1.0);
        if (!(zn > lo && zn < hi)) zn = 0.5 * (lo + hi);
        if (std::fabs(zn - z) <= 1e-15 * z) return zn;
        z = zn;
    }
    return z;
}

extern "C" int fredec_effective_bandwidth(const double *t, const double *sigma, int64_t N, double f_max,
                                          double *W_out) {
    if (!t || !sigma || !W_out || N < 2 || !(f_max > 0.0)) return fail(FREDEC_EINVAL, "bad bandwidth arguments");
    for (int64_t i = 0; i < N; ++i)
        if (!(sigma[i] > 0.0) || !std::isfinite(sigma[i]) || !std::isfinite(t[i]))
            return fail(FREDEC_EINVAL, "t must be finite and sigma positive");
    Stream s;
    FREDEC_CUDA_TRY(cudaStreamCreateWithFlags(&s.s, cudaStreamNonBlocking));
    DevBuf buf;
    if (int rc = buf.alloc((size_t)(2 * N + 1) * 8, s.s)) return rc;
    double *d = buf.as<double>();
    FREDEC_CUDA_TRY(cudaMemcpyAsync(d, t, N * 8, cudaMemcpyHostToDevice, s.s));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(d + N, sigma, N * 8, cudaMemcpyHostToDevice, s.s));
    if (int rc = bandwidth_dev(d, d + N, N, f_max, d + 2 * N, s.s)) return rc;
    FREDEC_CUDA_TRY(cudaMemcpyAsync(W_out, d + 2 * N, 8, cudaMemcpyDeviceToHost, s.s));
    FREDEC_CUDA_TRY(cudaStreamSynchronize(s.s));
    return FREDEC_OK;
}

extern "C" int fredec_cascade(const double *l_table, int32_t n_pool, int64_t N, const double *z_thr,
                              uint32_t *pass_bits, uint32_t *solutions, double *G_out, int64_t capacity,
                              int64_t *n_solutions) {
    if (n_pool < 0 || n_pool > FREDEC_MAX_POOL || !l_table || (n_pool > 0 && !z_thr) || N < 1 || capacity < 0 ||
        (capacity > 0 && (!solutions || !G_out)) || !n_solutions)
        return fail(FREDEC_EINVAL, "bad cascade arguments");
    for (int k = 0; k < n_pool; ++k)
        if (std::isnan(z_thr[k])) return fail(FREDEC_EINVAL, "z_thr must not be NaN");
    const int64_t nmask = (int64_t)1 << n_pool;
    Stream s;
    FREDEC_CUDA_TRY(cudaStreamCreateWithFlags(&s.s, cudaStreamNonBlocking));
    DevBuf lbuf;
    if (int rc = lbuf.alloc((size_t)nmask * 8, s.s)) return rc;
    FREDEC_CUDA_TRY(cudaMemcpyAsync(lbuf.ptr, l_table, nmask * 8, cudaMemcpyHostToDevice, s.s));
    std::vector<uint32_t> words(std::max<int64_t>(1, nmask / 32));
    std::vector<uint32_t> masks;
    std::vector<double> G;
    if (int rc = cascade_run(lbuf.as<double>(), n_pool, N, z_thr, l_table[0], pass_bits ? words.data() : nullptr,
                             &masks, &G, s.s))
        return rc;
    if (pass_bits) std::copy(words.begin(), words.end(), pass_bits);
    *n_solutions = (int64_t)masks.size();
    const int64_t nout = std::min<int64_t>(capacity, (int64_t)masks.size());
    for (int64_t i = 0; i < nout; ++i) {
        solutions[i] = masks[i];
        G_out[i] = G[i];
    }
    return FREDEC_OK;
}
