// Top-k local maxima of z (device), one or many series.
//
// A local maximum is z_j > z_{j-1} and z_j >= z_{j+1}; an end point counts when
// it exceeds its one neighbour (a single-point grid counts).  Maxima are ranked
// by decreasing z, ties to the lower index; missing ranks are -1.  Stage 1:
// every CTA takes a 4096-point chunk (thread t holds points t, t + 1024, ...,
// so the loads are coalesced), gathers its local maxima in shared memory (at
// most 2048: two maxima are never adjacent) and sorts them with a bitonic
// network; its first k, in rank order, are the chunk's candidates.  Stage 2:
// one CTA per series.  Few candidates (<= 512, or <= 2048 with k >= 16) are
// sorted the same way; otherwise (up to 1024 chunks) the chunks' sorted lists
// are merged by a k-round tournament (thread t holds the head of chunk t; each
// round a block argmax takes the best head and that chunk advances).  Series
// of more chunks use k rounds of warp selection over fixed slices, then a
// merge of the slices.
// 1024 threads per CTA: one compare-exchange per thread per sorting step.
// The order is strict and total, so the result does not depend on scheduling
// or on the order in which the maxima were gathered.  Every comparison is on
// integers: z is mapped once to an order-preserving 64-bit key (double
// comparisons run on the FP64 pipe, at 1/64 of the FP32 rate on this GPU).
#include <algorithm>
#include <cstring>
#include <vector>

#include "device_util.cuh"
#include "fredec_internal.cuh"

namespace fredec {

namespace {

constexpr int TK_THREADS = 1024;
constexpr int TK_WARPS = TK_THREADS / 32;
constexpr int TK_PER = 4;                        // points per thread
constexpr int TK_CHUNK = TK_THREADS * TK_PER;
constexpr int TK_SORT = TK_CHUNK / 2;            // sort capacity (maxima of a chunk)

// Order-preserving key of a non-NaN double: z1 < z2 exactly when
// key(z1) < key(z2) as unsigned integers (-0 is taken as +0).
__device__ __forceinline__ uint64_t order_key(double z) {
    uint64_t b = (uint64_t)__double_as_longlong(z);
    if (b == 0x8000000000000000ull) b = 0;
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ bool is_nan_bits(double z) {
    return ((uint64_t)__double_as_longlong(z) & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull;
}

// (k1, j1) ranks before (k2, j2); j < 0 is an empty slot, after everything.
__device__ __forceinline__ bool better(uint64_t k1, int64_t j1, uint64_t k2, int64_t j2) {
    if (j2 < 0) return j1 >= 0;
    if (j1 < 0) return false;
    return k1 > k2 || (k1 == k2 && j1 < j2);
}

// Sorts (kz, kj)[0..n) in shared memory into rank order; n a power of two.
__device__ void block_sort(uint64_t *kz, int64_t *kj, int n) {
    for (int size = 2; size <= n; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int i = threadIdx.x; i < n / 2; i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
                const bool first = (lo & size) == 0;   // this half-block in rank order
                const bool sw = first ? better(kz[hi], kj[hi], kz[lo], kj[lo]) : better(kz[lo], kj[lo], kz[hi], kj[hi]);
                if (sw) {
                    const uint64_t tz = kz[lo];
                    const int64_t tj = kj[lo];
                    kz[lo] = kz[hi];
                    kj[lo] = kj[hi];
                    kz[hi] = tz;
                    kj[hi] = tj;
                }
            }
        }
    __syncthreads();
}

__device__ __forceinline__ int pow2_at_least(int n) {
    int m = 2;
    while (m < n) m <<= 1;
    return m;
}

// Warp argmax of (z, j); every lane receives it.
__device__ __forceinline__ void warp_best(uint64_t &z, int64_t &j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t oz = __shfl_xor_sync(0xffffffffu, z, o);
        const int64_t oj = __shfl_xor_sync(0xffffffffu, j, o);
        if (better(oz, oj, z, j)) {
            z = oz;
            j = oj;
        }
    }
}

// One warp: the k best of the n candidates (cz, cj) (shared or global memory;
// the taken ones are marked j = -1), written to oz[0..k), oj[0..k).
__device__ void warp_select(const uint64_t *cz, int64_t *cj, int64_t n, int k, uint64_t *oz, int64_t *oj) {
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < k; ++r) {
        uint64_t bz = 0;
        int64_t bj = -1, bq = -1;
        for (int64_t q = lane; q < n; q += 32) {
            const int64_t j = cj[q];
            if (better(cz[q], j, bz, bj)) {
                bz = cz[q];
                bj = j;
                bq = q;
            }
        }
        const int64_t mine = bj;
        warp_best(bz, bj);
        if (bj >= 0 && mine == bj) cj[bq] = -1;   // the owning lane drops it
        __syncwarp();
        if (lane == 0) {
            oz[r] = bz;
            oj[r] = bj;
        }
    }
}

struct TopkArgs {
    const double *z;
    const int64_t *z_off;      // [S]
    const int64_t *nf;         // [S]
    const int32_t *chunk_series;
    const int64_t *chunk_begin; // first grid index of each chunk (series-local)
    const int64_t *chunk_off;  // [S+1] first chunk of each series
    int k;
    uint64_t *cand_z;          // [nchunks * k] order keys
    int64_t *cand_j;
    int64_t *out;              // [S * k]
    int64_t nf_single;         // single-series mode (chunk_series == nullptr)
    int64_t nchunks_single;
    const SeriesState *state;  // single-series mode, optional: stage 2 copies (chi2, W, t_c) to info
    double *info;
    const int32_t *err;        // with host: the call's bounded-wait status word (may be null)
    unsigned char *host;       // optional page-locked block: [status, err] int32, info at +8, indices at +32
};

__global__ void __launch_bounds__(TK_THREADS) topk_stage1(TopkArgs a) {
    __shared__ uint64_t kz[TK_SORT];
    __shared__ int64_t kj[TK_SORT];
    __shared__ int count;
    grid_dependency_wait();   // z
    const int64_t c = blockIdx.x;
    const int tid = threadIdx.x;
    const bool single = a.chunk_series == nullptr;
    const int s = single ? 0 : a.chunk_series[c];
    const double *z = a.z + (single ? 0 : a.z_off[s]);
    const int64_t n = single ? a.nf_single : a.nf[s];
    const int64_t cb = single ? c * TK_CHUNK : a.chunk_begin[c];
    if (tid == 0) count = 0;
    __syncthreads();
#pragma unroll
    for (int e = 0; e < TK_PER; ++e) {
        const int64_t j = cb + (int64_t)e * TK_THREADS + tid;
        if (j < n) {
            // the rule in double semantics: any comparison with a NaN is false
            const double zj = z[j];
            const double zl = j > 0 ? z[j - 1] : 0.0, zr = j + 1 < n ? z[j + 1] : 0.0;
            const uint64_t kc = order_key(zj);
            const bool lok = j > 0 && !is_nan_bits(zl), rok = j + 1 < n && !is_nan_bits(zr);
            bool m;
            if (n == 1) m = true;
            else if (j == 0) m = rok && kc > order_key(zr);
            else if (j == n - 1) m = lok && kc > order_key(zl);
            else m = lok && rok && kc > order_key(zl) && kc >= order_key(zr);
            if (m && !is_nan_bits(zj)) {
                const int at = atomicAdd(&count, 1);   // < TK_SORT: maxima are never adjacent
                kz[at] = kc;
                kj[at] = j;
            }
        }
    }
    __syncthreads();
    const int cnt = count, m = pow2_at_least(max(cnt, a.k));
    for (int q = cnt + tid; q < m; q += TK_THREADS) {
        kz[q] = 0;
        kj[q] = -1;
    }
    block_sort(kz, kj, m);
    for (int r = tid; r < a.k; r += TK_THREADS) {
        a.cand_z[c * a.k + r] = kz[r];
        a.cand_j[c * a.k + r] = kj[r];
    }
}

__global__ void __launch_bounds__(TK_THREADS) topk_stage2(TopkArgs a) {
    __shared__ uint64_t kz[TK_SORT];
    __shared__ int64_t kj[TK_SORT];
    __shared__ uint64_t oz[FREDEC_MAX_TOPK];
    __shared__ int64_t oj[FREDEC_MAX_TOPK];
    grid_dependency_wait();   // stage 1's candidates
    const int s = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool single = a.chunk_series == nullptr;
    const int64_t c0 = single ? 0 : a.chunk_off[s], c1 = single ? a.nchunks_single : a.chunk_off[s + 1];
    const int64_t nch = c1 - c0, ncand = nch * a.k;
    const uint64_t *cz = a.cand_z + c0 * a.k;
    int64_t *cj = a.cand_j + c0 * a.k;
    if (a.info && tid == 0) {
        a.info[0] = a.state->chi2;
        a.info[1] = a.state->W;
        a.info[2] = a.state->tc;
    }
    if (a.host && tid == 0) {
        int32_t *words = reinterpret_cast<int32_t *>(a.host);
        double *hinfo = reinterpret_cast<double *>(a.host + 8);
        words[0] = a.state->status;
        words[1] = a.err ? *a.err : FREDEC_OK;
        hinfo[0] = a.state->chi2;
        hinfo[1] = a.state->W;
        hinfo[2] = a.state->tc;
    }
    int64_t *htop = a.host ? reinterpret_cast<int64_t *>(a.host + 32) : nullptr;
    if (ncand <= 512 || (a.k >= 16 && ncand <= TK_SORT)) {
        const int m = pow2_at_least((int)ncand);
        for (int q = tid; q < m; q += TK_THREADS) {
            kz[q] = q < ncand ? cz[q] : 0;
            kj[q] = q < ncand ? cj[q] : -1;
        }
        block_sort(kz, kj, m);
        for (int r = tid; r < a.k; r += TK_THREADS) {
            a.out[(int64_t)s * a.k + r] = kj[r];
            if (htop) htop[r] = kj[r];
        }
        return;
    }
    if (nch <= TK_THREADS) {
        // head (hz, hj) of chunk tid and the entry after it (nz, nj), loaded
        // one round ahead so that the winner's advance waits for no load
        const bool own = tid < nch;
        const uint64_t *mz = cz + (int64_t)tid * a.k;
        const int64_t *mj = cj + (int64_t)tid * a.k;
        uint64_t hz = 0, nz = 0;
        int64_t hj = -1, nj = -1;
        if (own) {
            hz = mz[0];
            hj = mj[0];
            if (a.k > 1) {
                nz = mz[1];
                nj = mj[1];
            }
        }
        int ptr = 1;   // rank of (nz, nj) in chunk tid
        for (int r = 0; r < a.k; ++r) {
            uint64_t bz = hz;
            int64_t bj = hj;
            warp_best(bz, bj);
            if (lane == 0) {
                kz[warp] = bz;
                kj[warp] = bj;
            }
            __syncthreads();
            if (warp == 0) {
                bz = kz[lane];
                bj = kj[lane];
                warp_best(bz, bj);
                if (lane == 0) oj[r] = bj;
            }
            __syncthreads();
            if (hj >= 0 && hj == oj[r]) {   // the winning chunk advances
                hz = nz;
                hj = nj;
                ++ptr;
                nz = 0;
                nj = -1;
                if (ptr < a.k) {
                    nz = mz[ptr];
                    nj = mj[ptr];
                }
            }
        }
        for (int r = tid; r < a.k; r += TK_THREADS) {
            a.out[(int64_t)s * a.k + r] = oj[r];
            if (htop) htop[r] = oj[r];
        }
        return;
    }
    // many chunks: warp w selects the k best of [w ncand / 32, (w + 1) ncand / 32),
    // then one warp merges the 32k (<= TK_SORT)
    const int64_t q0 = ncand * warp / TK_WARPS, q1 = ncand * (warp + 1) / TK_WARPS;
    warp_select(cz + q0, cj + q0, q1 - q0, a.k, kz + warp * a.k, kj + warp * a.k);
    __syncthreads();
    if (warp == 0) {
        warp_select(kz, kj, (int64_t)TK_WARPS * a.k, a.k, oz, oj);
        __syncwarp();
        for (int r = lane; r < a.k; r += 32) {
            a.out[(int64_t)s * a.k + r] = oj[r];
            if (htop) htop[r] = oj[r];
        }
    }
}

}  // namespace

// Plan-time part of the segmented top-k: chunk metadata, uploaded once.
int topk_plan_bytes(const int64_t *nf_h, int S, int k, int64_t *nchunks_out) {
    int64_t nch = 0;
    for (int s = 0; s < S; ++s) nch += std::max<int64_t>(1, (nf_h[s] + TK_CHUNK - 1) / TK_CHUNK);
    *nchunks_out = nch;
    return (int)0;
}

size_t topk_plan_size(int S, int64_t nch, int k) { return nch * 4 + nch * 8 + (S + 1) * 8 + 2 * S * 8 + nch * k * 16 + 256; }

// Upload the metadata into dev (topk_plan_size bytes, synchronous) and return
// the argument block for topk_plan_launch.
int topk_plan_make(const int64_t *z_off_h, const int64_t *nf_h, int S, int k, int64_t *idx_out, const double *z,
                   unsigned char *dev, void *args_out) {
    std::vector<int32_t> cs;
    std::vector<int64_t> cb, coff(S + 1, 0);
    for (int s = 0; s < S; ++s) {
        const int64_t nc = std::max<int64_t>(1, (nf_h[s] + TK_CHUNK - 1) / TK_CHUNK);
        coff[s + 1] = coff[s] + nc;
        for (int64_t c = 0; c < nc; ++c) {
            cs.push_back(s);
            cb.push_back(c * TK_CHUNK);
        }
    }
    const int64_t nch = coff[S];
    unsigned char *p = dev;
    int64_t *d_cb = (int64_t *)p; p += nch * 8;
    int64_t *d_coff = (int64_t *)p; p += (S + 1) * 8;
    int64_t *d_zoff = (int64_t *)p; p += S * 8;
    int64_t *d_nf = (int64_t *)p; p += S * 8;
    uint64_t *d_cz = (uint64_t *)p; p += nch * k * 8;
    int64_t *d_cj = (int64_t *)p; p += nch * k * 8;
    int32_t *d_cs = (int32_t *)p;
    FREDEC_CUDA_TRY(cudaMemcpy(d_cb, cb.data(), nch * 8, cudaMemcpyHostToDevice));
    FREDEC_CUDA_TRY(cudaMemcpy(d_coff, coff.data(), (S + 1) * 8, cudaMemcpyHostToDevice));
    FREDEC_CUDA_TRY(cudaMemcpy(d_zoff, z_off_h, S * 8, cudaMemcpyHostToDevice));
    FREDEC_CUDA_TRY(cudaMemcpy(d_nf, nf_h, S * 8, cudaMemcpyHostToDevice));
    FREDEC_CUDA_TRY(cudaMemcpy(d_cs, cs.data(), nch * 4, cudaMemcpyHostToDevice));
    TopkArgs a{z, d_zoff, d_nf, d_cs, d_cb, d_coff, k, d_cz, d_cj, idx_out, 0, 0, nullptr, nullptr, nullptr, nullptr};
    static_assert(sizeof(TopkArgs) <= 256, "args block");
    std::memcpy(args_out, &a, sizeof(a));
    return FREDEC_OK;
}

// Kernel launches only (capturable).
int topk_plan_launch(const void *args, int64_t nch, int S, cudaStream_t st) {
    TopkArgs a;
    std::memcpy(&a, args, sizeof(a));
    topk_stage1<<<(unsigned)nch, TK_THREADS, 0, st>>>(a);
    topk_stage2<<<(unsigned)S, TK_THREADS, 0, st>>>(a);
    FREDEC_CUDA_TRY(cudaGetLastError());
    return FREDEC_OK;
}

int launch_topk(const double *z, const int64_t *z_off_h, const int64_t *nf_h, int S, int k, int64_t *idx_out,
                cudaStream_t st) {
    if (k <= 0 || S <= 0) return FREDEC_OK;
    std::vector<int32_t> cs;
    std::vector<int64_t> cb, coff(S + 1, 0);
    for (int s = 0; s < S; ++s) {
        const int64_t nc = std::max<int64_t>(1, (nf_h[s] + TK_CHUNK - 1) / TK_CHUNK);
        coff[s + 1] = coff[s] + nc;
        for (int64_t c = 0; c < nc; ++c) {
            cs.push_back(s);
            cb.push_back(c * TK_CHUNK);
        }
    }
    const int64_t nch = coff[S];
    DevBuf meta;
    const size_t bytes = nch * 4 + nch * 8 + (S + 1) * 8 + 2 * S * 8 + nch * k * 16 + 64;
    if (int rc = meta.alloc(bytes, st)) return rc;
    unsigned char *p = meta.as<unsigned char>();
    int64_t *d_cb = (int64_t *)p; p += nch * 8;
    int64_t *d_coff = (int64_t *)p; p += (S + 1) * 8;
    int64_t *d_zoff = (int64_t *)p; p += S * 8;
    int64_t *d_nf = (int64_t *)p; p += S * 8;
    uint64_t *d_cz = (uint64_t *)p; p += nch * k * 8;
    int64_t *d_cj = (int64_t *)p; p += nch * k * 8;
    int32_t *d_cs = (int32_t *)p;
    FREDEC_CUDA_TRY(cudaMemcpyAsync(d_cb, cb.data(), nch * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(d_coff, coff.data(), (S + 1) * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(d_zoff, z_off_h, S * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(d_nf, nf_h, S * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(d_cs, cs.data(), nch * 4, cudaMemcpyHostToDevice, st));
    TopkArgs a{z, d_zoff, d_nf, d_cs, d_cb, d_coff, k, d_cz, d_cj, idx_out, 0, 0, nullptr, nullptr, nullptr, nullptr};
    topk_stage1<<<(unsigned)nch, TK_THREADS, 0, st>>>(a);
    topk_stage2<<<(unsigned)S, TK_THREADS, 0, st>>>(a);
    FREDEC_CUDA_TRY(cudaGetLastError());
    // The host vectors are copied by stream-ordered copies from pageable
    // memory, which complete before cudaMemcpyAsync returns.
    return FREDEC_OK;
}

// Single series: chunk metadata is implicit, so nothing is uploaded from the
// host and the launch stays asynchronous (and capturable).
int launch_topk_single(const double *z, int64_t nf, int k, int64_t *idx_out, cudaStream_t st,
                       const SeriesState *state, double *info, const int32_t *err, unsigned char *host) {
    if (k <= 0) return FREDEC_OK;
    const int64_t nch = std::max<int64_t>(1, (nf + TK_CHUNK - 1) / TK_CHUNK);
    DevBuf cand;
    if (int rc = cand.alloc(nch * k * 16, st)) return rc;
    TopkArgs a{z, nullptr, nullptr, nullptr, nullptr, nullptr, k, cand.as<uint64_t>(),
               reinterpret_cast<int64_t *>(cand.as<uint64_t>() + nch * k), idx_out, nf, nch,
               (info || host) ? state : nullptr, state ? info : nullptr, err, state ? host : nullptr};
    FREDEC_CUDA_TRY(launch_pdl(topk_stage1, dim3((unsigned)nch), dim3(TK_THREADS), 0, st, a));
    FREDEC_CUDA_TRY(launch_pdl(topk_stage2, dim3(1), dim3(TK_THREADS), 0, st, a));
    FREDEC_CUDA_TRY(cudaGetLastError());
    return FREDEC_OK;
}

}  // namespace fredec
