// Top-k local maxima of z (device), one or many series.
//
// A local maximum is z_j > z_{j-1} and z_j >= z_{j+1}; an end point counts when
// it exceeds its one neighbour (a single-point grid counts).  Maxima are ranked
// by decreasing z, ties to the lower index; missing ranks are -1.  Stage 1:
// every CTA takes a 4096-point chunk (thread t holds points t, t + 256, ...,
// so the loads are coalesced); each warp finds its k best maxima by k rounds of
// a shuffle-only warp argmax, and one warp merges the CTA's 8k candidates the
// same way.  Stage 2: one CTA per series merges its chunks' candidates: each
// warp selects the k best of a fixed slice, one warp merges them.  Every step
// is a fixed-order selection over a strict total order, so the result does not
// depend on scheduling.
#include <algorithm>
#include <cstring>
#include <vector>

#include "fredec_internal.cuh"

namespace fredec {

namespace {

constexpr int TK_THREADS = 256;
constexpr int TK_WARPS = TK_THREADS / 32;
constexpr int TK_PER = 16;                       // points per thread (<= 32: a bit mask of live maxima)
constexpr int TK_CHUNK = TK_THREADS * TK_PER;

// (z1, j1) ranks before (z2, j2); j < 0 is an empty slot, after everything.
__device__ __forceinline__ bool better(double z1, int64_t j1, double z2, int64_t j2) {
    if (j2 < 0) return j1 >= 0;
    if (j1 < 0) return false;
    return z1 > z2 || (z1 == z2 && j1 < j2);
}

// Warp argmax of (z, j); every lane receives it.
__device__ __forceinline__ void warp_best(double &z, int64_t &j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double oz = __shfl_xor_sync(0xffffffffu, z, o);
        const int64_t oj = __shfl_xor_sync(0xffffffffu, j, o);
        if (better(oz, oj, z, j)) {
            z = oz;
            j = oj;
        }
    }
}

// One warp: the k best of the n candidates (cz, cj) (shared or global memory;
// the taken ones are marked j = -1), written to oj[0..k) and, unless it is
// null, oz[0..k).
__device__ void warp_select(const double *cz, int64_t *cj, int64_t n, int k, double *oz, int64_t *oj) {
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < k; ++r) {
        double bz = -INFINITY;
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
            if (oz) oz[r] = bz;
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
    double *cand_z;            // [nchunks * k]
    int64_t *cand_j;
    int64_t *out;              // [S * k]
    int64_t nf_single;         // single-series mode (chunk_series == nullptr)
    int64_t nchunks_single;
};

__global__ void __launch_bounds__(TK_THREADS) topk_stage1(TopkArgs a) {
    __shared__ double wz[TK_WARPS * FREDEC_MAX_TOPK];
    __shared__ int64_t wj[TK_WARPS * FREDEC_MAX_TOPK];
    const int64_t c = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool single = a.chunk_series == nullptr;
    const int s = single ? 0 : a.chunk_series[c];
    const double *z = a.z + (single ? 0 : a.z_off[s]);
    const int64_t n = single ? a.nf_single : a.nf[s];
    const int64_t cb = single ? c * TK_CHUNK : a.chunk_begin[c];
    double vz[TK_PER];
    uint32_t live = 0;   // bit e: point cb + e*TK_THREADS + tid is a local maximum not yet taken
#pragma unroll
    for (int e = 0; e < TK_PER; ++e) {
        const int64_t j = cb + (int64_t)e * TK_THREADS + tid;
        vz[e] = 0.0;
        if (j < n) {
            const double zj = z[j];
            bool m;
            if (n == 1) m = true;
            else if (j == 0) m = zj > z[1];
            else if (j == n - 1) m = zj > z[n - 2];
            else m = zj > z[j - 1] && zj >= z[j + 1];
            if (m && zj == zj) {
                vz[e] = zj;
                live |= 1u << e;
            }
        }
    }
    for (int r = 0; r < a.k; ++r) {
        double bz = -INFINITY;
        int64_t bj = -1;
        int be = -1;
#pragma unroll
        for (int e = 0; e < TK_PER; ++e) {
            const int64_t j = cb + (int64_t)e * TK_THREADS + tid;
            if ((live >> e & 1u) && better(vz[e], j, bz, bj)) {
                bz = vz[e];
                bj = j;
                be = e;
            }
        }
        const int64_t mine = bj;
        warp_best(bz, bj);
        if (bj >= 0 && mine == bj) live &= ~(1u << be);
        if (lane == 0) {
            wz[warp * a.k + r] = bz;
            wj[warp * a.k + r] = bj;
        }
    }
    __syncthreads();
    if (warp == 0) warp_select(wz, wj, (int64_t)TK_WARPS * a.k, a.k, a.cand_z + c * a.k, a.cand_j + c * a.k);
}

__global__ void __launch_bounds__(TK_THREADS) topk_stage2(TopkArgs a) {
    __shared__ double wz[TK_WARPS * FREDEC_MAX_TOPK];
    __shared__ int64_t wj[TK_WARPS * FREDEC_MAX_TOPK];
    const int s = blockIdx.x;
    const int warp = threadIdx.x >> 5;
    const bool single = a.chunk_series == nullptr;
    const int64_t c0 = single ? 0 : a.chunk_off[s], c1 = single ? a.nchunks_single : a.chunk_off[s + 1];
    const int64_t ncand = (c1 - c0) * a.k;
    // warp w: candidates [w ncand / 8, (w + 1) ncand / 8)
    const int64_t q0 = ncand * warp / TK_WARPS, q1 = ncand * (warp + 1) / TK_WARPS;
    warp_select(a.cand_z + c0 * a.k + q0, a.cand_j + c0 * a.k + q0, q1 - q0, a.k, wz + warp * a.k,
                wj + warp * a.k);
    __syncthreads();
    if (warp == 0) warp_select(wz, wj, (int64_t)TK_WARPS * a.k, a.k, nullptr, a.out + (int64_t)s * a.k);
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
    double *d_cz = (double *)p; p += nch * k * 8;
    int64_t *d_cj = (int64_t *)p; p += nch * k * 8;
    int32_t *d_cs = (int32_t *)p;
    FREDEC_CUDA_TRY(cudaMemcpy(d_cb, cb.data(), nch * 8, cudaMemcpyHostToDevice));
    FREDEC_CUDA_TRY(cudaMemcpy(d_coff, coff.data(), (S + 1) * 8, cudaMemcpyHostToDevice));
    FREDEC_CUDA_TRY(cudaMemcpy(d_zoff, z_off_h, S * 8, cudaMemcpyHostToDevice));
    FREDEC_CUDA_TRY(cudaMemcpy(d_nf, nf_h, S * 8, cudaMemcpyHostToDevice));
    FREDEC_CUDA_TRY(cudaMemcpy(d_cs, cs.data(), nch * 4, cudaMemcpyHostToDevice));
    TopkArgs a{z, d_zoff, d_nf, d_cs, d_cb, d_coff, k, d_cz, d_cj, idx_out, 0, 0};
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
    double *d_cz = (double *)p; p += nch * k * 8;
    int64_t *d_cj = (int64_t *)p; p += nch * k * 8;
    int32_t *d_cs = (int32_t *)p;
    FREDEC_CUDA_TRY(cudaMemcpyAsync(d_cb, cb.data(), nch * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(d_coff, coff.data(), (S + 1) * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(d_zoff, z_off_h, S * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(d_nf, nf_h, S * 8, cudaMemcpyHostToDevice, st));
    FREDEC_CUDA_TRY(cudaMemcpyAsync(d_cs, cs.data(), nch * 4, cudaMemcpyHostToDevice, st));
    TopkArgs a{z, d_zoff, d_nf, d_cs, d_cb, d_coff, k, d_cz, d_cj, idx_out, 0, 0};
    topk_stage1<<<(unsigned)nch, TK_THREADS, 0, st>>>(a);
    topk_stage2<<<(unsigned)S, TK_THREADS, 0, st>>>(a);
    FREDEC_CUDA_TRY(cudaGetLastError());
    // The host vectors are copied by stream-ordered copies from pageable
    // memory, which complete before cudaMemcpyAsync returns.
    return FREDEC_OK;
}

// Single series: chunk metadata is implicit, so nothing is uploaded from the
// host and the launch stays asynchronous (and capturable).
int launch_topk_single(const double *z, int64_t nf, int k, int64_t *idx_out, cudaStream_t st) {
    if (k <= 0) return FREDEC_OK;
    const int64_t nch = std::max<int64_t>(1, (nf + TK_CHUNK - 1) / TK_CHUNK);
    DevBuf cand;
    if (int rc = cand.alloc(nch * k * 16, st)) return rc;
    TopkArgs a{z, nullptr, nullptr, nullptr, nullptr, nullptr, k, cand.as<double>(),
               reinterpret_cast<int64_t *>(cand.as<double>() + nch * k), idx_out, nf, nch};
    topk_stage1<<<(unsigned)nch, TK_THREADS, 0, st>>>(a);
    topk_stage2<<<1, TK_THREADS, 0, st>>>(a);
    FREDEC_CUDA_TRY(cudaGetLastError());
    return FREDEC_OK;
}

}  // namespace fredec
