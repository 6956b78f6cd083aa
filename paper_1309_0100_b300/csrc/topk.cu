// Top-k local maxima of z (device), one or many series.
//
// A local maximum is z_j > z_{j-1} and z_j >= z_{j+1}; an end point counts when
// it exceeds its one neighbour (a single-point grid counts).  Maxima are ranked
// by decreasing z, ties to the lower index; missing ranks are -1.  Stage 1:
// every CTA selects the k best maxima of a 4096-point chunk (k rounds of a
// deterministic block argmax); stage 2: one CTA per series merges its chunks'
// candidates the same way.  The result does not depend on scheduling.
#include <algorithm>
#include <cstring>
#include <vector>

#include "fredec_internal.cuh"

namespace fredec {

namespace {

constexpr int TK_THREADS = 256;
constexpr int TK_PER = 16;
constexpr int TK_CHUNK = TK_THREADS * TK_PER;

__device__ __forceinline__ bool better(double z1, int64_t j1, double z2, int64_t j2) {
    if (j2 < 0) return j1 >= 0;
    if (j1 < 0) return false;
    return z1 > z2 || (z1 == z2 && j1 < j2);
}

// Block-wide best (z, j); every thread receives it.
__device__ void block_best(double &z, int64_t &j) {
    __shared__ double sz[32];
    __shared__ int64_t sj[32];
    for (int o = 16; o > 0; o >>= 1) {
        const double oz = __shfl_xor_sync(0xffffffffu, z, o);
        const int64_t oj = __shfl_xor_sync(0xffffffffu, j, o);
        if (better(oz, oj, z, j)) { z = oz; j = oj; }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) { sz[wid] = z; sj[wid] = j; }
    __syncthreads();
    z = sz[0];
    j = sj[0];
    for (int w = 1; w < nw; ++w)
        if (better(sz[w], sj[w], z, j)) { z = sz[w]; j = sj[w]; }
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
    const int64_t c = blockIdx.x;
    const bool single = a.chunk_series == nullptr;
    const int s = single ? 0 : a.chunk_series[c];
    const double *z = a.z + (single ? 0 : a.z_off[s]);
    const int64_t n = single ? a.nf_single : a.nf[s];
    const int64_t j0 = (single ? c * TK_CHUNK : a.chunk_begin[c]) + (int64_t)threadIdx.x * TK_PER;
    double vz[TK_PER];
    int64_t vj[TK_PER];
#pragma unroll
    for (int e = 0; e < TK_PER; ++e) {
        const int64_t j = j0 + e;
        vz[e] = -INFINITY;
        vj[e] = -1;
        if (j < n) {
            const double zj = z[j];
            bool m;
            if (n == 1) m = true;
            else if (j == 0) m = zj > z[1];
            else if (j == n - 1) m = zj > z[n - 2];
            else m = zj > z[j - 1] && zj >= z[j + 1];
            if (m && zj == zj) { vz[e] = zj; vj[e] = j; }
        }
    }
    for (int r = 0; r < a.k; ++r) {
        double bz = -INFINITY;
        int64_t bj = -1;
#pragma unroll
        for (int e = 0; e < TK_PER; ++e)
            if (better(vz[e], vj[e], bz, bj)) { bz = vz[e]; bj = vj[e]; }
        block_best(bz, bj);
#pragma unroll
        for (int e = 0; e < TK_PER; ++e)
            if (vj[e] == bj && bj >= 0) vj[e] = -1;
        if (threadIdx.x == 0) {
            a.cand_z[c * a.k + r] = bz;
            a.cand_j[c * a.k + r] = bj;
        }
    }
}

__global__ void __launch_bounds__(TK_THREADS) topk_stage2(TopkArgs a) {
    const int s = blockIdx.x;
    const bool single = a.chunk_series == nullptr;
    const int64_t c0 = single ? 0 : a.chunk_off[s], c1 = single ? a.nchunks_single : a.chunk_off[s + 1];
    const int64_t ncand = (c1 - c0) * a.k;
    for (int r = 0; r < a.k; ++r) {
        double bz = -INFINITY;
        int64_t bj = -1;
        for (int64_t q = threadIdx.x; q < ncand; q += blockDim.x) {
            const double cz = a.cand_z[c0 * a.k + q];
            const int64_t cj = a.cand_j[c0 * a.k + q];
            if (better(cz, cj, bz, bj)) { bz = cz; bj = cj; }
        }
        block_best(bz, bj);
        for (int64_t q = threadIdx.x; q < ncand; q += blockDim.x)
            if (a.cand_j[c0 * a.k + q] == bj && bj >= 0) a.cand_j[c0 * a.k + q] = -1;
        if (threadIdx.x == 0) a.out[(int64_t)s * a.k + r] = bj;
        __syncthreads();
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
