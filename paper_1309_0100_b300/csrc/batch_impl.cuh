// Persistent periodogram kernel for a batch of series: CTAs take work items
// (series, block of 32*F frequencies) from a device counter until the list is
// exhausted; each item runs the same block routine as the single-series
// kernel, with F fixed per base size P (a switch over the sizes of the class).
#pragma once

#include "pgram_impl.cuh"

namespace fredec {

// Frequencies per thread used by the batch kernels for each base size (mixed:
// p = 1, 3, 5 the widest that the 168 registers of three resident CTAs hold
// without spills; measured on the 4096-series workload, p = 1, 3, 5:
// 12 / 8 / 4 309.8 ms a replay, 16 / 12 / 6 286.8 ms, 20 / 12 / 6 284.8 ms;
// 20 / 14 / 8 and 24 / 16 / 8 spill; p = 7 stays at 4, where 6 moved short
// series past the single-series results by more than the mixed bar; p >= 13
// take 2, in a kernel of 240 registers without spills: with F = 1 for p >= 17,
// one unpacked FMA per sum and a seed per frequency, 512 series of p = 13..25
// took 168.6 ms a replay, with F = 2 126.6 ms) or the FP64 default.
__host__ __device__ constexpr int batch_fpt(int prec, int p) {
    return prec == FREDEC_MIXED ? (p == 1 ? 20 : p == 3 ? 12 : p == 5 ? 6 : p <= 7 ? 4 : p <= 11 ? 3 : 2)
                                : (p <= 5 ? 2 : 1);
}

struct BatchParams {
    PgramParams prm;
    const int2 *items;      // (series, block)
    int64_t n_items;
    unsigned long long *counter;
};

template <int PREC, int P, bool COMP>
__device__ __forceinline__ void batch_item(const BatchParams &bp, const SeriesDesc &d, const SeriesState &st,
                                           int64_t blk, unsigned char *smem, uint32_t &use0, uint32_t &use1) {
    constexpr int F = batch_fpt(PREC, P);
    if (st.status != FREDEC_OK) {
        for (int fs = threadIdx.x; fs < 32 * F; fs += blockDim.x) {
            const int64_t j = blk * 32 * F + fs;
            if (j < d.nf) bp.prm.z[d.z_off + j] = NAN;
        }
        return;
    }
    if constexpr (PREC == FREDEC_MIXED)
        pgram_block_cs<P, F, false, 1, COMP>(bp.prm, d, st, blk, smem, use0, use1);
    else
        pgram_block<PREC, P, F>(bp.prm, d, st, blk, smem, use0, use1);
}

// Shared memory of one batch item's block routine.
template <int PREC, int P, bool COMP>
size_t batch_item_smem(int warps) {
    constexpr int F = batch_fpt(PREC, P);
    if constexpr (PREC == FREDEC_MIXED) return PgramCsLayout<P, F, 1, COMP>::smem_bytes(warps);
    else return PgramLayout<PREC, P, F>::smem_bytes(warps);
}

// Batch plans take the kernels with compensated residual totals (COMP) from
// BATCH_COMP_MIN_FLUSHES tiles per warp on, not from COMP_MIN_FLUSHES as single
// series do: their four extra rows of shared memory (10 KB at F = 20) take the
// p <= 5 class from six to five CTAs per SM.  The first 256 series of the
// 4096-series workload (N up to 5000, 79 tiles on two-warp CTAs) took 16.34 ms
// a launch with COMP against 15.96 ms without; at 79 flushes the plain FP32
// running sums stay near the error of the block sums (their rounding grows as
// the square root of the flushes: the bound broke at 780).
constexpr int BATCH_COMP_MIN_FLUSHES = 256;
inline bool batch_comp(int64_t max_n, int warps) {
    return (max_n + 32LL * warps - 1) / (32LL * warps) > BATCH_COMP_MIN_FLUSHES;
}

// Resident CTAs of 128 threads asked from the compiler: 3 for the small-base
// class (about 170 registers), 2 when large base sizes are compiled in.
template <int PMAXC>
constexpr int batch_minb() { return PMAXC <= 5 ? 3 : 2; }

// COMP: compensated residual totals (mixed; plans holding a series of more
// than COMP_MIN_FLUSHES tiles per warp).
template <int PREC, int PMAXC, bool COMP>
__global__ void __launch_bounds__(128, batch_minb<PMAXC>()) pgram_batch_kernel(BatchParams bp) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ long long cur;
    pgram_cta_init<PREC>(smem);
    uint32_t use0 = 0u, use1 = 0u;
    for (;;) {
        if (threadIdx.x == 0) cur = (long long)atomicAdd(bp.counter, 1ull);
        __syncthreads();
        const long long it = cur;
        if (it >= bp.n_items) break;
        const int2 w = bp.items[it];
        const SeriesDesc d = bp.prm.desc[w.x];
        const SeriesState &st = bp.prm.state[w.x];
        switch (d.p) {
            case 1: batch_item<PREC, 1, COMP>(bp, d, st, w.y, smem, use0, use1); break;
            case 3: batch_item<PREC, 3, COMP>(bp, d, st, w.y, smem, use0, use1); break;
            case 5: batch_item<PREC, 5, COMP>(bp, d, st, w.y, smem, use0, use1); break;
#define C(P) case P: if constexpr (PMAXC >= P) batch_item<PREC, P, COMP>(bp, d, st, w.y, smem, use0, use1); break;
            C(7) C(9) C(11) C(13) C(15) C(17) C(19) C(21) C(23) C(25)
#undef C
            default: break;
        }
        __syncthreads();   // all threads have read cur before it is replaced
    }
}

template <int PREC, int PMAXC, bool COMP>
size_t batch_smem(int warps) {
    size_t m = 0;
    auto upd = [&](size_t v) { m = v > m ? v : m; };
    upd(batch_item_smem<PREC, 1, COMP>(warps));
    upd(batch_item_smem<PREC, 3, COMP>(warps));
    upd(batch_item_smem<PREC, 5, COMP>(warps));
#define C(P) if (PMAXC >= P) upd(batch_item_smem<PREC, P, COMP>(warps));
    C(7) C(9) C(11) C(13) C(15) C(17) C(19) C(21) C(23) C(25)
#undef C
    return m;
}

template <int PREC, int PMAXC, bool COMP>
int launch_batch_k(const BatchParams &bp, int warps, int grid, cudaStream_t st) {
    const size_t smem = batch_smem<PREC, PMAXC, COMP>(warps);
    auto kern = pgram_batch_kernel<PREC, PMAXC, COMP>;
    FREDEC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, warps * 32, smem, st>>>(bp);
    FREDEC_CUDA_TRY(cudaGetLastError());
    return FREDEC_OK;
}

template <int PREC, int PMAXC, bool COMP>
int batch_blocks_per_sm_k(int warps) {
    int n = 0;
    const size_t smem = batch_smem<PREC, PMAXC, COMP>(warps);
    auto kern = pgram_batch_kernel<PREC, PMAXC, COMP>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, warps * 32, smem) != cudaSuccess || n < 1) n = 1;
    return n;
}

// The FP64 kernels have no compensated variant (their sums are FP64).
template <int PREC, int PMAXC>
int launch_batch_t(const BatchParams &bp, int warps, int grid, bool comp, cudaStream_t st) {
    if constexpr (PREC == FREDEC_MIXED)
        if (comp) return launch_batch_k<PREC, PMAXC, true>(bp, warps, grid, st);
    return launch_batch_k<PREC, PMAXC, false>(bp, warps, grid, st);
}

template <int PREC, int PMAXC>
int batch_blocks_per_sm(int warps, bool comp) {
    if constexpr (PREC == FREDEC_MIXED)
        if (comp) return batch_blocks_per_sm_k<PREC, PMAXC, true>(warps);
    return batch_blocks_per_sm_k<PREC, PMAXC, false>(warps);
}

}  // namespace fredec
