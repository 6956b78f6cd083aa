// Re-evaluation of the bins that the mixed kernel flagged as ill-conditioned
// (a pivot of the 2x2 Schur complement below flag_tau times its column norm:
// near a base frequency, near f = 0, or where <c^2> or <s^2> is tiny).  There
// the FP32 sums lose too many digits to cancellation, so each flagged bin is
// recomputed with FP64-grade sums: one CTA per bin, its threads split the
// observations, every term takes its own float-float seed from the exact
// fixed-point phase and enters double-float running sums (about 1e-16 of the
// summed magnitudes, like FP64 sums, at a fraction of the FP64 pipe's cost on
// this GPU); the threads' sums are combined in float-float by a fixed-order
// block reduction, and the 2x2 solve is FP64.  Deterministic; the list order
// does not matter.  CTAs beyond the number of flagged bins exit at once.
#include <algorithm>

#include "pgram_impl.cuh"

namespace fredec {

namespace {

constexpr int FX_THREADS = 256;

struct FixupParams {
    const SeriesDesc *desc;
    const SeriesState *state;
    int nseries;                 // > 1: find the series of a global z index by binary search on z_off
    const unsigned char *rec64;  // float-float records (series offsets: desc.rec64_off)
    const int64_t *list;         // global z indices
    const int32_t *count;
    double *z, *coef;
    double *z_mirror;            // optional second destination of z
    int64_t nan_nf;              // > 0 (single series): if its prep failed, z[0..nan_nf) <- NaN instead
    double *dzdf;                // two-set records: dz/df of the re-evaluated bins
    int64_t cap;                 // entries of list, and the number of z values
    int32_t *err;                // optional: FREDEC_EINVAL when a listed index is out of range
};

// NSET = 2: the records carry the t'-weighted values as well; the kernel
// re-evaluates dz/df of the bin with the same float-float sums.
template <int P, int NSET>
__global__ void __launch_bounds__(FX_THREADS) fixup_kernel(FixupParams prm) {
    constexpr int Q0 = 2 * P + 4, Q = NSET * Q0 + (NSET == 2 ? 1 : 0);   // + <t'> with two sets
    __shared__ SeedTableFF tab;
    __shared__ ff red[FX_THREADS / 32][Q];
    __shared__ double S[Q];
    grid_dependency_wait();   // the periodogram kernel's flag list and z
    if (prm.nan_nf > 0 && prm.state[0].status != FREDEC_OK) {   // nothing was computed: z is NaN
        for (int64_t j = (int64_t)blockIdx.x * FX_THREADS + threadIdx.x; j < prm.nan_nf;
             j += (int64_t)gridDim.x * FX_THREADS)
            prm.z[j] = NAN;
        return;
    }
    const int32_t n = (int32_t)min((int64_t)*prm.count, prm.cap);
    if ((int32_t)blockIdx.x >= n) return;   // no flagged bin for this CTA
    fill_seed_table_ff(tab);
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int32_t it = blockIdx.x; it < n; it += gridDim.x) {
        const int64_t g = prm.list[it];
        int s = 0;
        if (prm.nseries > 1) {
            int lo = 0, hi = prm.nseries - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (prm.desc[mid].z_off <= g) lo = mid; else hi = mid - 1;
            }
            s = lo;
        }
        const SeriesDesc &d = prm.desc[s];
        const SeriesState &st = prm.state[s];
        if (d.p != P) continue;   // batches: another launch handles this base size
        const int64_t j = g - d.z_off;
        if (g < 0 || g >= prm.cap || j < 0 || j >= d.nf) {   // a listed index outside the outputs
            if (threadIdx.x == 0 && prm.err) atomicExch(prm.err, FREDEC_EINVAL);
            continue;
        }
        ff_acc fa[Q];
        const uint32_t *R0 = reinterpret_cast<const uint32_t *>(prm.rec64 + d.rec64_off);
        constexpr int RW = recff_words(P, NSET);
        for (int i = threadIdx.x; i < d.N; i += FX_THREADS) {
            const uint32_t *R = R0 + (int64_t)i * RW;
            const uint4 h = *reinterpret_cast<const uint4 *>(R);
            const uint64_t A = ((uint64_t)h.y << 32) | h.x, B = ((uint64_t)h.w << 32) | h.z;
            const float *Rf = reinterpret_cast<const float *>(R);
            ff sn, cs;
            ff_sincos_turns(tab, A + (uint64_t)j * B, &sn, &cs);
            const ff w = {Rf[4], Rf[5]}, wr = {Rf[6], Rf[7]};
            const ff wc = ff_mul(w, cs);
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const ff u = {Rf[8 + 2 * q], Rf[9 + 2 * q]};
                fa[q].add_prod(u, cs);
                fa[P + q].add_prod(u, sn);
            }
            fa[2 * P].add_prod(wr, cs);
            fa[2 * P + 1].add_prod(wr, sn);
            fa[2 * P + 2].add_prod(wc, cs);
            fa[2 * P + 3].add_prod(wc, sn);
            if constexpr (NSET == 2) {   // the t'-weighted set: w t', w r t', w psi_k t'
                const float *R2 = Rf + recff_words(P);
                const ff wt = {R2[0], R2[1]}, wrt = {R2[2], R2[3]};
                const ff wtc = ff_mul(wt, cs);
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const ff ut = {R2[4 + 2 * q], R2[5 + 2 * q]};
                    fa[Q0 + q].add_prod(ut, cs);
                    fa[Q0 + P + q].add_prod(ut, sn);
                }
                fa[Q0 + 2 * P].add_prod(wrt, cs);
                fa[Q0 + 2 * P + 1].add_prod(wrt, sn);
                fa[Q0 + 2 * P + 2].add_prod(wtc, cs);
                fa[Q0 + 2 * P + 3].add_prod(wtc, sn);
                fa[2 * Q0].add_prod(wt, {1.0f, 0.0f});   // <t'>
            }
        }
        // the threads' double-float sums combined in float-float (warp
        // butterflies, then over the warps in a fixed order), one conversion
        // to FP64 per sum
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            ff v = {fa[q].H, fa[q].L};
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                v = ff_add(v, {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
            if (lane == 0) red[wid][q] = v;
        }
        __syncthreads();
        if (threadIdx.x < Q) {
            ff v = red[0][threadIdx.x];
            for (int w = 1; w < FX_THREADS / 32; ++w) v = ff_add(v, red[w][threadIdx.x]);
            S[threadIdx.x] = ff_to_double(v);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double vcc = 0.0, vcs = 0.0, vss = 0.0;
            for (int q = 0; q < P; ++q) {
                vcc = fma(S[q], S[q], vcc);
                vcs = fma(S[q], S[P + q], vcs);
                vss = fma(S[P + q], S[P + q], vss);
            }
            const double CC = S[2 * P + 2];
            double a, b, ratio;
            prm.z[g] = solve2(CC, S[2 * P + 3], st.W - CC, vcc, vcs, vss, S[2 * P], S[2 * P + 1], &a, &b, &ratio);
            if constexpr (NSET == 2) prm.dzdf[g] = dz_df<P>(S, S + Q0, S[2 * Q0], a, b);
            if (prm.z_mirror) prm.z_mirror[g] = prm.z[g];
            if (prm.coef) {
                prm.coef[2 * g] = a;
                prm.coef[2 * g + 1] = b;
            }
        }
        __syncthreads();
    }
}

template <int P, int NSET>
void launch_fx(const FixupParams &prm, int grid, cudaStream_t st) {
    launch_pdl(fixup_kernel<P, NSET>, dim3(grid), dim3(FX_THREADS), 0, st, prm);
}

}  // namespace

namespace {

// z <- (N_H/2) ln(l_base / (l_base - 2 z)), the log form of Eq. zpowrel,
// N_H = N - 3 (n_base + 1) - 1 - npoly (the alternative model: the base and one
// trial frequency).  One grid row per series.
__global__ void log_form_kernel(const SeriesDesc *desc, const SeriesState *state, int nseries, double *z) {
    for (int s = blockIdx.y; s < nseries; s += gridDim.y) {
        const SeriesDesc d = desc[s];
        const double lb = state[s].chi2;
        const double NH = (double)((int64_t)d.N - 3 * ((int64_t)d.nb + 1) - 1 - d.npoly);
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < d.nf;
             j += (int64_t)gridDim.x * blockDim.x) {
            const double zd = z[d.z_off + j];
            const double ln = lb - 2.0 * zd;
            z[d.z_off + j] = isnan(zd) ? zd : (ln > 0.0 ? 0.5 * NH * log(lb / ln) : INFINITY);
        }
    }
}

}  // namespace

int launch_log_form(const SeriesDesc *desc, const SeriesState *state, int nseries, int64_t nf_max, double *z,
                    cudaStream_t st) {
    if (nseries <= 0 || nf_max <= 0) return FREDEC_OK;
    const unsigned gx = (unsigned)std::min<int64_t>(std::max<int64_t>(1, (nf_max + 255) / 256),
                                                    std::max(1, 2 * sm_count() / std::min(nseries, 2 * sm_count())));
    log_form_kernel<<<dim3(gx, (unsigned)std::min(nseries, 65535)), 256, 0, st>>>(desc, state, nseries, z);
    FREDEC_CUDA_TRY(cudaGetLastError());
    return FREDEC_OK;
}

int launch_fixup_bins(const SeriesDesc *desc, const SeriesState *state, int nseries, const void *rec64, int p,
                      const int64_t *list, const int32_t *count, int64_t max_items, double *z, double *coef,
                      cudaStream_t st, double *z_mirror, int64_t nan_nf, double *dzdf, int32_t *err) {
    FixupParams prm{desc, state, nseries, (const unsigned char *)rec64, list, count, z, coef, z_mirror,
                    nseries == 1 ? nan_nf : 0, dzdf, max_items, err};
    // one wave for up to 8 bins per SM (8 CTAs of 256 threads are resident per
    // SM): the flagged count is known only on the device, and CTAs beyond it
    // exit at once
    const int grid = (int)std::min<int64_t>(std::max<int64_t>(max_items, 1), 8LL * sm_count());
    switch (p) {
#define C(P) case P: if (dzdf) launch_fx<P, 2>(prm, grid, st); else launch_fx<P, 1>(prm, grid, st); break;
        C(1) C(3) C(5) C(7) C(9) C(11) C(13) C(15) C(17) C(19) C(21) C(23) C(25)
#undef C
        default: return fail(FREDEC_EINVAL, "unsupported base size");
    }
    FREDEC_CUDA_TRY(cudaGetLastError());
    return FREDEC_OK;
}

}  // namespace fredec
