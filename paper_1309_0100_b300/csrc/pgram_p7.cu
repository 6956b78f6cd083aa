// Instantiations of the periodogram kernels for P = 7 base columns.
#include "pgram_impl.cuh"

namespace fredec {

int launch_pgram_p7(int prec, int F, const PgramParams &prm, int64_t nblocks, int warps, cudaStream_t st,
                     const TailParams *tail) {
    if (prec == FREDEC_MIXED && F == 4) return launch_pgram_t<FREDEC_MIXED, 7, 4>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_MIXED && F == 6) return launch_pgram_t<FREDEC_MIXED, 7, 6>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_MIXED && F == 10) return launch_pgram_t<FREDEC_MIXED, 7, 10>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_FP64 && F == 1) return launch_pgram_t<FREDEC_FP64, 7, 1>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_FP64 && F == 2) return launch_pgram_t<FREDEC_FP64, 7, 2>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_FP64 && F == 4) return launch_pgram_t<FREDEC_FP64, 7, 4>(prm, nblocks, warps, st, tail);
    return -1;
}

size_t smem_pgram_p7(int prec, int F, int warps) {
    if (prec == FREDEC_MIXED && F == 4) return pgram_smem_t<FREDEC_MIXED, 7, 4>(warps);
    if (prec == FREDEC_MIXED && F == 6) return pgram_smem_t<FREDEC_MIXED, 7, 6>(warps);
    if (prec == FREDEC_MIXED && F == 10) return pgram_smem_t<FREDEC_MIXED, 7, 10>(warps);
    if (prec == FREDEC_FP64 && F == 1) return pgram_smem_t<FREDEC_FP64, 7, 1>(warps);
    if (prec == FREDEC_FP64 && F == 2) return pgram_smem_t<FREDEC_FP64, 7, 2>(warps);
    if (prec == FREDEC_FP64 && F == 4) return pgram_smem_t<FREDEC_FP64, 7, 4>(warps);
    return 0;
}

}  // namespace fredec
