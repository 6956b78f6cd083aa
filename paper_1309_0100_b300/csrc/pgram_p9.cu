// Instantiations of the periodogram kernels for P = 9 base columns.
#include "pgram_impl.cuh"

namespace fredec {

int launch_pgram_p9(int prec, int F, const PgramParams &prm, int64_t nblocks, int warps, cudaStream_t st,
                     const TailParams *tail) {
    if (prec == FREDEC_MIXED && F == 3) return launch_pgram_t<FREDEC_MIXED, 9, 3>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_MIXED && F == 5) return launch_pgram_t<FREDEC_MIXED, 9, 5>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_MIXED && F == 8) return launch_pgram_t<FREDEC_MIXED, 9, 8>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_FP64 && F == 1) return launch_pgram_t<FREDEC_FP64, 9, 1>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_FP64 && F == 2) return launch_pgram_t<FREDEC_FP64, 9, 2>(prm, nblocks, warps, st, tail);
    return -1;
}

size_t smem_pgram_p9(int prec, int F, int warps) {
    if (prec == FREDEC_MIXED && F == 3) return pgram_smem_t<FREDEC_MIXED, 9, 3>(warps);
    if (prec == FREDEC_MIXED && F == 5) return pgram_smem_t<FREDEC_MIXED, 9, 5>(warps);
    if (prec == FREDEC_MIXED && F == 8) return pgram_smem_t<FREDEC_MIXED, 9, 8>(warps);
    if (prec == FREDEC_FP64 && F == 1) return pgram_smem_t<FREDEC_FP64, 9, 1>(warps);
    if (prec == FREDEC_FP64 && F == 2) return pgram_smem_t<FREDEC_FP64, 9, 2>(warps);
    return 0;
}

}  // namespace fredec
