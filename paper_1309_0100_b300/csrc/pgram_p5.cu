// Instantiations of the periodogram kernels for P = 5 base columns.
#include "pgram_impl.cuh"

namespace fredec {

int launch_pgram_p5(int prec, int F, const PgramParams &prm, int64_t nblocks, int warps, cudaStream_t st,
                     const TailParams *tail) {
    if (prec == FREDEC_MIXED && F == 4) return launch_pgram_t<FREDEC_MIXED, 5, 4>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_MIXED && F == 8) return launch_pgram_t<FREDEC_MIXED, 5, 8>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_MIXED && F == 14) return launch_pgram_t<FREDEC_MIXED, 5, 14>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_FP64 && F == 2) return launch_pgram_t<FREDEC_FP64, 5, 2>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_FP64 && F == 4) return launch_pgram_t<FREDEC_FP64, 5, 4>(prm, nblocks, warps, st, tail);
    return -1;
}

size_t smem_pgram_p5(int prec, int F, int warps) {
    if (prec == FREDEC_MIXED && F == 4) return pgram_smem_t<FREDEC_MIXED, 5, 4>(warps);
    if (prec == FREDEC_MIXED && F == 8) return pgram_smem_t<FREDEC_MIXED, 5, 8>(warps);
    if (prec == FREDEC_MIXED && F == 14) return pgram_smem_t<FREDEC_MIXED, 5, 14>(warps);
    if (prec == FREDEC_FP64 && F == 2) return pgram_smem_t<FREDEC_FP64, 5, 2>(warps);
    if (prec == FREDEC_FP64 && F == 4) return pgram_smem_t<FREDEC_FP64, 5, 4>(warps);
    return 0;
}

}  // namespace fredec
