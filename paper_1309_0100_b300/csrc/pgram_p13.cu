// Instantiations of the periodogram kernels for P = 13 base columns.
#include "pgram_impl.cuh"

namespace fredec {

int launch_pgram_p13(int prec, int F, const PgramParams &prm, int64_t nblocks, int warps, cudaStream_t st,
                     const TailParams *tail) {
    if (prec == FREDEC_MIXED && F == 4) return launch_pgram_t<FREDEC_MIXED, 13, 4>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_MIXED && F == 6) return launch_pgram_t<FREDEC_MIXED, 13, 6>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_FP64 && F == 1) return launch_pgram_t<FREDEC_FP64, 13, 1>(prm, nblocks, warps, st, tail);
    return -1;
}

size_t smem_pgram_p13(int prec, int F, int warps) {
    if (prec == FREDEC_MIXED && F == 4) return pgram_smem_t<FREDEC_MIXED, 13, 4>(warps);
    if (prec == FREDEC_MIXED && F == 6) return pgram_smem_t<FREDEC_MIXED, 13, 6>(warps);
    if (prec == FREDEC_FP64 && F == 1) return pgram_smem_t<FREDEC_FP64, 13, 1>(warps);
    return 0;
}

}  // namespace fredec
