// Instantiations of the periodogram kernels for P = 1 base columns.
#include "pgram_impl.cuh"

namespace fredec {

int launch_pgram_p1(int prec, int F, const PgramParams &prm, int64_t nblocks, int warps, cudaStream_t st,
                     const TailParams *tail) {
    if (prec == FREDEC_MIXED && F == 12) return launch_pgram_t<FREDEC_MIXED, 1, 12>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_MIXED && F == 20) return launch_pgram_t<FREDEC_MIXED, 1, 20>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_MIXED && F == 32) return launch_pgram_t<FREDEC_MIXED, 1, 32>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_FP64 && F == 2) return launch_pgram_t<FREDEC_FP64, 1, 2>(prm, nblocks, warps, st, tail);
    if (prec == FREDEC_FP64 && F == 4) return launch_pgram_t<FREDEC_FP64, 1, 4>(prm, nblocks, warps, st, tail);
    return -1;
}

size_t smem_pgram_p1(int prec, int F, int warps) {
    if (prec == FREDEC_MIXED && F == 12) return pgram_smem_t<FREDEC_MIXED, 1, 12>(warps);
    if (prec == FREDEC_MIXED && F == 20) return pgram_smem_t<FREDEC_MIXED, 1, 20>(warps);
    if (prec == FREDEC_MIXED && F == 32) return pgram_smem_t<FREDEC_MIXED, 1, 32>(warps);
    if (prec == FREDEC_FP64 && F == 2) return pgram_smem_t<FREDEC_FP64, 1, 2>(warps);
    if (prec == FREDEC_FP64 && F == 4) return pgram_smem_t<FREDEC_FP64, 1, 4>(warps);
    return 0;
}

}  // namespace fredec
