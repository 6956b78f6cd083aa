// Instantiations of the periodogram kernels for P = 5 base columns.
#include "pgram_impl.cuh"

namespace fredec {

int launch_pgram_p5(int prec, int F, const PgramParams &prm, int64_t nblocks, int warps, int list_mode,
                     int grid_override, cudaStream_t st) {
    if (prec == FREDEC_MIXED && F == 6) return launch_pgram_t<FREDEC_MIXED, 5, 6>(prm, nblocks, warps, list_mode, grid_override, st);
    if (prec == FREDEC_MIXED && F == 10) return launch_pgram_t<FREDEC_MIXED, 5, 10>(prm, nblocks, warps, list_mode, grid_override, st);
    if (prec == FREDEC_FP64 && F == 2) return launch_pgram_t<FREDEC_FP64, 5, 2>(prm, nblocks, warps, list_mode, grid_override, st);
    if (prec == FREDEC_FP64 && F == 4) return launch_pgram_t<FREDEC_FP64, 5, 4>(prm, nblocks, warps, list_mode, grid_override, st);
    return -1;
}

size_t smem_pgram_p5(int prec, int F, int warps) {
    if (prec == FREDEC_MIXED && F == 6) return pgram_smem_t<FREDEC_MIXED, 5, 6>(warps);
    if (prec == FREDEC_MIXED && F == 10) return pgram_smem_t<FREDEC_MIXED, 5, 10>(warps);
    if (prec == FREDEC_FP64 && F == 2) return pgram_smem_t<FREDEC_FP64, 5, 2>(warps);
    if (prec == FREDEC_FP64 && F == 4) return pgram_smem_t<FREDEC_FP64, 5, 4>(warps);
    return 0;
}

}  // namespace fredec
