// Instantiations of the periodogram kernels for P = 1 base columns.
#include "pgram_impl.cuh"

namespace fredec {

int launch_pgram_p1(int prec, int F, const PgramParams &prm, int64_t nblocks, int warps, int list_mode,
                     int grid_override, cudaStream_t st) {
    if (prec == FREDEC_MIXED && F == 8) return launch_pgram_t<FREDEC_MIXED, 1, 8>(prm, nblocks, warps, list_mode, grid_override, st);
    if (prec == FREDEC_MIXED && F == 16) return launch_pgram_t<FREDEC_MIXED, 1, 16>(prm, nblocks, warps, list_mode, grid_override, st);
    if (prec == FREDEC_MIXED && F == 24) return launch_pgram_t<FREDEC_MIXED, 1, 24>(prm, nblocks, warps, list_mode, grid_override, st);
    if (prec == FREDEC_FP64 && F == 2) return launch_pgram_t<FREDEC_FP64, 1, 2>(prm, nblocks, warps, list_mode, grid_override, st);
    if (prec == FREDEC_FP64 && F == 4) return launch_pgram_t<FREDEC_FP64, 1, 4>(prm, nblocks, warps, list_mode, grid_override, st);
    return -1;
}

size_t smem_pgram_p1(int prec, int F, int warps) {
    if (prec == FREDEC_MIXED && F == 8) return pgram_smem_t<FREDEC_MIXED, 1, 8>(warps);
    if (prec == FREDEC_MIXED && F == 16) return pgram_smem_t<FREDEC_MIXED, 1, 16>(warps);
    if (prec == FREDEC_MIXED && F == 24) return pgram_smem_t<FREDEC_MIXED, 1, 24>(warps);
    if (prec == FREDEC_FP64 && F == 2) return pgram_smem_t<FREDEC_FP64, 1, 2>(warps);
    if (prec == FREDEC_FP64 && F == 4) return pgram_smem_t<FREDEC_FP64, 1, 4>(warps);
    return 0;
}

}  // namespace fredec
