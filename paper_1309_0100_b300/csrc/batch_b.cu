// Batch kernels for base sizes up to p = 15.
#include "batch_impl.cuh"

namespace fredec {

int launch_batch_p15(int prec, const BatchParams &bp, int warps, int grid, bool comp, cudaStream_t st) {
    return prec == FREDEC_MIXED ? launch_batch_t<FREDEC_MIXED, 15>(bp, warps, grid, comp, st)
                                : launch_batch_t<FREDEC_FP64, 15>(bp, warps, grid, comp, st);
}

int batch_occupancy_p15(int prec, int warps, bool comp) {
    return prec == FREDEC_MIXED ? batch_blocks_per_sm<FREDEC_MIXED, 15>(warps, comp)
                                : batch_blocks_per_sm<FREDEC_FP64, 15>(warps, comp);
}

}  // namespace fredec
