// Instantiations of the two-set periodogram kernels (z and dz/df per trial
// frequency) for base sizes 1, 3, 5, 7, 9, 11; dispatched by grad.cu.
#include "pgram_impl.cuh"

namespace fredec {

int launch_pgram_grad_a(int prec, int p, const PgramParams &prm, int64_t nblocks, int warps, cudaStream_t st,
                        const TailParams *tail) {
    switch (p) {
        case 1:
            return prec == FREDEC_MIXED ? launch_pgram_t<FREDEC_MIXED, 1, grad_fpt_mixed(1), false, 2>(prm, nblocks, warps, st, tail)
                                        : launch_pgram_t<FREDEC_FP64, 1, GRAD_FPT_FP64, false, 2>(prm, nblocks, warps, st, tail);
        case 3:
            return prec == FREDEC_MIXED ? launch_pgram_t<FREDEC_MIXED, 3, grad_fpt_mixed(3), false, 2>(prm, nblocks, warps, st, tail)
                                        : launch_pgram_t<FREDEC_FP64, 3, GRAD_FPT_FP64, false, 2>(prm, nblocks, warps, st, tail);
        case 5:
            return prec == FREDEC_MIXED ? launch_pgram_t<FREDEC_MIXED, 5, grad_fpt_mixed(5), false, 2>(prm, nblocks, warps, st, tail)
                                        : launch_pgram_t<FREDEC_FP64, 5, GRAD_FPT_FP64, false, 2>(prm, nblocks, warps, st, tail);
        case 7:
            return prec == FREDEC_MIXED ? launch_pgram_t<FREDEC_MIXED, 7, grad_fpt_mixed(7), false, 2>(prm, nblocks, warps, st, tail)
                                        : launch_pgram_t<FREDEC_FP64, 7, GRAD_FPT_FP64, false, 2>(prm, nblocks, warps, st, tail);
        case 9:
            return prec == FREDEC_MIXED ? launch_pgram_t<FREDEC_MIXED, 9, grad_fpt_mixed(9), false, 2>(prm, nblocks, warps, st, tail)
                                        : launch_pgram_t<FREDEC_FP64, 9, GRAD_FPT_FP64, false, 2>(prm, nblocks, warps, st, tail);
        case 11:
            return prec == FREDEC_MIXED ? launch_pgram_t<FREDEC_MIXED, 11, grad_fpt_mixed(11), false, 2>(prm, nblocks, warps, st, tail)
                                        : launch_pgram_t<FREDEC_FP64, 11, GRAD_FPT_FP64, false, 2>(prm, nblocks, warps, st, tail);
    }
    return -2;
}

size_t smem_pgram_grad_a(int prec, int p, int warps) {
    switch (p) {
        case 1:
            return prec == FREDEC_MIXED ? pgram_smem_t<FREDEC_MIXED, 1, grad_fpt_mixed(1), 2>(warps)
                                        : pgram_smem_t<FREDEC_FP64, 1, GRAD_FPT_FP64, 2>(warps);
        case 3:
            return prec == FREDEC_MIXED ? pgram_smem_t<FREDEC_MIXED, 3, grad_fpt_mixed(3), 2>(warps)
                                        : pgram_smem_t<FREDEC_FP64, 3, GRAD_FPT_FP64, 2>(warps);
        case 5:
            return prec == FREDEC_MIXED ? pgram_smem_t<FREDEC_MIXED, 5, grad_fpt_mixed(5), 2>(warps)
                                        : pgram_smem_t<FREDEC_FP64, 5, GRAD_FPT_FP64, 2>(warps);
        case 7:
            return prec == FREDEC_MIXED ? pgram_smem_t<FREDEC_MIXED, 7, grad_fpt_mixed(7), 2>(warps)
                                        : pgram_smem_t<FREDEC_FP64, 7, GRAD_FPT_FP64, 2>(warps);
        case 9:
            return prec == FREDEC_MIXED ? pgram_smem_t<FREDEC_MIXED, 9, grad_fpt_mixed(9), 2>(warps)
                                        : pgram_smem_t<FREDEC_FP64, 9, GRAD_FPT_FP64, 2>(warps);
        case 11:
            return prec == FREDEC_MIXED ? pgram_smem_t<FREDEC_MIXED, 11, grad_fpt_mixed(11), 2>(warps)
                                        : pgram_smem_t<FREDEC_FP64, 11, GRAD_FPT_FP64, 2>(warps);
    }
    return 0;
}

}  // namespace fredec
