// Instantiations of the two-set periodogram kernels (z and dz/df per trial
// frequency) for base sizes 13, 15, 17, 19, 21, 23, 25; dispatched by grad.cu.
#include "pgram_impl.cuh"

namespace fredec {

int launch_pgram_grad_b(int prec, int p, const PgramParams &prm, int64_t nblocks, int warps, cudaStream_t st,
                        const TailParams *tail) {
    switch (p) {
        case 13:
            return prec == FREDEC_MIXED ? launch_pgram_t<FREDEC_MIXED, 13, grad_fpt_mixed(13), false, 2>(prm, nblocks, warps, st, tail)
                                        : launch_pgram_t<FREDEC_FP64, 13, GRAD_FPT_FP64, false, 2>(prm, nblocks, warps, st, tail);
        case 15:
            return prec == FREDEC_MIXED ? launch_pgram_t<FREDEC_MIXED, 15, grad_fpt_mixed(15), false, 2>(prm, nblocks, warps, st, tail)
                                        : launch_pgram_t<FREDEC_FP64, 15, GRAD_FPT_FP64, false, 2>(prm, nblocks, warps, st, tail);
        case 17:
            return prec == FREDEC_MIXED ? launch_pgram_t<FREDEC_MIXED, 17, grad_fpt_mixed(17), false, 2>(prm, nblocks, warps, st, tail)
                                        : launch_pgram_t<FREDEC_FP64, 17, GRAD_FPT_FP64, false, 2>(prm, nblocks, warps, st, tail);
        case 19:
            return prec == FREDEC_MIXED ? launch_pgram_t<FREDEC_MIXED, 19, grad_fpt_mixed(19), false, 2>(prm, nblocks, warps, st, tail)
                                        : launch_pgram_t<FREDEC_FP64, 19, GRAD_FPT_FP64, false, 2>(prm, nblocks, warps, st, tail);
        case 21:
            return prec == FREDEC_MIXED ? launch_pgram_t<FREDEC_MIXED, 21, grad_fpt_mixed(21), false, 2>(prm, nblocks, warps, st, tail)
                                        : launch_pgram_t<FREDEC_FP64, 21, GRAD_FPT_FP64, false, 2>(prm, nblocks, warps, st, tail);
        case 23:
            return prec == FREDEC_MIXED ? launch_pgram_t<FREDEC_MIXED, 23, grad_fpt_mixed(23), false, 2>(prm, nblocks, warps, st, tail)
                                        : launch_pgram_t<FREDEC_FP64, 23, GRAD_FPT_FP64, false, 2>(prm, nblocks, warps, st, tail);
        case 25:
            return prec == FREDEC_MIXED ? launch_pgram_t<FREDEC_MIXED, 25, grad_fpt_mixed(25), false, 2>(prm, nblocks, warps, st, tail)
                                        : launch_pgram_t<FREDEC_FP64, 25, GRAD_FPT_FP64, false, 2>(prm, nblocks, warps, st, tail);
    }
    return -2;
}

size_t smem_pgram_grad_b(int prec, int p, int warps) {
    switch (p) {
        case 13:
            return prec == FREDEC_MIXED ? pgram_smem_t<FREDEC_MIXED, 13, grad_fpt_mixed(13), 2>(warps)
                                        : pgram_smem_t<FREDEC_FP64, 13, GRAD_FPT_FP64, 2>(warps);
        case 15:
            return prec == FREDEC_MIXED ? pgram_smem_t<FREDEC_MIXED, 15, grad_fpt_mixed(15), 2>(warps)
                                        : pgram_smem_t<FREDEC_FP64, 15, GRAD_FPT_FP64, 2>(warps);
        case 17:
            return prec == FREDEC_MIXED ? pgram_smem_t<FREDEC_MIXED, 17, grad_fpt_mixed(17), 2>(warps)
                                        : pgram_smem_t<FREDEC_FP64, 17, GRAD_FPT_FP64, 2>(warps);
        case 19:
            return prec == FREDEC_MIXED ? pgram_smem_t<FREDEC_MIXED, 19, grad_fpt_mixed(19), 2>(warps)
                                        : pgram_smem_t<FREDEC_FP64, 19, GRAD_FPT_FP64, 2>(warps);
        case 21:
            return prec == FREDEC_MIXED ? pgram_smem_t<FREDEC_MIXED, 21, grad_fpt_mixed(21), 2>(warps)
                                        : pgram_smem_t<FREDEC_FP64, 21, GRAD_FPT_FP64, 2>(warps);
        case 23:
            return prec == FREDEC_MIXED ? pgram_smem_t<FREDEC_MIXED, 23, grad_fpt_mixed(23), 2>(warps)
                                        : pgram_smem_t<FREDEC_FP64, 23, GRAD_FPT_FP64, 2>(warps);
        case 25:
            return prec == FREDEC_MIXED ? pgram_smem_t<FREDEC_MIXED, 25, grad_fpt_mixed(25), 2>(warps)
                                        : pgram_smem_t<FREDEC_FP64, 25, GRAD_FPT_FP64, 2>(warps);
    }
    return 0;
}

}  // namespace fredec
