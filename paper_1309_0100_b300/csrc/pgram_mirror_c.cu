// Mixed-precision periodogram kernels that also write z to a page-locked host
// mirror (pgram_impl.cuh, MIRROR), P = 13, 15, 17, 19, 21, 23, 25.  Kept out of the
// pgram_p*.cu units: see the note at pgram_block_cs.
#include "pgram_impl.cuh"

namespace fredec {

// -2: P not handled here.
int launch_pgram_mirror_c(int p, int F, const PgramParams &prm, int64_t nblocks, int warps, cudaStream_t st,
                     const TailParams *tail) {
    if (p == 13 && F == 4) return launch_pgram_t<FREDEC_MIXED, 13, 4, true>(prm, nblocks, warps, st, tail);
    if (p == 13 && F == 6) return launch_pgram_t<FREDEC_MIXED, 13, 6, true>(prm, nblocks, warps, st, tail);
    if (p == 15 && F == 2) return launch_pgram_t<FREDEC_MIXED, 15, 2, true>(prm, nblocks, warps, st, tail);
    if (p == 15 && F == 3) return launch_pgram_t<FREDEC_MIXED, 15, 3, true>(prm, nblocks, warps, st, tail);
    if (p == 17 && F == 2) return launch_pgram_t<FREDEC_MIXED, 17, 2, true>(prm, nblocks, warps, st, tail);
    if (p == 17 && F == 3) return launch_pgram_t<FREDEC_MIXED, 17, 3, true>(prm, nblocks, warps, st, tail);
    if (p == 19 && F == 2) return launch_pgram_t<FREDEC_MIXED, 19, 2, true>(prm, nblocks, warps, st, tail);
    if (p == 21 && F == 2) return launch_pgram_t<FREDEC_MIXED, 21, 2, true>(prm, nblocks, warps, st, tail);
    if (p == 23 && F == 2) return launch_pgram_t<FREDEC_MIXED, 23, 2, true>(prm, nblocks, warps, st, tail);
    if (p == 25 && F == 2) return launch_pgram_t<FREDEC_MIXED, 25, 2, true>(prm, nblocks, warps, st, tail);
    for (int q : {13, 15, 17, 19, 21, 23, 25})
        if (p == q) return -1;
    return -2;
}

}  // namespace fredec
