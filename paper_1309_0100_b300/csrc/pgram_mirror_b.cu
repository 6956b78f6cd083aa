// Mixed-precision periodogram kernels that also write z to a page-locked host
// mirror (pgram_impl.cuh, MIRROR), P = 7, 9, 11.  Kept out of the
// pgram_p*.cu units: see the note at pgram_block_cs.
#include "pgram_impl.cuh"

namespace fredec {

// -2: P not handled here.
int launch_pgram_mirror_b(int p, int F, const PgramParams &prm, int64_t nblocks, int warps, cudaStream_t st,
                     const TailParams *tail) {
    if (p == 7 && F == 4) return launch_pgram_t<FREDEC_MIXED, 7, 4, true>(prm, nblocks, warps, st, tail);
    if (p == 7 && F == 6) return launch_pgram_t<FREDEC_MIXED, 7, 6, true>(prm, nblocks, warps, st, tail);
    if (p == 7 && F == 10) return launch_pgram_t<FREDEC_MIXED, 7, 10, true>(prm, nblocks, warps, st, tail);
    if (p == 9 && F == 3) return launch_pgram_t<FREDEC_MIXED, 9, 3, true>(prm, nblocks, warps, st, tail);
    if (p == 9 && F == 5) return launch_pgram_t<FREDEC_MIXED, 9, 5, true>(prm, nblocks, warps, st, tail);
    if (p == 9 && F == 8) return launch_pgram_t<FREDEC_MIXED, 9, 8, true>(prm, nblocks, warps, st, tail);
    if (p == 11 && F == 4) return launch_pgram_t<FREDEC_MIXED, 11, 4, true>(prm, nblocks, warps, st, tail);
    if (p == 11 && F == 6) return launch_pgram_t<FREDEC_MIXED, 11, 6, true>(prm, nblocks, warps, st, tail);
    if (p == 11 && F == 8) return launch_pgram_t<FREDEC_MIXED, 11, 8, true>(prm, nblocks, warps, st, tail);
    for (int q : {7, 9, 11})
        if (p == q) return -1;
    return -2;
}

}  // namespace fredec
