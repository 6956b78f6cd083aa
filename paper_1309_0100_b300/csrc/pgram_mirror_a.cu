// Mixed-precision periodogram kernels that also write z to a page-locked host
// mirror (pgram_impl.cuh, MIRROR), P = 1, 3, 5.  Kept out of the
// pgram_p*.cu units: see the note at pgram_block_cs.
#include "pgram_impl.cuh"

namespace fredec {

// -2: P not handled here.
int launch_pgram_mirror_a(int p, int F, const PgramParams &prm, int64_t nblocks, int warps, cudaStream_t st,
                     const TailParams *tail) {
    if (p == 1 && F == 12) return launch_pgram_t<FREDEC_MIXED, 1, 12, true>(prm, nblocks, warps, st, tail);
    if (p == 1 && F == 20) return launch_pgram_t<FREDEC_MIXED, 1, 20, true>(prm, nblocks, warps, st, tail);
    if (p == 1 && F == 32) return launch_pgram_t<FREDEC_MIXED, 1, 32, true>(prm, nblocks, warps, st, tail);
    if (p == 3 && F == 8) return launch_pgram_t<FREDEC_MIXED, 3, 8, true>(prm, nblocks, warps, st, tail);
    if (p == 3 && F == 12) return launch_pgram_t<FREDEC_MIXED, 3, 12, true>(prm, nblocks, warps, st, tail);
    if (p == 3 && F == 20) return launch_pgram_t<FREDEC_MIXED, 3, 20, true>(prm, nblocks, warps, st, tail);
    if (p == 5 && F == 4) return launch_pgram_t<FREDEC_MIXED, 5, 4, true>(prm, nblocks, warps, st, tail);
    if (p == 5 && F == 8) return launch_pgram_t<FREDEC_MIXED, 5, 8, true>(prm, nblocks, warps, st, tail);
    if (p == 5 && F == 14) return launch_pgram_t<FREDEC_MIXED, 5, 14, true>(prm, nblocks, warps, st, tail);
    for (int q : {1, 3, 5})
        if (p == q) return -1;
    return -2;
}

}  // namespace fredec
