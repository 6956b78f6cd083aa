"""One series' periodogram sharded over ranks by frequency band, and the one
exchange step of that split: the merge of the per-rank top-k peaks.

The paper runs independent fitters side by side (Sect. 5); a residual
periodogram over a long grid splits the same way into bands of the grid,
each rank computing z on its own band (no data exchanged while computing).
The peaks (Sect. 4, Phase 1: the highest local maxima of the periodogram)
need one exchange: a local maximum z_j > z_{j-1}, z_j >= z_{j+1} at a band
edge depends on the neighbouring band, so every rank computes its band with a
halo of one bin on each inner side, reports the k highest local maxima among
its own bins, and the k (z, index) pairs of every rank (16 k bytes) are
gathered and merged: sorted by decreasing z, ties to the lower index, the
first k.  On the same z values the result is the single-rank top-k of the
whole grid (same local-maximum rule: an end point of the whole grid counts
when it exceeds its one neighbour).  A rank's z of a bin can differ from the
single-rank z by the path's rounding (the rotation recurrence restarts at
the band's own frequency blocks), so peaks whose z differ by less than the
path's tolerance may swap, as between two launch shapes.

This module is host logic over the library's calls: the periodogram and the
top-k run in the library's kernels on each rank's GPU; the merge handles k
pairs per rank.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = ["band", "halo", "own_from_halo", "merge_topk", "gather_merge", "sharded_topk"]


def band(rank: int, world: int, nf: int, align: int = 1) -> Tuple[int, int]:
    """[start, end) of rank's band of an nf-point grid: contiguous, covering
    the grid, boundaries at multiples of ``align`` bins (the last band takes
    the rest)."""
    if world < 1 or not 0 <= rank < world or nf < 0 or align < 1:
        raise ValueError("bad band arguments")
    units = -(-nf // align)
    lo = units * rank // world * align
    hi = nf if rank == world - 1 else units * (rank + 1) // world * align
    return min(lo, nf), min(hi, nf)


def halo(start: int, end: int, nf: int) -> Tuple[int, int]:
    """The bins a rank computes: its band plus one neighbour on each side
    that lies inside the grid."""
    return max(start - 1, 0), min(end + 1, nf)


def own_from_halo(idx_halo, z_at, h0: int, start: int, end: int, k: int) -> Tuple[np.ndarray, np.ndarray]:
    """A rank's own peaks from the top-(k+2) local maxima of its halo array
    (indices into the array of z on [h0, h1), -1 padded; z_at their values):
    the halo bins themselves, which the array's end-point rule may report,
    are dropped (at most two), leaving the k highest local maxima among the
    bins [start, end) -- every one of them has both of its grid neighbours in
    the array, so the rule applied there is the whole grid's.  Returns
    (z, global index), padded with (-inf, -1)."""
    out_v = np.full(k, -np.inf)
    out_i = np.full(k, -1, dtype=np.int64)
    r = 0
    for q, zq in zip(np.asarray(idx_halo, dtype=np.int64), np.asarray(z_at, dtype=np.float64)):
        g = h0 + int(q)
        if q < 0 or not start <= g < end:
            continue
        if r < k:
            out_v[r], out_i[r] = zq, g
            r += 1
    return out_v, out_i


def merge_topk(vals: Sequence[np.ndarray], idx: Sequence[np.ndarray], k: int) -> Tuple[np.ndarray, np.ndarray]:
    """Merge per-rank top-k lists (each padded with index -1) into the global
    top-k: decreasing z, ties to the lower index, padded with (-inf, -1)."""
    pairs = [(float(v), int(i)) for vs, ix in zip(vals, idx) for v, i in zip(vs, ix) if int(i) >= 0]
    pairs.sort(key=lambda p: (-p[0], p[1]))
    out_v = np.full(k, -np.inf)
    out_i = np.full(k, -1, dtype=np.int64)
    for r, (v, i) in enumerate(pairs[:k]):
        out_v[r] = v
        out_i[r] = i
    return out_v, out_i


def gather_merge(v: np.ndarray, i: np.ndarray, k: int, group=None) -> Tuple[np.ndarray, np.ndarray]:
    """The exchange step: all-gather every rank's k (z, index) pairs over the
    default process group (or ``group``) and merge them on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    mine = torch.stack([torch.as_tensor(v, dtype=torch.float64), torch.as_tensor(i, dtype=torch.float64)]).to(dev)
    bufs: List = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(bufs, mine, group=group)
    vals = [b[0].cpu().numpy() for b in bufs]
    idx = [b[1].cpu().numpy().astype(np.int64) for b in bufs]
    return merge_topk(vals, idx, k)


def sharded_topk(t, y, sigma, base_freqs, f0: float, df: float, nf: int, k: int, *, precision="mixed",
                 group=None, align: Optional[int] = None):
    """Rank's share of one series' residual periodogram and the global top-k
    peaks (the library's periodogram on this rank's band plus halo, then the
    exchange).  t, y, sigma, base_freqs: CUDA float64 tensors on this rank's
    device.  Returns (band start, band end, z of the band (CUDA tensor),
    global top-k indices, their z)."""
    import torch.distributed as dist
    import paper_1309_0100_b300 as F
    if not 1 <= k <= 62:
        raise ValueError("k must be in 1..62 (the device top-k takes k + 2 <= 64)")
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    start, end = band(rank, world, nf, align or 1)
    h0, h1 = halo(start, end, nf)
    out = F.periodogram_dev(t, y, sigma, base_freqs, f0 + h0 * df, df, h1 - h0, precision=precision)
    kk = min(k + 2, 64)
    top = F.topk_dev(out["z"], kk)
    zt = out["z"][top.clamp(min=0)]
    v, i = own_from_halo(top.cpu().numpy(), zt.cpu().numpy(), h0, start, end, k)
    gv, gi = gather_merge(v, i, k, group)
    return start, end, out["z"][start - h0:end - h0], gi, gv
