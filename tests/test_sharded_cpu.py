"""The exchange step of one series' periodogram sharded by frequency band
(paper_1309_0100_b300.sharded), on the CPU: band bookkeeping, the per-rank
peak list from a halo array, and the merge of the per-rank top-k over two
gloo ranks, against the single-rank local-maximum top-k of the whole grid
(helpers.local_max_topk) on periodograms from the oracle and on adversarial
arrays (plateaus and ties across band edges, NaN, end points)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from helpers import local_max_topk
from paper_1309_0100_b300 import sharded

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_topk(z, start, end, k):
    """What a rank reports: the local maxima of its halo array (the device
    top-k's rule, here the reference rule on the host) turned into its own
    peaks by sharded.own_from_halo."""
    h0, h1 = sharded.halo(start, end, z.size)
    zh = z[h0:h1]
    idx = np.asarray(local_max_topk(zh, min(k + 2, 64)), dtype=np.int64)
    vals = np.where(idx >= 0, zh[np.maximum(idx, 0)], -np.inf)
    return sharded.own_from_halo(idx, vals, h0, start, end, k)


def _arrays():
    rng = np.random.default_rng(7)
    out = [rng.standard_normal(101), rng.standard_normal(2)]
    z = rng.standard_normal(64)
    z[31] = z[32] = 9.0                       # a plateau across the middle band edge
    out.append(z)
    z = rng.standard_normal(64)
    z[32] = 8.0                               # a peak right at the start of the second band
    z[0] = 10.0                               # and a maximum at the grid's first end point
    out.append(z)
    z = np.round(rng.standard_normal(200), 1) # many ties, both sides of every edge
    z[99] = np.nan
    out.append(z)
    z = np.full(50, 3.0)                      # flat: no interior maximum
    z[-1] = 4.0
    out.append(z)
    return out


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_bands_cover_the_grid(world):
    for nf in (0, 1, 7, 1000, 1001):
        for align in (1, 32, 192):
            b = [sharded.band(r, world, nf, align) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == nf
            for (a0, a1), (c0, c1) in zip(b, b[1:]):
                assert a1 == c0 and a0 <= a1 and (a1 % align == 0 or a1 == nf)


@pytest.mark.parametrize("world", [2, 3, 4])
def test_merge_of_band_peaks_equals_whole_grid(world):
    for z in _arrays():
        for k in (1, 3, 5):
            parts = [_rank_topk(z, *sharded.band(r, world, z.size), k) for r in range(world)]
            v, i = sharded.merge_topk([p[0] for p in parts], [p[1] for p in parts], k)
            assert list(i) == local_max_topk(z, k), (world, k)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist
    import oracle
    import synth
    from paper_1309_0100_b300 import sharded as sh
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    # a residual periodogram: each rank evaluates only its band (plus halo) with the oracle
    s = synth.small_series(55, N=300, n_base=2, nf=3001, span=400.0, fmax=1.0)
    f = s.grid.array()
    start, end = sh.band(rank, ws, f.size)
    h0, h1 = sh.halo(start, end, f.size)
    zb, _ = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f[h0:h1])
    zfull = np.full(f.size, np.nan)
    zfull[h0:h1] = zb
    v, i = _rank_topk(zfull, start, end, 5)
    gv, gi = sh.gather_merge(v, i, 5)
    # adversarial arrays through the same exchange
    adv = [sh.gather_merge(*_rank_topk(z, *sh.band(rank, ws, z.size), 4), 4)[1].tolist() for z in _arrays()]
    dist.destroy_process_group()
    q.put((rank, gi.tolist(), adv))


def test_two_gloo_ranks_exchange():
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s = synth.small_series(55, N=300, n_base=2, nf=3001, span=400.0, fmax=1.0)
    z, _ = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, s.grid.array())
    want = local_max_topk(z, 5)
    want_adv = [local_max_topk(a, 4) for a in _arrays()]
    for rank, gi, adv in res:
        assert gi == want, rank                  # every rank holds the global top-k
        assert adv == want_adv, rank
