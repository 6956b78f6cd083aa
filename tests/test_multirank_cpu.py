"""The multi-GPU path of bench.py on CPU: two gloo ranks get disjoint
workloads (own series, own frequency band; weak scaling with no data-path
collective) and agree on the max-over-ranks time."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    s = bench.make_rank_workload(rank)
    band = (s.grid.f0, s.grid.f0 + (s.grid.nf - 1) * s.grid.df)
    local = 10.0 + rank
    m = bench.reduce_max(local, ws)
    bands = [None] * ws
    dist.all_gather_object(bands, band)
    seeds = [None] * ws
    dist.all_gather_object(seeds, float(s.y[0]))
    dist.destroy_process_group()
    q.put((rank, m, bands, seeds))


def test_two_gloo_ranks():
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
    for rank, m, bands, seeds in res:
        assert m == 11.0                       # max over ranks
        (a0, a1), (b0, b1) = bands
        assert a1 < b0                          # disjoint frequency bands
        assert seeds[0] != seeds[1]             # different series per rank
