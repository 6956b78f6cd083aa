"""Calls from several host threads at once (the library's per-thread streams,
page-locked scratch and error strings; its shared caches are guarded):
every result equals the same call made alone, bit for bit."""
import threading

import numpy as np
import pytest

import synth
from helpers import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    ensure_built()
    import paper_1309_0100_b300 as F
    return F


def test_host_threads_concurrent_calls(F):
    series = [synth.small_series(300 + k, N=400 + 150 * k, n_base=k % 4, nf=5000 + 700 * k, span=300.0)
              for k in range(6)]
    precs = ["mixed", "fp64", "mixed", "mixed", "fp64", "mixed"]

    def call(s, prec):
        return F.periodogram(s.t, s.y, s.sigma, s.base_freqs, s.grid.array(), precision=prec, topk=3)

    alone = [call(s, p) for s, p in zip(series, precs)]
    out = [[None] * len(series) for _ in range(3)]
    errors = []

    def worker(rep):
        try:
            for k in range(len(series)):
                out[rep][k] = call(series[k], precs[k])
        except Exception as e:   # reported below, from the main thread
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(r,)) for r in range(3)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    for rep in range(3):
        for k in range(len(series)):
            z, top = out[rep][k]
            assert np.array_equal(z, alone[k][0]), (rep, k)
            assert list(top) == list(alone[k][1]), (rep, k)
    # a failing call on one thread leaves its own error message and no other
    with pytest.raises(F.FredecError):
        F.periodogram(series[0].t, series[0].y, -series[0].sigma, series[0].base_freqs, series[0].grid.array())
