"""Batched periodograms (one plan, one persistent launch, CUDA graph replay)
must reproduce the single-series results for every series, with uneven
lengths, grid sizes and base sizes; replays are deterministic."""
import numpy as np
import pytest

import oracle
import synth
from helpers import cond_parity, ensure_built, local_max_topk, rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5}


@pytest.fixture(scope="module")
def F():
    ensure_built()
    import paper_1309_0100_b300 as F
    return F


def _batch(n=24, seed=0, nbs=(0, 1, 2, 3, 5, 7)):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nb = nbs[k % len(nbs)]
        N = int(rng.integers(2 * nb + 10, 700))
        nf = int(rng.integers(1, 3000))
        out.append(synth.small_series(500 + 7 * k + seed, N=N, n_base=nb, nf=nf, span=float(rng.uniform(50, 500)),
                                      fmax=float(rng.uniform(0.3, 2.0))))
    return out


@pytest.fixture(scope="module")
def batch_ref():
    """The batch and, per series, the oracle's z and conditioning ratios."""
    series = _batch()
    ref = [oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, s.grid.array(), want_ratio=True) for s in series]
    return series, ref


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_vs_oracle_and_single_series(F, prec, batch_ref):
    series, ref = batch_ref
    z, zo, top = F.periodogram_batch(series, precision=prec, topk=3)
    for k, s in enumerate(series):
        zr, c2, ratio = ref[k]
        got = z[zo[k]:zo[k] + s.grid.nf]
        r = cond_parity(got, zr, ratio, c2, TOL[prec], s.N)
        assert r["ok"], (k, r)
        zs = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, s.grid.array(), precision=prec)
        r = cond_parity(got, zs, ratio, c2, TOL[prec], s.N)   # the single-series path on the same bins
        assert r["ok"], (k, r)
        if prec == "fp64":
            assert list(top[k]) == local_max_topk(zr, 3)


def test_plan_replay_deterministic(F):
    import torch
    series = _batch(12, seed=5, nbs=(0, 1, 2))
    plan = F.BatchPlan(series, precision="mixed", topk=2)
    plan.run()
    torch.cuda.synchronize()
    z1, t1 = plan.download()
    plan.run()
    plan.run()
    torch.cuda.synchronize()
    z2, t2 = plan.download()
    assert np.array_equal(z1, z2) and np.array_equal(t1, t2)
    zb, zo, tb = F.periodogram_batch(series, precision="mixed", topk=2)
    assert rel_err(z1, zb) < 1e-5
    plan.close()


def test_batch_large_base_classes(F):
    """Base sizes p = 13, 19 and 25 select the larger compiled classes."""
    series = _batch(6, seed=9, nbs=(0,))
    rng = np.random.default_rng(17)
    for k, nb in enumerate((6, 9, 12, 6, 9, 12)):
        s = series[k]
        T = s.t.max() - s.t.min()
        s.base_freqs = np.sort(rng.uniform(0.02, 0.9, nb)) + np.arange(nb) * 4.0 / T   # separated by > 4/T
        s.t, s.y, s.sigma = s.t, s.y, s.sigma
    for prec in ("fp64", "mixed"):
        z, zo, _ = F.periodogram_batch(series, precision=prec)
        for k, s in enumerate(series):
            zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, s.grid.array(), want_ratio=True)
            r = cond_parity(z[zo[k]:zo[k] + s.grid.nf], zr, ratio, c2, TOL[prec], s.N)
            assert r["ok"], (prec, k, r)


def test_batch_long_series_error_distribution(F):
    """A plan holding series of more than 256 tiles per warp runs the batch
    kernel with compensated residual totals: the long series of the plan keep
    the error distribution of the single-series kernels (median below 4e-7,
    99th percentile below 3e-6 of the floor-relative error; measured 2.0e-7
    and 2.2e-7, 1.6e-6 and 1.8e-6), next to a short one.  The plain batch
    kernel gave medians of 5.0e-7 and 5.7e-7 and broke the element-wise bound
    on the 1e5-point series (2.0e-5 at one bin)."""
    series = [synth.small_series(40 + nb, N=N, n_base=nb, nf=300, span=3000.0, fmax=2.0)
              for N, nb in ((70000, 3), (100000, 5))] + [synth.small_series(7, N=300, n_base=1, nf=200)]
    z, zo, _ = F.periodogram_batch(series, precision="mixed")
    for k, s in enumerate(series):
        zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, s.grid.array(), want_ratio=True)
        zk = z[zo[k]:zo[k] + s.grid.nf]
        r = cond_parity(zk, zr, ratio, c2, TOL["mixed"], s.N)
        assert r["ok"], (k, r)
        if s.N > 10000:
            e = np.abs(zk - zr) / np.maximum(zr, 1e-3 * zr.max())
            assert np.median(e) < 4e-7 and np.quantile(e, 0.99) < 3e-6, (k, np.median(e), np.quantile(e, 0.99))
