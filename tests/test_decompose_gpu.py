"""GPU parity of the Phase 1 scan and of the whole decomposition (Sect. 4)
against the oracle pipeline on the same series.

The decisions of Phase 1 (peak ranking, thresholds) and Phase 3 (pass flags)
are integers decided by floating point.  The FP64 GPU periodogram agrees with
the oracle to ~1e-10 relative, so the decisions agree wherever the oracle's
margins exceed that; each case checks its margins first."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import pipeline as P
import paper_1309_0100_b300 as fx

from helpers import ensure_built

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _series(seed, N, span, freqs, amps, sig):
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0, span, N))
    s = np.full(N, sig)
    y = 0.3 + sum(a * np.cos(2 * np.pi * f * t + rng.uniform(0, 2 * np.pi)) for f, a in zip(freqs, amps))
    return t, y + s * rng.standard_normal(N), s


def _sec61():
    spec = json.load(open(os.path.join(GOLDEN, "sec61_lookalike.json")))
    rng = np.random.Generator(np.random.PCG64(spec["seed"]))
    per, win = spec["gap_period"], spec["window"]
    t = []
    while len(t) < spec["N"]:
        c = rng.uniform(0, spec["span"])
        if c % per < win:
            t.append(c)
    t = np.sort(np.asarray(t))
    y = sum(np.sin(2 * np.pi * f * t + ph) for f, ph in zip(spec["true_freqs"], spec["phases"]))
    sigma = np.full(t.size, spec["noise_rel"])
    return t, y + sigma * rng.standard_normal(t.size), sigma


def _thr(t, s, fmax, n=20):
    W = oracle.effective_bandwidth(t, s, fmax)
    z0 = oracle.fap_threshold(1, 1.0, W, 0.05)
    z1 = oracle.fap_threshold(1, 1.0, W, 0.1)
    zt = np.array([oracle.fap_threshold(c, 1.0, W, 0.05) for c in range(1, n + 1)])
    return z0, z1, zt


CASES = {
    "three": lambda: (_series(1, 300, 500.0, [0.0731, 0.2117, 0.3419], [5.0, 3.0, 1.5], 1.0), 0.5, 5000, {}),
    "half8": lambda: (_series(2, 300, 500.0, [0.1313, 0.3711], [10.0, 8.0], 1.0), 0.5, 5000, {"max_base": 1}),
    "half6": lambda: (_series(2, 300, 500.0, [0.1313, 0.3711], [10.0, 6.0], 1.0), 0.5, 5000, {"max_base": 1}),
    "cap2": lambda: (_series(1, 300, 500.0, [0.0731, 0.2117, 0.3419], [5.0, 3.0, 1.5], 1.0), 0.5, 5000,
                     {"max_pool": 2}),
    "sec61": lambda: (_sec61(), 2.0, 4000, {}),
    "noise": lambda: ((lambda r: (np.sort(r.uniform(0, 500, 300)), r.standard_normal(300), np.ones(300)))(
        np.random.default_rng(50)), 0.5, 5000, {}),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("precision", [fx.FP64, fx.MIXED])
def test_scan_parity(case, precision):
    (t, y, s), fmax, nf, kw = CASES[case]()
    df = fmax / nf
    z0, z1, _ = _thr(t, s, fmax)
    pool, pz, base, tr = P.phase1_scan(t, y, s, df, df, nf, z0, z1, **kw)
    gpool, gpz, gbase, gtr = fx.scan(t, y, s, df, df, nf, z0, z1, precision=precision, **kw)
    assert np.array_equal(gbase, base)
    assert np.array_equal(gpool, pool)
    assert gtr == tr
    np.testing.assert_allclose(gpz, pz, rtol=1e-8 if precision == fx.FP64 else 1e-4)


@pytest.mark.parametrize("case", ["three", "sec61", "noise"])
def test_decompose_parity_fp64(case):
    (t, y, s), fmax, nf, kw = CASES[case]()
    df = fmax / nf
    z0, z1, zt = _thr(t, s, fmax)
    ref = P.decompose(t, y, s, df, df, nf, z0, z1, zt, **kw)
    margin = np.abs(ref["slack"][1:])
    assert margin.size == 0 or margin.min() > 1e-6
    got = fx.decompose(t, y, s, df, df, nf, z0, z1, zt, **kw)
    assert np.array_equal(got["pool"], ref["pool"])
    np.testing.assert_allclose(got["l"], ref["l"], rtol=1e-9)
    assert np.array_equal(got["masks"], ref["masks"])
    np.testing.assert_allclose(got["G"], ref["G"], rtol=1e-9)
    T = t.max() - t.min()
    for a, b in zip(got["freqs"], ref["freqs"]):
        np.testing.assert_allclose(a, b, atol=1e-7 / T)
    # Phase 4 residual statistic (the oracle's residual periodogram at its own
    # fitted frequencies, equal to the GPU's to 1e-7/T)
    np.testing.assert_allclose(got["resid_z"], ref["resid_z"], rtol=1e-6)
    if case == "sec61":
        best = got["freqs"][int(np.argmin(got["G"]))]
        np.testing.assert_allclose(best, [0.9, 1.1], atol=1e-3)
    if case == "noise":
        assert got["pool"].size == 0 and got["n_solutions"] == 0 and got["l"].size == 1


def test_decompose_mixed_refine_same_solutions():
    (t, y, s), fmax, nf, kw = CASES["sec61"]()
    df = fmax / nf
    z0, z1, zt = _thr(t, s, fmax)
    ref = P.decompose(t, y, s, df, df, nf, z0, z1, zt)
    got = fx.decompose(t, y, s, df, df, nf, z0, z1, zt, precision=fx.MIXED, refine_precision=fx.MIXED)
    assert np.array_equal(got["pool"], ref["pool"])
    # FP32-accumulated sums: the error scales with the data's total power l_0
    np.testing.assert_allclose(got["l"], ref["l"], rtol=0, atol=1e-6 * ref["l"][0])
    assert np.array_equal(got["masks"], ref["masks"])
    # the residual statistic from the mixed periodogram at mixed-refined
    # frequencies: FP32 sums, the mixed path's 1e-5 bar with room for the
    # frequencies' own FP32-level offsets
    np.testing.assert_allclose(got["resid_z"], ref["resid_z"], rtol=1e-4)
