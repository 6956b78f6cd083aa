"""Pins of the oracle's Phase 1 scan and of the whole decomposition (Sect. 4)
on series whose answer is fixed by their construction, and on the paper's
double-frequency example (Sect. 6.1)."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import pipeline as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
FMAX, NF = 0.5, 5000
DF = FMAX / NF


def _series(seed, N, span, freqs, amps, sig):
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0, span, N))
    s = np.full(N, sig)
    y = 0.3 + sum(a * np.cos(2 * np.pi * f * t + rng.uniform(0, 2 * np.pi)) for f, a in zip(freqs, amps))
    return t, y + s * rng.standard_normal(N), s


def _thresholds(t, s, fmax, fap0=0.05, fap1=0.1):
    # A_n of Eq. zFAP is not given in the paper: A = 1 here
    W = oracle.effective_bandwidth(t, s, fmax)
    return oracle.fap_threshold(1, 1.0, W, fap0), oracle.fap_threshold(1, 1.0, W, fap1)


def test_local_maxima_rule():
    z = np.array([3.0, 1.0, 2.0, 2.0, 1.0, 5.0, 5.0, 4.0, 6.0])
    # 0 (end, above its neighbour), 2 (plateau start: > left, >= right),
    # 5 (plateau), 8 (end); ranked by z, ties to the lower index
    assert P.local_maxima(z) == [8, 5, 0, 2]
    assert P.local_maxima(np.array([1.0])) == [0]
    assert P.local_maxima(np.array([2.0, 2.0])) == []


def test_scan_three_sinusoids_in_amplitude_order():
    freqs = [0.0731, 0.2117, 0.3419]
    t, y, s = _series(1, 300, 500.0, freqs, [5.0, 3.0, 1.5], 1.0)
    z0, z1 = _thresholds(t, s, FMAX)
    pool, pz, base, trunc = P.phase1_scan(t, y, s, DF, DF, NF, z0, z1)
    assert base.size == 3 and not trunc
    np.testing.assert_allclose(base, freqs, atol=DF)       # SLICK order = amplitude order
    np.testing.assert_allclose(np.sort(pool), freqs, atol=DF)
    assert np.all(np.diff(pz) <= 0)
    # a cap keeps the candidates with the largest z (smallest FAP)
    pool2, pz2, _, trunc2 = P.phase1_scan(t, y, s, DF, DF, NF, z0, z1, max_pool=2)
    assert trunc2 and np.array_equal(pool2, pool[:2]) and np.array_equal(pz2, pz[:2])


@pytest.mark.parametrize("a2,enters", [(8.0, True), (6.0, False)])
def test_scan_half_height_rule(a2, enters):
    # one SLICK step: the second sinusoid's peak enters the pool (QUICK) only
    # when its z reaches half of the top peak's; z scales like amplitude^2
    t, y, s = _series(2, 300, 500.0, [0.1313, 0.3711], [10.0, a2], 1.0)
    z0, z1 = _thresholds(t, s, FMAX)
    pool, pz, base, _ = P.phase1_scan(t, y, s, DF, DF, NF, z0, z1, max_base=1)
    np.testing.assert_allclose(base, [0.1313], atol=DF)
    assert (np.abs(pool - 0.3711) < DF).any() == enters


@pytest.mark.parametrize("seed", range(3))
def test_scan_of_pure_noise_is_empty(seed):
    rng = np.random.default_rng(50 + seed)
    t = np.sort(rng.uniform(0, 500, 300))
    s = np.ones(300)
    y = rng.standard_normal(300)
    z0, z1 = _thresholds(t, s, FMAX)
    pool, _, base, _ = P.phase1_scan(t, y, s, DF, DF, NF, z0, z1)
    assert pool.size == 0 and base.size == 0


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
    return t, y + sigma * rng.standard_normal(t.size), sigma, spec


def test_decompose_sec61_finds_the_true_pair():
    # Sect. 6.1: the single periodogram peaks at the spurious 1.0; the
    # decomposition still finds the true pair 0.9 + 1.1, with the smallest G
    t, y, s, spec = _sec61()
    fmax, nf = 2.0, 4000
    df = fmax / nf
    W = oracle.effective_bandwidth(t, s, fmax)
    z0 = oracle.fap_threshold(1, 1.0, W, 0.05)
    z1 = oracle.fap_threshold(1, 1.0, W, 0.1)
    zt = np.array([oracle.fap_threshold(c, 1.0, W, 0.05) for c in range(1, 21)])
    r = P.decompose(t, y, s, df, df, nf, z0, z1, zt)
    assert abs(r["base"][0] - spec["expected_single_peak"]) < df
    for f in spec["true_freqs"]:
        assert (np.abs(r["pool"] - f) < df).any()
    best = r["freqs"][int(np.argmin(r["G"]))]
    np.testing.assert_allclose(best, spec["true_freqs"], atol=1e-3)
    masks = [int(m) for m in r["masks"]]
    for a in masks:
        for b in masks:
            assert a == b or (a & b) != a               # never nested
    # every solution's frequencies are a local minimum of chi2: dz/df ~ 0
    for f in r["freqs"]:
        _, g = oracle.tuple_grad(t, y, s, [f])
        assert np.max(np.abs(g)) * (t.max() - t.min()) < 1e-3 * oracle.l0(t, y, s)
    # Phase 4 residual statistic: the true pair leaves only noise behind, so its
    # residual periodogram's highest peak stays below the FAP_0 threshold;
    # it equals the log form of the residual periodogram's maximum
    best_i = int(np.argmin(r["G"]))
    assert r["resid_z"][best_i] < z0
    zres, lres = oracle.periodogram(t, y, s, r["freqs"][best_i], df * np.arange(1, nf + 1))
    NH = t.size - 3 * 3 - 1
    assert r["resid_z"][best_i] == pytest.approx(0.5 * NH * np.log(lres / (lres - 2 * zres.max())), rel=1e-12)
    # G = (l_S / l_0)(N-1)/(N-3m-1)
    for m, G in zip(masks, r["G"]):
        k = bin(m).count("1")
        assert G == pytest.approx(r["l"][m] / r["l"][0] * (t.size - 1) / (t.size - 3 * k - 1), rel=1e-14)
