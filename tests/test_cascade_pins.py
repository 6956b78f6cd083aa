"""Pins of the oracle's Phase 3 backward cascade, its non-nested solutions and
the FAP-threshold helper (Sect. 4, Eq. zpowrel, Eq. zFAP), each against a route
that does not enumerate the cascade's tests the way the oracle does."""
import itertools

import numpy as np
import pytest
from scipy.special import lambertw

import oracle
from synth import small_series


def _masks(n):
    return range(1 << n)


def _members(S, n):
    return [j for j in range(n) if S >> j & 1]


# ---------------------------------------------------------------------------
# FAP threshold: closed form through the Lambert W function.

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("fap", [0.1, 0.05, 1e-3, 1e-9])
def test_fap_threshold_matches_lambert_w(n, fap):
    A, W = 0.7, 250.0
    a = 1.5 * n - 1.0
    # A W^n e^{-z} z^a = fap  <=>  z = -a W_{-1}( -(fap/(A W^n))^{1/a} / a )
    c = fap / (A * W ** n)
    zc = float(np.real(-a * lambertw(-(c ** (1.0 / a)) / a, k=-1)))
    z = oracle.fap_threshold(n, A, W, fap)
    assert abs(z - zc) <= 1e-11 * zc
    assert z > a
    assert abs(oracle.fap_bound(n, A, W, z) / fap - 1.0) < 1e-10


def test_fap_threshold_when_every_z_passes():
    # M_n below the level everywhere on the decreasing branch: the branch start
    z = oracle.fap_threshold(2, 1e-9, 1.0, 0.5)
    assert z == pytest.approx(2.0)


# ---------------------------------------------------------------------------
# Every test is formed: sum_m C(n,m)(2^m - 1) = 3^n - 2^n (Sect. 4).

@pytest.mark.parametrize("n", range(0, 11))
def test_cascade_forms_every_relative_test(n):
    rng = np.random.default_rng(n)
    l = np.sort(rng.uniform(1.0, 2.0, 1 << n))[::-1].copy()
    _, _, tests = oracle.cascade(l, 10 ** 6, np.full(max(n, 1), 1.0))
    assert tests == 3 ** n - 2 ** n


# ---------------------------------------------------------------------------
# Multiplicative table: l[S] = l0 exp(-sum_{j in S} a_j).  Then
# ln(l[K]/l[S]) = sum of a_j over S\K, so the smallest z of layer k is
# (N_H/2) times the sum of the m-k smallest a_j of S.  S passes iff for every
# count c = 1..m that sum over the c smallest reaches zthr[c-1].

def _mult_table(a, l0=1e4):
    n = len(a)
    return np.array([l0 * np.exp(-sum(a[j] for j in _members(S, n))) for S in _masks(n)])


def _closed_form_pass(a, N, zthr):
    n = len(a)
    out = np.zeros(1 << n, dtype=np.uint8)
    for S in range(1, 1 << n):
        mem = sorted(a[j] for j in _members(S, n))
        m = len(mem)
        NH = N - 3 * m - 1
        if NH <= 0:
            continue
        csum = np.cumsum(mem)
        out[S] = all(0.5 * NH * csum[c - 1] >= zthr[c - 1] for c in range(1, m + 1))
    return out


def _mult_case(seed):
    # small N on half the seeds, so that N_H = N - 3m - 1 varies strongly with m
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(3, 9))
    a = rng.exponential(0.05, n) if seed % 2 else rng.exponential(0.6, n)
    N = int(rng.integers(3 * n - 2, 400)) if seed % 2 else int(rng.integers(3 * n - 2, 3 * n + 12))
    zthr = np.sort(rng.uniform(0.5, 6.0, n))
    return a, N, zthr


@pytest.mark.parametrize("seed", range(16))
def test_cascade_matches_multiplicative_closed_form(seed):
    a, N, zthr = _mult_case(seed)
    passed, slack, _ = oracle.cascade(_mult_table(a), N, zthr)
    ref = _closed_form_pass(a, N, zthr)
    tie = np.abs(slack) < 1e-9
    assert not tie.any()
    assert np.array_equal(passed, ref)
    assert np.array_equal(passed.astype(bool), slack >= 0)
    assert passed.any() and not passed.all()


# With linear thresholds zthr[c-1] = c * q the binding count is c = 1, so S
# passes iff every member has a_j >= 2q / N_H(m): S is inside
# J(m) = {j : a_j >= 2q/(N - 3m - 1)}.  J shrinks as m grows, hence a passing
# S (size m) has a passing strict superset iff S is inside J(m+1) and
# |J(m+1)| >= m+1.

@pytest.mark.parametrize("seed", range(5))
def test_cascade_solutions_match_linear_threshold_closed_form(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(4, 11))
    a = rng.exponential(0.05, n)
    N = int(rng.integers(3 * n + 5, 300))
    srt = np.sort(a)   # threshold between two members: no exact ties
    q = 0.5 * (srt[n // 2 - 1] + srt[n // 2]) * (N - 3 * (n // 2) - 1) / 2.0
    zthr = q * np.arange(1, n + 1)
    passed, slack, _ = oracle.cascade(_mult_table(a), N, zthr)
    assert not (np.abs(slack) < 1e-9).any()

    def J(m):
        NH = N - 3 * m - 1
        return {j for j in range(n) if NH > 0 and a[j] >= 2 * q / NH}

    expect = []
    for S in range(1, 1 << n):
        mem = set(_members(S, n))
        m = len(mem)
        if not mem <= J(m):
            continue
        assert passed[S]
        Jn = J(m + 1)
        if not (mem <= Jn and len(Jn) >= m + 1):
            expect.append(S)
    got = oracle.cascade_solutions(passed)
    assert list(got) == expect
    # no solution contains another (Sect. 4, Phase 4)
    for x, y in itertools.permutations(got, 2):
        assert (int(x) & int(y)) != int(x)


# ---------------------------------------------------------------------------
# A real series: two strong sinusoids and one spurious pool member.  The true
# pair is the only non-nested solution; the spurious member fails the test of
# adding it to the pair.

def test_cascade_on_series_keeps_the_true_pair():
    s = small_series(seed=7, N=240, n_base=0, span=400.0, n_sig=2, nf=16, fmax=0.5)
    f1, f2 = s.true_freqs[:2]
    pool = np.array([f1, f2, 0.3337])
    l = oracle.pool_table(s.t, s.y, s.sigma, pool)
    W = oracle.effective_bandwidth(s.t, s.sigma, 0.5)
    zthr = [oracle.fap_threshold(k, 1.0, W, 0.01) for k in (1, 2, 3)]
    passed, slack, _ = oracle.cascade(l, s.t.size, zthr)
    sols = oracle.cascade_solutions(passed)
    assert list(sols) == [0b011]
    ms, G = oracle.phase4_order(sols, l, s.t.size)
    assert G[0] < 1.0
    # monotone: each of the pair alone passes as well
    assert passed[0b001] and passed[0b010] and not passed[0b100]


def test_phase4_orders_by_size_then_chi2():
    l = np.array([10.0, 4.0, 5.0, 1.0, 3.0, 0.9, 0.8, 0.5])
    ms, G = oracle.phase4_order([0b110, 0b001, 0b100, 0b011], l, 100)
    assert list(ms) == [0b100, 0b001, 0b110, 0b011]
    assert G[0] == pytest.approx(3.0 / 10.0 * 99 / 96)


# ---------------------------------------------------------------------------
# A planted mistake in the cascade (N_H of the base model instead of the
# alternative) is caught by the closed-form pin.

def test_planted_cascade_mistake_is_caught():
    bad = oracle.Oracle(mutant=4)
    caught = False
    for seed in range(16):
        a, N, zthr = _mult_case(seed)
        passed, _, _ = oracle.cascade(_mult_table(a), N, zthr, lib=bad.lib)
        if not np.array_equal(passed, _closed_form_pass(a, N, zthr)):
            caught = True
    assert caught


# ---------------------------------------------------------------------------
# The normalised bandwidth W = f_max T_eff, T_eff = sqrt(4 pi Var_w(t))
# (Sect. 2), which every FAP threshold of the scan and the cascade uses, is
# pinned by closed forms of the weighted variance, not by its own formula.

def test_effective_bandwidth_equally_spaced_closed_form():
    # n equally spaced times on [0, T] with equal weights: the discrete
    # uniform variance T^2 (n + 1) / (12 (n - 1)); T_eff -> T sqrt(pi/3)
    T, fmax = 2000.0, 0.7
    for n in (2, 3, 10, 1001):
        t = np.linspace(0.0, T, n)
        W = oracle.effective_bandwidth(t, np.full(n, 0.3), fmax)
        assert W == pytest.approx(fmax * np.sqrt(4 * np.pi * T * T * (n + 1) / (12.0 * (n - 1))), rel=1e-13)
    t = np.linspace(0.0, T, 200001)
    assert oracle.effective_bandwidth(t, np.ones(t.size), 1.0) == pytest.approx(T * np.sqrt(np.pi / 3), rel=1e-5)


def test_effective_bandwidth_weights_closed_form():
    # two times with weights w1 = 1/s1^2, w2 = 1/s2^2: Var_w = w1 w2 T^2 / (w1 + w2)^2
    # (catches weights dropped, or 1/sigma used instead of 1/sigma^2)
    T = 37.5
    for s1, s2 in ((1.0, 1.0), (1.0, 3.0), (0.2, 5.0)):
        w1, w2 = 1 / s1 ** 2, 1 / s2 ** 2
        var = w1 * w2 * T * T / (w1 + w2) ** 2
        W = oracle.effective_bandwidth([0.0, T], [s1, s2], 2.0)
        assert W == pytest.approx(2.0 * np.sqrt(4 * np.pi * var), rel=1e-14)


def test_effective_bandwidth_shift_and_scale():
    # W does not depend on the time origin; it scales with f_max and with
    # the time unit (t -> a t, f_max -> f_max / a leaves W unchanged)
    rng = np.random.default_rng(11)
    t = np.sort(rng.uniform(0, 500, 300))
    sg = rng.lognormal(0, 0.5, 300)
    W = oracle.effective_bandwidth(t, sg, 1.3)
    assert oracle.effective_bandwidth(t + 2.45e6, sg, 1.3) == pytest.approx(W, rel=1e-9)
    assert oracle.effective_bandwidth(t, sg, 2.6) == pytest.approx(2 * W, rel=1e-14)
    assert oracle.effective_bandwidth(t * 24.0, sg, 1.3 / 24.0) == pytest.approx(W, rel=1e-13)
    assert oracle.effective_bandwidth(t, 7.0 * sg, 1.3) == pytest.approx(W, rel=1e-13)   # common sigma scale
