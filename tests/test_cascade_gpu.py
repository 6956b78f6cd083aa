"""GPU parity of the Phase 3 backward cascade and the Phase 4 ordering
(Sect. 4) against the oracle, on the same subtuple tables.

Pass flags are integers decided by floating point: the oracle forms
z = (N_H/2) ln(l_K/l_S) and compares it with the threshold, the GPU compares
l_K with l_S exp(2 z_thr/N_H).  Both decide identically except within a few
ulps of the threshold; every case below first checks (through the oracle's
slack) that no mask is that close, then requires bit-exact flags and identical
solution lists."""
import numpy as np
import pytest

import oracle
import paper_1309_0100_b300 as fx
from synth import small_series

from helpers import ensure_built

pytestmark = pytest.mark.gpu

TIE = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _mult_table(a, l0=1e4, noise=0.0, rng=None):
    logl = np.zeros(1)
    for aj in a:   # bit j of the index selects member j
        logl = np.concatenate([logl, logl - aj])
    l = l0 * np.exp(logl)
    if noise:
        l *= 1.0 + noise * rng.standard_normal(l.size)
    return l


def _compare(l, N, zthr):
    passed, slack, _ = oracle.cascade(l, N, zthr)
    assert not (np.abs(slack[1:]) < TIE * (1.0 + np.abs(np.nan_to_num(slack[1:], posinf=0, neginf=0)))).any()
    sols = oracle.cascade_solutions(passed)
    ms, G = oracle.phase4_order(sols, l, N)
    gm, gG, gpass = fx.cascade(l, N, zthr, want_pass=True)
    assert np.array_equal(gpass, passed)
    assert np.array_equal(gm, ms)
    np.testing.assert_allclose(gG, G, rtol=1e-14, atol=0)
    return gm


@pytest.mark.parametrize("seed", range(12))
def test_cascade_parity_random_tables(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(1, 13))
    a = rng.exponential(0.3 if seed % 2 else 0.04, n)
    N = int(rng.integers(3 * n + 2, 3 * n + 20)) if seed % 3 == 0 else int(rng.integers(3 * n + 2, 2000))
    l = _mult_table(a, noise=0.02, rng=rng)
    zthr = np.sort(rng.uniform(0.5, 8.0, n))
    _compare(l, N, zthr)


def test_cascade_empty_pool_and_tiny():
    gm, gG = fx.cascade(np.array([3.0]), 50, np.zeros(0))
    assert gm.size == 0 and gG.size == 0
    # one member: passes iff (N-4)/2 ln(l0/l1) >= zthr
    l = np.array([10.0, 5.0])
    N = 50
    z = 0.5 * (N - 4) * np.log(2.0)
    assert list(fx.cascade(l, N, [z - 1e-6])[0]) == [1]
    assert fx.cascade(l, N, [z + 1e-6])[0].size == 0


def test_cascade_degenerate_entries():
    rng = np.random.default_rng(9)
    n = 6
    l = _mult_table(rng.exponential(0.3, n), noise=0.01, rng=rng)
    l[0b000011] = 0.0            # a perfect fit
    l[0b000100] = np.nan         # a failed fit
    l[0b110000] = np.inf
    l[0b001000] = -1.0           # not a chi2
    zthr = np.full(n, 2.0)
    _compare(l, 30, zthr)
    # N too small for the larger tuples: N - 3m - 1 <= 0 fails them
    _compare(_mult_table(rng.exponential(0.5, n)), 12, np.full(n, 0.5))


def test_cascade_many_solutions_global_sort():
    # equal members and linear thresholds: every 7-subset of 14 is a solution
    # (C(14,7) = 3432 > 2048 takes the multi-launch sort); equal l within a
    # size, so the order falls back to the mask
    n = 14
    a = np.full(n, 0.1)
    N = 400
    NH7, NH8 = N - 22, N - 25
    q = 0.5 * (0.5 * NH7 * 0.1 + 0.5 * NH8 * 0.1)
    zthr = q * np.arange(1, n + 1)
    gm = _compare(_mult_table(a), N, zthr)
    assert gm.size == 3432
    assert all(bin(int(m)).count("1") == 7 for m in gm)


def test_cascade_on_refined_pool_table():
    s = small_series(seed=21, N=400, n_base=0, span=600.0, n_sig=4, nf=16, fmax=0.5)
    rng = np.random.default_rng(3)
    pool = np.concatenate([s.true_freqs[:4], rng.uniform(0.01, 0.5, 4)])
    # the table both cascades consume: the oracle's own local refinement of
    # every subtuple (Phase 2)
    l = np.empty(1 << pool.size)
    l[0] = oracle.l0(s.t, s.y, s.sigma)
    for S in range(1, 1 << pool.size):
        g = pool[[j for j in range(pool.size) if S >> j & 1]]
        l[S] = oracle.tuple_refine(s.t, s.y, s.sigma, g, max_iter=20, tol=1e-9)[1]
    W = oracle.effective_bandwidth(s.t, s.sigma, 0.5)
    zthr = np.array([oracle.fap_threshold(c, 1.0, W, 0.05) for c in range(1, pool.size + 1)])
    gm = _compare(l, s.t.size, zthr)
    assert gm.size >= 1


def test_fap_helpers_match_oracle():
    for n in (1, 2, 4, 9):
        for fap in (0.1, 1e-4):
            zo = oracle.fap_threshold(n, 0.6, 300.0, fap)
            zg = fx.fap_threshold(n, 0.6, 300.0, fap)
            assert abs(zg - zo) <= 1e-12 * zo
            assert fx.fap_bound(n, 0.6, 300.0, zg) == pytest.approx(fap, rel=1e-10)
    s = small_series(seed=4, N=300, n_base=0)
    W = fx.effective_bandwidth(s.t, s.sigma, 2.0)
    assert W == pytest.approx(oracle.effective_bandwidth(s.t, s.sigma, 2.0), rel=1e-13)


def _subtable(l, S):
    """Table over the subsets of S, indexed by the m-bit compressed mask."""
    mem = [j for j in range(32) if S >> j & 1]
    c = np.arange(1 << len(mem), dtype=np.int64)
    idx = np.zeros_like(c)
    for b, j in enumerate(mem):
        idx |= ((c >> b) & 1) << j
    return l[idx]


@pytest.mark.slow
def test_cascade_full_pool_24_sampled():
    # 2^24 subtuples (the largest pool): flags on sampled masks against the
    # oracle run on each mask's own sub-table; the solution list against the
    # maximal elements of the returned flags (superset-OR in numpy)
    rng = np.random.default_rng(24)
    n = 24
    a = np.concatenate([rng.uniform(0.2, 0.5, 5), rng.exponential(0.01, n - 5)])
    l = _mult_table(a, l0=5e3, noise=1e-3, rng=rng)
    N = 1000
    zthr = 6.0 + 4.0 * np.arange(1, n + 1)
    gm, gG, gpass = fx.cascade(l, N, zthr, want_pass=True)
    rand = rng.integers(1, 1 << n, 3000)
    rand = rand[[bin(int(x)).count("1") <= 12 for x in rand]][:600]
    sols = [int(m) for m in gm if bin(int(m)).count("1") <= 14][:50]
    sample = np.unique(np.concatenate([
        rand,
        [sum(1 << int(j) for j in rng.choice(n, int(k), replace=False)) for k in rng.integers(1, 9, 600)],
        np.asarray(sols, dtype=np.int64)]))
    for S in sample:
        S = int(S)
        sub = _subtable(l, S)
        p, slack, _ = oracle.cascade(sub, N, zthr)
        full = (1 << bin(S).count("1")) - 1
        if abs(slack[full]) > TIE:
            assert gpass[S] == p[full], hex(S)
    sup = gpass.astype(bool).copy()
    idx = np.arange(1 << n)
    for b in range(n):
        lo = (idx >> b & 1) == 0
        sup[idx[lo]] |= sup[idx[lo] | (1 << b)]
    strict = np.zeros_like(sup)
    for b in range(n):
        lo = (idx >> b & 1) == 0
        strict[idx[lo]] |= sup[idx[lo] | (1 << b)]
    maximal = np.flatnonzero(gpass.astype(bool) & ~strict)
    assert sorted(gm.tolist()) == sorted(maximal.tolist())
    key = [(bin(int(m)).count("1"), l[int(m)], int(m)) for m in gm]
    assert key == sorted(key)
