"""Pins of the FP64 CPU oracle against things other than itself.

Each test checks the oracle against an independent route that the paper and
the mathematics fix: the generalized Lomb-Scargle closed form for a constant
base (Section 2, Eq. H0), the Schuster periodogram for orthogonal columns,
library least squares (numpy lstsq, SVD based) on explicit design matrices,
exact rational arithmetic, invariances of the least-squares statistic,
finite differences, and an independent nonlinear least-squares solver
(scipy) for the local refinement of Section 3.  A planted-mistake test checks
that each plausible oracle bug fails at least one of them.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(k):
    return np.random.Generator(np.random.PCG64(4242 + k))


def _series(k=0, N=60, span=80.0):
    rng = _rng(k)
    t = np.sort(rng.uniform(0, span, N))
    sigma = rng.lognormal(0, 0.5, N)
    y = 1.3 + 3 * np.sin(2 * np.pi * t / 7.3 + 0.4) + 2 * np.cos(2 * np.pi * t / 19.0) + sigma * rng.standard_normal(N)
    return t, y, sigma


# ----------------------------------------------------------------------------
# Closed forms

def gls_z(t, y, sigma, f):
    """Generalized (floating-mean) Lomb-Scargle written from the 2x2 Schur
    complement of weighted mean-removed sums; z = p * chi2_0 / 2."""
    w = 1.0 / sigma ** 2
    W = w.sum()
    out = []
    for fj in f:
        c = np.cos(2 * np.pi * fj * t)
        s = np.sin(2 * np.pi * fj * t)
        Y = (w * y).sum() / W
        C = (w * c).sum() / W
        S = (w * s).sum() / W
        YY = (w * y * y).sum() / W - Y * Y
        YC = (w * y * c).sum() / W - Y * C
        YS = (w * y * s).sum() / W - Y * S
        CC = (w * c * c).sum() / W - C * C
        SS = (w * s * s).sum() / W - S * S
        CS = (w * c * s).sum() / W - C * S
        D = CC * SS - CS * CS
        p = (SS * YC * YC + CC * YS * YS - 2 * CS * YC * YS) / (YY * D)
        out.append(p * W * YY / 2)
    return np.array(out)


def test_gls_closed_form_constant_base():
    t, y, sigma = _series(1)
    f = np.linspace(0.003, 0.9, 157)
    z, c2 = oracle.periodogram(t, y, sigma, [], f)
    zg = gls_z(t, y, sigma, f)
    assert np.max(np.abs(z - zg) / np.maximum(zg, 1e-3 * zg.max())) < 1e-10
    w = 1 / sigma ** 2
    assert c2 == pytest.approx((w * (y - (w * y).sum() / w.sum()) ** 2).sum(), rel=1e-12)


def test_schuster_special_case():
    """Uniform sampling, equal weights, Fourier frequencies k/(N dt): the
    columns are orthogonal and z = w |sum y e^{i w t}|^2 / N."""
    N = 48
    s = synth.uniform_series(3, N=N, dt=0.5)
    sigma = np.full(N, 1.7)
    ks = np.arange(1, N // 2)
    f = ks / (N * 0.5)
    z, _ = oracle.periodogram(s.t, s.y, sigma, [], f)
    ref = np.abs(np.exp(2j * np.pi * np.outer(f, s.t)) @ s.y) ** 2 / N / 1.7 ** 2
    np.testing.assert_allclose(z, ref, rtol=1e-11)


def test_exact_rational_tiny_case():
    """t = 0..7, f = 1/4: cos and sin take values in {0, +-1} exactly, so the
    normal equations can be solved in exact rational arithmetic."""
    t = np.arange(8.0)
    y = np.array([3, -1, 4, 1, -5, 9, 2, -6], dtype=float)
    sigma = np.array([1, 2, 1, 1, 2, 1, 1, 2], dtype=float)
    w = [Fraction(1, int(s * s)) for s in sigma]
    cs = [[1, 0, -1, 0][i % 4] for i in range(8)]
    sn = [[0, 1, 0, -1][i % 4] for i in range(8)]

    def chi2(cols):
        k = len(cols)
        G = [[sum(w[i] * cols[a][i] * cols[b][i] for i in range(8)) for b in range(k)] for a in range(k)]
        r = [sum(w[i] * cols[a][i] * int(y[i]) for i in range(8)) for a in range(k)]
        # Gauss-Jordan elimination in exact arithmetic
        M = [G[a][:] + [r[a]] for a in range(k)]
        for c in range(k):
            piv = next(a for a in range(c, k) if M[a][c] != 0)
            M[c], M[piv] = M[piv], M[c]
            for a in range(k):
                if a != c and M[a][c] != 0:
                    fac = M[a][c] / M[c][c]
                    M[a] = [u - fac * v for u, v in zip(M[a], M[c])]
        th = [M[a][k] / M[a][a] for a in range(k)]
        return sum(w[i] * (int(y[i]) - sum(th[a] * cols[a][i] for a in range(k))) ** 2 for i in range(8))

    one = [1] * 8
    zexact = (chi2([one]) - chi2([one, cs, sn])) / 2
    z, c2 = oracle.periodogram(t, y, sigma, [], [0.25])
    assert c2 == pytest.approx(float(chi2([one])), rel=1e-14)
    assert z[0] == pytest.approx(float(zexact), rel=1e-13)


def test_brute_force_lstsq_with_base():
    """Joint refit with fixed base frequencies equals an explicit library
    least-squares solve of the full design matrix."""
    t, y, sigma = _series(2, N=40)
    base = np.array([1 / 7.3, 1 / 19.0, 0.31])
    f = np.linspace(0.01, 1.2, 41)
    z, c2, coef = oracle.periodogram(t, y, sigma, base, f, want_coef=True)
    sw = 1 / sigma

    def cols(freqs):
        A = [np.ones_like(t)]
        for g in freqs:
            A += [np.cos(2 * np.pi * g * t), np.sin(2 * np.pi * g * t)]
        return np.stack(A, 1)

    def lsq(freqs):
        A = cols(freqs) * sw[:, None]
        x, *_ = np.linalg.lstsq(A, y * sw, rcond=None)
        return ((y * sw - A @ x) ** 2).sum(), x

    l0, _ = lsq(base)
    assert c2 == pytest.approx(l0, rel=1e-11)
    for j, fj in enumerate(f):
        l1, x = lsq(list(base) + [fj])
        assert z[j] == pytest.approx((l0 - l1) / 2, rel=1e-9, abs=1e-9 * l0)
        np.testing.assert_allclose(coef[j], x[-2:], rtol=1e-7, atol=1e-9 * np.abs(x).max())


def test_high_precision_small_z():
    """Small z under a large chi2 (big offset and noise): the oracle's z agrees
    with a 40-digit normal-equation solve to 1e-12 relative, i.e. it does not
    lose digits to the cancellation of chi2_base - chi2_new."""
    import mpmath as mp
    mp.mp.dps = 40
    rng = _rng(21)
    N = 40
    t = np.sort(rng.uniform(0, 50, N))
    sigma = rng.lognormal(0, 0.3, N)
    y = 1e3 + 30 * rng.standard_normal(N) + 0.05 * np.sin(2 * np.pi * 0.31 * t)
    base = np.array([0.123])
    f = np.array([0.31, 0.05, 0.77])
    z, c2 = oracle.periodogram(t, y, sigma, base, f)

    def chi2(freqs):
        cols = [[mp.mpf(1)] * N]
        for g in freqs:
            cols.append([mp.cos(2 * mp.pi * mp.mpf(g) * mp.mpf(ti)) for ti in t])
            cols.append([mp.sin(2 * mp.pi * mp.mpf(g) * mp.mpf(ti)) for ti in t])
        w = [1 / mp.mpf(s) ** 2 for s in sigma]
        k = len(cols)
        G = mp.matrix(k, k)
        r = mp.matrix(k, 1)
        for a in range(k):
            r[a] = mp.fsum(w[i] * cols[a][i] * mp.mpf(y[i]) for i in range(N))
            for b in range(k):
                G[a, b] = mp.fsum(w[i] * cols[a][i] * cols[b][i] for i in range(N))
        th = mp.lu_solve(G, r)
        return mp.fsum(w[i] * (mp.mpf(y[i]) - mp.fsum(th[a] * cols[a][i] for a in range(k))) ** 2 for i in range(N))

    l0 = chi2(list(base))
    for j, fj in enumerate(f):
        zmp = (l0 - chi2(list(base) + [fj])) / 2
        assert float(abs(z[j] - zmp) / abs(zmp)) < 1e-12, (j, z[j], float(zmp))
    assert float(abs(c2 - l0) / l0) < 1e-13


# ----------------------------------------------------------------------------
# Invariants

def test_bounds_and_base_frequency_zero():
    t, y, sigma = _series(3)
    base = np.array([1 / 7.3])
    f = np.concatenate([np.linspace(0.001, 1.0, 300), base])
    z, c2 = oracle.periodogram(t, y, sigma, base, f)
    assert np.all(z >= -1e-12 * c2)
    assert np.all(z <= c2 / 2 * (1 + 1e-12))
    assert abs(z[-1]) <= 1e-10 * c2            # f = base frequency adds nothing


def test_shift_scale_permutation_invariance():
    t, y, sigma = _series(4)
    base = np.array([1 / 19.0])
    f = np.linspace(0.002, 0.8, 97)
    z, _ = oracle.periodogram(t, y, sigma, base, f)
    fl = 1e-3 * z.max()
    zs, _ = oracle.periodogram(t + 1234.5, y, sigma, base, f)
    assert np.max(np.abs(zs - z) / np.maximum(z, fl)) < 1e-8
    za, _ = oracle.periodogram(t, 3.0 * y, sigma, base, f)
    np.testing.assert_allclose(za, 9.0 * z, rtol=1e-9, atol=1e-9 * z.max())
    zb, _ = oracle.periodogram(t, y, 2.0 * sigma, base, f)
    np.testing.assert_allclose(zb, z / 4.0, rtol=1e-9, atol=1e-9 * z.max())
    perm = _rng(9).permutation(t.size)
    zp, _ = oracle.periodogram(t[perm], y[perm], sigma[perm], base, f)
    np.testing.assert_allclose(zp, z, rtol=1e-9, atol=1e-9 * z.max())


def test_aliasing_uniform_sampling():
    dt = 0.7
    s = synth.uniform_series(5, N=50, dt=dt, t0=3.0)
    sigma = _rng(5).lognormal(0, 0.3, 50)
    f = np.linspace(0.01, 0.69, 61)
    z, _ = oracle.periodogram(s.t, s.y, sigma, [], f)
    z1, _ = oracle.periodogram(s.t, s.y, sigma, [], f + 1 / dt)
    z2, _ = oracle.periodogram(s.t, s.y, sigma, [], 1 / dt - f)
    fl = 1e-3 * z.max()
    assert np.max(np.abs(z1 - z) / np.maximum(z, fl)) < 1e-8
    assert np.max(np.abs(z2 - z) / np.maximum(z, fl)) < 1e-8


def test_analytic_peak_noiseless_sinusoid():
    """Noiseless y = c + A cos(2 pi f0 t + phi) on a constant base: the trial
    frequency f0 removes all residual, so z(f0) = chi2_base/2 = max z."""
    rng = _rng(6)
    t = np.sort(rng.uniform(0, 50, 70))
    sigma = rng.lognormal(0, 0.4, 70)
    f0 = 0.237
    y = 2.0 + 1.5 * np.cos(2 * np.pi * f0 * t + 0.9)
    f = np.concatenate([np.linspace(0.01, 0.5, 200), [f0]])
    z, c2 = oracle.periodogram(t, y, sigma, [], f)
    assert z[-1] == pytest.approx(c2 / 2, rel=1e-11)
    assert np.all(z[:-1] <= z[-1] * (1 + 1e-12))


# ----------------------------------------------------------------------------
# Tuples

def test_pool_table_vs_lstsq_and_monotone():
    t, y, sigma = _series(7, N=45)
    pool = np.array([1 / 7.3, 1 / 19.0, 0.33, 0.51, 0.077])
    tab = oracle.pool_table(t, y, sigma, pool)
    sw = 1 / sigma
    for mask in range(1 << pool.size):
        fr = [pool[k] for k in range(pool.size) if mask >> k & 1]
        A = [np.ones_like(t)]
        for g in fr:
            A += [np.cos(2 * np.pi * g * t), np.sin(2 * np.pi * g * t)]
        A = np.stack(A, 1) * sw[:, None]
        x, *_ = np.linalg.lstsq(A, y * sw, rcond=None)
        assert tab[mask] == pytest.approx(((y * sw - A @ x) ** 2).sum(), rel=1e-9)
        for k in range(pool.size):      # nested models can only fit better
            if mask >> k & 1:
                assert tab[mask] <= tab[mask & ~(1 << k)] * (1 + 1e-12)
    z, l0 = oracle.tuple_eval(t, y, sigma, [[pool[0]], [pool[1], pool[3]], []])
    assert l0 == pytest.approx(tab[0], rel=1e-13)
    np.testing.assert_allclose(z, [(tab[0] - tab[1]) / 2, (tab[0] - tab[0b1010]) / 2, 0.0], atol=1e-9 * tab[0])


# ----------------------------------------------------------------------------
# Gradients

def test_periodogram_grad_vs_finite_differences():
    t, y, sigma = _series(8)
    base = np.array([1 / 19.0])
    f = np.array([0.05, 0.137, 0.2, 0.41])
    g = oracle.periodogram_grad(t, y, sigma, base, f)
    T = t.max() - t.min()
    h = 1e-7 / T
    zp, _ = oracle.periodogram(t, y, sigma, base, f + h)
    zm, _ = oracle.periodogram(t, y, sigma, base, f - h)
    fd = (zp - zm) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6 * np.abs(g).max())


def test_tuple_grad_vs_finite_differences():
    t, y, sigma = _series(10)
    tup = [[0.137, 0.052], [0.31]]
    z, g = oracle.tuple_grad(t, y, sigma, tup)
    T = t.max() - t.min()
    h = 1e-7 / T
    flat = np.concatenate([np.asarray(x) for x in tup])
    fd = np.empty_like(flat)
    k = 0
    for tp in tup:
        for q in range(len(tp)):
            a = list(tp); b = list(tp)
            a[q] += h; b[q] -= h
            fd[k] = (oracle.tuple_eval(t, y, sigma, [a])[0][0] - oracle.tuple_eval(t, y, sigma, [b])[0][0]) / (2 * h)
            k += 1
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6 * np.abs(g).max())
    z2, _ = oracle.tuple_eval(t, y, sigma, tup)
    np.testing.assert_allclose(z, z2, rtol=1e-13)


def test_vjp_vs_finite_differences():
    """z is a ratio of quadratic forms in y with y-independent Gram, so the
    central difference in y is exact up to rounding."""
    t, y, sigma = _series(11, N=30)
    base = np.array([1 / 7.3])
    f = np.array([0.05, 0.21, 0.33])
    v = np.array([0.7, -1.2, 0.4])
    g = oracle.periodogram_vjp(t, y, sigma, base, f, v)
    h = 1e-4
    fd = np.empty_like(y)
    for i in range(y.size):
        yp = y.copy(); yp[i] += h
        ym = y.copy(); ym[i] -= h
        fd[i] = (v @ oracle.periodogram(t, yp, sigma, base, f)[0] - v @ oracle.periodogram(t, ym, sigma, base, f)[0]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-7 * np.abs(g).max())


# ----------------------------------------------------------------------------
# Local refinement (Section 3)

def test_refine_matches_independent_nonlinear_solver():
    from scipy.optimize import least_squares
    rng = _rng(12)
    t = np.sort(rng.uniform(0, 120, 90))
    sigma = rng.lognormal(0, 0.3, 90)
    ftrue = np.array([0.0813, 0.231])
    y = 0.5 + 4 * np.sin(2 * np.pi * ftrue[0] * t + 1) + 2.5 * np.cos(2 * np.pi * ftrue[1] * t) + 0.5 * sigma * rng.standard_normal(90)
    T = t.max() - t.min()
    f0 = ftrue + np.array([0.15, -0.2]) / T
    fr, l, it = oracle.tuple_refine(t, y, sigma, f0, max_iter=60, tol=1e-12)
    assert 0 < it < 60

    def res(p):
        mu = p[0] + sum(p[1 + 3 * k] * np.cos(2 * np.pi * p[3 + 3 * k] * t) + p[2 + 3 * k] * np.sin(2 * np.pi * p[3 + 3 * k] * t) for k in range(2))
        return (y - mu) / sigma

    _, th = oracle.tuple_l(t, y, sigma, f0, want_theta=True)
    p0 = [th[0], th[1], th[2], f0[0], th[3], th[4], f0[1]]
    sol = least_squares(res, p0, xtol=1e-15, ftol=1e-15, gtol=1e-15, method="lm")
    np.testing.assert_allclose(fr, [sol.x[3], sol.x[6]], atol=1e-8 / T)
    assert l == pytest.approx((sol.fun ** 2).sum(), rel=1e-10)
    # stationary point: the oracle's own gradient vanishes there
    _, g = oracle.tuple_grad(t, y, sigma, [list(fr)])
    _, g0 = oracle.tuple_grad(t, y, sigma, [list(f0)])
    assert np.abs(g).max() < 1e-6 * np.abs(g0).max()


# ----------------------------------------------------------------------------
# Section 6.1 look-alike: aliasing makes the single-frequency periodogram peak
# at a wrong frequency between the two true ones.

def test_section61_lookalike():
    spec = json.load(open(os.path.join(GOLDEN, "sec61_lookalike.json")))
    rng = np.random.Generator(np.random.PCG64(spec["seed"]))
    per, win = spec["gap_period"], spec["window"]
    t = []
    while len(t) < spec["N"]:
        c = rng.uniform(0, spec["span"])
        if c % per < win:
            t.append(c)
    t = np.sort(np.asarray(t))
    ft = spec["true_freqs"]
    y = sum(np.sin(2 * np.pi * f * t + ph) for f, ph in zip(ft, spec["phases"]))
    sigma = np.full(t.size, spec["noise_rel"])
    y = y + sigma * rng.standard_normal(t.size)
    f = np.linspace(0.5, 1.5, 2001)
    z, c2 = oracle.periodogram(t, y, sigma, [], f)
    assert abs(f[np.argmax(z)] - spec["expected_single_peak"]) < 0.01
    # the true pair explains the data better than any pair containing the
    # spurious peak frequency (grid search over the partner)
    zt, _ = oracle.tuple_eval(t, y, sigma, [ft])
    partners = np.linspace(0.5, 1.5, 201)
    zalt, _ = oracle.tuple_eval(t, y, sigma, [[spec["expected_single_peak"], p] for p in partners])
    assert zt[0] > zalt.max()


# ----------------------------------------------------------------------------
# Planted mistakes must be caught by the pins above.

@pytest.mark.parametrize("mutant", [0, 1, 2, 3])
def test_planted_oracle_mistakes_are_caught(mutant):
    o = oracle.Oracle(mutant=mutant) if mutant else oracle.Oracle()
    t, y, sigma = _series(1)
    f = np.linspace(0.003, 0.9, 57)
    z, _ = oracle.periodogram(t, y, sigma, [], f, lib=o.lib)
    zg = gls_z(t, y, sigma, f)
    gls_ok = np.max(np.abs(z - zg) / np.maximum(zg, 1e-3 * zg.max())) < 1e-10
    tg = np.sort(_rng(3).uniform(0, 30, 40)) + 1.0
    yy = 2 + np.sin(2 * np.pi * 0.3 * tg + 0.2)
    # phase sign error: visible in the fitted sine coefficient
    _, _, coef = oracle.periodogram(tg, yy, np.ones(40), [], [0.3], lib=o.lib, want_coef=True)
    coef_ok = abs(coef[0, 1] - np.cos(0.2)) < 1e-9
    assert (gls_ok and coef_ok) == (mutant == 0)
