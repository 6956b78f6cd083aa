"""Pins of the oracle's polynomial-trend base model (Sect. 2: the constant of
Eq. H0 extended to a time polynomial) and of the log-form statistic of
Eq. zpowrel."""
import numpy as np
import pytest

import oracle
from synth import small_series


def _lstsq_chi2(A, b):
    x, *_ = np.linalg.lstsq(A, b, rcond=None)
    r = b - A @ x
    return float(r @ r)


@pytest.mark.parametrize("trend", [1, 2, 3])
@pytest.mark.parametrize("n_base", [0, 2])
def test_trend_periodogram_matches_lstsq(trend, n_base):
    s = small_series(seed=40 + trend, N=36, n_base=n_base, span=60.0)
    f = np.linspace(0.013, 0.9, 23)
    z, c2 = oracle.periodogram_trend(s.t, s.y, s.sigma, s.base_freqs, trend, f)
    sw = 1.0 / s.sigma
    tau = s.t / 60.0
    cols = [sw * tau ** d for d in range(trend + 1)]
    for g in s.base_freqs:
        cols += [sw * np.cos(2 * np.pi * g * s.t), sw * np.sin(2 * np.pi * g * s.t)]
    B = np.array(cols).T
    b = sw * s.y
    cb = _lstsq_chi2(B, b)
    assert c2 == pytest.approx(cb, rel=1e-10)
    for j, fj in enumerate(f):
        A = np.column_stack([B, sw * np.cos(2 * np.pi * fj * s.t), sw * np.sin(2 * np.pi * fj * s.t)])
        assert z[j] == pytest.approx(0.5 * (cb - _lstsq_chi2(A, b)), rel=1e-8, abs=1e-10 * cb)


@pytest.mark.parametrize("trend", [1, 2, 3])
def test_trend_invariance(trend):
    # adding any polynomial of degree <= trend to y changes neither z nor chi2
    s = small_series(seed=50 + trend, N=120, n_base=1, span=300.0)
    f = np.linspace(0.005, 0.5, 80)
    z0, c0 = oracle.periodogram_trend(s.t, s.y, s.sigma, s.base_freqs, trend, f)
    rng = np.random.default_rng(trend)
    coef = rng.normal(0, 5, trend + 1)
    u = (s.t - 150.0) / 150.0
    y2 = s.y + sum(c * u ** d for d, c in enumerate(coef))
    z1, c1 = oracle.periodogram_trend(s.t, y2, s.sigma, s.base_freqs, trend, f)
    assert c1 == pytest.approx(c0, rel=1e-9)
    np.testing.assert_allclose(z1, z0, rtol=1e-7, atol=1e-9 * c0)


def test_trend_zero_is_the_constant_base():
    s = small_series(seed=3, N=80, n_base=1)
    f = np.linspace(0.01, 0.5, 50)
    z0, c0 = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f)
    zt, ct = oracle.periodogram_trend(s.t, s.y, s.sigma, s.base_freqs, 0, f)
    assert ct == c0
    np.testing.assert_array_equal(zt, z0)


def test_linear_trend_is_removed_only_with_a_trend_base():
    # a strong linear drift leaks into the lowest frequencies of the constant
    # base periodogram; with a degree-1 base it is gone
    s = small_series(seed=8, N=200, n_base=0, span=400.0)
    y = s.y + 0.05 * (s.t - 200.0)
    f = np.linspace(0.5 / 400, 0.02, 40)
    zc, _ = oracle.periodogram_trend(s.t, y, s.sigma, [], 0, f)
    zt, _ = oracle.periodogram_trend(s.t, y, s.sigma, [], 1, f)
    zref, _ = oracle.periodogram_trend(s.t, s.y, s.sigma, [], 1, f)
    assert zc[0] > 10 * zt[0]
    np.testing.assert_allclose(zt, zref, rtol=1e-6, atol=1e-9 * zref.max())


def test_log_form_against_fitted_chi2():
    # (N_H/2) ln(l_base / l_new) with l_new fitted directly (constant base,
    # one trial frequency: N_H = N - 3*1 - 1)
    s = small_series(seed=11, N=90, n_base=0, span=200.0)
    f = np.array([0.0371, 0.1234, 0.31])
    z, c2 = oracle.periodogram(s.t, s.y, s.sigma, [], f)
    zl = oracle.log_form(z, c2, s.t.size, 1)
    for j, fj in enumerate(f):
        l_new = oracle.tuple_l(s.t, s.y, s.sigma, [fj])
        assert zl[j] == pytest.approx(0.5 * (s.t.size - 4) * np.log(c2 / l_new), rel=1e-9)
