"""GPU parity of the polynomial-trend base model (the constant of Eq. H0
extended to a time polynomial, Sect. 2) and of the log-form statistic of
Eq. zpowrel, against the FP64 oracle.

Tolerances as for the constant base: z relative (floor 1e-3 of the highest
peak) 1e-10 for the FP64 path, 1e-5 for the mixed path, over bins whose trial
columns keep >= 1% of their norm after projection (low frequencies are nearly
collinear with the polynomial columns and are excluded, counted)."""
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


def _trend_series(seed, N, nb, trend, nf, span=300.0, fmax=1.0):
    s = synth.small_series(seed, N=N, n_base=nb, nf=nf, span=span, fmax=fmax)
    rng = np.random.default_rng(seed)
    u = (s.t - span / 2) / (span / 2)
    s.y = s.y + sum(rng.normal(0, 3) * u ** d for d in range(1, trend + 1))
    return s


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("trend,nb,N,nf", [(1, 0, 200, 700), (2, 0, 333, 1000), (3, 0, 150, 513),
                                           (1, 2, 400, 900), (2, 3, 260, 777), (3, 5, 500, 1201),
                                           (1, 11, 120, 300)])
def test_trend_parity(F, prec, trend, nb, N, nf):
    s = _trend_series(300 + 10 * trend + nb, N, nb, trend, nf)
    f = s.grid.array()
    zr, c2, ratio = oracle.periodogram_trend(s.t, s.y, s.sigma, s.base_freqs, trend, f, want_ratio=True)
    z, top, info = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision=prec, topk=5, want_info=True,
                                 trend=trend)
    r = cond_parity(z, zr, ratio, c2, TOL[prec], s.N)
    assert r["ok"], r
    assert info[0] == pytest.approx(c2, rel=1e-11)
    ref_top = local_max_topk(zr, 5)
    zs = sorted(zr[[j for j in ref_top if j >= 0]], reverse=True)
    if np.all(np.abs(np.diff(zs)) > 10 * TOL[prec] * zs[0]):
        assert list(top) == ref_top


def _dlog_dz(z, chi2, N, nb, trend):
    """d(log form)/dz = N_H / (chi2_base - 2 z): scales the conditioning term
    of the difference form to the log form."""
    return (N - 3 * (nb + 1) - 1 - trend) / (chi2 - 2.0 * np.asarray(z))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("trend,nb", [(0, 0), (0, 2), (2, 1)])
def test_log_form_statistic(F, prec, trend, nb):
    s = _trend_series(400 + nb, 300, nb, trend, 800)
    f = s.grid.array()
    zr, c2, ratio = oracle.periodogram_trend(s.t, s.y, s.sigma, s.base_freqs, trend, f, want_ratio=True)
    zl_ref = oracle.log_form(zr, c2, s.t.size, nb + 1, trend)
    zl, top = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision=prec, topk=5, trend=trend,
                            statistic="log")
    zd, topd = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision=prec, topk=5, trend=trend)
    r = cond_parity(zl, zl_ref, ratio, c2, TOL[prec], s.N, cond_scale=_dlog_dz(zr, c2, s.N, nb, trend))
    assert r["ok"], r
    assert list(top) == list(topd)     # the log form is monotone in z


def test_trend_device_generic_batch_noalloc(F):
    import torch
    dev = torch.device("cuda:0")
    s = _trend_series(500, 700, 2, 2, 2000)
    f = s.grid.array()
    zr, c2, ratio = oracle.periodogram_trend(s.t, s.y, s.sigma, s.base_freqs, 2, f, want_ratio=True)
    tt = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64), device=dev)
    r = F.periodogram_dev(tt(s.t), tt(s.y), tt(s.sigma), tt(s.base_freqs), s.grid.f0, s.grid.df, s.grid.nf,
                          precision="fp64", trend=2)
    assert cond_parity(r["z"].cpu().numpy(), zr, ratio, c2, TOL["fp64"], s.N)["ok"]
    # non-uniform grid (the generic kernel)
    fg = np.sort(np.random.default_rng(1).uniform(0.001, 1.0, 500))
    zg_r, cg, rg = oracle.periodogram_trend(s.t, s.y, s.sigma, s.base_freqs, 2, fg, want_ratio=True)
    zg = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, fg, precision="fp64", trend=2)
    assert cond_parity(zg, zg_r, rg, cg, TOL["fp64"], s.N)["ok"]
    # batch: every series with the same trend degree, log form
    ser = [_trend_series(600 + k, 150 + 97 * k, k % 3, 1, 300 + 50 * k) for k in range(5)]
    zb, zo, topb = F.periodogram_batch(ser, precision="mixed", topk=3, trend=1, statistic="log")
    for k, sk in enumerate(ser):
        fk = sk.grid.array()
        zk, ck, rk = oracle.periodogram_trend(sk.t, sk.y, sk.sigma, sk.base_freqs, 1, fk, want_ratio=True)
        zlk = oracle.log_form(zk, ck, sk.t.size, len(sk.base_freqs) + 1, 1)
        r = cond_parity(zb[zo[k]:zo[k] + fk.size], zlk, rk, ck, TOL["mixed"], sk.N,
                        cond_scale=_dlog_dz(zk, ck, sk.N, len(sk.base_freqs), 1))
        assert r["ok"], (k, r)
    # the no-allocation entry point
    lib = F.lib()
    zn = torch.empty(s.grid.nf, dtype=torch.float64, device=dev)
    o = F._opts("fp64", 0, 0, 0, 0.0, 2, 0)
    dt, dy, ds, db = tt(s.t), tt(s.y), tt(s.sigma), tt(s.base_freqs)   # alive until the stream is synchronised
    F._check(lib.fredec_periodogram_noalloc_dev(F._dptr(dt), F._dptr(dy), F._dptr(ds), s.t.size, F._dptr(db),
                                                len(s.base_freqs), s.grid.f0, s.grid.df, s.grid.nf,
                                                F.ctypes.byref(o), F._dptr(zn), None, None))
    torch.cuda.synchronize()
    assert cond_parity(zn.cpu().numpy(), zr, ratio, c2, TOL["fp64"], s.N)["ok"]


@pytest.mark.parametrize("trend", [1, 3])
def test_trend_invariance_on_gpu(F, trend):
    s = _trend_series(700, 500, 1, 0, 1500)
    f = s.grid.array()
    u = (s.t - 100.0) / 77.0
    y2 = s.y + sum(c * u ** d for d, c in enumerate([5.0, -2.0, 0.7, 0.3][:trend + 1]))
    z1 = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision="fp64", trend=trend)
    z2 = F.periodogram(s.t, y2, s.sigma, s.base_freqs, f, precision="fp64", trend=trend)
    assert rel_err(z2, z1) < 1e-8


def test_trend_argument_checks(F):
    s = synth.small_series(1, N=40, n_base=11, nf=10)
    f = s.grid.array()
    with pytest.raises(F.FredecError):
        F.periodogram(s.t, s.y, s.sigma, [], f, trend=4)
    with pytest.raises(F.FredecError):          # 1 + 3 + 22 columns > 25
        F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, trend=3)
    with pytest.raises(F.FredecError):          # N_H <= 0 for the log form
        F.periodogram(s.t[:7], s.y[:7], s.sigma[:7], [], f, trend=3, statistic="log")
