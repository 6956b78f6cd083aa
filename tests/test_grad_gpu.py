"""GPU parity of the frequency derivative dz/df of the residual periodogram
(fredec_periodogram_grad / _grad_dev) against the oracle's envelope-theorem
gradient and against central finite differences of the oracle's z (step
1e-7/T), in FP64 and mixed precision, through the C ABI.

Bound per bin (the conditioning reading of the z tests carried over): with
g* the oracle's gradient, floor = 1e-3 max |g*| and ratio the oracle's
smaller remaining-norm ratio of the two trial columns,
    |g - g*| <= tol max(|g*|, floor) + C_COND EPS64 sqrt(N) 2 pi T chi2_base / ratio^2,
since g = dz/df is at most about 2 pi T chi2_base (z <= chi2_base / 2 moves by
that over a frequency step of 1/T).  tol = 1e-8 (FP64), 1e-4 (mixed: the
t'-weighted sums in FP32 carry the rounding of the FP32 cos/sin values, about
1e-7 of the largest |dz/df|, i.e. 1e-4 at the floor); bins with a condition
above 1e12 (ratio < 1e-6) are left out, as for z.  Against central finite
differences of the oracle's z (step 1e-7/T) the FP64 path meets 1e-6 plus the
same conditioning term (the differences inherit the oracle's own rounding,
amplified near a base frequency).
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import C_COND, EPS64, MIN_RATIO_COND, cond_parity, ensure_built

pytestmark = pytest.mark.gpu

TOL_G = {"fp64": 1e-8, "mixed": 1e-4}
TOL_FD = {"fp64": 1e-6, "mixed": 1e-4}
TOL_Z = {"fp64": 1e-10, "mixed": 1e-5}


@pytest.fixture(scope="module")
def F():
    ensure_built()
    import paper_1309_0100_b300 as F
    return F


# The mixed path re-evaluates its ill-conditioned bins in float-float
# arithmetic, whose sin/cos carry up to about 1e-15 absolute error (FP64: 1.1e-16);
# its conditioning term uses this epsilon.
EPS_FF = 2e-15


def grad_parity(g, gr, ratio, chi2, T, N, tol, eps=EPS64, extra=0.0):
    """Element-wise |g - g*| <= tol max(|g*|, floor) + C_COND eps sqrt(N) 2 pi T
    chi2 / ratio^2 + extra (extra: a per-bin allowance for the reference's own
    error, e.g. the rounding of finite differences)."""
    g, gr, ratio = (np.asarray(a, dtype=np.float64) for a in (g, gr, ratio))
    keep = ratio >= MIN_RATIO_COND
    den = np.maximum(np.abs(gr), 1e-3 * np.max(np.abs(gr)))
    bound = tol * den + C_COND * eps * np.sqrt(N) * 2 * np.pi * T * chi2 / np.maximum(ratio, MIN_RATIO_COND) ** 2 \
        + extra
    d = np.abs(g - gr)
    bad = keep & ~(d <= bound)
    return {"ok": not bad.any(), "excluded": int((~keep).sum()), "rel": float(np.max(d[keep] / den[keep])),
            "worst": float(np.max(d[keep] / bound[keep])), "first_bad": int(np.flatnonzero(bad)[0]) if bad.any() else -1}


def _check(F, s, prec, f0, df, nf):
    f = f0 + df * np.arange(nf)
    T = s.t.max() - s.t.min()
    z, g, info = F.periodogram_grad(s.t, s.y, s.sigma, s.base_freqs, f0, df, nf, precision=prec, want_info=True)
    zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, want_ratio=True)
    gr = oracle.periodogram_grad(s.t, s.y, s.sigma, s.base_freqs, f)
    rz = cond_parity(z, zr, ratio, c2, TOL_Z[prec], s.N)
    assert rz["ok"], ("z", prec, rz)
    rg = grad_parity(g, gr, ratio, c2, T, s.N, TOL_G[prec], eps=EPS64 if prec == "fp64" else EPS_FF)
    assert rg["ok"], ("dz/df", prec, rg)
    assert info[0] == pytest.approx(c2, rel=1e-11)
    return z, g, zr, gr, ratio, rg


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nb,N,nf", [(0, 60, 300), (1, 257, 700), (3, 1000, 640), (5, 300, 513), (12, 90, 77),
                                     (2, 3000, 200)])
def test_grad_vs_oracle(F, prec, nb, N, nf):
    s = synth.small_series(700 + nb, N=N, n_base=nb, nf=nf, span=300.0, fmax=0.8)
    _, _, _, _, _, rg = _check(F, s, prec, s.grid.f0, s.grid.df, nf)
    print(f"dz/df {prec} nb={nb} N={N}: largest relative error {rg['rel']:.2e}, error / bound {rg['worst']:.3f}")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_grad_vs_finite_differences(F, prec):
    """Central differences of the oracle's z at step h = 1e-7/T around
    sampled bins (peaks, slopes, troughs, and bins next to a base frequency)
    agree with dz/df to 1e-6 (FP64; mixed 1e-4) of max(|dz/df|, 1e-3 max
    |dz/df|), plus the conditioning term next to a base frequency and twice
    the differences' own rounding, estimated as |FD(h) - FD(2h)| (the
    truncation error, about (2 pi 1e-7)^2 / 6 of dz/df, is negligible)."""
    s = synth.small_series(711, N=500, n_base=2, nf=4000, span=400.0, fmax=0.5)
    T = s.t.max() - s.t.min()
    f = s.grid.array()
    z, g = F.periodogram_grad(s.t, s.y, s.sigma, s.base_freqs, s.grid.f0, s.grid.df, s.grid.nf, precision=prec)
    gr = oracle.periodogram_grad(s.t, s.y, s.sigma, s.base_freqs, f)
    near = np.clip([int(np.argmin(np.abs(f - b))) + d for b in s.base_freqs for d in (-3, 3)], 5, f.size - 6)
    picks = np.unique(np.concatenate([np.arange(5, f.size - 5, 157), near, [int(np.argmax(z))]]))
    h = 1e-7 / T

    def fd_at(step):
        zp, c2 = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f[picks] + step)
        zm, _ = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f[picks] - step)
        return (zp - zm) / (2 * step), c2

    fd, c2 = fd_at(h)
    noise = 2 * np.abs(fd - fd_at(2 * h)[0])
    _, _, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f[picks], want_ratio=True)
    r = grad_parity(g[picks], fd, ratio, c2, T, s.N, TOL_FD[prec], eps=EPS64 if prec == "fp64" else EPS_FF,
                    extra=noise)
    assert r["ok"], (prec, r, int(picks[r["first_bad"]]) if r["first_bad"] >= 0 else -1)
    # the oracle's own gradient agrees with its finite differences (the FP64 bar)
    assert grad_parity(gr[picks], fd, ratio, c2, T, s.N, 1e-6, extra=noise)["ok"]



@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_grad_next_to_base_frequency(F, prec):
    """Uniform grids closing in on a base frequency by factors of ten: every
    bin with a condition below 1e12 meets the bound (on the mixed path these
    bins are re-evaluated in float-float, dz/df included)."""
    s = synth.small_series(712, N=600, n_base=2, nf=10, span=400.0, fmax=0.5)
    T = s.t.max() - s.t.min()
    for k in range(1, 6):
        df = 10.0 ** -k / T
        f0 = s.base_freqs[0] + 0.37 * df - 32 * df
        _check(F, s, prec, f0, df, 65)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_grad_z_equals_periodogram(F, prec):
    """The z of the derivative pass is the periodogram's z; the device variant
    gives the host variant's results bit for bit; a polynomial trend works."""
    import torch
    s = synth.small_series(713, N=800, n_base=3, nf=5000, span=500.0)
    z, g = F.periodogram_grad(s.t, s.y, s.sigma, s.base_freqs, s.grid.f0, s.grid.df, s.grid.nf, precision=prec)
    zp = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, s.grid.array(), precision=prec)
    floor = 1e-3 * np.max(zp)
    assert np.max(np.abs(z - zp) / np.maximum(zp, floor)) < 2 * TOL_Z[prec]
    dev = torch.device("cuda:0")
    tt = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64), device=dev)
    r = F.periodogram_grad_dev(tt(s.t), tt(s.y), tt(s.sigma), tt(s.base_freqs), s.grid.f0, s.grid.df, s.grid.nf,
                               precision=prec)
    torch.cuda.synchronize()
    assert np.array_equal(r["z"].cpu().numpy(), z) and np.array_equal(r["dzdf"].cpu().numpy(), g)
    # trend: finite differences of the oracle's trend periodogram
    zt, gt = F.periodogram_grad(s.t, s.y, s.sigma, s.base_freqs, s.grid.f0, s.grid.df, 400, precision=prec, trend=2)
    f = s.grid.array()[:400]
    T = s.t.max() - s.t.min()
    h = 1e-7 / T
    picks = np.arange(3, 400, 37)
    fdt = lambda step: (oracle.periodogram_trend(s.t, s.y, s.sigma, s.base_freqs, 2, f[picks] + step)[0] -
                        oracle.periodogram_trend(s.t, s.y, s.sigma, s.base_freqs, 2, f[picks] - step)[0]) / (2 * step)
    fd = fdt(h)
    noise = 2 * np.abs(fd - fdt(2 * h))
    ztr, c2t, rt = oracle.periodogram_trend(s.t, s.y, s.sigma, s.base_freqs, 2, f, want_ratio=True)
    rz = cond_parity(zt, ztr, rt, c2t, TOL_Z[prec], s.N)
    assert rz["ok"], rz
    r = grad_parity(gt[picks], fd, rt[picks], c2t, T, s.N, TOL_FD[prec], eps=EPS64 if prec == "fp64" else EPS_FF,
                    extra=noise)
    assert r["ok"], r


def test_grad_full_size_sampled(F):
    """The N = 2000, 1e6-frequency residual periodogram: z and dz/df on the
    whole grid, checked against the oracle on a strided sample plus the
    neighbourhoods of the highest peaks; at each peak dz/df changes sign."""
    s = synth.residual_n2000_p7()
    f = s.grid.array()
    T = s.t.max() - s.t.min()
    for prec in ("fp64", "mixed"):
        z, g = F.periodogram_grad(s.t, s.y, s.sigma, s.base_freqs, s.grid.f0, s.grid.df, s.grid.nf, precision=prec)
        top = np.argsort(z)[-3:]
        idx = np.unique(np.concatenate([np.arange(0, f.size, 9973)] + [np.arange(j - 2, j + 3) for j in top]))
        zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f[idx], want_ratio=True)
        gr = oracle.periodogram_grad(s.t, s.y, s.sigma, s.base_freqs, f[idx])
        rg = grad_parity(g[idx], gr, ratio, c2, T, s.N, TOL_G[prec], eps=EPS64 if prec == "fp64" else EPS_FF)
        assert rg["ok"], (prec, rg)
        for j in top:
            if 0 < j < f.size - 1 and z[j] >= z[j - 1] and z[j] >= z[j + 1]:
                assert g[j - 1] > 0 > g[j + 1] or g[j - 1] >= 0 >= g[j + 1], (prec, j)


def test_grad_tail_split(F):
    """A two-set launch whose last wave of CTAs is part-filled (1954 blocks of
    128 frequencies on two CTAs per SM) runs its last blocks as an even split
    of their tiles over a wave of tail CTAs: z and dz/df on the bins of the
    tail agree with the oracle, and two calls agree bit for bit."""
    s = synth.small_series(715, N=2000, n_base=3, nf=250_000, span=3000.0, fmax=2.0)
    f = s.grid.array()
    T = s.t.max() - s.t.min()
    runs = [F.periodogram_grad(s.t, s.y, s.sigma, s.base_freqs, s.grid.f0, s.grid.df, s.grid.nf, precision="mixed")
            for _ in range(2)]
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    z, g = runs[0]
    tail = int(0.12 * f.size)
    idx = np.unique(np.concatenate([np.linspace(f.size - tail, f.size - 1, 200).astype(int),
                                    np.linspace(0, f.size - tail - 1, 50).astype(int)]))
    zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f[idx], want_ratio=True)
    gr = oracle.periodogram_grad(s.t, s.y, s.sigma, s.base_freqs, f[idx])
    rz = cond_parity(z[idx], zr, ratio, c2, TOL_Z["mixed"], s.N)
    assert rz["ok"], rz
    rg = grad_parity(g[idx], gr, ratio, c2, T, s.N, TOL_G["mixed"], eps=EPS_FF)
    assert rg["ok"], rg


def test_grad_argument_checks(F):
    import ctypes
    s = synth.small_series(714, N=100, n_base=2, nf=50)
    base = np.array([s.base_freqs[0], s.base_freqs[0]])
    with pytest.raises(F.FredecError) as ei:                  # singular base model
        F.periodogram_grad(s.t, s.y, s.sigma, base, s.grid.f0, s.grid.df, s.grid.nf)
    assert ei.value.code == 4
    L = F.lib()
    z = np.empty(50)
    g = np.empty(50)
    dp = ctypes.POINTER(ctypes.c_double)
    args = lambda o: (s.t.ctypes.data_as(dp), s.y.ctypes.data_as(dp), s.sigma.ctypes.data_as(dp), s.N,
                      s.base_freqs.ctypes.data_as(dp), len(s.base_freqs), s.grid.f0, s.grid.df, 50, ctypes.byref(o),
                      z.ctypes.data_as(dp), g.ctypes.data_as(dp), None)
    for kw in ({"topk": 3}, {"statistic": 1}, {"fpt": 7}):
        o = F._opts("fp64", kw.get("topk", 0), kw.get("fpt", 0), 0, 0.0, 0, kw.get("statistic", 0))
        assert L.fredec_periodogram_grad(*args(o)) == 1, kw
    o = F._opts("fp64")
    bad = s.sigma.copy()
    bad[3] = -1.0
    assert L.fredec_periodogram_grad(s.t.ctypes.data_as(dp), s.y.ctypes.data_as(dp), bad.ctypes.data_as(dp), s.N,
                                     s.base_freqs.ctypes.data_as(dp), len(s.base_freqs), s.grid.f0, s.grid.df, 50,
                                     ctypes.byref(o), z.ctypes.data_as(dp), g.ctypes.data_as(dp), None) == 1
