"""GPU parity of the residual periodogram (FP64 and mixed paths) against the
FP64 CPU oracle, through the C ABI.

Tolerances (z relative, with the floor of 1e-3 of the highest peak):
FP64 path 1e-10, mixed path 1e-5, plus a term that scales with the
conditioning of the bin's two trial columns (helpers.cond_parity: an FP64
normal-equation method loses about EPS64 sqrt(N) / ratio^2 of chi2_base).
Only bins whose 2x2 system has a condition number above 1e12 (oracle ratio
< 1e-6) are left out; every other bin is compared element by element.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import cond_parity, ensure_built, local_max_topk, rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5}


def _assert_cond(z, zr, ratio, chi2, prec, N, what=""):
    r = cond_parity(z, zr, ratio, chi2, TOL[prec], N)
    assert r["ok"], (prec, what, r)
    return r


@pytest.fixture(scope="module")
def F():
    ensure_built()
    import paper_1309_0100_b300 as F
    return F


def _compare(F, s, f, prec, topk=5, **kw):
    zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, want_ratio=True)
    z, top, info = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision=prec, topk=topk, want_info=True, **kw)
    r = _assert_cond(z, zr, ratio, c2, prec, s.N)
    assert info[0] == pytest.approx(c2, rel=1e-11)
    return z, zr, top, r["rel_err"]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nb,N,nf", [(0, 37, 300), (1, 129, 257), (2, 300, 1000), (3, 1000, 700), (5, 260, 333),
                                     (7, 90, 150), (12, 64, 101),
                                     # prep paths: one point per thread up to 16 x 128 points, then the
                                     # per-width loop kernel (base widths 9 and 11)
                                     (4, 777, 400), (5, 2048, 200), (5, 2049, 200)])
def test_parity_small(F, prec, nb, N, nf):
    s = synth.small_series(100 + nb, N=N, n_base=nb, nf=nf, span=200.0, fmax=1.5)
    f = s.grid.array()
    z, zr, top, _ = _compare(F, s, f, prec)
    ref_top = local_max_topk(zr, 5)
    # peak indices must agree wherever the oracle's ranking is not a near-tie
    zs = sorted(zr[[j for j in ref_top if j >= 0]], reverse=True)
    gaps = np.diff(zs) if len(zs) > 1 else np.array([-1.0])
    if np.all(np.abs(gaps) > 10 * TOL[prec] * zs[0]):
        assert list(top) == ref_top


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("N", [5000, 40000, 70000])
def test_prep_paths_long_series(F, prec, N):
    # the base fit of one series: a thread-block cluster of up to 16 CTAs for
    # N <= 65536 (5000: about 2.5 points per thread; 40000: about 20), the
    # one-warp chunk kernels above; parity of z and chi2_base either way
    s = synth.small_series(900 + N % 97, N=N, n_base=3, nf=48, span=3000.0, fmax=0.5)
    _compare(F, s, s.grid.array(), prec)


def _long_series_errors(F, N, nb):
    s = synth.small_series(40 + nb, N=N, n_base=nb, nf=300, span=3000.0, fmax=2.0)
    f = s.grid.array()
    zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, want_ratio=True)
    z = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision="mixed", topk=0)
    _assert_cond(z, zr, ratio, c2, "mixed", s.N, f"N={N}")
    return np.abs(z - zr) / np.maximum(zr, 1e-3 * zr.max())


@pytest.mark.parametrize("N,nb", [(70000, 3), (100000, 5)])
def test_mixed_long_series_error_distribution(F, N, nb):
    """Long series (more than 64 tiles per warp) take the kernels whose
    residual sums end in compensated CTA-level totals: beyond the element-wise
    bound, the bulk of the bins keeps the error of the FP32 block sums
    (measured: medians 2.0e-7 and 2.5e-7, 99th percentiles 1.6e-6 and 2.1e-6).
    With one FP32 running sum per warp over all tiles the N = 7e4 case gave a
    median of 5.0e-7 and a 99th percentile of 3.5e-6, and the N = 1e5 case
    broke the element-wise bound (2.0e-5 at one bin)."""
    e = _long_series_errors(F, N, nb)
    assert np.median(e) < 4e-7 and np.quantile(e, 0.99) < 3e-6, (np.median(e), np.quantile(e, 0.99))


@pytest.mark.parametrize("N,nb,fpt,warps,nf", [(2000, 3, 10, 4, 1_000_000), (2000, 3, 6, 4, 300_000),
                                               (2000, 3, 10, 2, 1_000_000), (777, 1, 12, 4, 300_000),
                                               (70000, 3, 6, 4, 100_000)])
def test_tail_split(F, N, nb, fpt, warps, nf):
    """Grids whose last wave of CTAs is part-filled run their last blocks as an
    even split of the blocks' tiles over a wave of tail CTAs; a CTA that
    completes a shared block adds the parts in a fixed order (the last case
    with compensated residual totals).  The bins of the tail (and a sample of
    the rest) agree with the oracle, two calls agree bit for bit, and so do the
    host-pointer calls with a pageable and a page-locked z_out (whose kernels
    write z to host memory themselves)."""
    import torch
    s = synth.small_series(61 + nb, N=N, n_base=nb, nf=nf, span=3000.0, fmax=2.0)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda:0")
    t, y, sg, b = (dev(a) for a in (s.t, s.y, s.sigma, s.base_freqs))
    zs = []
    for _ in range(2):
        z = torch.empty(nf, dtype=torch.float64, device="cuda:0")
        F.periodogram_dev(t, y, sg, b, s.grid.f0, s.grid.df, nf, precision="mixed", fpt=fpt, warps=warps, out=z)
        zs.append(z.cpu().numpy())
    assert np.array_equal(zs[0], zs[1])
    f = s.grid.array()
    zh = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision="mixed", fpt=fpt, warps=warps)
    pinned = torch.full((nf,), -1.0, dtype=torch.float64).pin_memory().numpy()
    F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision="mixed", fpt=fpt, warps=warps, out=pinned)
    assert np.array_equal(pinned, zh)
    tail = int(0.12 * nf)
    ns = 60 if N > 10000 else 240
    idx = np.unique(np.concatenate([np.linspace(nf - tail, nf - 1, ns).astype(int),
                                    np.linspace(0, nf - tail - 1, ns // 4).astype(int)]))
    zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, s.grid.array()[idx], want_ratio=True)
    r = cond_parity(zs[0][idx], zr, ratio, c2, TOL["mixed"], s.N,
                    floor_frac=1e-3 * np.max(zs[0]) / max(np.max(zr), 1e-300))
    assert r["ok"], r


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_seasonal_n200_full_grid(F, prec):
    s = synth.seasonal_n200()
    f = s.grid.array()
    z, zr, top, err = _compare(F, s, f, prec)
    assert list(top) == local_max_topk(zr, 5)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_residual_n2000_full_size_sampled(F, prec):
    """Full 1e6-point grid on the GPU in the benchmark launch shape (the shapes
    its tuner picks: 6 frequencies per thread in mixed precision, 4 in FP64,
    4 warps); the oracle evaluates a strided sample plus the neighbourhoods of
    the top-5 peaks."""
    s = synth.residual_n2000_p7()
    f = s.grid.array()
    z, top = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision=prec, topk=5,
                           fpt=6 if prec == "mixed" else 4, warps=4)
    idx = np.unique(np.concatenate([np.arange(0, f.size, 997), np.arange(f.size - 3, f.size)]))
    zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f[idx], want_ratio=True)
    _assert_cond(z[idx], zr, ratio, c2, prec, s.N)
    for j in top:
        nb = np.arange(max(j - 2, 0), min(j + 3, f.size))
        zn, _ = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f[nb])
        assert nb[np.argmax(zn)] == j
        assert abs(z[j] - zn[np.argmax(zn)]) <= TOL[prec] * zn.max()
    if prec == "mixed":
        z64, top64 = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision="fp64", topk=5)
        assert list(top) == list(top64)
        assert rel_err(z, z64) < TOL["mixed"]


def test_edge_grids(F):
    s = synth.small_series(7, N=50, n_base=2)
    for f in [np.array([0.0]), np.array([0.37]), np.linspace(0.0, 0.5, 33), np.array([s.base_freqs[0], 0.2])]:
        for prec in ("fp64", "mixed"):
            z = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision=prec)
            zr, c2 = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f)
            assert np.all(np.abs(z - zr) <= 1e-8 * c2 + TOL[prec] * np.abs(zr)), (f, prec, z, zr)
    z = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, np.zeros(0))
    assert z.size == 0


def test_non_uniform_grid(F):
    s = synth.small_series(8, N=120, n_base=1)
    f = np.sort(np.random.default_rng(3).uniform(0.01, 1.0, 400))
    zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, want_ratio=True)
    z = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f)
    _assert_cond(z, zr, ratio, c2, "fp64", s.N)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_grid_nearly_uniform(F, prec):
    # the host API starts the uniform-grid pipeline when 65 evenly spaced
    # entries fit f0 + j df, and checks every entry meanwhile: one entry moved
    # between the sampled ones must still give the periodogram at the
    # frequencies given (the generic-grid kernel), a NaN there an error
    s = synth.small_series(9, N=300, n_base=2, nf=6401, fmax=1.0)
    f = s.grid.array().copy()
    f[1234] += 0.3 * s.grid.df                     # 1234 is not a multiple of 6400/64
    zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, want_ratio=True)
    z, top = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision=prec, topk=3)
    _assert_cond(z, zr, ratio, c2, prec, s.N)
    zu = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, s.grid.array(), precision=prec)
    assert abs(z[1234] - zu[1234]) > 1e-6 * abs(zu[1234])   # not the uniform grid's value
    f[2345] = np.nan
    with pytest.raises(F.FredecError):
        F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision=prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_page_locked_output(F, prec):
    # a page-locked z_out is written by the kernels during the computation
    # (no copy afterwards); a fine grid around the base frequencies makes the
    # mixed path re-evaluate flagged bins, which write it too
    import torch
    s = synth.small_series(21, N=800, n_base=2, nf=30, span=2000.0, fmax=0.05)
    lo, hi = min(s.base_freqs) * 0.9, max(s.base_freqs) * 1.1
    f = lo + (hi - lo) / 4000 * np.arange(4001)
    zp, topp = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision=prec, topk=5)
    pinned = torch.full((f.size,), -1.0, dtype=torch.float64).pin_memory().numpy()
    zz, top = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision=prec, topk=5, out=pinned)
    assert np.array_equal(zz, zp) and np.array_equal(pinned, zp) and list(top) == list(topp)
    zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, want_ratio=True)
    _assert_cond(zz, zr, ratio, c2, prec, s.N)


def test_singular_base_and_determinism(F):
    s = synth.small_series(9, N=80, n_base=2)
    with pytest.raises(F.FredecError) as ei:
        F.periodogram(s.t, s.y, s.sigma, [0.1, 0.1], s.grid.array())
    assert ei.value.code == 4
    f = s.grid.array()
    for prec in ("fp64", "mixed"):
        a = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision=prec)
        b = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision=prec)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_launch_shapes_agree(F, prec):
    """Every compiled (frequencies per thread, warps) shape meets the bound
    against the oracle on every bin, and the shapes agree with each other on
    every bin, with no bin left out."""
    s = synth.small_series(11, N=400, n_base=3, nf=2000)
    f = s.grid.array()
    zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, want_ratio=True)
    first = None
    for fpt in {"fp64": (1, 2, 4), "mixed": (4, 6, 10)}[prec]:
        for warps in (1, 2, 3, 4, 6, 8):   # 3 and 6: slices of the CTA-level sums that are not powers of two
            z = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision=prec, fpt=fpt, warps=warps)
            r = _assert_cond(z, zr, ratio, c2, prec, s.N, (fpt, warps))
            assert r["excluded"] == 0
            if first is None:
                first = z
            else:   # every bin: the summation order is the only difference between shapes
                r = cond_parity(z, first, ratio, c2, TOL[prec], s.N)
                assert r["ok"] and r["excluded"] == 0, (fpt, warps, r)


@pytest.mark.parametrize("nb", [4, 5, 6])
def test_mixed_shapes_wide_bases_long_series(F, nb):
    """Base widths 9, 11 and 13 (odd frequencies per thread among the
    compiled shapes of width 9) on a series long enough for several flushes of the CTA-level
    slow sums at every CTA width (2600 points: 82 tiles of one warp, 11 of
    eight) and a ragged last tile: every shape meets the bound against the
    oracle on every bin, and any two shapes agree within twice it (each is
    within the bound of the oracle; their summation orders differ)."""
    s = synth.small_series(40 + nb, N=2600, n_base=nb, nf=1500, span=400.0, fmax=1.2)
    f = s.grid.array()
    zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, want_ratio=True)
    p = 2 * nb + 1
    first = None
    for fpt in {9: (3, 5, 8), 11: (4, 6, 8), 13: (4, 6)}[p]:   # the compiled mixed shapes of these widths
        for warps in (1, 2, 4, 8):
            z = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision="mixed", fpt=fpt, warps=warps)
            _assert_cond(z, zr, ratio, c2, "mixed", s.N, (fpt, warps))
            if first is None:
                first = z
            else:
                r = cond_parity(z, first, ratio, c2, 2 * TOL["mixed"], s.N)
                assert r["ok"], (fpt, warps, r)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("where", ["base", "zero"])
def test_conditioning_sweep(F, prec, where):
    """Uniform grids closing in on a base frequency (or on f = 0) by factors
    of ten: the trial columns' remaining norms after projection run from
    about 1e-6 to 1 of their own norms, i.e. conditions of the 2x2 system up
    to 1e12.  Every bin below 1e12 is compared with the oracle under the
    conditioning-scaled bound; on the mixed path these are the bins that the
    float-float re-evaluation computes."""
    s = synth.small_series(41, N=600, n_base=2, nf=10, span=400.0, fmax=0.5)
    T = s.t.max() - s.t.min()
    checked = excluded = 0
    lowest, worst = 1.0, 0.0
    for k in range(1, 7):
        df = 10.0 ** -k / T
        f0 = (s.base_freqs[1] if where == "base" else 0.0) + 0.37 * df - (32 * df if where == "base" else 0.0)
        f = f0 + df * np.arange(65)
        zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, want_ratio=True)
        z = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision=prec)
        r = _assert_cond(z, zr, ratio, c2, prec, s.N, (where, k))
        checked += r["checked"]
        excluded += r["excluded"]
        kept = ratio[ratio >= 1e-6]
        lowest = min(lowest, kept.min() if kept.size else 1.0)
        worst = max(worst, r["worst"])
    assert checked > 250 and lowest < 1e-4, (checked, excluded, lowest)
    print(f"conditioning sweep {where} {prec}: {checked} bins compared, {excluded} left out (cond > 1e12), "
          f"smallest ratio compared {lowest:.2e}, largest error / bound {worst:.3f}")


def test_device_path_matches_host_path(F):
    import torch
    s = synth.small_series(12, N=333, n_base=2, nf=5000)
    dev = torch.device("cuda:0")
    tt = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64), device=dev)
    for prec in ("fp64", "mixed"):
        out = F.periodogram_dev(tt(s.t), tt(s.y), tt(s.sigma), tt(s.base_freqs), s.grid.f0, s.grid.df, s.grid.nf,
                                precision=prec, topk=3)
        torch.cuda.synchronize()
        zh, toph = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, s.grid.array(), precision=prec, topk=3)
        assert np.array_equal(out["z"].cpu().numpy(), zh)
        assert list(out["topk"].cpu().numpy()) == list(toph)


def test_invariants_on_gpu(F):
    s = synth.small_series(13, N=200, n_base=1, nf=800)
    f = s.grid.array()
    z = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f)
    zs = F.periodogram(s.t + 5000.25, s.y, s.sigma, s.base_freqs, f)
    assert rel_err(zs, z) < 1e-9
    za = F.periodogram(s.t, 2.5 * s.y, s.sigma, s.base_freqs, f)
    assert rel_err(za, 6.25 * z) < 1e-11
    c2 = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, want_info=True)[1][0]
    assert np.all(z >= -1e-12 * c2) and np.all(z <= 0.5 * c2 * (1 + 1e-12))
