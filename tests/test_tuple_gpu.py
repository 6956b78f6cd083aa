"""GPU parity of the multifrequency tuple statistics (constant base) against
the FP64 oracle: z for arbitrary tuples, the all-subtuple l table of a
candidate pool, dz/df (adjoint sums) against the oracle and against central
finite differences of z (step 1e-7/T), and Gauss-Newton refinement."""
import numpy as np
import pytest

import oracle
import synth
from helpers import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    ensure_built()
    import paper_1309_0100_b300 as F
    return F


def _series(k, N=300, span=200.0):
    rng = np.random.default_rng(900 + k)
    t = np.sort(rng.uniform(0, span, N))
    sigma = rng.lognormal(0, 0.4, N)
    fr = np.array([0.0731, 0.151, 0.33, 0.0123])
    y = 2.0 + sum(a * np.sin(2 * np.pi * f * t + p) for a, f, p in zip([4, 3, 2, 1.5], fr, [0.1, 1.2, 2.2, 0.7]))
    return t, y + sigma * rng.standard_normal(N), sigma, fr


def test_tuple_eval_vs_oracle(F):
    t, y, s, fr = _series(1)
    tuples = [[fr[0]], [fr[0], fr[1]], [fr[2], fr[1], 0.47], list(fr), [0.2, 0.21, 0.4, 0.41, 0.6]]
    z, l0 = F.tuple_eval(t, y, s, tuples)
    zr, l0r = oracle.tuple_eval(t, y, s, tuples)
    assert l0 == pytest.approx(l0r, rel=1e-12)
    np.testing.assert_allclose(z, zr, rtol=1e-10)


@pytest.mark.parametrize("n,N", [(5, 120), (8, 257)])
def test_pool_table_vs_oracle(F, n, N):
    t, y, s, fr = _series(2 + n, N=N)
    pool = np.concatenate([fr, np.linspace(0.05, 0.45, n - 4) + 0.003])[:n]
    tab = F.pool_subtuples_eval(t, y, s, pool)
    ref = oracle.pool_table(t, y, s, pool)
    np.testing.assert_allclose(tab, ref, rtol=1e-10)


def test_pool_table_pool16_sampled(F):
    s = synth.pool16_n1000()
    tab = F.pool_subtuples_eval(s.t, s.y, s.sigma, s.pool)
    assert tab.size == 1 << 16
    rng = np.random.default_rng(4)
    for mask in np.concatenate([[0, 1, 0xFFFF, 0x003F], rng.integers(0, 1 << 16, 40)]):
        fr = [s.pool[k] for k in range(16) if int(mask) >> k & 1]
        lr = oracle.tuple_l(s.t, s.y, s.sigma, fr)
        assert tab[mask] == pytest.approx(lr, rel=1e-9), mask


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("mixed", 1e-8)])
def test_tuple_grad_vs_oracle_and_fd(F, prec, tol):
    """dz/df against the oracle's envelope-theorem gradient and against
    central finite differences of the oracle's z (step 1e-7/T) to 1e-6 of
    max(|dz/df|, 1e-3 max |dz/df|); the mixed path sums in float-float."""
    t, y, s, fr = _series(3)
    tuples = [[fr[0] + 0.0004], [fr[0] - 0.0003, fr[1] + 0.0002], [fr[2] + 0.0001, 0.47, fr[3]],
              [fr[0], fr[1], fr[2], fr[3] - 0.0002, 0.21]]
    z, g = F.tuple_grad(t, y, s, tuples, precision=prec)
    zr, gr = oracle.tuple_grad(t, y, s, tuples)
    assert np.max(np.abs(z - zr) / zr) < 1e-10
    assert np.max(np.abs(g - gr)) <= tol * np.max(np.abs(gr))
    T = t.max() - t.min()
    h = 1e-7 / T
    k = 0
    for tp in tuples:
        for q in range(len(tp)):
            a = list(tp); b = list(tp)
            a[q] += h; b[q] -= h
            fd = (oracle.tuple_eval(t, y, s, [a])[0][0] - oracle.tuple_eval(t, y, s, [b])[0][0]) / (2 * h)
            assert abs(fd - g[k]) <= 1e-6 * max(abs(g[k]), 1e-3 * np.max(np.abs(g))), (prec, k, fd, g[k])
            k += 1


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_tuple_grad_dev_and_autograd(F, prec):
    """The device entry point equals the host one; TupleZFn (device tensors
    through forward and backward) gives the oracle's gradient."""
    import torch
    from paper_1309_0100_b300.autograd import tuple_z
    t, y, s, fr = _series(4, N=400)
    tuples = [[fr[0] + 0.0002], [fr[1] - 0.0001, fr[2] + 0.0003], [fr[0], fr[1], fr[2], fr[3] + 0.0001]]
    flat = np.concatenate([np.asarray(tp, dtype=np.float64) for tp in tuples])
    off = np.cumsum([0] + [len(tp) for tp in tuples]).astype(np.int64)
    dev = torch.device("cuda:0")
    tt = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    zd, gd = F.tuple_grad_dev(tt(t), tt(y), tt(s), tt(flat), off, precision=prec)
    torch.cuda.synchronize()
    zh, gh = F.tuple_grad(t, y, s, tuples, precision=prec)
    assert np.array_equal(zd.cpu().numpy(), zh) and np.array_equal(gd.cpu().numpy(), gh)
    freqs = tt(flat).requires_grad_(True)
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device=dev)
    zt = tuple_z(freqs, tt(t), tt(y), tt(s), torch.as_tensor(off), precision=prec)
    assert zt.is_cuda
    (zt * w).sum().backward()
    zr, gr = oracle.tuple_grad(t, y, s, tuples)
    want = np.repeat(w.cpu().numpy(), np.diff(off)) * gr
    np.testing.assert_allclose(zt.detach().cpu().numpy(), zr, rtol=1e-10)
    assert np.max(np.abs(freqs.grad.cpu().numpy() - want)) <= 1e-8 * np.max(np.abs(want))
    # a repeated frequency: NaN for that tuple only (device entry points read nothing back)
    bad = np.array([fr[0], fr[0], fr[1]])
    zb, gb = F.tuple_grad_dev(tt(t), tt(y), tt(s), tt(bad), np.array([0, 2, 3], dtype=np.int64), precision=prec)
    torch.cuda.synchronize()
    zb, gb = zb.cpu().numpy(), gb.cpu().numpy()
    assert np.isnan(zb[0]) and np.isnan(gb[:2]).all() and np.isfinite(zb[1]) and np.isfinite(gb[2])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_tuple_refine_vs_oracle(F, prec):
    t, y, s, fr = _series(5)
    T = t.max() - t.min()
    starts = [[fr[0] + 0.2 / T], [fr[0] - 0.15 / T, fr[1] + 0.25 / T], [fr[0] + 0.1 / T, fr[1], fr[2] - 0.2 / T]]
    got_f, got_l, its = F.tuple_refine(t, y, s, starts, max_iter=30, tol=1e-10, precision=prec)
    for st, gf, gl in zip(starts, got_f, got_l):
        rf, rl, _ = oracle.tuple_refine(t, y, s, st, max_iter=60, tol=1e-12)
        ftol = (1e-7 if prec == "fp64" else 1e-4) / T
        assert np.max(np.abs(gf - rf)) < ftol, (gf - rf) * T
        assert gl == pytest.approx(rl, rel=1e-10 if prec == "fp64" else 1e-6)


def _separated(rng, m, lo=0.02, step=0.028):
    """m frequencies on a jittered grid (well apart at the series' resolution)."""
    base = lo + step * np.sort(rng.choice(20, m, replace=False))
    return list(base + rng.uniform(-0.004, 0.004, m))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_many_tuples_every_size_vs_oracle(F, prec):
    """Eight tuples of every size 1..20: the warp-per-tuple kernels run over
    several size ranges, with one sweep of the Gram blocks or several, and
    with groups of lanes splitting the points for the smallest Grams.  z and
    dz/df against the oracle."""
    t, y, s, fr = _series(6, N=500, span=300.0)
    rng = np.random.default_rng(7)
    tuples = [_separated(rng, m) for m in range(1, 21) for _ in range(8)]
    z, g = F.tuple_grad(t, y, s, tuples, precision=prec)
    zr, gr = oracle.tuple_grad(t, y, s, tuples)
    np.testing.assert_allclose(z, zr, rtol=1e-10)
    k = 0
    for tp in tuples:
        m = len(tp)
        gk, gkr = g[k:k + m], gr[k:k + m]
        assert np.max(np.abs(gk - gkr)) <= 1e-8 * np.max(np.abs(gkr)), (prec, m)
        k += m
    ze, _ = F.tuple_eval(t, y, s, tuples)
    np.testing.assert_allclose(ze, zr, rtol=1e-10)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_long_series_few_tuples_cta_kernel(F, prec):
    """A long series with a few tuples takes the CTA-per-tuple kernel (the
    whole CTA on one tuple's pass): z, dz/df and refinement against the
    oracle."""
    t, y, s, fr = _series(7, N=10000, span=2000.0)
    T = t.max() - t.min()
    tuples = [[fr[0] + 0.02 / T], [fr[0], fr[1] - 0.03 / T], [fr[0], fr[1], fr[2] + 0.01 / T, fr[3]]]
    z, g = F.tuple_grad(t, y, s, tuples, precision=prec)
    zr, gr = oracle.tuple_grad(t, y, s, tuples)
    np.testing.assert_allclose(z, zr, rtol=1e-10)
    assert np.max(np.abs(g - gr)) <= 1e-8 * np.max(np.abs(gr))
    starts = [[fr[0] + 0.2 / T], [fr[0] - 0.15 / T, fr[1] + 0.25 / T]]
    got_f, got_l, _ = F.tuple_refine(t, y, s, starts, max_iter=30, tol=1e-10, precision=prec)
    for st, gf, gl in zip(starts, got_f, got_l):
        rf, rl, _ = oracle.tuple_refine(t, y, s, st, max_iter=60, tol=1e-12)
        assert np.max(np.abs(gf - rf)) < (1e-7 if prec == "fp64" else 1e-4) / T, (gf - rf) * T
        assert gl == pytest.approx(rl, rel=1e-10 if prec == "fp64" else 1e-6)


def test_tensor_core_gram_wide_weight_range(F):
    """Tuples of 11 to 15 frequencies (Grams of 46 to 62 columns: the
    float-float passes on the tensor cores, columns split into bf16 digits
    relative to each column's largest value) on a series whose 1/sigma spans
    two decades, so that most values sit far below their column's scale: z and
    dz/df of the mixed path against the oracle."""
    rng = np.random.default_rng(11)
    N = 600
    t = np.sort(rng.uniform(0, 400.0, N))
    sigma = 10.0 ** rng.uniform(-1.0, 1.0, N)
    y = 3.0 + 2.0 * np.sin(2 * np.pi * 0.05 * t) + 1.5 * np.cos(2 * np.pi * 0.17 * t) + sigma * rng.standard_normal(N)
    tuples = [_separated(rng, m) for m in (11, 12, 13, 14, 15) for _ in range(3)]
    z, g = F.tuple_grad(t, y, sigma, tuples, precision="mixed")
    zr, gr = oracle.tuple_grad(t, y, sigma, tuples)
    np.testing.assert_allclose(z, zr, rtol=1e-10)
    k = 0
    for tp in tuples:
        m = len(tp)
        assert np.max(np.abs(g[k:k + m] - gr[k:k + m])) <= 1e-8 * np.max(np.abs(gr[k:k + m])), m
        k += m
