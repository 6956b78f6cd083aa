"""GPU parity of the adjoint dL/dy of the residual periodogram (envelope
theorem: dz_j/dy_i = w_i (mu_j(t_i) - mu_base(t_i))) against the oracle's
VJP and against finite differences of z; and the torch.autograd route."""
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


def _dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda:0")


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 1e-5)])
@pytest.mark.parametrize("nb,N,nf", [(0, 50, 300), (2, 333, 1000), (5, 130, 4099)])
def test_vjp_vs_oracle(F, prec, tol, nb, N, nf):
    s = synth.small_series(200 + nb, N=N, n_base=nb, nf=nf, span=150.0)
    f = s.grid.array()
    v = np.random.default_rng(nb).standard_normal(nf)
    ref = oracle.periodogram_vjp(s.t, s.y, s.sigma, s.base_freqs, f, v)
    got = F.periodogram_vjp(s.t, s.y, s.sigma, s.base_freqs, s.grid.f0, s.grid.df, nf, v, precision=prec)
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref)), np.max(np.abs(got - ref)) / np.max(np.abs(ref))


def test_vjp_one_hot_at_peak_vs_oracle(F):
    """v = one-hot at the highest peak: the oracle needs a single fit."""
    s = synth.small_series(210, N=3000, n_base=3, nf=20000, span=2000.0)
    f = s.grid.array()
    z, top = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision="mixed", topk=1)
    v = np.zeros(f.size)
    v[top[0]] = 1.0
    ref = oracle.periodogram_vjp(s.t, s.y, s.sigma, s.base_freqs, f[top[0]:top[0] + 1], v[top[0]:top[0] + 1])
    for prec, tol in (("fp64", 1e-9), ("mixed", 1e-5)):
        got = F.periodogram_vjp(s.t, s.y, s.sigma, s.base_freqs, s.grid.f0, s.grid.df, f.size, v, precision=prec)
        assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


def test_autograd_matches_finite_differences(F):
    import torch
    from paper_1309_0100_b300.autograd import periodogram_z
    s = synth.small_series(220, N=40, n_base=1, nf=64, span=60.0)
    t, sg, b = _dev(torch, s.t), _dev(torch, s.sigma), _dev(torch, s.base_freqs)
    y = _dev(torch, s.y).requires_grad_(True)
    v = torch.as_tensor(np.random.default_rng(1).standard_normal(64), device="cuda:0")
    z = periodogram_z(y, t, sg, b, s.grid.f0, s.grid.df, 64)
    (z * v).sum().backward()
    g = y.grad.cpu().numpy()
    fd = np.empty(40)
    h = 1e-4
    for i in range(40):
        yp = s.y.copy(); yp[i] += h
        ym = s.y.copy(); ym[i] -= h
        zp = F.periodogram(s.t, yp, s.sigma, s.base_freqs, s.grid.array())
        zm = F.periodogram(s.t, ym, s.sigma, s.base_freqs, s.grid.array())
        fd[i] = v.cpu().numpy() @ (zp - zm) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-8 * np.abs(g).max())
