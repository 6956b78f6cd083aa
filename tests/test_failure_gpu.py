"""Failure detection without faulting the GPU: a bounded device wait that
nothing completes reports FREDEC_ETIMEOUT and leaves the context usable;
injected allocation failures report FREDEC_ENOMEM; invalid device inputs give
non-finite outputs, not a fault."""
import ctypes

import numpy as np
import pytest

import synth
from helpers import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    ensure_built()
    import paper_1309_0100_b300 as F
    return F


def test_bounded_wait_reports_timeout_and_context_survives(F):
    st = ctypes.c_int32(-1)
    assert F.lib().fredec_selftest_wait_timeout(ctypes.byref(st)) == 0
    assert st.value == 5          # FREDEC_ETIMEOUT
    s = synth.small_series(1, N=64, n_base=1, nf=100)
    z = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, s.grid.array())
    assert np.all(np.isfinite(z))


def test_injected_allocation_failure(F, monkeypatch):
    s = synth.small_series(2, N=64, n_base=1, nf=100)
    monkeypatch.setenv("FREDEC_FAIL_ALLOC", "1")
    with pytest.raises(F.FredecError) as ei:
        F.periodogram(s.t, s.y, s.sigma, s.base_freqs, s.grid.array())
    assert ei.value.code == 2
    monkeypatch.delenv("FREDEC_FAIL_ALLOC")
    z = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, s.grid.array())
    assert np.all(np.isfinite(z))


@pytest.mark.parametrize("prec,topk", [("fp64", 0), ("fp64", 3), ("mixed", 0), ("mixed", 3)])
def test_device_path_singular_base_gives_nan(F, prec, topk):
    # the NaN fill runs in its own kernel (FP64) or in the re-evaluation launch (mixed)
    import torch
    s = synth.small_series(3, N=80, n_base=2, nf=50)
    tt = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64), device="cuda:0")
    r = F.periodogram_dev(tt(s.t), tt(s.y), tt(s.sigma), tt([0.1, 0.1]), s.grid.f0, s.grid.df, s.grid.nf,
                          precision=prec, topk=topk)
    torch.cuda.synchronize()
    assert np.all(np.isnan(r["z"].cpu().numpy()))
    if topk:
        assert r["topk"].cpu().tolist() == [-1] * topk


def test_split_launch_singular_base_gives_nan(F):
    """A grid large enough for the tail split of the mixed launch (1e6
    frequencies at F = 10 with four warps): with a singular base model both
    periodogram launches return at once and the whole of z is NaN."""
    import torch
    s = synth.small_series(4, N=2000, n_base=3, nf=1_000_000, span=3000.0, fmax=2.0)
    tt = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64), device="cuda:0")
    r = F.periodogram_dev(tt(s.t), tt(s.y), tt(s.sigma), tt([0.1, 0.1, 0.2]), s.grid.f0, s.grid.df, s.grid.nf,
                          precision="mixed", topk=3, fpt=10, warps=4)
    torch.cuda.synchronize()
    assert np.all(np.isnan(r["z"].cpu().numpy()))
    assert r["topk"].cpu().tolist() == [-1] * 3


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_device_path_info_with_and_without_topk(F, prec):
    # info comes from the top-k launch when there is one, else from its own kernel
    import torch
    s = synth.small_series(4, N=300, n_base=1, nf=3000)
    tt = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64), device="cuda:0")
    args = (tt(s.t), tt(s.y), tt(s.sigma), tt(s.base_freqs), s.grid.f0, s.grid.df, s.grid.nf)
    a = F.periodogram_dev(*args, precision=prec, topk=5)
    b = F.periodogram_dev(*args, precision=prec, topk=0)
    torch.cuda.synchronize()
    ia, ib = a["info"].cpu().numpy(), b["info"].cpu().numpy()
    assert np.array_equal(ia, ib) and np.all(np.isfinite(ia)) and ia[0] > 0 and ia[1] > 0
