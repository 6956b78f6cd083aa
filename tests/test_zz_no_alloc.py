"""The no-allocation periodogram entry point, through the C ABI.

fredec_periodogram_noalloc_dev serves callers that cannot allocate device
memory when they call (their memory is reserved up front by their own
allocator, or allocation is forbidden after start-up): its scratch is a fixed
16 MiB device array inside the library.  Its results must match the regular
stream-ordered entry point, call after call, since every call reuses (and
must re-clear) the same array.  This file is collected last so that a run
stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth
from helpers import ensure_built, rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5}


@pytest.fixture(scope="module")
def F():
    ensure_built()
    import paper_1309_0100_b300 as F
    return F


def _dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda:0")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_matches_regular_entry_point(F, prec):
    import torch
    L = F.lib()
    series = [synth.small_series(31, N=700, n_base=3, nf=20000, span=400.0),
              synth.small_series(32, N=257, n_base=1, nf=4999, span=90.0)]
    for s in series:      # two different problems, each called twice in a row
        t, y, sg, b = (_dev(torch, a) for a in (s.t, s.y, s.sigma, s.base_freqs))
        ref = F.periodogram_dev(t, y, sg, b, s.grid.f0, s.grid.df, s.grid.nf, precision=prec)
        o = F._opts(prec)
        for call in range(2):
            z = torch.full((s.grid.nf,), -1.0, dtype=torch.float64, device="cuda:0")
            info = torch.empty(3, dtype=torch.float64, device="cuda:0")
            stream = torch.cuda.current_stream()
            rc = L.fredec_periodogram_noalloc_dev(t.data_ptr(), y.data_ptr(), sg.data_ptr(), s.N,
                                                  b.data_ptr() if b.numel() else None, b.numel(),
                                                  float(s.grid.f0), float(s.grid.df), int(s.grid.nf),
                                                  ctypes.byref(o), z.data_ptr(), info.data_ptr(),
                                                  int(stream.cuda_stream))
            assert rc == 0, L.fredec_last_error().decode()
            torch.cuda.synchronize()
            zr = ref["z"].cpu().numpy()
            assert rel_err(z.cpu().numpy(), zr) < TOL[prec], (prec, call)
            np.testing.assert_allclose(info.cpu().numpy(), ref["info"].cpu().numpy(), rtol=1e-12)


def test_noalloc_rejects_oversized_problem(F):
    import torch
    L = F.lib()
    N = 100_000
    rng = np.random.default_rng(5)
    t = _dev(torch, np.sort(rng.uniform(0, 1000, N)))
    y = _dev(torch, rng.standard_normal(N))
    sg = _dev(torch, np.ones(N))
    b = _dev(torch, np.linspace(0.01, 0.2, 12))
    z = torch.empty(10, dtype=torch.float64, device="cuda:0")
    o = F._opts("fp64")
    rc = L.fredec_periodogram_noalloc_dev(t.data_ptr(), y.data_ptr(), sg.data_ptr(), N, b.data_ptr(), 12, 0.01, 0.01,
                                          10, ctypes.byref(o), z.data_ptr(), None, None)
    assert rc == 1
    assert "bytes of scratch" in L.fredec_last_error().decode()
