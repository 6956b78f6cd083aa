"""The no-allocation periodogram entry point, through the C ABI.

fredec_periodogram_noalloc_dev serves callers that cannot allocate device
memory when they call (their memory is reserved up front by their own
allocator, or allocation is forbidden after start-up): its scratch is a fixed
16 MiB device array inside the library.  Its results must match the regular
stream-ordered entry point, call after call, since every call reuses (and
must re-clear) the same array: z with its NaN pattern, and info.  The cases
cover both precisions, the polynomial trend, the log-form statistic and a
singular base model (z all NaN on both entry points).  The scratch-size
formula of the header is checked against the library's own accounting just
under and just over the 16 MiB limit.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes
import re

import numpy as np
import pytest

import oracle
import synth
from helpers import cond_parity, ensure_built, rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5}
LIMIT = 16 << 20


@pytest.fixture(scope="module")
def F():
    ensure_built()
    import paper_1309_0100_b300 as F
    return F


def _dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda:0")


def _noalloc(F, torch, t, y, sg, b, s, o, nf=None, f0=None, df=None):
    """One call of the no-allocation entry point on torch's current stream;
    returns (rc, z, info) after synchronising."""
    L = F.lib()
    nf = s.grid.nf if nf is None else nf
    z = torch.full((max(nf, 1),), -1.0, dtype=torch.float64, device="cuda:0")
    info = torch.empty(3, dtype=torch.float64, device="cuda:0")
    rc = L.fredec_periodogram_noalloc_dev(t.data_ptr(), y.data_ptr(), sg.data_ptr(), t.numel(),
                                          b.data_ptr() if b.numel() else None, b.numel(),
                                          float(s.grid.f0 if f0 is None else f0),
                                          float(s.grid.df if df is None else df), int(nf),
                                          ctypes.byref(o), z.data_ptr(), info.data_ptr(),
                                          int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, z.cpu().numpy()[:nf], info.cpu().numpy()


def _same_as_regular(z, zr, prec):
    assert np.array_equal(np.isnan(z), np.isnan(zr))
    fin = ~np.isnan(zr)
    if fin.any():
        assert rel_err(z[fin], zr[fin]) < TOL[prec]


@pytest.mark.parametrize("prec,trend,stat", [("fp64", 0, "diff"), ("mixed", 0, "diff"), ("fp64", 1, "diff"),
                                             ("mixed", 1, "log"), ("fp64", 0, "log"), ("mixed", 2, "diff")])
def test_noalloc_matches_regular_entry_point(F, prec, trend, stat):
    import torch
    series = [synth.small_series(31, N=700, n_base=3, nf=20000, span=400.0),
              synth.small_series(32, N=257, n_base=1, nf=4999, span=90.0)]
    for s in series:      # two different problems, each called twice in a row
        t, y, sg, b = (_dev(torch, a) for a in (s.t, s.y, s.sigma, s.base_freqs))
        ref = F.periodogram_dev(t, y, sg, b, s.grid.f0, s.grid.df, s.grid.nf, precision=prec, trend=trend,
                                statistic=stat)
        torch.cuda.synchronize()
        zr, ir = ref["z"].cpu().numpy(), ref["info"].cpu().numpy()
        o = F._opts(prec, 0, 0, 0, 0.0, trend, stat)
        for call in range(2):
            rc, z, info = _noalloc(F, torch, t, y, sg, b, s, o)
            assert rc == 0, F.lib().fredec_last_error().decode()
            _same_as_regular(z, zr, prec)
            np.testing.assert_allclose(info, ir, rtol=1e-12)


def test_noalloc_vs_oracle(F):
    """The default case also against the oracle (conditioning-scaled bound)."""
    import torch
    s = synth.small_series(33, N=300, n_base=2, nf=3000, span=200.0)
    t, y, sg, b = (_dev(torch, a) for a in (s.t, s.y, s.sigma, s.base_freqs))
    zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, s.grid.array(), want_ratio=True)
    for prec in ("fp64", "mixed"):
        for call in range(2):
            rc, z, info = _noalloc(F, torch, t, y, sg, b, s, F._opts(prec))
            assert rc == 0
            r = cond_parity(z, zr, ratio, c2, TOL[prec], s.N)
            assert r["ok"], (prec, call, r)
            assert info[0] == pytest.approx(c2, rel=1e-11)


def test_noalloc_singular_base(F):
    """Duplicate base frequencies: the base fit fails; both entry points give
    an all-NaN z (device entry points read nothing back), call after call."""
    import torch
    s = synth.small_series(34, N=200, n_base=2, nf=500, span=100.0)
    base = np.array([s.base_freqs[0], s.base_freqs[0]])
    t, y, sg, b = (_dev(torch, a) for a in (s.t, s.y, s.sigma, base))
    for prec in ("fp64", "mixed"):
        ref = F.periodogram_dev(t, y, sg, b, s.grid.f0, s.grid.df, s.grid.nf, precision=prec)
        torch.cuda.synchronize()
        zr = ref["z"].cpu().numpy()
        assert np.isnan(zr).all()
        for call in range(2):
            rc, z, _ = _noalloc(F, torch, t, y, sg, b, s, F._opts(prec))
            assert rc == 0
            assert np.isnan(z).all(), (prec, call)
        # and a regular problem right after it still gives the regular result
        s2 = synth.small_series(35, N=200, n_base=2, nf=500, span=100.0)
        t2, y2, sg2, b2 = (_dev(torch, a) for a in (s2.t, s2.y, s2.sigma, s2.base_freqs))
        ref2 = F.periodogram_dev(t2, y2, sg2, b2, s2.grid.f0, s2.grid.df, s2.grid.nf, precision=prec)
        torch.cuda.synchronize()
        rc, z, _ = _noalloc(F, torch, t2, y2, sg2, b2, s2, F._opts(prec))
        assert rc == 0
        _same_as_regular(z, ref2["z"].cpu().numpy(), prec)


def _r256(x):
    return (x + 255) // 256 * 256


def _scratch_bytes(N, n_base, nf, prec, trend=0, reeval=True):
    """The header's scratch formula of the no-allocation entry point."""
    p = (1 + trend + 2 * n_base) | 1
    c = -(-N // 32)
    r = 8 * (6 + 2 * -(-p // 2)) if prec == "fp64" else 4 * (8 + 4 * -(-(p + 2) // 4))
    b = 6912 + _r256(4 * c) + _r256(8 * c * (p * (p + 1) // 2 + p + 4)) + _r256(8 * p * N) + _r256(r * N)
    if prec == "mixed" and reeval:
        b += _r256(16 * -(-(8 + 2 * p) // 4) * N) + _r256(8 * nf + 8)
    return b


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_scratch_formula_at_the_limit(F, prec):
    """Problems just under and just over 16 MiB by the header's formula: the
    first runs and matches the regular entry point, the second is rejected
    before anything runs, with the formula's byte count in the message."""
    import torch
    nb, nf = 3, 64
    lo, hi = 1000, 400000
    while hi - lo > 1:                       # largest N that fits
        mid = (lo + hi) // 2
        lo, hi = (mid, hi) if _scratch_bytes(mid, nb, nf, prec) <= LIMIT else (lo, mid)
    n_fit = lo
    assert _scratch_bytes(n_fit, nb, nf, prec) <= LIMIT < _scratch_bytes(n_fit + 1, nb, nf, prec)
    for N, fits in ((n_fit, True), (n_fit + 1, False)):
        s = synth.small_series(36, N=N, n_base=nb, nf=nf, span=3000.0, fmax=0.2)
        t, y, sg, b = (_dev(torch, a) for a in (s.t, s.y, s.sigma, s.base_freqs))
        rc, z, _ = _noalloc(F, torch, t, y, sg, b, s, F._opts(prec))
        msg = F.lib().fredec_last_error().decode()
        if fits:
            assert rc == 0, msg
            ref = F.periodogram_dev(t, y, sg, b, s.grid.f0, s.grid.df, s.grid.nf, precision=prec)
            torch.cuda.synchronize()
            _same_as_regular(z, ref["z"].cpu().numpy(), prec)
        else:
            assert rc == 1 and np.all(z == -1.0), msg        # nothing was written
            need = int(re.search(r"needs (\d+) bytes", msg).group(1))
            assert need == _scratch_bytes(N, nb, nf, prec), (need, msg)


def test_noalloc_rejects_bad_arguments_before_running(F):
    """Checks shared with the regular entry point: a non-finite f0 or df, an
    unknown launch shape, a top-k request; z is left untouched."""
    import torch
    s = synth.small_series(37, N=100, n_base=1, nf=50, span=50.0)
    t, y, sg, b = (_dev(torch, a) for a in (s.t, s.y, s.sigma, s.base_freqs))
    for kw, over in (({}, {"f0": float("nan")}), ({}, {"df": float("inf")}), ({"fpt": 7}, {}),
                     ({"topk": 3}, {})):
        o = F._opts("mixed", kw.get("topk", 0), kw.get("fpt", 0))
        rc, z, _ = _noalloc(F, torch, t, y, sg, b, s, o, **over)
        assert rc == 1 and np.all(z == -1.0), (kw, over)
