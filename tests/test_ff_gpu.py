"""Float-float arithmetic on the GPU: the FF sin/cos against the FP64 path's,
and the mixed path's re-evaluated (flagged) bins, which use FF sums, against the
FP64 path at FP64-grade tolerance."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from helpers import cond_parity, ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    ensure_built()
    import paper_1309_0100_b300 as F
    return F


def test_ff_sincos_selftest(F):
    rng = np.random.default_rng(64)
    ph = rng.integers(0, 2 ** 63, 200000, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, 200000,
                                                                                       dtype=np.uint64)
    edges = [0, 1, (1 << 56) - 1, 1 << 56, (1 << 56) + 1, 1 << 63, (1 << 64) - 1] + [k << 56 for k in range(256)] \
        + [(k << 56) - 1 for k in range(1, 256)]
    ph = np.ascontiguousarray(np.concatenate([ph, np.asarray(edges, dtype=np.uint64)]))
    err = np.zeros(1)
    F._check(F.lib().fredec_selftest_ff_sincos(ph.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), ph.size,
                                                 err.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    assert err[0] < 2e-14, err[0]   # float-float resolution (about 48 bits)


def test_flagged_bins_are_fp64_grade(F):
    # a grid crowded around the base frequencies and f = 0: many bins are
    # flagged for re-evaluation (pivot ratio below 0.2, i.e. oracle ratio
    # below about 0.45); there the mixed result must be FP64-grade, against
    # the oracle (1e-9 plus the conditioning term) and against the FP64 path
    s = synth.small_series(77, N=2000, n_base=3, span=3000.0, nf=10, fmax=0.5)
    f = np.concatenate([g + np.linspace(-2e-4, 2e-4, 401) for g in s.base_freqs] + [np.linspace(1e-6, 2e-4, 200)])
    f = np.sort(np.abs(f))
    zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, want_ratio=True)
    z64 = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision="fp64")
    zmx = F.periodogram(s.t, s.y, s.sigma, s.base_freqs, f, precision="mixed")
    flagged = ratio < 0.3
    assert flagged.sum() > 400 and (ratio[flagged] < 1e-2).sum() > 20
    r = cond_parity(zmx[flagged], zr[flagged], ratio[flagged], c2, 1e-9, s.N,
                    floor_frac=1e-3 * np.max(zr) / np.max(zr[flagged]))
    assert r["ok"], r
    r = cond_parity(zmx, zr, ratio, c2, 1e-5, s.N)     # every bin at the mixed bar
    assert r["ok"], r
    mid = (ratio < 0.05) & (ratio >= 1e-3)
    floor = 1e-3 * np.max(zr)
    den = np.maximum(np.abs(z64), floor)
    assert np.max(np.abs(zmx - z64)[mid] / den[mid]) < 1e-9
