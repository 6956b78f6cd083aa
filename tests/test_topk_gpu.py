"""Top-k local maxima on the device (the candidate peaks of Sect. 4, Phase 1)
through fredec_topk_dev, against the oracle's rule (oracle.pipeline.local_maxima,
pinned in test_pipeline_pins.py) on adversarial arrays: ties and plateaus,
NaNs, signed zeros and infinities, end points, fewer maxima than k, sizes
around the 4096-point chunks of the first stage, and every merge of the second
(one sort of all candidates, the k-round tournament over the chunks' lists,
the warp selection for more than 1024 chunks).  Index work: the comparison is
exact.
"""
import numpy as np
import pytest

from helpers import ensure_built
from oracle import pipeline as P

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 7, 100, 4095, 4096, 4097, 8191, 8192, 8193, 16385, 70001, 1_000_003]
KS = [1, 5, 8, 9, 64]


@pytest.fixture(scope="module")
def F():
    ensure_built()
    import paper_1309_0100_b300 as F
    return F


def _ref(z, k):
    r = P.local_maxima(z)[:k]
    return r + [-1] * (k - len(r))


def _arrays(n, rng):
    yield "quantised", rng.integers(0, 4, n).astype(np.float64)          # many ties, plateaus
    x = np.linspace(0.0, 40.0 * np.pi, n)
    yield "smooth", np.sin(x) * (1.0 + 0.1 * np.cos(0.37 * x)) + 1e-3 * rng.standard_normal(n)
    z = rng.standard_normal(n)
    z[rng.random(n) < 0.05] = np.nan
    yield "nan", z
    z = rng.choice(np.array([-0.0, 0.0, 1.0, -np.inf, np.inf]), n)
    yield "zeros_inf", z
    yield "constant", np.full(n, 2.5)
    z = np.arange(n, dtype=np.float64)
    yield "increasing", z                                                   # one maximum: the last point
    yield "decreasing", z[::-1].copy()                                      # one maximum: the first point


@pytest.mark.parametrize("n", SIZES)
def test_topk_matches_rule(F, n):
    import torch
    rng = np.random.default_rng(1309 + n)
    for label, z in _arrays(n, rng):
        zd = torch.as_tensor(z, device="cuda")
        for k in KS:
            got = F.topk_dev(zd, k).cpu().tolist()
            assert got == _ref(z, k), (label, n, k)


def test_topk_many_equal_peaks(F):
    # equal peak heights: ranks go to the lower index, across chunks
    import torch
    n = 50_000
    z = np.zeros(n)
    z[np.arange(3, n - 1, 97)] = 1.0
    zd = torch.as_tensor(z, device="cuda")
    for k in (5, 8, 64):
        assert F.topk_dev(zd, k).cpu().tolist() == _ref(z, k)


def test_topk_many_chunks(F):
    # more than 1024 chunks of 4096 points: the warp-selection merge
    import torch
    rng = np.random.default_rng(7)
    n = 4_500_001
    x = np.linspace(0.0, 3000.0 * np.pi, n)
    z = np.abs(np.sin(x)) * (1.0 + 0.2 * np.sin(0.013 * x)) + 1e-4 * rng.standard_normal(n)
    zd = torch.as_tensor(z, device="cuda")
    for k in (1, 5, 64):
        assert F.topk_dev(zd, k).cpu().tolist() == _ref(z, k)


def test_topk_empty_and_errors(F):
    import torch
    empty = torch.empty(0, dtype=torch.float64, device="cuda")
    assert F.topk_dev(empty, 4).cpu().tolist() == [-1, -1, -1, -1]
    z = torch.zeros(10, dtype=torch.float64, device="cuda")
    for k in (0, 65):
        with pytest.raises(RuntimeError):
            F.topk_dev(z, k)
