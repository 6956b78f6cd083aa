"""Shared test helpers: building the library, and the parity metrics."""
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def ensure_built():
    """Build libfredec.so in-tree if it is missing or stale (nvcc is in the image)."""
    from paper_1309_0100_b300 import _build
    return _build.build()


def rel_err(z, zref, mask=None, floor_frac=1e-3):
    """max_j |z_j - z*_j| / max(z*_j, floor_frac * max z*) over the masked bins
    (the relative-error reading: bins far below the highest peak are compared
    against a floor of 1e-3 of it)."""
    z = np.asarray(z, dtype=np.float64)
    zref = np.asarray(zref, dtype=np.float64)
    if mask is None:
        mask = np.ones(zref.shape, dtype=bool)
    floor = floor_frac * np.max(np.abs(zref))
    den = np.maximum(np.abs(zref), floor)
    return float(np.max(np.abs(z - zref)[mask] / den[mask])) if mask.any() else 0.0


def local_max_topk(z, k):
    """Reference top-k local maxima (same definition as the library)."""
    z = np.asarray(z)
    n = z.size
    cand = []
    for j in range(n):
        if n == 1:
            m = True
        elif j == 0:
            m = z[0] > z[1]
        elif j == n - 1:
            m = z[-1] > z[-2]
        else:
            m = z[j] > z[j - 1] and z[j] >= z[j + 1]
        if m:
            cand.append((-z[j], j))
    cand.sort()
    out = [j for _, j in cand[:k]]
    return out + [-1] * (k - len(out))
