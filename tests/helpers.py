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


# ---------------------------------------------------------------------------
# z parity with a bound that scales with the conditioning of the trial columns
#
# The oracle reports, per bin, ratio = the smaller remaining-norm / original-
# norm of the two trial columns after projection on the base (and on each
# other).  A normal-equation method forms the 2x2 Schur complement
# S = G - V^T V from sums whose rounding error is about gamma ||c||^2, with
# gamma the relative error of an N-term FP64 (or double-float) sum, about
# EPS64 sqrt(N) for random rounding.  S itself is ratio^2 ||c||^2, so its
# relative error is gamma / ratio^2 and z = rho^T S^{-1} rho / 2 <= chi2_base / 2
# moves by at most about (gamma / ratio^2) chi2_base / 2.  The bound per bin is
#     |z - z*| <= tol max(z*, floor) + C_COND EPS64 sqrt(N) chi2_base / ratio^2,
# C_COND = 8 (16x the estimate above).  Bins whose 2x2 system has a
# condition number above 1e12 (ratio < 1e-6) are the only ones left out:
# there the drop rule of degenerate columns (ratio < 1e-7 on either side) may
# decide differently in the two methods.
EPS64 = 2.0 ** -52
C_COND = 8.0
MIN_RATIO_COND = 1e-6


def cond_parity(z, zref, ratio, chi2, tol, N, floor_frac=1e-3, cond_scale=None):
    """Element-wise check of z against the oracle's zref with the
    conditioning-scaled bound above.  Returns a dict: 'ok' (all compared bins
    within the bound), 'checked', 'excluded' (bins with ratio < 1e-6),
    'worst' (largest |z - z*| / bound over the compared bins) and 'rel_err'
    (the plain relative error of the compared bins, floor_frac floor).
    cond_scale (per bin, optional) multiplies the conditioning term: the
    derivative of a statistic computed from z (the log form) with respect
    to z."""
    z = np.asarray(z, dtype=np.float64)
    zref = np.asarray(zref, dtype=np.float64)
    ratio = np.asarray(ratio, dtype=np.float64)
    keep = ratio >= MIN_RATIO_COND
    floor = floor_frac * np.max(np.abs(zref)) if zref.size else 0.0
    den = np.maximum(np.abs(zref), floor)
    with np.errstate(divide="ignore"):
        cond_term = C_COND * EPS64 * np.sqrt(N) * chi2 / np.maximum(ratio, MIN_RATIO_COND) ** 2
    if cond_scale is not None:
        cond_term = cond_term * np.abs(np.asarray(cond_scale, dtype=np.float64))
    bound = tol * den + cond_term
    diff = np.abs(z - zref)
    bad = keep & ~(diff <= bound)          # NaN fails
    worst = float(np.max(diff[keep] / bound[keep])) if keep.any() else 0.0
    rel = float(np.max(diff[keep] / den[keep])) if keep.any() else 0.0
    return {"ok": not bad.any(), "checked": int(keep.sum()), "excluded": int((~keep).sum()), "worst": worst,
            "rel_err": rel, "first_bad": int(np.flatnonzero(bad)[0]) if bad.any() else -1}
