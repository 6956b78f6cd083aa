"""Oracle of the whole FREDEC decomposition (Sect. 4): Phase 1 scan, Phase 2
local fits of every subtuple, Phase 3 backward cascade, Phase 4 ordering.

TEST INFRASTRUCTURE ONLY (imported by the tests, never by the product path).
Plain Python driving the FP64 oracle functions of oracle.c: every periodogram
is the QR definition, every subtuple is refined by the QR Gauss-Newton oracle.

Readings taken where Sect. 4 is silent:
  * the statistic of Phase 1 is the log form of Eq. zpowrel for one added
    frequency, z = (N - 3(m+1) - 1)/2 ln(l_base / l_new), with
    l_new = l_base - 2 z_diff from the difference-form periodogram;
  * "periodogram peaks" are local maxima (z_j > z_{j-1}, z_j >= z_{j+1}; an end
    point counts when it exceeds its one neighbour), ranked by decreasing z
    (ties to the lower index); the 64 highest are considered;
  * the top peak enters the base and the pool when its z reaches z_thr0 (FAP_0);
    otherwise the scan stops.  The other considered peaks enter the pool when
    their z reaches z_thr1 (FAP_1) and half of the top peak's z;
  * a candidate closer than merge_dist (default 0.5/T, T = span of t) to a
    pool member is the same candidate: the one with the larger z is kept;
  * at the end the pool is ordered by decreasing z (ties to the lower
    frequency) and cut to max_pool (default N/10, at most 20);
  * the scan also stops after max_base base frequencies (default 12, and at
    most (N-3)/2 so that the base model stays overdetermined);
  * Phase 4's residual statistic of a solution is the log-form z of the
    highest local maximum of the residual periodogram whose base is the
    solution's fitted frequencies, on the scan's grid (N_H = N - 3(m+1) - 1);
    NaN for solutions of more than 12 frequencies.
"""
from __future__ import annotations

import numpy as np

from . import (cascade, cascade_solutions, l0, periodogram, phase4_order, tuple_refine)

MAX_SIDE = 64


def local_maxima(z):
    """Indices of the local maxima of z ranked by decreasing z, ties to the
    lower index."""
    z = np.asarray(z, dtype=np.float64)
    nf = z.size
    if nf == 0:
        return []
    if nf == 1:
        return [0] if not np.isnan(z[0]) else []
    ok = np.zeros(nf, dtype=bool)
    ok[0] = z[0] > z[1]
    ok[-1] = z[-1] > z[-2]
    ok[1:-1] = (z[1:-1] > z[:-2]) & (z[1:-1] >= z[2:])
    idx = np.flatnonzero(ok)
    order = np.lexsort((idx, -z[idx]))
    return [int(j) for j in idx[order]]


def log_form(z_diff, l_base, N, m_alt):
    """(N - 3 m_alt - 1)/2 ln(l_base / (l_base - 2 z_diff))."""
    NH = N - 3 * m_alt - 1
    l_new = l_base - 2.0 * np.asarray(z_diff, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(l_new > 0, 0.5 * NH * np.log(l_base / l_new), np.inf)


def phase1_scan(t, y, sigma, f0, df, nf, z_thr0, z_thr1, *, max_pool=0, max_base=12,
                half=0.5, merge_dist=0.0):
    """Phase 1 (SLICK/QUICK).  Returns (pool freqs, pool z, base freqs,
    truncated)."""
    t = np.asarray(t, dtype=np.float64)
    N = t.size
    T = float(t.max() - t.min())
    md = merge_dist if merge_dist > 0 else 0.5 / T
    cap = max_pool if max_pool > 0 else N // 10
    cap = min(cap, 20)
    max_base = min(max_base, max(0, (N - 3) // 2))
    grid = f0 + df * np.arange(nf)
    base, pool = [], []          # pool: list of [f, z]

    def add(f, z):
        near = [k for k, (g, _) in enumerate(pool) if abs(g - f) < md]
        if not near:
            pool.append([f, z])
            return
        k = min(near, key=lambda q: abs(pool[q][0] - f))
        if z > pool[k][1]:
            pool[k] = [f, z]

    while len(base) < max_base:
        zd, lb = periodogram(t, y, sigma, base, grid)
        peaks = local_maxima(zd)[:MAX_SIDE]
        if not peaks:
            break
        zl = log_form(zd[peaks], lb, N, len(base) + 1)
        if not zl[0] >= z_thr0:
            break
        ftop = float(grid[peaks[0]])
        base.append(ftop)
        add(ftop, float(zl[0]))
        for j, zj in zip(peaks[1:], zl[1:]):
            if zj >= z_thr1 and zj >= half * zl[0]:
                add(float(grid[j]), float(zj))
    pool.sort(key=lambda r: (-r[1], r[0]))
    truncated = len(pool) > cap
    pool = pool[:cap]
    return (np.array([r[0] for r in pool]), np.array([r[1] for r in pool]), np.array(base), truncated)


def decompose(t, y, sigma, f0, df, nf, z_thr0, z_thr1, z_thr, *, max_pool=0, max_base=12,
              half=0.5, merge_dist=0.0, refine_iter=20, refine_tol=1e-9):
    """Phases 1-4.  Returns a dict with the pool, the subtuple table, the
    refined frequencies of every subtuple, the pass flags and slack of the
    cascade, and the solutions in Phase 4 order with G and their refined
    frequencies (increasing)."""
    t, y, sigma = (np.asarray(a, dtype=np.float64) for a in (t, y, sigma))
    N = t.size
    pool, pool_z, base, trunc = phase1_scan(t, y, sigma, f0, df, nf, z_thr0, z_thr1, max_pool=max_pool,
                                            max_base=max_base, half=half, merge_dist=merge_dist)
    n = pool.size
    l = np.empty(1 << n)
    fref = np.zeros((1 << n, n))
    l[0] = l0(t, y, sigma)
    for S in range(1, 1 << n):
        mem = [j for j in range(n) if S >> j & 1]
        f, lS, _ = tuple_refine(t, y, sigma, pool[mem], max_iter=refine_iter, tol=refine_tol)
        l[S] = lS
        fref[S, mem] = f
    passed, slack, _ = cascade(l, N, z_thr[:max(n, 1)] if n else np.zeros(1))
    sols = cascade_solutions(passed)
    masks, G = phase4_order(sols, l, N)
    freqs = [np.sort(fref[int(S)][[j for j in range(n) if int(S) >> j & 1]]) for S in masks]
    grid = f0 + df * np.arange(nf)
    resid = []
    for fs in freqs:
        if fs.size > 12:
            resid.append(np.nan)
            continue
        zd, lb = periodogram(t, y, sigma, fs, grid)
        pk = local_maxima(zd)
        resid.append(float(log_form(zd[pk[0]], lb, N, fs.size + 1)) if pk else np.nan)
    return dict(pool=pool, pool_z=pool_z, base=base, truncated=trunc, l=l, f=fref, passed=passed,
                slack=slack, masks=masks, G=G, freqs=freqs, resid_z=np.array(resid))
