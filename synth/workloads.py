"""Seeded synthetic time series shaped like the paper's workloads.

The paper analyses radial-velocity archives and an artificial two-sinusoid
series (Section 6) that are not available here, so these generators stand in
for them with the sizes named by the five benchmark workloads (workload k
draws its seeds with k):

  1  seasonal_n200      single series, N=200, seasonal gaps, constant base, 20000-point grid
  2  residual_n2000_p7  residual periodogram, N=2000, base = constant + 3 fixed sinusoids, 1e6 grid
  3  batch_4096         4096 independent series of uneven length and grid size (batched launch)
  4  pool16_n1000       N=1000, six sinusoids, a 16-frequency candidate pool (tuple sweep)
  5  nightly_n1e5_p11   survey-like N=1e5 nightly cadence, base = constant + 5 sinusoids, 1e7 grid

Everything is float64 numpy arrays.  A frequency grid is always uniform
``f_j = f0 + j*df`` (j = 0..nf-1) and is described by (f0, df, nf); the
explicit array can be made with :func:`grid_array`.

Only numpy's PCG64 generator is used.  Seeds follow
``13090100 + 1000*k + rep`` for workload k.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

__all__ = [
    "Series", "Grid", "Workload", "seed_for", "grid_array",
    "seasonal_n200", "residual_n2000_p7", "batch_4096", "pool16_n1000", "nightly_n1e5_p11",
    "small_series", "uniform_series", "make_workload",
]

SEED_BASE = 13090100


def seed_for(workload: int, rep: int = 0) -> int:
    return SEED_BASE + 1000 * int(workload) + int(rep)


@dataclass
class Grid:
    f0: float
    df: float
    nf: int

    def array(self) -> np.ndarray:
        return grid_array(self.f0, self.df, self.nf)


@dataclass
class Series:
    t: np.ndarray
    y: np.ndarray
    sigma: np.ndarray
    base_freqs: np.ndarray            # frequencies held fixed in the base model
    grid: Optional[Grid] = None
    true_freqs: np.ndarray = field(default_factory=lambda: np.zeros(0))
    pool: Optional[np.ndarray] = None  # candidate pool (tuple workloads)

    @property
    def N(self) -> int:
        return int(self.t.shape[0])


@dataclass
class Workload:
    name: str
    series: List[Series]


def grid_array(f0: float, df: float, nf: int) -> np.ndarray:
    return f0 + df * np.arange(nf, dtype=np.float64)


def _loguniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size))


def _sinusoids(rng, t, periods, amps):
    y = np.zeros_like(t)
    for P, A in zip(periods, amps):
        y += A * np.sin(2.0 * np.pi * t / P + rng.uniform(0.0, 2.0 * np.pi))
    return y


def seasonal_n200(rep: int = 0) -> Series:
    """N=200 over 1000 d with seasonal gaps (t mod 365 < 240), periods 13.7 d and
    87 d (amplitudes 5 and 3), offset 1, sigma ~ LogNormal(0, 0.3); constant base;
    grid f_j = j*5e-5, j = 1..20000 (0 < f <= 1 /d)."""
    rng = np.random.Generator(np.random.PCG64(seed_for(1, rep)))
    t = []
    while len(t) < 200:
        c = rng.uniform(0.0, 1000.0)
        if c % 365.0 < 240.0:
            t.append(c)
    t = np.sort(np.asarray(t))
    sigma = rng.lognormal(0.0, 0.3, t.size)
    y = 1.0 + _sinusoids(rng, t, [13.7, 87.0], [5.0, 3.0]) + sigma * rng.standard_normal(t.size)
    return Series(t, y, sigma, np.zeros(0), Grid(5e-5, 5e-5, 20000),
                  true_freqs=np.array([1 / 13.7, 1 / 87.0]))


def residual_n2000_p7(rep: int = 0, nf: int = 1_000_000) -> Series:
    """N=2000 over 3000 d, sigma ~ LogNormal(0, 0.5); four sinusoids with periods
    log-uniform in [2, 500] d and amplitudes U[1, 10]; base = constant + the first
    three of them; grid f_j = j*2e-6, j = 1..1e6 (0 < f <= 2 /d)."""
    rng = np.random.Generator(np.random.PCG64(seed_for(2, rep)))
    N = 2000
    t = np.sort(rng.uniform(0.0, 3000.0, N))
    sigma = rng.lognormal(0.0, 0.5, N)
    periods = _loguniform(rng, 2.0, 500.0, 4)
    amps = rng.uniform(1.0, 10.0, 4)
    y = _sinusoids(rng, t, periods, amps) + sigma * rng.standard_normal(N)
    df = 2.0 / 1_000_000
    return Series(t, y, sigma, 1.0 / periods[:3], Grid(df, df, nf), true_freqs=1.0 / periods)


def batch_4096(rep: int = 0, n_series: int = 4096, nf_lo: int = 10_000, nf_hi: int = 100_000,
               n_lo: int = 50, n_hi: int = 5000) -> Workload:
    """4096 independent series: N_s ~ U{50..5000}, span T_s ~ U[100, 5000] d, uniform
    times, 0-3 injected sinusoids (periods log-uniform in [2, T_s/2], amplitudes
    U[1, 10]), sigma ~ LogNormal(0, 0.4); base = constant + the first
    min(k_inj, U{0..2}) injected frequencies; nf_s ~ U{1e4..1e5}, f_j = j/nf_s."""
    rng = np.random.Generator(np.random.PCG64(seed_for(3, rep)))
    out = []
    for _ in range(n_series):
        N = int(rng.integers(n_lo, n_hi + 1))
        T = rng.uniform(100.0, 5000.0)
        t = np.sort(rng.uniform(0.0, T, N))
        sigma = rng.lognormal(0.0, 0.4, N)
        k = int(rng.integers(0, 4))
        periods = _loguniform(rng, 2.0, T / 2.0, k)
        amps = rng.uniform(1.0, 10.0, k)
        y = _sinusoids(rng, t, periods, amps) + sigma * rng.standard_normal(N)
        nb = min(k, int(rng.integers(0, 3)))
        nf = int(rng.integers(nf_lo, nf_hi + 1))
        out.append(Series(t, y, sigma, 1.0 / periods[:nb], Grid(1.0 / nf, 1.0 / nf, nf),
                          true_freqs=1.0 / periods))
    return Workload("batched", out)


def pool16_n1000(rep: int = 0, N: int = 1000, n_pool: int = 16) -> Series:
    """N=1000 over 2000 d, sigma ~ LogNormal(0, 0.4); six sinusoids (periods
    log-uniform in [2, 500] d, amplitudes U[1, 10]).  Pool of 16: the six true
    frequencies, six yearly/daily aliases (|f +- 1/365.25|, |1 - f|) of randomly
    chosen true ones and four noise frequencies U(0, 1), each perturbed by
    U(-0.3, 0.3)/T."""
    rng = np.random.Generator(np.random.PCG64(seed_for(4, rep)))
    T = 2000.0
    t = np.sort(rng.uniform(0.0, T, N))
    sigma = rng.lognormal(0.0, 0.4, N)
    periods = _loguniform(rng, 2.0, 500.0, 6)
    amps = rng.uniform(1.0, 10.0, 6)
    y = _sinusoids(rng, t, periods, amps) + sigma * rng.standard_normal(N)
    ftrue = 1.0 / periods
    pool = list(ftrue)
    while len(pool) < 12:
        f = ftrue[int(rng.integers(0, 6))]
        kind = int(rng.integers(0, 3))
        pool.append(abs(f + 1 / 365.25) if kind == 0 else abs(f - 1 / 365.25) if kind == 1 else abs(1.0 - f))
    pool += list(rng.uniform(0.0, 1.0, 4))
    pool = np.asarray(pool[:n_pool]) + rng.uniform(-0.3, 0.3, n_pool) / T
    return Series(t, y, sigma, np.zeros(0), None, true_freqs=ftrue, pool=np.abs(pool))


def nightly_n1e5_p11(rep: int = 0, N: int = 100_000, nf: int = 10_000_000) -> Series:
    """Survey-like series: 4000 nights, each kept with probability 0.7, with three
    60-night gaps per year at random places; points uniform inside a 0.3 d window
    of each kept night, counts chosen so that N is exact; sigma ~ LogNormal(0, 0.4);
    five sinusoids with periods log-uniform in [0.3, 1000] d; base = constant +
    those five; grid f_j = j*1e-6, j = 1..1e7 (0 < f <= 10 /d)."""
    rng = np.random.Generator(np.random.PCG64(seed_for(5, rep)))
    nights = np.arange(4000)
    keep = rng.uniform(size=4000) < 0.7
    for year in range(int(np.ceil(4000 / 365.25))):
        for _ in range(3):
            start = int(year * 365.25 + rng.uniform(0.0, 365.25))
            keep[start:start + 60] = False
    kept = nights[keep]
    counts = np.full(kept.size, N // kept.size)
    counts[rng.choice(kept.size, N - counts.sum(), replace=False)] += 1
    t = np.concatenate([n + rng.uniform(0.0, 0.3, c) for n, c in zip(kept, counts)])
    t = np.sort(t)
    sigma = rng.lognormal(0.0, 0.4, N)
    periods = _loguniform(rng, 0.3, 1000.0, 5)
    amps = rng.uniform(1.0, 10.0, 5)
    y = _sinusoids(rng, t, periods, amps) + sigma * rng.standard_normal(N)
    df = 10.0 / 10_000_000
    return Series(t, y, sigma, 1.0 / periods, Grid(df, df, nf), true_freqs=1.0 / periods)


def small_series(seed: int, N: int = 64, n_base: int = 1, span: float = 100.0,
                 n_sig: int = 2, nf: int = 300, fmax: float = 1.0) -> Series:
    """Small irregular series for parity tests (sizes the oracle finishes fast)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + seed))
    t = np.sort(rng.uniform(0.0, span, N))
    sigma = rng.lognormal(0.0, 0.4, N)
    periods = _loguniform(rng, 2.0, span / 2.0, max(n_sig, n_base))
    amps = rng.uniform(1.0, 10.0, periods.size)
    y = 0.7 + _sinusoids(rng, t, periods, amps) + sigma * rng.standard_normal(N)
    df = fmax / nf
    return Series(t, y, sigma, 1.0 / periods[:n_base], Grid(df, df, nf), true_freqs=1.0 / periods)


def uniform_series(seed: int, N: int = 64, dt: float = 1.0, t0: float = 0.0) -> Series:
    """Evenly sampled series (for the aliasing and Schuster special cases)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + seed))
    t = t0 + dt * np.arange(N, dtype=np.float64)
    sigma = np.ones(N)
    y = rng.standard_normal(N) + 2.0 * np.cos(2 * np.pi * 0.13 * t / dt + 0.4)
    return Series(t, y, sigma, np.zeros(0), None)


def make_workload(k: int, rep: int = 0, **kw):
    return {1: seasonal_n200, 2: residual_n2000_p7, 3: batch_4096, 4: pool16_n1000, 5: nightly_n1e5_p11}[k](rep, **kw)
