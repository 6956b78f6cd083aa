"""Python access to the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check and
by the bench's CPU-baseline leg, never by the product path.  The shared library
is built from oracle.c with the host C compiler on first use (or by
``build()``); nothing here imports the CUDA package.

All functions take and return float64 numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(path: str = _LIB, mutant: int = 0) -> str:
    """Compile oracle.c into a shared library.  ``mutant`` > 0 plants one known
    mistake (used only by the tests that check the pins catch it)."""
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
           f"-DORACLE_MUTANT={int(mutant)}", "-o", path, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    return path


def _needs_build(path: str) -> bool:
    return not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC)


class Oracle:
    """ctypes view of one compiled oracle library."""

    def __init__(self, path: Optional[str] = None, mutant: int = 0):
        if path is None:
            if mutant:
                path = os.path.join(tempfile.mkdtemp(prefix="oracle_mut"), f"liboracle_m{mutant}.so")
                build(path, mutant)
            else:
                path = _LIB
                if _needs_build(path):
                    build(path)
        self.lib = ctypes.CDLL(path)
        L = self.lib
        L.oracle_periodogram.argtypes = [_dp, _dp, _dp, ctypes.c_int64, _dp, ctypes.c_int, _dp,
                                         ctypes.c_int64, _dp, _dp, _dp, _dp]
        L.oracle_periodogram_grad.argtypes = [_dp, _dp, _dp, ctypes.c_int64, _dp, ctypes.c_int, _dp,
                                              ctypes.c_int64, _dp]
        L.oracle_periodogram_vjp.argtypes = [_dp, _dp, _dp, ctypes.c_int64, _dp, ctypes.c_int, _dp,
                                             ctypes.c_int64, _dp, _dp]
        L.oracle_l0.argtypes = [_dp, _dp, _dp, ctypes.c_int64]
        L.oracle_l0.restype = ctypes.c_double
        L.oracle_tuple_l.argtypes = [_dp, _dp, _dp, ctypes.c_int64, _dp, ctypes.c_int, _dp]
        L.oracle_tuple_l.restype = ctypes.c_double
        L.oracle_tuple_eval.argtypes = [_dp, _dp, _dp, ctypes.c_int64, _dp, _i64p, ctypes.c_int64, _dp, _dp]
        L.oracle_pool_table.argtypes = [_dp, _dp, _dp, ctypes.c_int64, _dp, ctypes.c_int, _dp]
        L.oracle_tuple_grad.argtypes = [_dp, _dp, _dp, ctypes.c_int64, _dp, _i64p, ctypes.c_int64, _dp, _dp]
        L.oracle_tuple_refine.argtypes = [_dp, _dp, _dp, ctypes.c_int64, _dp, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, _dp]
        L.oracle_tuple_refine.restype = ctypes.c_int
        L.oracle_periodogram_trend.argtypes = [_dp, _dp, _dp, ctypes.c_int64, _dp, ctypes.c_int, ctypes.c_int,
                                               _dp, ctypes.c_int64, _dp, _dp, _dp]
        L.oracle_fap_bound.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.oracle_fap_bound.restype = ctypes.c_double
        L.oracle_fap_threshold.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.oracle_fap_threshold.restype = ctypes.c_double
        L.oracle_cascade.argtypes = [_dp, ctypes.c_int, ctypes.c_int64, _dp, ctypes.c_char_p, _dp, _i64p]
        L.oracle_cascade_solutions.argtypes = [ctypes.c_char_p, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_uint32), ctypes.c_int64]
        L.oracle_cascade_solutions.restype = ctypes.c_int64


_default: Optional[Oracle] = None


def _lib() -> ctypes.CDLL:
    global _default
    if _default is None:
        _default = Oracle()
    return _default.lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp) if a is not None else None


def periodogram(t, y, sigma, base_freqs, fgrid, *, lib=None, want_coef=False, want_ratio=False):
    """z_j = (chi2_base - chi2_j)/2 for every trial frequency (residual
    periodogram, joint refit of the base amplitudes).  Returns z, chi2_base and,
    on request, coef (nf, 2: a_j, b_j in raw time) and ratio (nf)."""
    L = lib or _lib()
    t, y, sigma, base, f = map(_d, (t, y, sigma, base_freqs, fgrid))
    nf = f.size
    z = np.empty(nf)
    c2 = np.zeros(1)
    coef = np.empty((nf, 2)) if want_coef else None
    ratio = np.empty(nf) if want_ratio else None
    rc = L.oracle_periodogram(_p(t), _p(y), _p(sigma), t.size, _p(base), base.size, _p(f), nf,
                              _p(z), _p(c2), _p(coef), _p(ratio))
    if rc:
        raise ValueError("oracle_periodogram rejected its arguments")
    out = [z, float(c2[0])]
    if want_coef:
        out.append(coef)
    if want_ratio:
        out.append(ratio)
    return tuple(out)


def periodogram_trend(t, y, sigma, base_freqs, trend, fgrid, *, lib=None, want_ratio=False):
    """Residual periodogram whose base model has a polynomial of degree
    ``trend`` in time instead of the constant.  Returns z, chi2_base and, on
    request, the trial columns' conditioning ratio."""
    L = lib or _lib()
    t, y, sigma, base, f = map(_d, (t, y, sigma, base_freqs, fgrid))
    z = np.empty(f.size)
    c2 = np.zeros(1)
    ratio = np.empty(f.size) if want_ratio else None
    if L.oracle_periodogram_trend(_p(t), _p(y), _p(sigma), t.size, _p(base), base.size, int(trend), _p(f),
                                  f.size, _p(z), _p(c2), _p(ratio)):
        raise ValueError("oracle_periodogram_trend rejected its arguments")
    return (z, float(c2[0]), ratio) if want_ratio else (z, float(c2[0]))


def log_form(z, chi2_base, N, n_alt, trend=0):
    """Log form of Eq. zpowrel: (N_H/2) ln(l_base / (l_base - 2 z)) with
    N_H = N - 3 n_alt - 1 - trend (n_alt frequencies in the alternative
    model, a polynomial of degree trend in place of the constant)."""
    NH = N - 3 * n_alt - 1 - trend
    l_new = chi2_base - 2.0 * np.asarray(z, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(l_new > 0, 0.5 * NH * np.log(chi2_base / l_new), np.inf)


def periodogram_grad(t, y, sigma, base_freqs, fgrid, *, lib=None):
    L = lib or _lib()
    t, y, sigma, base, f = map(_d, (t, y, sigma, base_freqs, fgrid))
    g = np.empty(f.size)
    if L.oracle_periodogram_grad(_p(t), _p(y), _p(sigma), t.size, _p(base), base.size, _p(f), f.size, _p(g)):
        raise ValueError("oracle_periodogram_grad rejected its arguments")
    return g


def periodogram_vjp(t, y, sigma, base_freqs, fgrid, v, *, lib=None):
    L = lib or _lib()
    t, y, sigma, base, f, v = map(_d, (t, y, sigma, base_freqs, fgrid, v))
    out = np.empty(t.size)
    if L.oracle_periodogram_vjp(_p(t), _p(y), _p(sigma), t.size, _p(base), base.size, _p(f), f.size,
                                _p(v), _p(out)):
        raise ValueError("oracle_periodogram_vjp rejected its arguments")
    return out


def l0(t, y, sigma, *, lib=None) -> float:
    L = lib or _lib()
    t, y, sigma = map(_d, (t, y, sigma))
    return float(L.oracle_l0(_p(t), _p(y), _p(sigma), t.size))


def tuple_l(t, y, sigma, freqs, *, lib=None, want_theta=False):
    L = lib or _lib()
    t, y, sigma, f = map(_d, (t, y, sigma, freqs))
    th = np.empty(2 * f.size + 1)
    l = float(L.oracle_tuple_l(_p(t), _p(y), _p(sigma), t.size, _p(f), f.size, _p(th)))
    return (l, th) if want_theta else l


def _csr(tuples: Sequence[Sequence[float]]):
    off = np.zeros(len(tuples) + 1, dtype=np.int64)
    for k, tp in enumerate(tuples):
        off[k + 1] = off[k] + len(tp)
    flat = np.concatenate([np.asarray(tp, dtype=np.float64) for tp in tuples]) if off[-1] else np.zeros(0)
    return np.ascontiguousarray(flat), off


def tuple_eval(t, y, sigma, tuples, *, lib=None):
    """z_k = (l_0 - l_k)/2 for each tuple (constant base).  Returns z, l_0."""
    L = lib or _lib()
    t, y, sigma = map(_d, (t, y, sigma))
    flat, off = _csr(tuples)
    z = np.empty(len(tuples))
    l0v = np.zeros(1)
    if L.oracle_tuple_eval(_p(t), _p(y), _p(sigma), t.size, _p(flat), off.ctypes.data_as(_i64p),
                           len(tuples), _p(z), _p(l0v)):
        raise ValueError("oracle_tuple_eval rejected its arguments")
    return z, float(l0v[0])


def pool_table(t, y, sigma, pool, *, lib=None):
    """l_table[mask] for every subset of the pool; entry 0 is l_0."""
    L = lib or _lib()
    t, y, sigma, pool = map(_d, (t, y, sigma, pool))
    out = np.empty(1 << pool.size)
    if L.oracle_pool_table(_p(t), _p(y), _p(sigma), t.size, _p(pool), pool.size, _p(out)):
        raise ValueError("oracle_pool_table rejected its arguments")
    return out


def tuple_grad(t, y, sigma, tuples, *, lib=None):
    """z and dz/df (flattened in the tuples' order) for each tuple."""
    L = lib or _lib()
    t, y, sigma = map(_d, (t, y, sigma))
    flat, off = _csr(tuples)
    z = np.empty(len(tuples))
    g = np.empty(flat.size)
    if L.oracle_tuple_grad(_p(t), _p(y), _p(sigma), t.size, _p(flat), off.ctypes.data_as(_i64p),
                           len(tuples), _p(z), _p(g)):
        raise ValueError("oracle_tuple_grad rejected its arguments")
    return z, g


def tuple_refine(t, y, sigma, freqs, *, max_iter=50, tol=1e-10, lib=None):
    """Gauss-Newton refinement of one tuple.  Returns (freqs, l, iterations)."""
    L = lib or _lib()
    t, y, sigma = map(_d, (t, y, sigma))
    f = _d(freqs).copy()
    lout = np.zeros(1)
    it = L.oracle_tuple_refine(_p(t), _p(y), _p(sigma), t.size, _p(f), f.size, int(max_iter),
                               float(tol), _p(lout))
    if it < 0:
        raise ValueError("oracle_tuple_refine rejected its arguments")
    return f, float(lout[0]), int(it)


# ---------------------------------------------------------------------------
# Phase 3 backward cascade, non-nested solutions, Phase 4 ordering (Sect. 4)

def fap_bound(n, A, W, z, *, lib=None) -> float:
    """M_n(z) = A W^n exp(-z) z^(3n/2-1) (Eq. zFAP; A supplied by the caller)."""
    L = lib or _lib()
    return float(L.oracle_fap_bound(int(n), float(A), float(W), float(z)))


def fap_threshold(n, A, W, fap, *, lib=None) -> float:
    """z with M_n(z) = fap on the decreasing branch of M_n."""
    L = lib or _lib()
    return float(L.oracle_fap_threshold(int(n), float(A), float(W), float(fap)))


def effective_bandwidth(t, sigma, f_max) -> float:
    """W = f_max T_eff with T_eff = sqrt(4 pi Var(t)), Var the weighted
    variance of the times with weights 1/sigma^2 (Sect. 2)."""
    t, sigma = map(_d, (t, sigma))
    w = 1.0 / sigma ** 2
    tm = np.sum(w * t) / np.sum(w)
    var = np.sum(w * (t - tm) ** 2) / np.sum(w)
    return float(f_max * np.sqrt(4.0 * np.pi * var))


def cascade(l_table, N, zthr, *, lib=None):
    """Phase 3 on a subtuple table.  Returns (pass (uint8, 2^n), slack (2^n),
    number of tests formed)."""
    L = lib or _lib()
    l = _d(l_table)
    n = int(l.size).bit_length() - 1
    if l.size != 1 << n:
        raise ValueError("l_table length must be a power of two")
    zt = _d(zthr)
    if zt.size < n:
        raise ValueError("need one threshold per number of added frequencies")
    ps = ctypes.create_string_buffer(l.size)
    slack = np.empty(l.size)
    nt = np.zeros(1, dtype=np.int64)
    if L.oracle_cascade(_p(l), n, int(N), _p(zt), ps, _p(slack), nt.ctypes.data_as(_i64p)):
        raise ValueError("oracle_cascade rejected its arguments")
    return np.frombuffer(ps.raw, dtype=np.uint8).copy(), slack, int(nt[0])


def cascade_solutions(passed, *, lib=None) -> np.ndarray:
    """Passing masks contained in no other passing mask, in increasing order."""
    L = lib or _lib()
    passed = np.ascontiguousarray(np.asarray(passed, dtype=np.uint8))
    n = int(passed.size).bit_length() - 1
    buf = ctypes.create_string_buffer(passed.tobytes(), passed.size)
    cnt = L.oracle_cascade_solutions(buf, n, None, 0)
    out = np.zeros(max(cnt, 1), dtype=np.uint32)
    L.oracle_cascade_solutions(buf, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), cnt)
    return out[:cnt]


def phase4_order(masks, l_table, N):
    """Phase 4 as far as the paper defines it: the solutions grouped by their
    number of frequencies m and, within a group, in increasing chi2; with the
    goodness of fit G = (l_S / l_0) (N - 1) / (N - 3m - 1) (ratio of reduced
    chi2 of H_m and H_0).  Returns (masks, G) in that order."""
    rows = []
    for S in masks:
        S = int(S)
        m = bin(S).count("1")
        rows.append((m, float(l_table[S]), S))
    rows.sort()
    l0v = float(l_table[0])
    ms = np.array([r[2] for r in rows], dtype=np.uint32)
    G = np.array([(r[1] / l0v) * (N - 1) / (N - 3 * r[0] - 1) for r in rows])
    return ms, G
