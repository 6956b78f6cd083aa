"""B300-native FREDEC hot path: residual and multifrequency periodograms.

A thin Python binding of libfredec.so (C ABI declared in include/fredec.h).
This module only marshals arguments: every step of the computation runs in
the library's CUDA kernels.  numpy arrays go through the host-pointer entry
points; CUDA torch tensors through the stream-ordered ``*_dev`` entry points
on torch's current stream.

If the shared library has not been built, every call raises: there is no
CPU fallback.  Build it with ``python -m paper_1309_0100_b300._build``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

__all__ = [
    "FredecError", "FP64", "MIXED", "lib", "version", "periodogram", "periodogram_dev", "periodogram_grad",
    "periodogram_grad_dev",
    "periodogram_vjp", "periodogram_vjp_dev", "tuple_eval", "pool_subtuples_eval", "tuple_grad", "tuple_grad_dev",
    "tuple_refine", "pool_refine", "periodogram_batch", "BatchPlan", "tune", "profile_events", "pipe_peaks", "LIB_PATH",
    "fap_bound", "fap_threshold", "effective_bandwidth", "cascade", "scan", "decompose", "Z_DIFF", "Z_LOG",
]

FP64 = 0
MIXED = 1
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libfredec.so")

_c_dp = ctypes.POINTER(ctypes.c_double)
_c_i64p = ctypes.POINTER(ctypes.c_int64)
_c_i32p = ctypes.POINTER(ctypes.c_int32)
_vp = ctypes.c_void_p


class FredecError(RuntimeError):
    STATUS = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ESINGULAR", 5: "ETIMEOUT"}

    def __init__(self, code: int, msg: str):
        self.code = code
        self.status = self.STATUS.get(code, str(code))
        super().__init__(f"fredec {self.status}: {msg}")


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("topk", ctypes.c_int32), ("fpt", ctypes.c_int32),
                ("warps", ctypes.c_int32), ("flag_tau", ctypes.c_double), ("trend", ctypes.c_int32),
                ("statistic", ctypes.c_int32)]


class ScanOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("max_pool", ctypes.c_int32), ("max_base", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("z_thr0", ctypes.c_double), ("z_thr1", ctypes.c_double),
                ("half", ctypes.c_double), ("merge_dist", ctypes.c_double)]


class DecomposeOpts(ctypes.Structure):
    _fields_ = [("scan", ScanOpts), ("z_thr", ctypes.POINTER(ctypes.c_double)),
                ("refine_precision", ctypes.c_int32), ("refine_iter", ctypes.c_int32),
                ("refine_tol", ctypes.c_double)]


MAX_TUPLE = 20
MAX_NBASE = 12

_lib_handle = None


def lib() -> ctypes.CDLL:
    """The loaded libfredec.so (raises if it was not built)."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(LIB_PATH):
        raise FredecError(3, f"{LIB_PATH} is missing: build it with python -m paper_1309_0100_b300._build")
    L = ctypes.CDLL(LIB_PATH)
    d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int32
    sig = {
        "fredec_opts_init": (None, [ctypes.POINTER(Opts)]),
        "fredec_last_error": (ctypes.c_char_p, []),
        "fredec_version": (ctypes.c_char_p, []),
        "fredec_periodogram": (ctypes.c_int, [_c_dp, _c_dp, _c_dp, i64, _c_dp, i32, _c_dp, i64, _c_dp]),
        "fredec_periodogram_ex": (ctypes.c_int, [_c_dp, _c_dp, _c_dp, i64, _c_dp, i32, _c_dp, i64,
                                                 ctypes.POINTER(Opts), _c_dp, _c_dp, _c_i64p, _c_dp]),
        "fredec_periodogram_dev": (ctypes.c_int, [_vp, _vp, _vp, i64, _vp, i32, d, d, i64, ctypes.POINTER(Opts),
                                                  _vp, _vp, _vp, _vp, _vp]),
        "fredec_periodogram_vjp_dev": (ctypes.c_int, [_vp, _vp, _vp, i64, _vp, i32, d, d, i64, _vp, _vp, _vp, i32,
                                                      _vp, _vp]),
        "fredec_periodogram_vjp": (ctypes.c_int, [_c_dp, _c_dp, _c_dp, i64, _c_dp, i32, d, d, i64, _c_dp, i32,
                                                  _c_dp]),
        "fredec_tuple_eval": (ctypes.c_int, [_c_dp, _c_dp, _c_dp, i64, _c_dp, _c_i64p, i64, _c_dp, _c_dp]),
        "fredec_pool_subtuples_eval": (ctypes.c_int, [_c_dp, _c_dp, _c_dp, i64, _c_dp, i32, _c_dp]),
        "fredec_tuple_grad": (ctypes.c_int, [_c_dp, _c_dp, _c_dp, i64, _c_dp, _c_i64p, i64, i32, _c_dp, _c_dp]),
        "fredec_tuple_grad_dev": (ctypes.c_int, [_vp, _vp, _vp, i64, _vp, _c_i64p, i64, i32, _vp, _vp, _vp]),
        "fredec_tuple_refine": (ctypes.c_int, [_c_dp, _c_dp, _c_dp, i64, _c_dp, _c_i64p, i64, i32, d, i32, _c_dp,
                                               _c_i32p]),
        "fredec_periodogram_batch": (ctypes.c_int, [_c_dp, _c_dp, _c_dp, _c_i64p, i64, _c_dp, _c_i64p, _c_dp, _c_dp,
                                                    _c_i64p, _c_i64p, ctypes.POINTER(Opts), _c_dp, _c_i64p]),
        "fredec_batch_plan_create": (ctypes.c_int, [ctypes.POINTER(_vp), _c_dp, _c_dp, _c_dp, _c_i64p, i64, _c_dp,
                                                    _c_i64p, _c_dp, _c_dp, _c_i64p, _c_i64p, ctypes.POINTER(Opts)]),
        "fredec_batch_plan_run": (ctypes.c_int, [_vp, _vp]),
        "fredec_batch_plan_outputs": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _c_i64p,
                                                     _c_i64p]),
        "fredec_batch_plan_download": (ctypes.c_int, [_vp, _c_dp, _c_i64p]),
        "fredec_batch_plan_destroy": (None, [_vp]),
        "fredec_tune": (ctypes.c_int, [i32, i32, i64, i64, _c_i32p, _c_i32p]),
        "fredec_profile_events": (ctypes.c_int, [_vp, _vp]),
        "fredec_pool_refine": (ctypes.c_int, [_c_dp, _c_dp, _c_dp, i64, _c_dp, i32, ctypes.POINTER(ctypes.c_uint32),
                                              i64, i32, d, i32, _c_dp, _c_dp, _c_i32p]),
        "fredec_pipe_peaks": (ctypes.c_int, [_c_dp]),
        "fredec_topk_dev": (ctypes.c_int, [_vp, i64, i32, _vp, _vp]),
        "fredec_selftest_wait_timeout": (ctypes.c_int, [_c_i32p]),
        "fredec_selftest_ff_sincos": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), i64, _c_dp]),
        "fredec_periodogram_noalloc_dev": (ctypes.c_int, [_vp, _vp, _vp, i64, _vp, i32, d, d, i64,
                                                          ctypes.POINTER(Opts), _vp, _vp, _vp]),
        "fredec_periodogram_grad_dev": (ctypes.c_int, [_vp, _vp, _vp, i64, _vp, i32, d, d, i64,
                                                       ctypes.POINTER(Opts), _vp, _vp, _vp, _vp]),
        "fredec_periodogram_grad": (ctypes.c_int, [_c_dp, _c_dp, _c_dp, i64, _c_dp, i32, d, d, i64,
                                                   ctypes.POINTER(Opts), _c_dp, _c_dp, _c_dp]),
        "fredec_fap_bound": (d, [i32, d, d, d]),
        "fredec_fap_threshold": (d, [i32, d, d, d]),
        "fredec_effective_bandwidth": (ctypes.c_int, [_c_dp, _c_dp, i64, d, _c_dp]),
        "fredec_cascade": (ctypes.c_int, [_c_dp, i32, i64, _c_dp, ctypes.POINTER(ctypes.c_uint32),
                                          ctypes.POINTER(ctypes.c_uint32), _c_dp, i64, _c_i64p]),
        "fredec_scan_opts_init": (None, [ctypes.POINTER(ScanOpts)]),
        "fredec_decompose_opts_init": (None, [ctypes.POINTER(DecomposeOpts)]),
        "fredec_scan": (ctypes.c_int, [_c_dp, _c_dp, _c_dp, i64, d, d, i64, ctypes.POINTER(ScanOpts), _c_dp, _c_dp,
                                       _c_i32p, _c_dp, _c_i32p, _c_i32p]),
        "fredec_decompose": (ctypes.c_int, [_c_dp, _c_dp, _c_dp, i64, d, d, i64, ctypes.POINTER(DecomposeOpts),
                                            _c_dp, _c_i32p, _c_dp, ctypes.POINTER(ctypes.c_uint32), _c_dp, _c_dp,
                                            _c_dp, i64, _c_i64p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib_handle = L
    return L


def version() -> str:
    return lib().fredec_version().decode()


def _check(rc: int):
    if rc != 0:
        raise FredecError(rc, lib().fredec_last_error().decode())


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _p(a: Optional[np.ndarray]):
    if a is None:
        return None
    if a.dtype == np.float64:
        return a.ctypes.data_as(_c_dp)
    if a.dtype == np.int64:
        return a.ctypes.data_as(_c_i64p)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_c_i32p)
    raise TypeError(a.dtype)


def _prec(precision) -> int:
    if isinstance(precision, str):
        return {"fp64": FP64, "mixed": MIXED}[precision.lower()]
    return int(precision)


Z_DIFF = 0   # statistic: (l_base - l_new)/2
Z_LOG = 1    # statistic: log form (N_H/2) ln(l_base/l_new)


def _stat(statistic) -> int:
    if isinstance(statistic, str):
        return {"diff": Z_DIFF, "log": Z_LOG}[statistic.lower()]
    return int(statistic)


def _opts(precision=FP64, topk=0, fpt=0, warps=0, flag_tau=0.0, trend=0, statistic=Z_DIFF) -> Opts:
    o = Opts()
    lib().fredec_opts_init(ctypes.byref(o))
    o.precision = _prec(precision)
    o.topk = int(topk)
    o.fpt = int(fpt)
    o.warps = int(warps)
    o.flag_tau = float(flag_tau)
    o.trend = int(trend)
    o.statistic = _stat(statistic)
    return o


# ---------------------------------------------------------------------------
# Residual periodogram

def periodogram(t, y, sigma, base_freqs, f_grid, *, precision=FP64, topk=0, want_coef=False, want_info=False,
                fpt=0, warps=0, flag_tau=0.0, trend=0, statistic=Z_DIFF, out=None):
    """z(f) for every trial frequency (host arrays in, host arrays out).
    ``trend``: degree of the base model's time polynomial (0 = constant);
    ``statistic``: "diff" (default) or "log" (log form of Eq. zpowrel).

    Returns z, or a tuple (z, [topk_idx], [info], [coef]) when extras are
    requested.  info = (chi2_base, sum of weights, time origin t_c); coef
    (nf, 2) = fitted amplitudes of cos/sin of 2 pi f (t - t_c).
    """
    t, y, sigma, f = map(_f64, (t, y, sigma, f_grid))
    base = _f64(base_freqs)
    nf = f.size
    z = out if out is not None else np.empty(nf)
    if z.dtype != np.float64 or z.size != nf or not z.flags.c_contiguous:
        raise TypeError("out must be a contiguous float64 array of size nf")
    top = np.empty(max(int(topk), 1), dtype=np.int64) if topk else None
    info = np.empty(3) if want_info else None
    coef = np.empty((nf, 2)) if want_coef else None
    o = _opts(precision, topk, fpt, warps, flag_tau, trend, statistic)
    _check(lib().fredec_periodogram_ex(_p(t), _p(y), _p(sigma), t.size, _p(base) if base.size else None, base.size,
                                       _p(f), nf, ctypes.byref(o), _p(z), _p(info), _p(top), _p(coef)))
    if not (topk or want_info or want_coef):
        return z
    out = [z]
    if topk:
        out.append(top[:topk])
    if want_info:
        out.append(info)
    if want_coef:
        out.append(coef)
    return tuple(out)


def _dptr(x) -> int:
    return 0 if x is None else int(x.data_ptr())


def _stream(torch, stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def periodogram_dev(t, y, sigma, base_freqs, f0: float, df: float, nf: int, *, precision=FP64, topk=0,
                    want_coef=False, fpt=0, warps=0, flag_tau=0.0, trend=0, statistic=Z_DIFF, out=None,
                    stream=None):
    """Device path on the uniform grid f_j = f0 + j df (torch CUDA tensors,
    float64, contiguous).  Enqueued on torch's current stream (or ``stream``).
    Returns dict with z, info (3), and optionally topk (int64) and coef."""
    import torch
    dev = t.device
    for x in (t, y, sigma, base_freqs):
        if x.dtype != torch.float64 or not x.is_cuda or not x.is_contiguous():
            raise TypeError("periodogram_dev wants contiguous float64 CUDA tensors")
    z = out if out is not None else torch.empty(nf, dtype=torch.float64, device=dev)
    info = torch.empty(3, dtype=torch.float64, device=dev)
    top = torch.empty(max(topk, 1), dtype=torch.int64, device=dev) if topk else None
    coef = torch.empty((nf, 2), dtype=torch.float64, device=dev) if want_coef else None
    o = _opts(precision, topk, fpt, warps, flag_tau, trend, statistic)
    _check(lib().fredec_periodogram_dev(_dptr(t), _dptr(y), _dptr(sigma), t.numel(),
                                        _dptr(base_freqs) if base_freqs.numel() else None, base_freqs.numel(),
                                        float(f0), float(df), int(nf), ctypes.byref(o), _dptr(z), _dptr(info),
                                        _dptr(top), _dptr(coef), _stream(torch, stream)))
    res = {"z": z, "info": info}
    if topk:
        res["topk"] = top[:topk]
    if want_coef:
        res["coef"] = coef
    return res


def periodogram_grad(t, y, sigma, base_freqs, f0: float, df: float, nf: int, *, precision=FP64, trend=0,
                     want_info=False):
    """z and dz/df on the uniform grid f_j = f0 + j df (host arrays in and
    out).  Returns (z, dzdf) or (z, dzdf, info)."""
    t, y, sigma = map(_f64, (t, y, sigma))
    base = _f64(base_freqs)
    z = np.empty(max(int(nf), 1))
    g = np.empty(max(int(nf), 1))
    info = np.empty(3)
    o = _opts(precision, 0, 0, 0, 0.0, trend, Z_DIFF)
    _check(lib().fredec_periodogram_grad(_p(t), _p(y), _p(sigma), t.size, _p(base) if base.size else None,
                                         base.size, float(f0), float(df), int(nf), ctypes.byref(o), _p(z), _p(g),
                                         _p(info)))
    return (z[:nf], g[:nf], info) if want_info else (z[:nf], g[:nf])


def periodogram_grad_dev(t, y, sigma, base_freqs, f0: float, df: float, nf: int, *, precision=FP64, trend=0,
                         warps=0, out=None, out_grad=None, stream=None):
    """Device path of periodogram_grad (contiguous float64 CUDA tensors, torch's
    current stream or ``stream``).  Returns dict with z, dzdf and info."""
    import torch
    dev = t.device
    for x in (t, y, sigma, base_freqs):
        if x.dtype != torch.float64 or not x.is_cuda or not x.is_contiguous():
            raise TypeError("periodogram_grad_dev wants contiguous float64 CUDA tensors")
    z = out if out is not None else torch.empty(nf, dtype=torch.float64, device=dev)
    g = out_grad if out_grad is not None else torch.empty(nf, dtype=torch.float64, device=dev)
    info = torch.empty(3, dtype=torch.float64, device=dev)
    o = _opts(precision, 0, 0, warps, 0.0, trend, Z_DIFF)
    _check(lib().fredec_periodogram_grad_dev(_dptr(t), _dptr(y), _dptr(sigma), t.numel(),
                                             _dptr(base_freqs) if base_freqs.numel() else None, base_freqs.numel(),
                                             float(f0), float(df), int(nf), ctypes.byref(o), _dptr(z), _dptr(g),
                                             _dptr(info), _stream(torch, stream)))
    return {"z": z, "dzdf": g, "info": info}


def topk_dev(z, k: int, *, stream=None):
    """Top-k local maxima of a contiguous float64 CUDA tensor z (device kernels;
    ranks by decreasing z, ties to the lower index, -1 where fewer exist)."""
    import torch
    if z.dtype != torch.float64 or not z.is_cuda or not z.is_contiguous():
        raise TypeError("topk_dev wants a contiguous float64 CUDA tensor")
    out = torch.empty(max(int(k), 1), dtype=torch.int64, device=z.device)
    _check(lib().fredec_topk_dev(_dptr(z) if z.numel() else None, z.numel(), int(k), _dptr(out),
                                 _stream(torch, stream)))
    return out


def periodogram_vjp_dev(t, y, sigma, base_freqs, f0, df, nf, coef, info, v, *, precision=FP64, out=None,
                        stream=None):
    """dL/dy = sum_j v_j dz_j/dy on the device (inputs from a forward call)."""
    import torch
    g = out if out is not None else torch.empty_like(y)
    _check(lib().fredec_periodogram_vjp_dev(_dptr(t), _dptr(y), _dptr(sigma), t.numel(),
                                            _dptr(base_freqs) if base_freqs.numel() else None, base_freqs.numel(),
                                            float(f0), float(df), int(nf), _dptr(coef), _dptr(info), _dptr(v),
                                            _prec(precision), _dptr(g), _stream(torch, stream)))
    return g


def periodogram_vjp(t, y, sigma, base_freqs, f0, df, nf, v, *, precision=FP64):
    t, y, sigma, base, v = map(_f64, (t, y, sigma, base_freqs, v))
    g = np.empty(t.size)
    _check(lib().fredec_periodogram_vjp(_p(t), _p(y), _p(sigma), t.size, _p(base) if base.size else None, base.size,
                                        float(f0), float(df), int(nf), _p(v), _prec(precision), _p(g)))
    return g


# ---------------------------------------------------------------------------
# Tuples

def _csr(tuples: Sequence[Sequence[float]]):
    off = np.zeros(len(tuples) + 1, dtype=np.int64)
    for k, tp in enumerate(tuples):
        off[k + 1] = off[k] + len(tp)
    flat = np.concatenate([np.asarray(tp, dtype=np.float64) for tp in tuples]) if off[-1] else np.zeros(1)
    return np.ascontiguousarray(flat), off


def tuple_eval(t, y, sigma, tuples):
    """z_k = (l_0 - l(S_k))/2 for each tuple (constant base). Returns (z, l0)."""
    t, y, sigma = map(_f64, (t, y, sigma))
    flat, off = _csr(tuples)
    z = np.empty(max(len(tuples), 1))
    l0 = np.empty(1)
    _check(lib().fredec_tuple_eval(_p(t), _p(y), _p(sigma), t.size, _p(flat), _p(off), len(tuples), _p(z), _p(l0)))
    return z[:len(tuples)], float(l0[0])


def pool_subtuples_eval(t, y, sigma, pool):
    """l_table[mask] for all subsets of the pool (entry 0 = l_0)."""
    t, y, sigma, pool = map(_f64, (t, y, sigma, pool))
    out = np.empty(1 << pool.size)
    _check(lib().fredec_pool_subtuples_eval(_p(t), _p(y), _p(sigma), t.size, _p(pool), pool.size, _p(out)))
    return out


def tuple_grad(t, y, sigma, tuples, *, precision=FP64):
    """(z, dz/df flattened in tuple order)."""
    t, y, sigma = map(_f64, (t, y, sigma))
    flat, off = _csr(tuples)
    z = np.empty(max(len(tuples), 1))
    g = np.empty(max(int(off[-1]), 1))
    _check(lib().fredec_tuple_grad(_p(t), _p(y), _p(sigma), t.size, _p(flat), _p(off), len(tuples),
                                   _prec(precision), _p(z), _p(g)))
    return z[:len(tuples)], g[:int(off[-1])]


def tuple_grad_dev(t, y, sigma, freqs, offsets, *, precision=FP64, stream=None):
    """Device path of tuple_grad: t, y, sigma, freqs contiguous float64 CUDA
    tensors (freqs flattened in CSR order), offsets a host int64 array or CPU
    tensor of n_tuples + 1 entries.  Returns (z, dzdf) CUDA tensors, enqueued
    on torch's current stream (or ``stream``)."""
    import torch
    for x in (t, y, sigma, freqs):
        if x.dtype != torch.float64 or not x.is_cuda or not x.is_contiguous():
            raise TypeError("tuple_grad_dev wants contiguous float64 CUDA tensors")
    off = _i64(offsets.cpu().numpy() if hasattr(offsets, "cpu") else offsets)
    n = off.size - 1
    z = torch.empty(max(n, 1), dtype=torch.float64, device=t.device)
    g = torch.empty(max(freqs.numel(), 1), dtype=torch.float64, device=t.device)
    _check(lib().fredec_tuple_grad_dev(_dptr(t), _dptr(y), _dptr(sigma), t.numel(),
                                       _dptr(freqs) if freqs.numel() else None, _p(off), n, _prec(precision),
                                       _dptr(z), _dptr(g), _stream(torch, stream)))
    return z[:n], g[:freqs.numel()]


def tuple_refine(t, y, sigma, tuples, *, max_iter=20, tol=1e-9, precision=FP64):
    """Gauss-Newton refinement of every tuple.  Returns (list of refined
    frequency arrays, l, iterations)."""
    t, y, sigma = map(_f64, (t, y, sigma))
    flat, off = _csr(tuples)
    flat = flat.copy()
    n = len(tuples)
    l = np.empty(max(n, 1))
    it = np.empty(max(n, 1), dtype=np.int32)
    _check(lib().fredec_tuple_refine(_p(t), _p(y), _p(sigma), t.size, _p(flat), _p(off), n, int(max_iter),
                                     float(tol), _prec(precision), _p(l), _p(it)))
    return [flat[off[k]:off[k + 1]].copy() for k in range(n)], l[:n], it[:n]


def pool_refine(t, y, sigma, pool, masks=None, *, max_iter=20, tol=1e-9, precision=FP64):
    """Refine subtuples of a pool (all 2^n - 1 non-empty ones by default).
    Returns (masks, f (n_masks, n_pool), l, iterations)."""
    t, y, sigma, pool = map(_f64, (t, y, sigma, pool))
    n = pool.size
    if masks is None:
        masks = np.arange(1, 1 << n, dtype=np.uint32)
    masks = np.ascontiguousarray(np.asarray(masks, dtype=np.uint32))
    f = np.empty((max(masks.size, 1), n))
    l = np.empty(max(masks.size, 1))
    it = np.empty(max(masks.size, 1), dtype=np.int32)
    _check(lib().fredec_pool_refine(_p(t), _p(y), _p(sigma), t.size, _p(pool), n,
                                    masks.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), masks.size, int(max_iter),
                                    float(tol), _prec(precision), _p(f), _p(l), _p(it)))
    return masks, f[:masks.size], l[:masks.size], it[:masks.size]


# ---------------------------------------------------------------------------
# Phase 3 backward cascade, Phase 4 ordering, FAP levels

def fap_bound(n, A, W, z) -> float:
    """M_n(z) = A W^n exp(-z) z^(3n/2 - 1) (Eq. zFAP, A supplied by the caller)."""
    return float(lib().fredec_fap_bound(int(n), float(A), float(W), float(z)))


def fap_threshold(n, A, W, fap) -> float:
    """The z at which M_n(z) = fap on the decreasing branch."""
    return float(lib().fredec_fap_threshold(int(n), float(A), float(W), float(fap)))


def effective_bandwidth(t, sigma, f_max) -> float:
    """W = f_max sqrt(4 pi Var_w(t)) (weights 1/sigma^2)."""
    t, sigma = map(_f64, (t, sigma))
    out = np.zeros(1)
    _check(lib().fredec_effective_bandwidth(_p(t), _p(sigma), t.size, float(f_max), _p(out)))
    return float(out[0])


def cascade(l_table, N, z_thr, *, want_pass=False, capacity=None):
    """Phase 3 on a subtuple table: the non-nested passing combinations in the
    order of Phase 4.  Returns (masks, G) and, with want_pass, the pass flags
    as a uint8 array over all masks."""
    l = _f64(l_table)
    n = int(l.size).bit_length() - 1
    if l.size != 1 << n:
        raise ValueError("l_table length must be a power of two")
    zt = _f64(z_thr)
    if zt.size < n:
        raise ValueError("need one threshold per number of added frequencies")
    words = np.zeros(max(1, l.size // 32), dtype=np.uint32)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    cnt = np.zeros(1, dtype=np.int64)
    cap = 1 << 16 if capacity is None else int(capacity)
    while True:
        masks = np.zeros(max(cap, 1), dtype=np.uint32)
        G = np.empty(max(cap, 1))
        _check(lib().fredec_cascade(_p(l), n, int(N), _p(zt) if zt.size else None,
                                    words.ctypes.data_as(u32p) if want_pass else None,
                                    masks.ctypes.data_as(u32p), _p(G), cap, _p(cnt)))
        if capacity is not None or cnt[0] <= cap:
            break
        cap = int(cnt[0])
    k = min(int(cnt[0]), cap)
    out = (masks[:k], G[:k])
    if want_pass:
        bits = np.unpackbits(words.view(np.uint8), bitorder="little")[: l.size]
        out = out + (bits.astype(np.uint8),)
    return out


def _scan_opts(z_thr0, z_thr1, precision, max_pool, max_base, half, merge_dist):
    o = ScanOpts()
    lib().fredec_scan_opts_init(ctypes.byref(o))
    o.precision = _prec(precision)
    o.max_pool = int(max_pool)
    o.max_base = int(max_base)
    o.z_thr0 = float(z_thr0)
    o.z_thr1 = float(z_thr1)
    o.half = float(half)
    o.merge_dist = float(merge_dist)
    return o


def scan(t, y, sigma, f0, df, nf, z_thr0, z_thr1, *, precision=FP64, max_pool=0, max_base=0, half=0.5,
         merge_dist=0.0):
    """Phase 1 scan.  Returns (pool, pool_z, base, truncated)."""
    t, y, sigma = map(_f64, (t, y, sigma))
    o = _scan_opts(z_thr0, z_thr1, precision, max_pool, max_base, half, merge_dist)
    pool = np.zeros(MAX_TUPLE)
    pz = np.zeros(MAX_TUPLE)
    base = np.zeros(MAX_NBASE)
    npool = np.zeros(1, dtype=np.int32)
    nbase = np.zeros(1, dtype=np.int32)
    tr = np.zeros(1, dtype=np.int32)
    _check(lib().fredec_scan(_p(t), _p(y), _p(sigma), t.size, float(f0), float(df), int(nf), ctypes.byref(o),
                             _p(pool), _p(pz), _p(npool), _p(base), _p(nbase), _p(tr)))
    k, b = int(npool[0]), int(nbase[0])
    return pool[:k].copy(), pz[:k].copy(), base[:b].copy(), bool(tr[0])


def decompose(t, y, sigma, f0, df, nf, z_thr0, z_thr1, z_thr, *, precision=FP64, refine_precision=FP64,
              max_pool=0, max_base=0, half=0.5, merge_dist=0.0, refine_iter=20, refine_tol=1e-9,
              capacity=4096):
    """Phases 1-4.  Returns a dict: pool, l (Phase 2 table), masks, G, freqs
    (list of increasing arrays), n_solutions."""
    t, y, sigma = map(_f64, (t, y, sigma))
    zt = np.zeros(MAX_TUPLE)
    z_thr = _f64(z_thr)
    zt[:min(MAX_TUPLE, z_thr.size)] = z_thr[:MAX_TUPLE]
    o = DecomposeOpts()
    lib().fredec_decompose_opts_init(ctypes.byref(o))
    o.scan = _scan_opts(z_thr0, z_thr1, precision, max_pool, max_base, half, merge_dist)
    o.z_thr = zt.ctypes.data_as(_c_dp)
    o.refine_precision = _prec(refine_precision)
    o.refine_iter = int(refine_iter)
    o.refine_tol = float(refine_tol)
    pool = np.zeros(MAX_TUPLE)
    npool = np.zeros(1, dtype=np.int32)
    cap_pool = min(MAX_TUPLE, t.size // 10 if max_pool == 0 else max_pool)
    l = np.zeros(1 << max(cap_pool, 0))
    masks = np.zeros(max(capacity, 1), dtype=np.uint32)
    G = np.zeros(max(capacity, 1))
    F = np.zeros((max(capacity, 1), MAX_TUPLE))
    rz = np.zeros(max(capacity, 1))
    cnt = np.zeros(1, dtype=np.int64)
    _check(lib().fredec_decompose(_p(t), _p(y), _p(sigma), t.size, float(f0), float(df), int(nf), ctypes.byref(o),
                                  _p(pool), _p(npool), _p(l), masks.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                  _p(G), _p(F), _p(rz), int(capacity), _p(cnt)))
    n = int(npool[0])
    k = min(int(cnt[0]), capacity)
    return dict(pool=pool[:n].copy(), l=l[:1 << n].copy(), masks=masks[:k].copy(), G=G[:k].copy(),
                freqs=[F[i, :bin(int(masks[i])).count("1")].copy() for i in range(k)], resid_z=rz[:k].copy(),
                n_solutions=int(cnt[0]))


# ---------------------------------------------------------------------------
# Batches

def _batch_arrays(series):
    """CSR arrays from a list of objects with t, y, sigma, base_freqs, grid(f0, df, nf)."""
    obs = np.zeros(len(series) + 1, dtype=np.int64)
    bo = np.zeros(len(series) + 1, dtype=np.int64)
    zo = np.zeros(len(series) + 1, dtype=np.int64)
    for k, s in enumerate(series):
        obs[k + 1] = obs[k] + s.t.size
        bo[k + 1] = bo[k] + len(s.base_freqs)
        zo[k + 1] = zo[k] + s.grid.nf
    cat = lambda xs: np.ascontiguousarray(np.concatenate(xs)) if len(xs) else np.zeros(1)
    t = cat([s.t for s in series])
    y = cat([s.y for s in series])
    sg = cat([s.sigma for s in series])
    base = cat([np.asarray(s.base_freqs, dtype=np.float64) for s in series]) if bo[-1] else np.zeros(1)
    f0 = _f64([s.grid.f0 for s in series])
    df = _f64([s.grid.df for s in series])
    nf = _i64([s.grid.nf for s in series])
    return t, y, sg, obs, base, bo, f0, df, nf, zo


def periodogram_batch(series, *, precision=FP64, topk=0, flag_tau=0.0, trend=0, statistic=Z_DIFF):
    """One call for many series (objects with t, y, sigma, base_freqs, grid).
    Returns (z_concat, z_offsets, topk (n_series, k) or None)."""
    t, y, sg, obs, base, bo, f0, df, nf, zo = _batch_arrays(series)
    z = np.empty(max(int(zo[-1]), 1))
    top = np.empty(max(len(series) * topk, 1), dtype=np.int64) if topk else None
    o = _opts(precision, topk, 0, 0, flag_tau, trend, statistic)
    _check(lib().fredec_periodogram_batch(_p(t), _p(y), _p(sg), _p(obs), len(series), _p(base), _p(bo), _p(f0),
                                          _p(df), _p(nf), _p(zo[:-1].copy()), ctypes.byref(o), _p(z), _p(top)))
    return z[:int(zo[-1])], zo, (top.reshape(len(series), topk) if topk else None)


class BatchPlan:
    """Device-resident batch with a captured CUDA graph (see fredec.h)."""

    def __init__(self, series, *, precision=FP64, topk=0, flag_tau=0.0, trend=0, statistic=Z_DIFF):
        t, y, sg, obs, base, bo, f0, df, nf, zo = _batch_arrays(series)
        self.n_series = len(series)
        self.topk = topk
        self.z_offsets = zo
        self._h = _vp()
        o = _opts(precision, topk, 0, 0, flag_tau, trend, statistic)
        _check(lib().fredec_batch_plan_create(ctypes.byref(self._h), _p(t), _p(y), _p(sg), _p(obs), len(series),
                                              _p(base), _p(bo), _p(f0), _p(df), _p(nf), _p(zo[:-1].copy()),
                                              ctypes.byref(o)))
        zp, tp = _vp(), _vp()
        ztot, terms = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().fredec_batch_plan_outputs(self._h, ctypes.byref(zp), ctypes.byref(tp), ctypes.byref(ztot),
                                               ctypes.byref(terms)))
        self.z_total = ztot.value
        self.terms = terms.value
        self.z_ptr = zp.value
        self.topk_ptr = tp.value

    def run(self, stream=None):
        import torch
        _check(lib().fredec_batch_plan_run(self._h, _stream(torch, stream)))

    def download(self):
        z = np.empty(max(self.z_total, 1))
        top = np.empty(max(self.n_series * self.topk, 1), dtype=np.int64)
        _check(lib().fredec_batch_plan_download(self._h, _p(z), _p(top) if self.topk else None))
        return z[:self.z_total], (top.reshape(self.n_series, self.topk) if self.topk else None)

    def close(self):
        if self._h:
            lib().fredec_batch_plan_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def profile_events(ev_start=None, ev_stop=None):
    """Record torch.cuda.Event pairs around the main periodogram kernel of the
    following calls on this thread (None, None switches it off)."""
    h = lambda e: None if e is None else ctypes.c_void_p(int(e.cuda_event))
    _check(lib().fredec_profile_events(h(ev_start), h(ev_stop)))


def pipe_peaks():
    """Measured FP32 FMA, FP64 FMA and MUFU sine lane-op rates (per second)."""
    out = np.empty(3)
    _check(lib().fredec_pipe_peaks(_p(out)))
    return {"ffma_per_s": out[0], "dfma_per_s": out[1], "mufu_per_s": out[2]}


def tune(precision, n_base, N, nf):
    """Time the compiled launch shapes and remember the best; returns (fpt, warps)."""
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().fredec_tune(_prec(precision), int(n_base), int(N), int(nf), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value
