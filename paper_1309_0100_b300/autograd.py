"""torch.autograd.Function wrappers over the C ABI (device tensors, torch's
current stream).  The forward and backward passes are the library's kernels;
this module only routes tensors.

PeriodogramFn: y -> z on a uniform grid; backward is the VJP kernel
    dL/dy_i = w_i sum_j (dL/dz_j) (mu_j(t_i) - mu_base(t_i)).
TupleZFn: tuple frequencies -> z per tuple; backward uses
    dz/df_k = sum_i w_i r_i 2 pi t_i (-a_k sin + b_k cos)  (adjoint sums).
"""
from __future__ import annotations

import numpy as np
import torch

from . import FP64, _prec, periodogram_dev, periodogram_vjp_dev, tuple_grad_dev


class PeriodogramFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, t, sigma, base, f0, df, nf, precision):
        out = periodogram_dev(t, y, sigma, base, f0, df, nf, precision=precision, want_coef=True)
        ctx.save_for_backward(t, y, sigma, base, out["coef"], out["info"])
        ctx.grid = (f0, df, nf, _prec(precision))
        return out["z"]

    @staticmethod
    def backward(ctx, gz):
        t, y, sigma, base, coef, info = ctx.saved_tensors
        f0, df, nf, prec = ctx.grid
        g = periodogram_vjp_dev(t, y, sigma, base, f0, df, nf, coef, info, gz.contiguous().to(torch.float64),
                                precision=prec)
        return g, None, None, None, None, None, None, None


def periodogram_z(y, t, sigma, base, f0, df, nf, precision=FP64):
    """Differentiable residual periodogram z(f_j), j < nf (gradient w.r.t. y)."""
    return PeriodogramFn.apply(y, t, sigma, base, f0, df, nf, precision)


class TupleZFn(torch.autograd.Function):
    """Tuple frequencies (CUDA tensor, CSR order) -> z per tuple.  The forward
    pass runs the library's tuple kernel on the device (fredec_tuple_grad_dev:
    z and dz/df in one pass, kept for backward); the offsets stay on the host,
    since they size the launch."""

    @staticmethod
    def forward(ctx, freqs, t, y, sigma, offsets, precision):
        off = np.ascontiguousarray(np.asarray(offsets.cpu() if hasattr(offsets, "cpu") else offsets,
                                              dtype=np.int64))
        z, g = tuple_grad_dev(t, y, sigma, freqs.detach().contiguous(), off, precision=precision)
        ctx.save_for_backward(g)
        ctx.rep = torch.as_tensor(np.repeat(np.arange(off.size - 1), np.diff(off)), device=freqs.device)
        return z

    @staticmethod
    def backward(ctx, gz):
        (g,) = ctx.saved_tensors
        return gz[ctx.rep] * g, None, None, None, None, None


def tuple_z(freqs, t, y, sigma, offsets, precision=FP64):
    """Differentiable multifrequency statistic z per tuple (gradient w.r.t. the
    tuple frequencies, CSR layout given by offsets)."""
    return TupleZFn.apply(freqs, t, y, sigma, offsets, precision)
