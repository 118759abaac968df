"""torch.autograd wrappers over the C ABI.

OpApply / OpAdjoint: y = A x and x = A^T y, each with the other kernel as its
backward (the operators are exact transposes of each other).
UnrolledSolve: x = K unrolled Algorithm 3 iterations (TV, dual APG prox)
as a function of lambda and the blur kernel h, with the library's
hand-written reverse pass as the backward.  Every computation is a libnys
call; this module only marshals tensors.
"""
from __future__ import annotations

import torch

from . import api


class OpApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, op):
        ctx.op = op
        return api.op_apply(op, x.contiguous())

    @staticmethod
    def backward(ctx, gy):
        return api.op_adjoint(ctx.op, gy.contiguous()), None


class OpAdjoint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, op):
        ctx.op = op
        return api.op_adjoint(op, y.contiguous())

    @staticmethod
    def backward(ctx, gx):
        return api.op_apply(ctx.op, gx.contiguous()), None


def op_apply(op: api.Operator, x: torch.Tensor) -> torch.Tensor:
    return OpApply.apply(x, op)


def op_adjoint(op: api.Operator, y: torch.Tensor) -> torch.Tensor:
    return OpAdjoint.apply(y, op)


class UnrolledSolve(torch.autograd.Function):
    """x_K(lambda, h) for fixed data y; lam is a 0-d tensor, h a (kh, kw)
    float64 tensor (or None to keep the operator's kernel)."""

    @staticmethod
    def forward(ctx, lam, h, unroll: api.Unroll, y):
        if h is not None:
            unroll.op.set_kernel(h.detach().double().cpu().numpy())
        unroll.set_lambda(float(lam))
        ctx.unroll = unroll
        ctx.lam_like = (lam.device, lam.dtype)
        ctx.h_like = (h.device, h.dtype) if h is not None else None
        return unroll.forward(y)

    @staticmethod
    def backward(ctx, xbar):
        dlam, dh = ctx.unroll.backward(xbar)
        dlam = dlam.to(device=ctx.lam_like[0], dtype=ctx.lam_like[1])
        dh_out = None
        if ctx.h_like is not None and dh is not None:
            dh_out = dh.to(device=ctx.h_like[0], dtype=ctx.h_like[1])
        return dlam, dh_out, None, None


def unrolled_solve(unroll: api.Unroll, y: torch.Tensor, lam: torch.Tensor, h: torch.Tensor | None = None):
    return UnrolledSolve.apply(lam, h, unroll, y)
