"""Differentiation through the simultaneous solve: a torch.autograd.Function.

Forward: X = A^{-1} B with any of the simultaneous methods (kr_solve).
Backward (reverse mode, for a real loss L): with G = dL/dX in torch's complex
convention (dL/dRe X + i dL/dIm X), the adjoint system A^H Lambda = G is solved
with the same method (kr_adjoint_solve: the A^H products the BiCG family already
has), and

    dL/dB = Lambda,        dL/dA_ij = - sum_c Lambda_ic conj(X_jc)   (stored (i, j) only),

the latter by kr_grad_values.  Parameters that enter A linearly (e.g. the
convection velocities of a convection-diffusion operator) get their gradient
from torch's chain rule through the returned value gradient.
"""
from __future__ import annotations

import torch

from . import kr_adjoint_solve, kr_grad_values, kr_op_update_values, kr_solve


class KrylovSolve(torch.autograd.Function):
    """X = KrylovSolve.apply(vals, B, op, method, tol, maxit)."""

    @staticmethod
    def forward(ctx, vals, B, op, method="egl_bicg", tol=1e-8, maxit=1000):
        kr_op_update_values(op, vals)
        X, info = kr_solve(op, method, B.contiguous(), tol=tol, maxit=maxit)
        if info.status != "OK":
            raise RuntimeError("forward solve did not converge: %s" % (info,))
        ctx.op, ctx.method, ctx.tol, ctx.maxit = op, method, tol, maxit
        ctx.save_for_backward(X)
        ctx.vals_device = vals.device
        return X

    @staticmethod
    def backward(ctx, G):
        (X,) = ctx.saved_tensors
        Lam, info = kr_adjoint_solve(ctx.op, ctx.method, G.contiguous(), tol=ctx.tol, maxit=ctx.maxit)
        if info.status != "OK":
            raise RuntimeError("adjoint solve did not converge: %s" % (info,))
        dvals = kr_grad_values(ctx.op, Lam, X).to(ctx.vals_device)
        return dvals, Lam, None, None, None, None


def krylov_solve(vals, B, op, method="egl_bicg", tol=1e-8, maxit=1000):
    return KrylovSolve.apply(vals, B, op, method, tol, maxit)
