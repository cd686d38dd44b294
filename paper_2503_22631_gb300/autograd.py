"""Differentiable x = f(A) b through a Krylov handle (PyTorch autograd).

The forward pass is one ``krylov_apply``; the backward pass is one
``krylov_apply_adjoint`` for the input vector and, for f(z) = exp(-t z), one
``krylov_spmv`` with a fused dot product for the time parameter:

* f(A)^T = f(A^T) for a matrix function (Sec. 1: f(A) is defined by the Cauchy
  integral over a contour enclosing the spectrum), so grad_b = f(A^T) g is the
  same restarted method run on A^T;
* d/dt exp(-t A) b = -A exp(-t A) b, so grad_t = -<g, A x> with x the forward
  result.

These are the gradients of the exact function, evaluated with the method's
approximations of f(A) b and f(A^T) g; they match finite differences of the
approximate forward pass to the accuracy the restart loop is run to.
"""
from __future__ import annotations

import torch

from ._lib import F_EXP_NEG


class KrylovExpm(torch.autograd.Function):
    """x = f(A) b for a ``Krylov`` handle; differentiable in b and (for exp) in t.

    ``t`` is a float or a 0-d tensor; when it is a tensor its value is set on
    the handle before the forward and the backward products.
    """

    @staticmethod
    def forward(ctx, b, t, handle, tol, max_cycles):
        tv = float(t) if not isinstance(t, torch.Tensor) else float(t.detach().cpu())
        if handle.f == F_EXP_NEG:
            handle.set_param(tv)
        x = handle.apply(b.detach().to(torch.float64).contiguous(), tol=tol, max_cycles=max_cycles)
        ctx.handle, ctx.t, ctx.tol, ctx.max_cycles = handle, tv, tol, max_cycles
        ctx.t_is_tensor = isinstance(t, torch.Tensor)
        ctx.t_meta = (t.dtype, t.device) if ctx.t_is_tensor else None
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        h = ctx.handle
        g = g.detach().to(torch.float64).contiguous()
        grad_b = grad_t = None
        if ctx.needs_input_grad[0]:
            if h.f == F_EXP_NEG:
                h.set_param(ctx.t)
            grad_b = h.apply(g, tol=ctx.tol, max_cycles=ctx.max_cycles, adjoint=True)
        if ctx.t_is_tensor and ctx.needs_input_grad[1]:
            if h.f != F_EXP_NEG:
                raise ValueError("the t-derivative is defined for f(z) = exp(-t z) only")
            _, dot = h.spmv(x, dot_with=g)
            dtype, device = ctx.t_meta
            grad_t = torch.tensor(-dot, dtype=dtype, device=device)
        return grad_b, grad_t, None, None, None


def krylov_expm(b, t, handle, tol=0.0, max_cycles=1):
    """Functional form of ``KrylovExpm.apply``."""
    return KrylovExpm.apply(b, t, handle, tol, max_cycles)
