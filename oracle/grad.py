"""Gradients of a loss through x = exp(-t A) b, plain FP64 (test infrastructure only).

The paper approximates f(A) b; it has no backward pass.  The differentiable
form follows from two facts about the matrix function of Sec. 1 (defined by the
Cauchy integral over a contour around the spectrum):

* f(A)^T = f(A^T), so the vector-Jacobian product in b is
  grad_b = f(A)^T g = f(A^T) g, i.e. the same restarted method run on A^T;
* for f(z) = exp(-t z), d/dt exp(-t A) b = -A exp(-t A) b, so
  grad_t = <g, -A x> = -<g, A x>.

For the loss L = ||x - y||^2 the upstream gradient is g = 2 (x - y).  Both
products are taken with the oracle's restarted method (``krylov.restarted``),
the same algorithm the forward pass uses.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import dense
from .krylov import TRUNC, csr_matvec, restarted


@dataclass
class LossGrad:
    loss: float
    x: np.ndarray
    grad_b: np.ndarray
    grad_t: float


def expm_loss_grad(A, b, y, t, m, k, s, zeta, seed, mode=TRUNC, tol=0.0, max_cycles=1):
    """L = ||exp(-tA) b - y||^2 with its gradients in b and t (see module notes)."""
    fwd = restarted(A, b, dense.EXP_NEG, t, m, k, s, zeta, seed, mode=mode, tol=tol, max_cycles=max_cycles)
    x = fwd.x
    g = 2.0 * (x - y)
    adj = restarted(A.transpose(), g, dense.EXP_NEG, t, m, k, s, zeta, seed, mode=mode, tol=tol,
                    max_cycles=max_cycles)
    grad_t = -float(np.dot(g, csr_matvec(A, x)))
    loss = float(np.dot(x - y, x - y))
    return LossGrad(loss=loss, x=x, grad_b=adj.x, grad_t=grad_t)
