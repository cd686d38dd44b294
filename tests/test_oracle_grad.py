"""Pins of the oracle's loss gradients through exp(-t A) b (no GPU).

The reference values do not come from the oracle's own formulas: the Kronecker
closed form of the grid operator's exponential gives the exact forward value and
the exact adjoint, and central differences of the exact loss give d/dt.  The
operator is nonsymmetric (upwind convection), so using A where A^T belongs fails.
"""
import numpy as np
import pytest

import workloads as W
from oracle import grad as G
from oracle import truth as TR

N, BETA, T = 8, (20.0, 0.0, 0.0), 5e-3


@pytest.fixture(scope="module")
def case():
    A = W.convdiff3d(N, BETA)
    b = W.rhs_normal(A.n, 1)
    y = W.rhs_normal(A.n, 2)
    r = G.expm_loss_grad(A, b, y, T, 20, 2, 60, 8, 3, tol=1e-14, max_cycles=40)
    return A, b, y, r


def _exact_loss(b, y, t):
    x = TR.kron_expm_apply(N, 3, BETA, t, b)
    return float(np.dot(x - y, x - y))


def test_forward_and_adjoint_match_kronecker(case):
    A, b, y, r = case
    f = TR.kron_expm_apply(N, 3, BETA, T, b)
    gb = 2.0 * TR.kron_expm_apply(N, 3, BETA, T, f - y, transpose=True)
    assert np.linalg.norm(r.x - f) / np.linalg.norm(f) <= 1e-12
    assert np.linalg.norm(r.grad_b - gb) / np.linalg.norm(gb) <= 1e-12
    # the untransposed product is far away: the pin separates A from A^T
    wrong = 2.0 * TR.kron_expm_apply(N, 3, BETA, T, f - y)
    assert np.linalg.norm(wrong - gb) / np.linalg.norm(gb) > 0.1


def test_grad_b_matches_exact_directional_difference(case):
    """L is quadratic in b, so a central difference is exact up to rounding."""
    A, b, y, r = case
    d = W.rhs_normal(A.n, 3)
    eps = 0.5
    fd = (_exact_loss(b + eps * d, y, T) - _exact_loss(b - eps * d, y, T)) / (2 * eps)
    assert abs(np.dot(r.grad_b, d) - fd) <= 1e-10 * abs(fd)


def test_grad_t_matches_central_difference(case):
    A, b, y, r = case
    h = 1e-6
    fd = (_exact_loss(b, y, T + h) - _exact_loss(b, y, T - h)) / (2 * h)
    assert r.grad_t < 0.0
    assert abs(r.grad_t - fd) <= 1e-6 * abs(fd)


def test_loss_value(case):
    A, b, y, r = case
    assert abs(r.loss - _exact_loss(b, y, T)) <= 1e-12 * r.loss
