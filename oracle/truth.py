"""Closed-form references for f(A) b that involve no Krylov code.

* Grid operators of ``workloads.convdiff`` are Kronecker sums of 1D
  tridiagonal matrices, A = A_x (+) A_y (+) A_z, so
      exp(-t A) = E_z (x) E_y (x) E_x,   E_d = exp(-t A_d),
  applied to b as mode products on the (Nz, Ny, Nx) grid array.  E_d is an
  N x N dense exponential, so the reference costs O(N^4) even at n = N^3 = 2M.
  The transpose gives exp(-t A)^T = exp(-t A^T) for the adjoint.
* Sine modes are eigenvectors of the 5-point Laplacian with eigenvalues
  (4/h^2)(sin^2(p pi h/2) + sin^2(q pi h/2)).
* Tiny matrices: f(A) b through the dense eigendecomposition (symmetric A) or
  the dense function of the full matrix.
"""
import numpy as np

from . import dense


def tridiag_1d(N, beta_d):
    """1D factor of the upwind convection-diffusion operator along one axis."""
    inv_h = float(N + 1)
    lo = -inv_h**2 - (beta_d * inv_h if beta_d >= 0 else 0.0)
    hi = -inv_h**2 - (-beta_d * inv_h if beta_d < 0 else 0.0)
    d = 2.0 * inv_h**2 + abs(beta_d) * inv_h
    return np.diag(np.full(N, d)) + np.diag(np.full(N - 1, lo), -1) + np.diag(np.full(N - 1, hi), 1)


def kron_expm_apply(N, dim, beta, t, b, transpose=False):
    """exp(-t A) b (or exp(-t A)^T b) for A = convdiff(N, dim, beta) exactly
    (to the accuracy of the N x N exponentials)."""
    E = []
    for d in range(dim):
        Ed = dense.expm(-t * tridiag_1d(N, beta[d]))
        E.append(Ed.T if transpose else Ed)
    X = np.asarray(b, dtype=np.float64).reshape((N,) * dim)
    # axis dim-1 is x (d = 0), axis 0 is the slowest direction
    for d in range(dim):
        axis = dim - 1 - d
        X = np.moveaxis(np.tensordot(E[d], X, axes=([1], [axis])), 0, axis)
    return X.reshape(-1)


def sine_mode_exp(N, c, p, q, t):
    """exp(-t A) b for b = sum_l c_l phi_{p_l q_l} on the 5-point Laplacian."""
    h = 1.0 / (N + 1)
    ii = np.arange(1, N + 1)
    lam = (4.0 / h**2) * (np.sin(p * np.pi * h / 2) ** 2 + np.sin(q * np.pi * h / 2) ** 2)
    out = np.zeros((N, N))
    for cl, pl, ql, ll in zip(c, p, q, lam):
        out += cl * np.exp(-t * ll) * np.outer(np.sin(ql * np.pi * ii * h), np.sin(pl * np.pi * ii * h))
    return out.reshape(-1)


def phi1_neg(x):
    """phi_1(-x) = (1 - e^{-x}) / x elementwise (1 at x = 0), from expm1."""
    x = np.asarray(x, dtype=np.float64)
    safe = np.where(x == 0.0, 1.0, x)
    return np.where(x == 0.0, 1.0, -np.expm1(-safe) / safe)


def sine_mode_phi1(N, c, p, q, t):
    """phi_1(-t A) b for b = sum_l c_l phi_{p_l q_l} on the 5-point Laplacian."""
    h = 1.0 / (N + 1)
    ii = np.arange(1, N + 1)
    lam = (4.0 / h**2) * (np.sin(np.asarray(p) * np.pi * h / 2) ** 2 + np.sin(np.asarray(q) * np.pi * h / 2) ** 2)
    out = np.zeros((N, N))
    for cl, pl, ql, ll in zip(c, p, q, lam):
        out += cl * phi1_neg(t * ll) * np.outer(np.sin(ql * np.pi * ii * h), np.sin(pl * np.pi * ii * h))
    return out.reshape(-1)


def sine_mode_cos(N, c, p, q, t):
    """cos(t sqrt(A)) b for b = sum_l c_l phi_{p_l q_l} on the 5-point Laplacian."""
    h = 1.0 / (N + 1)
    ii = np.arange(1, N + 1)
    lam = (4.0 / h**2) * (np.sin(np.asarray(p) * np.pi * h / 2) ** 2 + np.sin(np.asarray(q) * np.pi * h / 2) ** 2)
    out = np.zeros((N, N))
    for cl, pl, ql, ll in zip(c, p, q, lam):
        out += cl * np.cos(t * np.sqrt(ll)) * np.outer(np.sin(ql * np.pi * ii * h), np.sin(pl * np.pi * ii * h))
    return out.reshape(-1)


def dense_fAb(Adense, b, fkind, t=1.0, symmetric=False):
    """f(A) b on a small dense matrix."""
    if symmetric:
        lam, Q = np.linalg.eigh(Adense)
        if fkind == dense.EXP_NEG:
            fl = np.exp(-t * lam)
        elif fkind == dense.PHI1_NEG:
            fl = phi1_neg(t * lam)
        elif fkind == dense.COS_SQRT:
            fl = np.cos(t * np.sqrt(lam))
        elif fkind == dense.INVSQRT:
            fl = lam ** -0.5
        else:
            fl = 1.0 / lam
        return Q @ (fl * (Q.T @ b))
    return dense.f_dense(fkind, Adense, t) @ b
