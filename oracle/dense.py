"""Small dense FP64 routines used by the oracle's projected problem.

* ``qr_positive``  thin Householder QR with a positive diagonal in T
  (App. A: the paper notes LAPACK's dgeqrf does not fix the sign of t_11 and
  compensates with sign(t_11); forcing diag(T) > 0 makes T unique instead).
* ``expm``         exp(A) by scaling and squaring with the [13/13] Pade
  approximant (N. J. Higham, "The scaling and squaring method for the matrix
  exponential revisited", SIAM J. Matrix Anal. Appl. 26(4), 2005; the method
  the paper uses for exp, App. A).
* ``invsqrtm``     A^{-1/2} by the Denman-Beavers iteration with determinant
  scaling (E. D. Denman, A. N. Beavers, 1976; N. J. Higham, "Functions of
  Matrices", 2008, Sec. 6.3 and 6.5).  Not in the paper: the inverse square
  root workload is an extension.
* ``phi1m``        phi_1(A) = sum_k A^k / (k+1)!  (the paper's phi function,
  Sec. 5, phi_1(z) = (e^z - 1)/z) as the top-right block of exp of the block
  triangular [[A, I], [0, 0]], whose exponential is [[e^A, phi_1(A)], [0, I]]
  (the series of the two sides agree term by term; the identity is the usual
  way to evaluate phi functions with an exponential, see Hochbruck and
  Ostermann, "Exponential integrators", Acta Numerica 2010, which the paper
  cites for phi_1).
* ``cossqrtm``     cos(t sqrt(A)) (the membrane example of Sec. 5, cos(nu t sqrt(L)))
  as the top-left block of exp(t [[0, I], [-A, 0]]): that matrix propagates
  u'' = -A u, whose solution is u(t) = cos(t sqrt(A)) u(0) + ..., and the
  series of both sides agree term by term.
* ``f_dense``      f(H) for the five supported kinds.
"""
import math
from fractions import Fraction

import numpy as np

EXP_NEG = 0      # f(z) = exp(-t z)
INVSQRT = 1      # f(z) = z^{-1/2}
INV = 2          # f(z) = 1/z
PHI1_NEG = 3     # f(z) = phi_1(-t z) = (1 - e^{-t z}) / (t z)
COS_SQRT = 4     # f(z) = cos(t sqrt(z))


def qr_positive(U):
    """Thin QR U = Q T (U is s x c with s >= c) by Householder reflections,
    then the sign of every row of T (and column of Q) flipped so diag(T) > 0."""
    U = np.array(U, dtype=np.float64)
    s, c = U.shape
    Rw = U.copy()
    Q = np.eye(s)
    for j in range(c):
        x = Rw[j:, j].copy()
        nx = np.linalg.norm(x)
        if nx == 0.0:
            continue
        alpha = -nx if x[0] >= 0 else nx
        v = x.copy()
        v[0] -= alpha
        nv = np.linalg.norm(v)
        if nv == 0.0:
            continue
        v /= nv
        Rw[j:, :] -= 2.0 * np.outer(v, v @ Rw[j:, :])
        Q[:, j:] -= 2.0 * np.outer(Q[:, j:] @ v, v)
    T = np.triu(Rw[:c, :])
    Q = Q[:, :c]
    d = np.where(np.diag(T) < 0, -1.0, 1.0)
    return Q * d[None, :], T * d[:, None]


def _pade13_coefficients():
    """b_k = (26-k)! 13! / (26! k! (13-k)!), k = 0..13 (diagonal Pade for exp)."""
    q = 13
    f = math.factorial
    return [float(Fraction(f(2 * q - k) * f(q), f(2 * q) * f(k) * f(q - k))) for k in range(q + 1)]


# theta_13 of Higham (2005), Table 2.3: the largest ||A||_1 for which the
# degree-13 approximant meets unit roundoff in backward error.
THETA_13 = 5.371920351148152


def expm(A):
    """exp(A): scale by 2^-s so ||A||_1 <= theta_13, evaluate r_13, square s times."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    if n == 0:
        return A.copy()
    norm1 = np.abs(A).sum(axis=0).max()
    s = 0 if norm1 <= THETA_13 else int(math.ceil(math.log2(norm1 / THETA_13)))
    B = A / (2.0 ** s)
    b = _pade13_coefficients()
    P = np.eye(n)
    N = b[0] * P
    D = b[0] * P
    for k in range(1, 14):
        P = P @ B
        N = N + b[k] * P
        D = D + ((-1) ** k) * b[k] * P
    E = np.linalg.solve(D, N)
    for _ in range(s):
        E = E @ E
    return E


def invsqrtm(A, tol=1e-14, max_iter=100):
    """A^{-1/2} for A with no eigenvalues on the closed negative real axis.

    Scaled Denman-Beavers: Y_0 = A, Z_0 = I,
        mu = |det(Y) det(Z)|^{-1/(2n)},
        Y <- (mu Y + (mu Z)^{-1}) / 2,  Z <- (mu Z + (mu Y)^{-1}) / 2,
    so Y -> A^{1/2} and Z -> A^{-1/2}.  Scaling is applied in the first eight
    iterations; the iteration stops when the relative change of Y falls below
    tol or stops decreasing once below 1e-8 (rounding level).  Raises if it
    does not converge.
    """
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    Y = A.copy()
    Z = np.eye(n)
    prev = np.inf
    for it in range(max_iter):
        sy, ly = np.linalg.slogdet(Y)
        sz, lz = np.linalg.slogdet(Z)
        mu = math.exp(-(ly + lz) / (2.0 * n)) if it < 8 else 1.0
        Yn = 0.5 * (mu * Y + np.linalg.inv(mu * Z))
        Zn = 0.5 * (mu * Z + np.linalg.inv(mu * Y))
        diff = np.linalg.norm(Yn - Y, 1) / max(np.linalg.norm(Yn, 1), 1e-300)
        Y, Z = Yn, Zn
        # converged, or stagnated at the rounding level of the iteration
        if mu == 1.0 and (diff < tol or (diff < 1e-8 and diff >= 0.5 * prev)):
            break
        prev = diff if mu == 1.0 else np.inf
        if not np.all(np.isfinite(Z)):
            raise FloatingPointError("Denman-Beavers iteration produced non-finite values")
    else:
        raise RuntimeError("Denman-Beavers iteration did not converge")
    return Z


def phi1m(A):
    """phi_1(A): the top-right n x n block of exp([[A, I], [0, 0]])."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    Z = np.zeros((2 * n, 2 * n))
    Z[:n, :n] = A
    Z[:n, n:] = np.eye(n)
    return expm(Z)[:n, n:]


def cossqrtm(A, t=1.0):
    """cos(t sqrt(A)): the top-left n x n block of exp(t [[0, I], [-A, 0]])."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    Z = np.zeros((2 * n, 2 * n))
    Z[:n, n:] = t * np.eye(n)
    Z[n:, :n] = -t * A
    return expm(Z)[:n, :n]


def f_dense(kind, H, t=1.0):
    """f(H) for f(z) = exp(-t z), z^{-1/2}, 1/z, phi_1(-t z) or cos(t sqrt(z)) (dense, FP64)."""
    if kind == EXP_NEG:
        return expm(-t * H)
    if kind == PHI1_NEG:
        return phi1m(-t * H)
    if kind == COS_SQRT:
        return cossqrtm(H, t)
    if kind == INVSQRT:
        return invsqrtm(H)
    if kind == INV:
        return np.linalg.inv(H)
    raise ValueError(kind)
