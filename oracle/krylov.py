"""Restarted Krylov methods for f(A)b, plain FP64 loops (test infrastructure only).

Three orthogonalization modes share one restart driver (Algorithm 2):

CLASSICAL  the classical restarted Arnoldi method (Sec. 2.2, the ``restart``
           method of Sec. 5): full modified Gram-Schmidt in every cycle,
           f_m = beta V_m f(H_m) e_1 with beta = ||b||.
RGS        the paper's randomized restart: Algorithm 1 (randomized Arnoldi,
           sketch-orthogonalization by MGS in sketch space, one basis update per
           step) inside Algorithm 2.  ``k >= m`` is the paper's method exactly;
           ``k < m`` restricts the sketch orthogonalization to the last k
           sketches.
TRUNC      truncated (incomplete) orthogonalization against the last k basis
           vectors (classical Gram-Schmidt, all coefficients from the same
           unmodified vector), followed by basis whitening of the sketched
           basis (App. A, Eq. A.1) and the restart of Algorithm 2.

Readings where the paper is silent (each one is listed in the design notes):
* TRUNC projection coefficients are <w_i, p> / <w_i, w_i>, i.e. projections;
  they equal the plain dots whenever w_i has unit norm.
* The whitened restart: with S W_{m+1} = Q T, T = [[T_m, t], [0, tau]],
  the whitened basis W_m T_m^{-1} satisfies the exact Arnoldi-like relation
      A (W_m T_m^{-1}) = (W_m T_m^{-1}) X + v rho e_m^T,
      X   = T_m R_m T_m^{-1} + (r_{m+1,m} / T_m[m,m]) t e_m^T      (Eq. A.1),
      v   = (w_{m+1} - W_m T_m^{-1} t) / tau,
      rho = r_{m+1,m} tau / T_m[m,m].
  The next cycle starts from w_1 = v without renormalization, so the coupling
  entry of Algorithm 2's block matrix is gamma = rho * T^{next}[1,1], and the
  first cycle's scale is beta = ||b|| * T^{(1)}[1,1].
* "t_m" in Eq. A.1 is T_m[m,m], the last diagonal entry of T_m.
* Stopping test ||y|| <= tol * ||x|| (relative); tol = 0 runs max_cycles.
* Happy breakdown: r_{j+1,j} <= 1e-14 * ||A w_j|| ends the cycle after j
  columns; the decomposition is then exact and the method stops.
* RGS cycles c >= 2 normalize the start vector by alpha' = ||S w_{m+1}||
  (= 1 up to rounding) and discard alpha', as Algorithm 2 does.
* Reduced-precision storage of the basis (TRUNC only, ``store``): every basis
  vector is rounded to the storage precision when it is stored (the start
  vector w_1 and each new w_{j+1} = p / r_{j+1,j}); every later use -- the next
  product, the window dots and updates, the sketch, the restart vector and
  x += W z -- reads the stored value, and all arithmetic stays FP64.  The
  Arnoldi-like relation of Sec. 2.2 (Eq. 5) then holds for the stored vectors
  up to the storage rounding of each new column, which is the perturbation a
  float32 or bfloat16 basis makes to the method.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import dense
from .sketch import SparseSign

CLASSICAL = "classical"
RGS = "rgs"
TRUNC = "trunc"

BREAKDOWN_REL = 1e-14

F64, F32, BF16 = "f64", "f32", "bf16"


def round_storage(v, store):
    """v rounded to the storage format `store` and returned as float64:
    F64 (or None) leaves v as is; F32 rounds to IEEE binary32; BF16 rounds to
    bfloat16 (binary32's sign, exponent and top 7 fraction bits) to nearest
    with ties to even, from the binary32 value."""
    if store is None or store == F64:
        return np.asarray(v, dtype=np.float64)
    f = np.asarray(v, dtype=np.float64).astype(np.float32)
    if store == F32:
        return f.astype(np.float64)
    if store != BF16:
        raise ValueError(f"unknown storage format {store!r}")
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)  # ties go to the even upper half
    r = ((u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def csr_matvec(A, x):
    """y = A x for a CSR matrix: y_i = sum_q val[q] x[col[q]] over row i, in
    storage order."""
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    return np.bincount(rows, weights=A.val * x[A.col_idx], minlength=A.n)


@dataclass
class CycleInfo:
    m_eff: int
    update_norm: float
    x_norm: float
    kappa_T: float = float("nan")
    sketch_orth_err: float = float("nan")
    R: np.ndarray | None = None
    T: np.ndarray | None = None
    X: np.ndarray | None = None
    W: np.ndarray | None = None
    U: np.ndarray | None = None
    z: np.ndarray | None = None


@dataclass
class Result:
    x: np.ndarray
    cycles: int
    breakdown: bool
    H: np.ndarray
    beta: float
    info: list = field(default_factory=list)


def _arnoldi_classical(A, w1, m):
    """Arnoldi with modified Gram-Schmidt (Sec. 2.2)."""
    n = w1.size
    V = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    V[:, 0] = w1
    for j in range(m):
        p = csr_matvec(A, V[:, j])
        pn = np.linalg.norm(p)
        for i in range(j + 1):
            H[i, j] = V[:, i] @ p
            p = p - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(p)
        if H[j + 1, j] <= BREAKDOWN_REL * pn:
            return V[:, : j + 1], H[: j + 1, : j + 1], j + 1, True
        V[:, j + 1] = p / H[j + 1, j]
    return V, H, m, False


def _arnoldi_randomized(A, S, w_start, m, k):
    """Algorithm 1 (randomized Arnoldi); the sketch Gram-Schmidt runs over the
    last k sketches (all of them when k >= m).  Returns alpha, W_{m+1},
    R_underline, U = S W_{m+1}, the number of columns and the breakdown flag."""
    n = w_start.size
    Sb = S.apply(w_start)
    alpha = np.linalg.norm(Sb)
    W = np.zeros((n, m + 1))
    Us = np.zeros((S.s, m + 1))
    R = np.zeros((m + 1, m))
    Us[:, 0] = Sb / alpha
    W[:, 0] = w_start / alpha
    for j in range(m):
        w = csr_matvec(A, W[:, j])
        u = S.apply(w)
        un = np.linalg.norm(u)
        window = range(max(0, j - k + 1), j + 1)
        for i in window:
            R[i, j] = Us[:, i] @ u
            u = u - R[i, j] * Us[:, i]
        for i in window:
            w = w - R[i, j] * W[:, i]
        R[j + 1, j] = np.linalg.norm(u)
        if R[j + 1, j] <= BREAKDOWN_REL * un:
            return alpha, W[:, : j + 1], R[: j + 1, : j + 1], Us[:, : j + 1], j + 1, True
        W[:, j + 1] = w / R[j + 1, j]
        Us[:, j + 1] = u / R[j + 1, j]
    return alpha, W, R, Us, m, False


def _arnoldi_truncated(A, w1, m, k, store=None):
    """Incomplete Arnoldi: classical Gram-Schmidt against the last k vectors.
    Stored vectors are rounded to `store` (see round_storage)."""
    n = w1.size
    W = np.zeros((n, m + 1))
    R = np.zeros((m + 1, m))
    W[:, 0] = round_storage(w1, store)
    for j in range(m):
        p = csr_matvec(A, W[:, j])
        pn = np.linalg.norm(p)
        window = range(max(0, j - k + 1), j + 1)
        h = {i: (W[:, i] @ p) / (W[:, i] @ W[:, i]) for i in window}
        for i in window:
            p = p - h[i] * W[:, i]
            R[i, j] = h[i]
        R[j + 1, j] = np.linalg.norm(p)
        if R[j + 1, j] <= BREAKDOWN_REL * pn:
            return W[:, : j + 1], R[: j + 1, : j + 1], j + 1, True
        W[:, j + 1] = round_storage(p / R[j + 1, j], store)
    return W, R, m, False


def _append_block(H, X, gamma):
    """H_{cm} = [[H_{(c-1)m}, 0], [gamma e_1 e_last^T, X]] (Algorithm 2)."""
    a = H.shape[0]
    b = X.shape[0]
    Hn = np.zeros((a + b, a + b))
    Hn[:a, :a] = H
    Hn[a:, a:] = X
    if a > 0:
        Hn[a, a - 1] = gamma
    return Hn


def restarted(A, b, fkind, t, m, k, s, zeta, seed, mode=TRUNC, tol=0.0, max_cycles=1,
              sketch=None, keep=False, abs_tol=False, store=None):
    """Approximate f(A) b by the restarted method of the chosen mode.

    A       workloads.Csr; b: (n,) float64.
    fkind   oracle.dense.EXP_NEG (exp(-t z)), PHI1_NEG (phi_1(-t z)), COS_SQRT (cos(t sqrt(z))), INVSQRT or INV.
    m, k    restart length and orthogonalization window.
    s, zeta sketch rows and nonzeros per sketch column; seed keys the sketch.
    tol     stop once ||y|| <= tol * ||x|| (or <= tol if abs_tol).
    keep    keep per-cycle matrices (R, T, X, W, U, z) in the result's info.
    store   TRUNC only: storage format of the basis (F64 = None, F32, BF16).
    """
    if store not in (None, F64) and mode != TRUNC:
        raise ValueError("reduced-precision storage is modelled for the TRUNC mode only")
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    if mode != CLASSICAL and sketch is None:
        sketch = SparseSign(n, s, zeta, seed)
    S = sketch
    x = np.zeros(n)
    H = np.zeros((0, 0))
    beta = None
    coupling = 0.0  # coupling term of the previous cycle, before the T[1,1] factor
    start = b.copy()
    info = []
    breakdown = False
    cycles = 0
    for c in range(1, max_cycles + 1):
        cycles = c
        ci = CycleInfo(0, 0.0, 0.0)
        if mode == CLASSICAL:
            if c == 1:
                beta = np.linalg.norm(b)
                w1 = b / beta
            else:
                w1 = start
            V, Hbar, me, brk = _arnoldi_classical(A, w1, m)
            X = Hbar[:me, :me]
            H = _append_block(H, X, coupling)
            basis = V[:, :me]
            coef_map = np.eye(me)
            if not brk:
                coupling = Hbar[me, me - 1]
                start = V[:, me]
            if keep:
                ci.R, ci.W = Hbar, V
        elif mode == RGS:
            alpha, W, Rbar, Us, me, brk = _arnoldi_randomized(A, S, start, m, k)
            if c == 1:
                beta = alpha
            X = Rbar[:me, :me]
            H = _append_block(H, X, coupling)
            basis = W[:, :me]
            coef_map = np.eye(me)
            if not brk:
                coupling = Rbar[me, me - 1]
                start = W[:, me]
            G = Us.T @ Us
            ci.sketch_orth_err = np.linalg.norm(G - np.eye(G.shape[0]))
            if keep:
                ci.R, ci.W, ci.U = Rbar, W, Us
        else:  # TRUNC + whitening
            if c == 1:
                eta = np.linalg.norm(b)
                w1 = b / eta
            else:
                w1 = start
            W, Rbar, me, brk = _arnoldi_truncated(A, w1, m, k, store)
            ncols = me if brk else me + 1
            U = S.apply(W[:, :ncols])
            Q, T = dense.qr_positive(U)
            Tm = T[:me, :me]
            Tm_inv = np.linalg.inv(Tm)
            X = Tm @ Rbar[:me, :me] @ Tm_inv
            if not brk:
                tvec = T[:me, me]
                tau = T[me, me]
                r = Rbar[me, me - 1]
                X = X + (r / Tm[me - 1, me - 1]) * np.outer(tvec, np.eye(me)[me - 1])
            if c == 1:
                beta = eta * T[0, 0]
                H = _append_block(H, X, 0.0)
            else:
                H = _append_block(H, X, coupling * T[0, 0])
            basis = W[:, :me]
            coef_map = Tm_inv
            if not brk:
                g = Tm_inv @ tvec
                start = (W[:, me] - W[:, :me] @ g) / tau
                coupling = r * tau / Tm[me - 1, me - 1]
            ci.kappa_T = np.linalg.cond(T)
            G = Q.T @ Q
            ci.sketch_orth_err = np.linalg.norm(G - np.eye(G.shape[0]))
            if keep:
                ci.R, ci.W, ci.U, ci.T, ci.X = Rbar, W, U, T, X
        F = dense.f_dense(fkind, H, t)
        off = H.shape[0] - me
        z = beta * (coef_map @ F[off:, 0])
        y = basis @ z
        x = x + y
        ci.m_eff = me
        ci.update_norm = float(np.linalg.norm(y))
        ci.x_norm = float(np.linalg.norm(x))
        if keep:
            ci.z = z
        info.append(ci)
        if brk:
            breakdown = True
            break
        limit = tol if abs_tol else tol * ci.x_norm
        if ci.update_norm <= limit:
            break
    return Result(x=x, cycles=cycles, breakdown=breakdown, H=H, beta=beta, info=info)
