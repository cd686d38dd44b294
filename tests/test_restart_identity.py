"""The restart of a whitened basis (the reading of App. A, Eq. A.1, for a
restarted cycle): with S W_{m+1} = Q T and T = [[T_m, t], [0, tau]],

    A (W_m T_m^-1) = (W_m T_m^-1) X + v rho e_m^T,
    X = T_m R_m T_m^-1 + (r_{m+1,m} / T_m[m,m]) t e_m^T,
    v = (w_{m+1} - W_m T_m^-1 t) / tau,  rho = r_{m+1,m} tau / T_m[m,m],

follows from the Arnoldi-like relation A W_m = W_m R_m + w_{m+1} r_{m+1,m}
e_m^T (Eq. 5) by algebra alone: it holds for ANY invertible upper-triangular
T, so the sketch decides the conditioning of W_m T_m^-1, not whether the
restart is exact.  Checked on CPU with numpy, independent of the oracle."""
import numpy as np


def arnoldi(A, b, m):
    n = len(b)
    W = np.zeros((n, m + 1))
    R = np.zeros((m + 1, m))
    W[:, 0] = b / np.linalg.norm(b)
    for j in range(m):
        p = A @ W[:, j]
        for i in range(j + 1):
            R[i, j] = W[:, i] @ p
            p -= R[i, j] * W[:, i]
        R[j + 1, j] = np.linalg.norm(p)
        W[:, j + 1] = p / R[j + 1, j]
    return W, R


def test_restart_identity_for_any_upper_triangular_T():
    rng = np.random.default_rng(31)
    n, m = 60, 12
    A = rng.standard_normal((n, n)) + 5.0 * np.eye(n)
    W, R = arnoldi(A, rng.standard_normal(n), m)
    Rm, r = R[:m, :], R[m, m - 1]
    assert np.linalg.norm(A @ W[:, :m] - W @ R) <= 1e-12 * np.linalg.norm(A)
    for trial in range(5):
        T = np.triu(rng.standard_normal((m + 1, m + 1))) + np.diag(rng.uniform(0.5, 2.0, m + 1))
        Tm, t, tau = T[:m, :m], T[:m, m], T[m, m]
        Tinv = np.linalg.inv(Tm)
        What = W[:, :m] @ Tinv
        e_m = np.eye(m)[-1]
        X = Tm @ Rm @ Tinv + (r / Tm[-1, -1]) * np.outer(t, e_m)
        v = (W[:, m] - W[:, :m] @ (Tinv @ t)) / tau
        rho = r * tau / Tm[-1, -1]
        lhs = A @ What
        rhs = What @ X + rho * np.outer(v, e_m)
        assert np.linalg.norm(lhs - rhs) <= 1e-10 * np.linalg.norm(lhs)
