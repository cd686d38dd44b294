"""Randomized properties of the oracle's dense routines and sparse sign
embedding (hypothesis; CPU only).  Each property is a fact of the mathematics
that holds for every input in the drawn family, not a re-typed formula."""
import math

import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

from oracle import dense as D  # noqa: E402
from oracle import sketch as OS  # noqa: E402

SETTINGS = dict(max_examples=25, deadline=None, derandomize=True)


@settings(**SETTINGS)
@given(s=st.integers(1, 40), c=st.integers(1, 12), seed=st.integers(0, 2**32 - 1),
       spread=st.floats(0.0, 8.0))
def test_qr_positive_factorizes_with_orthonormal_q(s, c, seed, spread):
    """U = Q T, Q^T Q = I, T upper triangular with positive diagonal, for
    full-column-rank U (s >= c) whose column scales span up to 10^8."""
    if s < c:
        s, c = c, s
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((s, c)) * 10.0 ** rng.uniform(-spread / 2, spread / 2, size=c)
    Q, T = D.qr_positive(U)
    assert np.linalg.norm(Q @ T - U) <= 1e-13 * np.linalg.norm(U)
    assert np.linalg.norm(Q.T @ Q - np.eye(c)) <= 1e-13 * c
    assert np.all(np.diag(T) > 0) and np.all(np.tril(T, -1) == 0)


@settings(**SETTINGS)
@given(n=st.integers(1, 10), seed=st.integers(0, 2**32 - 1), scale=st.floats(1e-3, 60.0),
       a=st.floats(-3.0, 3.0), b=st.floats(-3.0, 3.0))
def test_expm_group_and_shift_properties(n, seed, scale, a, b):
    """exp((a + b) X) = exp(a X) exp(b X) (commuting arguments), and
    exp(X + c I) = e^c exp(X): catches a wrong scaling or squaring count,
    which breaks the group law at some norms."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n)) * scale / max(1.0, math.sqrt(n))
    X = X / max(1.0, np.abs(X).sum(axis=0).max() / scale)
    lhs = D.expm((a + b) * X)
    rhs = D.expm(a * X) @ D.expm(b * X)
    tol = 1e-12 * max(1.0, np.linalg.norm(D.expm(abs(a) * X), 2) * np.linalg.norm(D.expm(abs(b) * X), 2)) \
        * (1.0 + scale * (abs(a) + abs(b)))
    assert np.linalg.norm(lhs - rhs) <= tol * max(1.0, np.linalg.norm(rhs))
    c = 0.7
    assert np.allclose(D.expm(X + c * np.eye(n)), math.exp(c) * D.expm(X), rtol=1e-12,
                       atol=1e-12 * np.abs(D.expm(X)).max())


@settings(**SETTINGS)
@given(n=st.integers(1, 8), seed=st.integers(0, 2**32 - 1), cond=st.floats(0.0, 6.0))
def test_invsqrtm_squares_to_the_inverse(n, seed, cond):
    """Z = A^{-1/2} for SPD A with condition number up to 10^6: Z is
    symmetric and Z A Z = I."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = 10.0 ** rng.uniform(0.0, cond, size=n)
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    Z = D.invsqrtm(A)
    assert np.linalg.norm(Z - Z.T) <= 1e-10 * np.linalg.norm(Z)
    assert np.linalg.norm(Z @ A @ Z - np.eye(n)) <= 1e-8


@settings(**SETTINGS)
@given(n=st.integers(1, 600), s=st.integers(1, 400), zeta=st.integers(1, 32), seed=st.integers(0, 2**64 - 1))
def test_sketch_columns_are_unit_signed_and_distinct(n, s, zeta, seed):
    """Every column: zeta distinct rows in [0, s), signs +-1, so ||S e_j|| = 1
    (Eq. 3), for any seed and any zeta <= min(s, 32)."""
    zeta = min(zeta, s)
    rows, signs = OS.sketch_columns(n, s, zeta, seed)
    assert rows.shape == (n, zeta) and rows.min() >= 0 and rows.max() < s
    assert all(len(set(r)) == zeta for r in rows.tolist())
    assert set(np.unique(signs).tolist()) <= {-1.0, 1.0}
