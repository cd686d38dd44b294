"""The incremental evaluation of exp(-t H) for the block lower-bidiagonal H of
Algorithm 2, checked on CPU against scipy's expm, independent of the library.

The GPU needs only the last block row of exp(-t H_{cm}) each cycle.  It uses
scaling and squaring with a degree-14 Taylor polynomial on B = -t H / 2^s,
||B||_1 <= 0.5 (the first omitted term, 0.5^15 / 15! e^0.5, is below 2^-53),
and keeps the block rows of every scale level: the powers of a block lower
triangular matrix are block lower triangular, so block row c of a square
needs only block rows <= c of the factor, and a new cycle adds one block row
per level instead of recomputing the whole exponential.
"""
import math

import numpy as np
import scipy.linalg as sla

DEG = 14


def block_bidiagonal(rng, c, m, scale):
    H = np.zeros((c * m, c * m))
    for a in range(c):
        X = rng.standard_normal((m, m)) * scale / m + scale * np.eye(m)
        H[a * m:(a + 1) * m, a * m:(a + 1) * m] = X
        if a > 0:
            H[a * m, a * m - 1] = rng.standard_normal() * scale
    return H


def squarings_for(B):
    nrm = np.abs(B).sum(axis=0).max()
    return max(0, math.ceil(math.log2(nrm / 0.5))) if nrm > 0.5 else 0


def taylor(B):
    n = B.shape[0]
    S = np.eye(n)
    for k in range(DEG, 0, -1):  # Horner: I + B/k (I + B/(k+1) (...))
        S = np.eye(n) + (B @ S) / k
    return S


def test_taylor_degree_bound():
    assert 0.5 ** (DEG + 1) / math.factorial(DEG + 1) * math.exp(0.5) < 2.0 ** -53


def test_taylor_scaling_and_squaring_matches_expm():
    rng = np.random.default_rng(3)
    for t in (1e-3, 1e-2, 1e-1):
        H = block_bidiagonal(rng, 4, 10, 300.0)
        B = -t * H
        s = squarings_for(B)
        E = taylor(B / 2.0 ** s)
        for _ in range(s):
            E = E @ E
        ref = sla.expm(B)
        assert np.abs(E - ref).max() <= 1e-12 * np.abs(ref).max()


def test_block_rows_of_every_level_need_only_earlier_rows():
    """Block row c of the result from the stored block rows <= c at every
    scale level: the same as the full evaluation, so a cycle adds one block
    row per level."""
    rng = np.random.default_rng(4)
    c, m, t = 5, 6, 2e-2
    H = block_bidiagonal(rng, c, m, 200.0)
    B = -t * H
    s = squarings_for(B)
    Bs = B / 2.0 ** s
    full = [taylor(Bs)]
    for _ in range(s):
        full.append(full[-1] @ full[-1])
    levels = [np.zeros_like(B) for _ in range(s + 1)]  # block rows filled cycle by cycle
    for a in range(c):
        rows = slice(a * m, (a + 1) * m)
        lead = slice(0, (a + 1) * m)
        # level 0: the Taylor polynomial of the leading block (the principal
        # submatrix of a block lower triangular matrix's polynomial is the
        # polynomial of its principal submatrix)
        levels[0][rows, lead] = taylor(Bs[lead, lead])[rows]
        for lv in range(1, s + 1):
            prev = levels[lv - 1]
            levels[lv][rows, lead] = prev[rows, lead] @ prev[lead, lead]
        for lv in range(s + 1):
            ref = full[lv]
            assert np.abs(levels[lv][rows] - ref[rows]).max() <= 1e-13 * np.abs(ref[rows]).max()
    last = levels[s][(c - 1) * m:, :]
    exact = sla.expm(B)[(c - 1) * m:, :]
    assert np.abs(last - exact).max() <= 1e-12 * np.abs(exact).max()


def test_cos_sqrt_series_bound():
    """cos(sqrt(-x)) = sum_k x^k / (2k)! for the double-angle form: degree 14
    on ||B||_1 <= 4 leaves a first omitted term of 4^15 / 30! = 4.05e-24."""
    assert 4.0 ** 15 / math.factorial(30) < 4.1e-24
    rng = np.random.default_rng(8)
    A = rng.standard_normal((12, 12))
    A = A @ A.T
    A *= 4.0 / np.abs(A).sum(axis=0).max()  # ||A||_1 = 4, spectrum in [0, 4]
    S = np.zeros_like(A)
    term = np.eye(12)
    for k in range(DEG + 1):
        S += term
        term = -term @ A / ((2 * k + 1) * (2 * k + 2))
    w, V = np.linalg.eigh(A)
    ref = (V * np.cos(np.sqrt(np.maximum(w, 0.0)))) @ V.T
    assert np.abs(S - ref).max() <= 1e-14


def test_phi1_extra_column_from_the_horner_iterate_and_squarings():
    """phi_1(-tH) e_1 as the extra column of exp([[-tH, e_1], [0, 0]]): after
    the Taylor-Horner steps on B = -tH / 2^s the column is S2 w (w = e_1 2^-s,
    S2 the iterate before the last step, which equals sum_i B^i / (i+1)!),
    and a squaring of [[E, g], [0, 1]] maps g to E g + g."""
    rng = np.random.default_rng(9)
    H = block_bidiagonal(rng, 3, 8, 150.0)
    n = H.shape[0]
    t = 3e-2
    B = -t * H
    s = squarings_for(B)
    Bs = B / 2.0 ** s
    S = np.eye(n)
    S2 = None
    for k in range(DEG, 0, -1):
        if k == 1:
            S2 = S
        S = np.eye(n) + (Bs @ S) / k
    series = sum(np.linalg.matrix_power(Bs, i) / math.factorial(i + 1) for i in range(DEG))
    assert np.abs(S2 - series).max() <= 1e-15 * np.abs(series).max()
    w = np.zeros(n)
    w[0] = 2.0 ** -s
    E, g = S, S2 @ w
    for _ in range(s):
        E, g = E @ E, E @ g + g
    aug = np.zeros((n + 1, n + 1))
    aug[:n, :n] = B
    aug[0, n] = 1.0
    ref = sla.expm(aug)[:n, n]
    assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()
    lam, V = np.linalg.eig(B)  # phi_1 by its definition (e^z - 1) / z on the eigenvalues
    direct = np.real(V @ (np.expm1(lam) / lam * np.linalg.solve(V, np.eye(n)[:, 0])))
    assert np.abs(g - direct).max() <= 1e-8 * np.abs(direct).max()


def test_cos_sqrt_by_series_and_double_angle_steps():
    """cos(t sqrt(H)) from the series on B = -t^2 H / 4^s (||B||_1 <= 4) and s
    steps C <- 2 C^2 - I (cos(2x) = 2 cos(x)^2 - 1), against cos(t sqrt(lambda))
    on the eigendecomposition of a symmetric positive semidefinite H."""
    rng = np.random.default_rng(10)
    n = 16
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = rng.uniform(0.0, 5e4, n)
    H = (Q * lam) @ Q.T
    t = 0.05
    B = -(t * t) * H
    nrm = np.abs(B).sum(axis=0).max()
    s = max(0, math.ceil(0.5 * math.log2(nrm / 4.0))) if nrm > 4.0 else 0
    Bs = B / 4.0 ** s
    assert np.abs(Bs).sum(axis=0).max() <= 4.0
    C = np.eye(n)
    for k in range(DEG, 0, -1):  # Horner for sum_k Bs^k / (2k)!
        C = np.eye(n) + (Bs @ C) / ((2 * k - 1) * (2 * k))
    for _ in range(s):
        C = 2.0 * C @ C - np.eye(n)
    ref = (Q * np.cos(t * np.sqrt(lam))) @ Q.T
    assert np.abs(C - ref).max() <= 1e-10
