"""Pins of the CPU oracle against things other than itself (runs without a GPU).

Each test ties one oracle routine to an independent fact: a library routine
used as a special case, a closed form, an invariant the paper states, or brute
force on tiny inputs.  The comment on each names the mistake it would catch.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sl

import workloads as W
from oracle import dense as D
from oracle import krylov as K
from oracle import philox as PH
from oracle import sketch as OS
from oracle import truth as TR


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- Philox ----
def _triton_randint4x(seed, offsets):
    os.environ["TRITON_INTERPRET"] = "1"
    triton = pytest.importorskip("triton")
    import torch
    import triton.language as tl

    @triton.jit
    def kern(out_ptr, off_ptr, seed, N: tl.constexpr):
        i = tl.arange(0, N)
        off = tl.load(off_ptr + i)
        a, b, c, d = tl.randint4x(seed, off, 10)
        tl.store(out_ptr + i * 4 + 0, a)
        tl.store(out_ptr + i * 4 + 1, b)
        tl.store(out_ptr + i * 4 + 2, c)
        tl.store(out_ptr + i * 4 + 3, d)

    N = len(offsets)
    out = torch.zeros(4 * N, dtype=torch.int32)
    off = torch.tensor(offsets, dtype=torch.int64)
    kern[(1,)](out, off, seed, N)
    return (out.numpy().astype(np.int64) & 0xFFFFFFFF).reshape(N, 4)


def test_philox_matches_independent_implementation():
    """Triton's Philox4x32-10 (counter (lo, hi, 0, 0) of a 64-bit offset, key
    from the 64-bit seed) must agree word for word: catches a wrong multiplier,
    Weyl constant, word order or key schedule."""
    for seed in (0, 1, 0xDEADBEEF, 0x1234_5678_9ABC_DEF0):
        offs = [0, 1, 2, 3, 12345, (1 << 32) + 5, (7 << 32) + 99, (63 << 32) + 4_000_000]
        ref = _triton_randint4x(seed, offs)
        c0 = np.array([o & 0xFFFFFFFF for o in offs], dtype=np.uint64)
        c1 = np.array([o >> 32 for o in offs], dtype=np.uint64)
        got = np.stack(PH.philox4x32_10(c0, c1, 0, 0, seed & 0xFFFFFFFF, seed >> 32), axis=1).astype(np.int64)
        assert np.array_equal(got, ref)


def test_philox_known_answer_vectors():
    """The published known-answer vectors of Philox4x32-10
    (tests/golden/philox4x32_10_kat.txt): an all-zero, an all-ones and a
    digits-of-pi counter/key, so a wrong constant fails without any other
    implementation to compare with."""
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    lines = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(lines) == 3
    for words in lines:
        v = [int(w, 16) for w in words]
        got = [int(w) for w in PH.philox4x32_10(*v[:6])]
        assert got == v[6:]


# ---------------------------------------------------------------- sketch ----
def test_sketch_columns_invariants():
    """Eq. (3): zeta distinct rows per column, +-1/sqrt(zeta) entries, so every
    column of S has norm exactly 1."""
    for n, s, zeta in [(3000, 160, 8), (2000, 17, 4), (500, 40, 32), (400, 8, 8), (1000, 60, 1)]:
        rows, signs = OS.sketch_columns(n, s, zeta, 99)
        assert rows.shape == (n, zeta)
        assert rows.min() >= 0 and rows.max() < s
        assert all(len(set(r)) == zeta for r in rows)
        assert set(np.unique(signs)) <= {-1.0, 1.0}
        S = OS.SparseSign(n, s, zeta, 99).dense()
        assert np.allclose(np.linalg.norm(S, axis=0), 1.0, atol=1e-15)
    # subsets of columns reproduce the full generation (counter-based)
    rows, signs = OS.sketch_columns(5000, 60, 8, 7)
    r2, s2 = OS.sketch_columns(5000, 60, 8, 7, cols=np.arange(1000, 1200))
    assert np.array_equal(rows[1000:1200], r2) and np.array_equal(signs[1000:1200], s2)


def test_sketch_uniform_rows_and_balanced_signs():
    """Rows uniform over [0, s) and Rademacher signs: chi-square and binomial
    checks on 2e5 columns (catches a biased row map such as v % s without
    rejection at large s, or a sign bit tied to the row)."""
    for n, s in [(200_000, 1000), (300_000, 20000)]:
        rows, signs = OS.sketch_columns(n, s, 1, 2024)
        counts = np.bincount(rows.ravel(), minlength=s)
        expected = n / s
        chi2 = ((counts - expected) ** 2 / expected).sum()
        # chi-square with s-1 dof: mean s-1, sd sqrt(2(s-1)); allow 5 sd.  At
        # s = 20000, v % s without rejection would double the weight of rows
        # below 12768.
        assert abs(chi2 - (s - 1)) < 5 * math.sqrt(2 * (s - 1))
    frac_neg = np.mean(signs < 0)
    assert abs(frac_neg - 0.5) < 5 * math.sqrt(0.25 / signs.size)
    # sign independent of row parity
    odd = rows.ravel() % 2 == 1
    assert abs(np.mean(signs.ravel()[odd] < 0) - 0.5) < 5 * math.sqrt(0.25 / odd.sum())


def test_sketch_column_from_known_answer_words():
    """Column 0 under seed 0 uses the Philox counter (0, 0, 0, 0) and key
    (0, 0), whose output words are the first published known-answer vector
    6627e8d5 e169c58d bc57ac4c 9b00dbd8.  Taking 16-bit chunks low half first
    (e8d5, 6627, c58d, e169, ac4c, bc57, dbd8, 9b00), a candidate row
    (chunk & 0x7fff) mod s and a sign from bit 15, worked by hand:
    s = 160 (no chunk reaches the rejection limit 32640) gives rows
    117, 71, 45, 137, 140, 87, 152, 32 with signs - + - - - - - -;
    s = 20000 (limit 20000 rejects 26837, 26151, 24937 and 23512) gives
    17805, 11340, 15447, 6912, all negative.  Pins the chunk order, the mask,
    the sign bit and the rejection rule of the generator's definition."""
    rows, signs = OS.sketch_columns(1, 160, 8, 0)
    assert rows[0].tolist() == [117, 71, 45, 137, 140, 87, 152, 32]
    assert signs[0].tolist() == [-1.0, 1.0, -1.0, -1.0, -1.0, -1.0, -1.0, -1.0]
    rows, signs = OS.sketch_columns(1, 20000, 4, 0)
    assert rows[0].tolist() == [17805, 11340, 15447, 6912]
    assert signs[0].tolist() == [-1.0] * 4


def test_sketch_stream_from_independent_philox():
    """Columns away from 0, seeds with both key words set and sizes that need
    several counter blocks: rebuilt one candidate at a time from Triton's
    Philox4x32-10 words for counter (column, block, 0, 0) and key
    (seed mod 2^32, seed div 2^32).  Pins which counter and key words carry
    the column, the block and the seed."""
    cases = [(0x1234_5678_9ABC_DEF0, 20000, 8), (77, 160, 8), (2**40 + 3, 3001, 16)]
    cols = [1, 2, 12345, 1_000_003]
    for seed, s, zeta in cases:
        rows, signs = OS.sketch_columns(cols[-1] + 1, s, zeta, seed, cols=np.array(cols))
        lim = 32768 - 32768 % s
        for ci, col in enumerate(cols):
            want_r, want_s, block = [], [], 0
            while len(want_r) < zeta:
                words = _triton_randint4x(seed, [col + (block << 32)])[0]
                for w in words:
                    for chunk in (int(w) & 0xFFFF, int(w) >> 16):
                        v, row = chunk & 0x7FFF, (chunk & 0x7FFF) % s
                        if len(want_r) < zeta and v < lim and row not in want_r:
                            want_r.append(row)
                            want_s.append(-1.0 if chunk >> 15 else 1.0)
                block += 1
            assert rows[ci].tolist() == want_r and signs[ci].tolist() == want_s


def test_sketch_is_an_embedding_in_expectation():
    """Eq. (1): E ||S x||^2 = ||x||^2 over the random S; mean over 400 seeds
    within 4 standard errors."""
    rng = np.random.default_rng(0)
    x = rng.standard_normal(300)
    vals = [np.linalg.norm(OS.SparseSign(300, 40, 4, sd).apply(x)) ** 2 / np.dot(x, x) for sd in range(400)]
    vals = np.array(vals)
    assert abs(vals.mean() - 1.0) < 4 * vals.std() / math.sqrt(len(vals))


def test_sketch_apply_matches_dense_product():
    """S applied column-wise equals the dense S matrix product (catches a
    missing 1/sqrt(zeta) or a sign flip in apply)."""
    Sk = OS.SparseSign(700, 50, 8, 3)
    V = np.random.default_rng(1).standard_normal((700, 3))
    dense = np.zeros((50, 700))
    for j in range(700):
        for q in range(8):
            dense[Sk.rows[j, q], j] += Sk.signs[j, q] / math.sqrt(8)
    assert np.allclose(Sk.apply(V), dense @ V, rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------- dense -----
def test_qr_positive_is_cholesky_factor():
    """T with positive diagonal is unique: it equals the Cholesky factor of
    U^T U, and Q T = U with orthonormal Q."""
    rng = np.random.default_rng(2)
    for s, c in [(60, 31), (160, 41), (20, 20), (5, 1)]:
        U = rng.standard_normal((s, c)) * rng.uniform(0.1, 10, size=c)
        Q, T = D.qr_positive(U)
        assert np.allclose(Q @ T, U, atol=1e-12 * np.abs(U).max())
        assert np.allclose(Q.T @ Q, np.eye(c), atol=1e-13)
        assert np.all(np.diag(T) > 0) and np.allclose(np.tril(T, -1), 0)
        L = np.linalg.cholesky(U.T @ U)
        assert rel(T, L.T) < 1e-10


@pytest.mark.parametrize("scale", [1e-3, 0.3, 4.0, 40.0, 400.0])
def test_expm_matches_scipy(scale):
    """Degree-13 Pade scaling and squaring against scipy's expm."""
    rng = np.random.default_rng(int(scale * 1000) % 97)
    A = rng.standard_normal((25, 25)) / 5.0 * scale
    A = A - np.diag(np.full(25, 1.2 * scale))  # keep exp(A) of moderate size
    assert rel(D.expm(A), sl.expm(A)) < 1e-12


def test_expm_closed_forms():
    """Rotation generator, a Jordan block, and exp(A) exp(-A) = I."""
    th = 2.7
    R = D.expm(np.array([[0.0, th], [-th, 0.0]]))
    assert np.allclose(R, [[math.cos(th), math.sin(th)], [-math.sin(th), math.cos(th)]], atol=1e-15)
    lam = -3.0
    J = lam * np.eye(4) + np.diag(np.ones(3), 1)
    E = D.expm(J)
    ref = math.exp(lam) * np.array([[1, 1, 1 / 2, 1 / 6], [0, 1, 1, 1 / 2], [0, 0, 1, 1], [0, 0, 0, 1]])
    assert np.allclose(E, ref, rtol=1e-14, atol=1e-16)
    A = np.random.default_rng(5).standard_normal((12, 12))
    assert np.allclose(D.expm(A) @ D.expm(-A), np.eye(12), atol=1e-12)


@pytest.mark.parametrize("th", [10.6, 21.2, 42.4, 84.8])
def test_expm_rotation_at_scaling_boundaries(th):
    """exp of [[0, th], [-th, 0]] is the rotation by th.  The angles sit just
    below 2^j * 2 theta_13, where scaling by 2^-s with s = ceil(log2(||A||_1 /
    theta_13)) brings the norm to theta_13 but one fewer halving leaves it
    near 2 theta_13, where the degree-13 approximant on the imaginary axis is
    off by ~1e-8 (catches a floor for the ceil, or one squaring too few)."""
    R = D.expm(np.array([[0.0, th], [-th, 0.0]]))
    ref = np.array([[math.cos(th), math.sin(th)], [-math.sin(th), math.cos(th)]])
    assert np.abs(R - ref).max() < 1e-14 * th


def test_qr_positive_column_nearly_along_e1():
    """Householder QR is backward stable only when the reflector is formed
    with alpha = -sign(x_1) ||x|| (no cancellation in x_1 - alpha); columns
    whose trailing parts are tiny relative to the leading entry expose a wrong
    sign choice as a large ||Q T - U|| or a non-orthogonal Q."""
    rng = np.random.default_rng(11)
    for sgn in (1.0, -1.0):
        U = 1e-9 * rng.standard_normal((30, 6))
        U[np.arange(6), np.arange(6)] += sgn * np.array([1.0, 2.0, 0.5, 3.0, 1.5, 0.7])
        Q, T = D.qr_positive(U)
        assert np.linalg.norm(Q @ T - U) < 1e-14 * np.linalg.norm(U)
        assert np.linalg.norm(Q.T @ Q - np.eye(6)) < 1e-14
        assert np.all(np.diag(T) > 0) and np.allclose(np.tril(T, -1), 0)


def test_invsqrtm():
    """Z^2 A = I, and agreement with the eigendecomposition for SPD A and with
    scipy's sqrtm for a non-symmetric matrix with positive spectrum."""
    rng = np.random.default_rng(3)
    B = rng.standard_normal((30, 30))
    S = B @ B.T + 1e-3 * np.eye(30)
    lam, Q = np.linalg.eigh(S)
    Z = D.invsqrtm(S)
    assert rel(Z, Q @ np.diag(lam ** -0.5) @ Q.T) < 1e-10
    N = np.eye(20) * 5 + rng.standard_normal((20, 20)) * 0.5
    Z = D.invsqrtm(N)
    assert rel(Z @ Z @ N, np.eye(20)) < 1e-12
    assert rel(Z, np.linalg.inv(sl.sqrtm(N))) < 1e-11


def test_phi1m_closed_forms():
    """phi_1 on a diagonal (expm1(l)/l, 1 at l = 0), on a 2 x 2 Jordan block
    (phi_1' on the superdiagonal), and A phi_1(A) = e^A - I for a random A."""
    lam = np.array([-30.0, -2.5, -1e-9, 0.0, 1e-9, 0.7, 3.0])
    P = D.phi1m(np.diag(lam))
    ref = np.where(lam == 0.0, 1.0, np.expm1(lam) / np.where(lam == 0.0, 1.0, lam))
    assert np.allclose(np.diag(P), ref, rtol=1e-14, atol=0)
    assert np.abs(P - np.diag(np.diag(P))).max() == 0.0
    l = -1.7
    J = np.array([[l, 1.0], [0.0, l]])
    dphi = (l * math.exp(l) - math.exp(l) + 1.0) / l**2
    assert np.allclose(D.phi1m(J), [[math.expm1(l) / l, dphi], [0.0, math.expm1(l) / l]], rtol=1e-14, atol=1e-16)
    A = np.random.default_rng(11).standard_normal((14, 14))
    assert rel(A @ D.phi1m(A), D.expm(A) - np.eye(14)) < 1e-12
    # f_dense applies the parameter: phi_1(-t H)
    H = np.diag([2.0, 5.0])
    assert np.allclose(np.diag(D.f_dense(D.PHI1_NEG, H, 0.3)), -np.expm1(-0.3 * np.array([2.0, 5.0])) / (0.3 * np.array([2.0, 5.0])), rtol=1e-14)


def test_phi1m_matches_eigendecomposition():
    S = W.poisson2d(6).to_dense()
    lam, Q = np.linalg.eigh(S)
    t = 3e-3
    ref = Q @ np.diag(-np.expm1(-t * lam) / (t * lam)) @ Q.T
    assert rel(D.f_dense(D.PHI1_NEG, S, t), ref) < 1e-13


def test_cossqrtm_closed_forms():
    """cos(t sqrt(l)) on a diagonal (cos(0) = 1; a negative l gives cosh), the
    Jordan block: d/dl cos(t sqrt(l)) = -t sin(t sqrt(l)) / (2 sqrt(l)) on the
    superdiagonal, and the double-angle identity C(4A) = 2 C(A)^2 - I."""
    t = 0.9
    lam = np.array([0.0, 0.3, 2.0, 17.0, 150.0, -0.5])
    C = D.cossqrtm(np.diag(lam), t)
    ref = np.where(lam >= 0, np.cos(t * np.sqrt(np.abs(lam))), np.cosh(t * np.sqrt(np.abs(lam))))
    assert np.allclose(np.diag(C), ref, rtol=1e-13, atol=1e-14)
    l = 3.0
    J = np.array([[l, 1.0], [0.0, l]])
    d = -t * math.sin(t * math.sqrt(l)) / (2 * math.sqrt(l))
    assert np.allclose(D.cossqrtm(J, t), [[math.cos(t * math.sqrt(l)), d], [0.0, math.cos(t * math.sqrt(l))]],
                       rtol=1e-13, atol=1e-15)
    A = W.convdiff(5, 2, (3.0, 1.0)).to_dense() * 1e-2
    C1 = D.cossqrtm(A, 1.0)
    assert rel(D.cossqrtm(4.0 * A, 1.0), 2.0 * C1 @ C1 - np.eye(A.shape[0])) < 1e-12
    assert rel(D.f_dense(D.COS_SQRT, A, 2.0), D.cossqrtm(4.0 * A, 1.0)) < 1e-12


def test_cossqrtm_matches_eigendecomposition():
    S = W.poisson2d(6).to_dense()
    lam, Q = np.linalg.eigh(S)
    t = 0.05
    assert rel(D.f_dense(D.COS_SQRT, S, t), Q @ np.diag(np.cos(t * np.sqrt(lam))) @ Q.T) < 1e-12


# ---------------------------------------------------------------- truth -----
def test_kronecker_truth_matches_dense_exponential():
    """exp(-tA) of the Kronecker-sum grid operator applied by mode products
    equals the dense exponential of the assembled CSR matrix (velocities of
    both signs, so the upwind side and the |beta| on the diagonal count)."""
    for N, dim, beta, t in [(6, 3, (50.0, 50.0, 50.0), 1e-2), (9, 2, (0.0, 0.0), 1e-3), (5, 3, (20.0, 0.0, 0.0), 5e-3),
                              (7, 2, (-30.0, 15.0), 2e-3), (5, 3, (-10.0, 40.0, -25.0), 4e-3)]:
        A = W.convdiff(N, dim, beta)
        b = np.random.default_rng(N).standard_normal(A.n)
        ref = sl.expm(-t * A.to_dense()) @ b
        assert rel(TR.kron_expm_apply(N, dim, beta, t, b), ref) < 1e-12
        refT = sl.expm(-t * A.to_dense()).T @ b
        assert rel(TR.kron_expm_apply(N, dim, beta, t, b, transpose=True), refT) < 1e-12


def test_sine_modes_are_eigenvectors():
    N = 16
    A = W.poisson2d(N)
    b, c, p, q = W.sine_mode_mixture_2d(N, 5, 1)
    assert rel(TR.sine_mode_exp(N, c, p, q, 3e-3), sl.expm(-3e-3 * A.to_dense()) @ b) < 1e-12


def test_csr_matvec_matches_dense():
    A = W.convdiff3d(7, (50.0, 10.0, 0.0))
    x = np.random.default_rng(4).standard_normal(A.n)
    assert rel(K.csr_matvec(A, x), A.to_dense() @ x) < 1e-15


def test_workload_sizes_match_configurations():
    """Matrix sizes quoted for the workloads (n, nnz)."""
    A = W.poisson2d(64)
    assert (A.n, A.nnz) == (4096, 20224)
    B = W.convdiff3d(12)
    assert B.nnz == 7 * 12**3 - 6 * 12**2
    assert set(np.unique(W.convdiff3d(4).val)) == {-275.0, -25.0, 900.0}  # h=1/5, beta/h=250
    F = W.fem_p1_kuhn(6, 1.0, 1)
    Fd = F.to_dense()
    assert np.allclose(Fd, Fd.T) and np.linalg.eigvalsh(Fd).min() > 0
    assert np.diff(F.row_ptr).max() == 15
    N = 5  # interior nodes per axis: diagonal + 6 axis + 6 face-diagonal + 2 body-diagonal couplings
    assert F.nnz == N**3 + 6 * N * N * (N - 1) + 6 * N * (N - 1) ** 2 + 2 * (N - 1) ** 3


# ---------------------------------------------------------------- Krylov ----
MODES = [K.TRUNC, K.RGS, K.CLASSICAL]


@pytest.mark.parametrize("mode", MODES)
def test_restarted_converges_to_kronecker_truth(mode):
    """Algorithm 2 in every orthogonalization mode reaches exp(-tA)b of the
    closed form (non-symmetric 3D convection-diffusion)."""
    N, beta, t = 10, (50.0, 50.0, 50.0), 3e-3
    A = W.convdiff3d(N, beta)
    b = W.rhs_uniform(A.n, 1)
    k = 2 if mode == K.TRUNC else 20
    r = K.restarted(A, b, D.EXP_NEG, t, 20, k, 80, 8, 5, mode=mode, tol=1e-13, max_cycles=40)
    assert rel(r.x, TR.kron_expm_apply(N, 3, beta, t, b)) < 1e-11


@pytest.mark.parametrize("mode", MODES)
def test_sine_mixture_closed_form(mode):
    N, t = 32, 1e-3
    A = W.poisson2d(N)
    b, c, p, q = W.sine_mode_mixture_2d(N, 20, 4)
    k = 2 if mode == K.TRUNC else 30
    r = K.restarted(A, b, D.EXP_NEG, t, 30, k, 60, 8, 6, mode=mode, tol=1e-13, max_cycles=30)
    assert rel(r.x, TR.sine_mode_exp(N, c, p, q, t)) < 1e-11


@pytest.mark.parametrize("mode", MODES)
def test_single_mode_breaks_down_exactly(mode):
    N = 20
    A = W.poisson2d(N)
    b, c, p, q = W.sine_mode_mixture_2d(N, 1, 2)
    r = K.restarted(A, b, D.EXP_NEG, 2e-3, 10, 2 if mode == K.TRUNC else 10, 30, 4, 1, mode=mode, max_cycles=5)
    assert r.breakdown and r.cycles == 1 and r.info[0].m_eff == 1
    assert rel(r.x, TR.sine_mode_exp(N, c, p, q, 2e-3)) < 1e-13


@pytest.mark.parametrize("mode", MODES)
def test_near_breakdown_is_not_breakdown(mode):
    """b = phi_{1,1} + 1e-7 phi_{12,12}: after one step the residual is about
    1e-5 of ||A w_1||, far above rounding, so the first step is NOT a happy
    breakdown, and one cycle reproduces the closed form of the sine modes to
    rounding; a breakdown test that is too loose stops after one column with
    an error of order 1e-7."""
    N = 24
    A = W.poisson2d(N)
    c, p, q = np.array([1.0, 1e-7]), np.array([1, 12]), np.array([1, 12])
    h = 1.0 / (N + 1)
    ii = np.arange(1, N + 1)
    b = sum(cl * np.outer(np.sin(ql * np.pi * ii * h), np.sin(pl * np.pi * ii * h))
            for cl, pl, ql in zip(c, p, q)).reshape(-1)
    k = 2 if mode == K.TRUNC else 10
    r = K.restarted(A, b, D.EXP_NEG, 1e-3, 10, k, 30, 4, 1, mode=mode, max_cycles=1)
    assert r.info[0].m_eff > 1
    assert rel(r.x, TR.sine_mode_exp(N, c, p, q, 1e-3)) < 1e-12


def test_stopping_is_invariant_to_the_scale_of_b():
    """f(A)(a b) = a f(A) b and the stopping test ||y|| <= tol ||x|| is
    relative (Sec. 4 estimate compared with the iterate's norm), so scaling b
    by 1e6 or 1e-6 changes neither the number of cycles nor x / a."""
    A = W.poisson2d(32)
    b = W.rhs_normal(A.n, 4, normalize=True)
    runs = [K.restarted(A, a * b, D.EXP_NEG, 1e-3, 10, 2, 40, 8, 3, mode=K.TRUNC, tol=1e-8, max_cycles=60)
            for a in (1.0, 1e6, 1e-6)]
    assert runs[0].cycles > 2
    assert all(r.cycles == runs[0].cycles for r in runs)
    assert rel(runs[1].x / 1e6, runs[0].x) < 1e-13 and rel(runs[2].x / 1e-6, runs[0].x) < 1e-13


@pytest.mark.parametrize("mode", MODES)
def test_update_norm_is_the_norm_of_the_update(mode):
    """The stopping quantity of cycle c is ||x_c - x_{c-1}|| (the norm of the
    correction y added in that cycle), checked by running one cycle fewer."""
    A = W.convdiff(14, 2, (30.0, 10.0))
    b = W.rhs_uniform(A.n, 6)
    k = 2 if mode == K.TRUNC else 12
    r3 = K.restarted(A, b, D.EXP_NEG, 2e-2, 12, k, 48, 8, 3, mode=mode, max_cycles=3)
    r2 = K.restarted(A, b, D.EXP_NEG, 2e-2, 12, k, 48, 8, 3, mode=mode, max_cycles=2)
    assert r3.cycles == 3
    d = np.linalg.norm(r3.x - r2.x)
    assert d > 1e-6 * np.linalg.norm(r3.x)
    assert abs(r3.info[2].update_norm - d) <= 1e-12 * d
    assert abs(r3.info[2].x_norm - np.linalg.norm(r3.x)) <= 1e-14 * np.linalg.norm(r3.x)


@pytest.mark.parametrize("fkind", [D.EXP_NEG, D.INV, D.INVSQRT, D.PHI1_NEG, D.COS_SQRT])
def test_exact_when_m_reaches_n(fkind):
    """With m = n the Krylov space is the whole space: one cycle is exact."""
    A = W.fem_p1_kuhn(4, 1.0, 2)  # 27 unknowns, SPD
    b = np.random.default_rng(7).standard_normal(A.n)
    r = K.restarted(A, b, fkind, 0.05, A.n, A.n, A.n + 10, 4, 9, mode=K.TRUNC, max_cycles=1)
    ref = TR.dense_fAb(A.to_dense(), b, fkind, 0.05, symmetric=True)
    assert rel(r.x, ref) < 1e-10


def test_inverse_residual():
    """f = 1/z: the restarted result solves A x = b (true residual)."""
    A = W.convdiff(20, 2, (10.0, 5.0))
    b = W.rhs_normal(A.n, 2)
    r = K.restarted(A, b, D.INV, 1.0, 30, 2, 90, 8, 3, mode=K.TRUNC, tol=1e-12, max_cycles=200)
    assert np.linalg.norm(b - K.csr_matvec(A, r.x)) / np.linalg.norm(b) < 1e-9


def test_arnoldi_like_relations():
    """Eq. (5) A W_m = W_{m+1} R_m for every mode; RGS sketches orthonormal
    (Algorithm 1); whitened TRUNC: the restart decomposition
    A (W_m T_m^-1) = (W_m T_m^-1) X + v rho e_m^T holds (Eq. A.1 reading)."""
    A = W.convdiff3d(8, (50.0, 50.0, 50.0))
    b = W.rhs_uniform(A.n, 3)
    m = 12
    Ad = A.to_dense()
    for mode, k in [(K.TRUNC, 2), (K.RGS, m), (K.RGS, 3), (K.CLASSICAL, m)]:
        r = K.restarted(A, b, D.EXP_NEG, 1e-3, m, k, 4 * m, 8, 3, mode=mode, max_cycles=2, keep=True)
        for ci in r.info:
            Wm, Rb = ci.W, ci.R
            res = np.linalg.norm(Ad @ Wm[:, :m] - Wm @ Rb) / (np.linalg.norm(Ad) * np.linalg.norm(Wm))
            assert res < 1e-14
            if mode == K.RGS and k >= m:  # full sketch orthogonalization
                assert ci.sketch_orth_err < 1e-12
        if mode == K.TRUNC:
            # the next start vector v has S v = q_{m+1} (the last column of Q),
            # so the second cycle's T[1,1] = ||S v|| is 1 up to rounding and the
            # coupling rho T^{next}[1,1] reduces to rho
            assert abs(r.info[1].T[0, 0] - 1.0) < 1e-12
        if mode == K.TRUNC:
            ci = r.info[0]
            T = ci.T
            Tm = T[:m, :m]
            What = ci.W[:, :m] @ np.linalg.inv(Tm)
            v = (ci.W[:, m] - ci.W[:, :m] @ np.linalg.solve(Tm, T[:m, m])) / T[m, m]
            rho = ci.R[m, m - 1] * T[m, m] / Tm[-1, -1]
            lhs = Ad @ What
            rhs = What @ ci.X + np.outer(v, np.eye(m)[-1]) * rho
            assert rel(lhs, rhs) < 1e-12
            Sk = OS.SparseSign(A.n, 4 * m, 8, 3)
            SW = Sk.apply(What)
            assert np.allclose(SW.T @ SW, np.eye(m), atol=1e-12)
            assert abs(np.linalg.norm(Sk.apply(v)) - 1.0) < 1e-12


@pytest.mark.parametrize("mode", [K.TRUNC, K.RGS])
def test_orthogonalization_window_holds_exactly_k_vectors(mode):
    """The truncated orthogonalization of step j involves exactly the last k
    vectors: column j of R is zero above row j - k + 1 and nonzero on the k
    rows of the window, and the new vector (TRUNC: w_{j+1}; RGS: its sketch
    u_{j+1}) is orthogonal to the window's vectors but not to the one just
    outside it (a non-symmetric operator, so no three-term recurrence makes
    older vectors orthogonal by accident).  Catches a window one too wide or
    one too narrow."""
    A = W.convdiff(16, 2, (60.0, 25.0))
    b = W.rhs_uniform(A.n, 5)
    m, k = 10, 3
    r = K.restarted(A, b, D.EXP_NEG, 1e-3, m, k, 80, 8, 5, mode=mode, max_cycles=1, keep=True)
    ci = r.info[0]
    R = ci.R
    V = ci.W if mode == K.TRUNC else ci.U
    V = V / np.linalg.norm(V, axis=0)
    outside = []
    for j in range(m):
        lo = max(0, j - k + 1)
        assert np.all(R[:lo, j] == 0.0)
        assert np.all(R[lo:j + 1, j] != 0.0)
        assert np.abs(V[:, lo:j + 1].T @ V[:, j + 1]).max() < 1e-12
        if lo > 0:
            outside.append(abs(V[:, lo - 1] @ V[:, j + 1]))
    assert max(outside) > 1e-3


def test_interpolation_property():
    """Proposition (Eqs. 7-8): the restarted result equals q(A) b where q
    interpolates f at the eigenvalues of H_{km} (Newton divided differences,
    Horner form), independently of the basis."""
    A = W.convdiff(12, 1, (30.0,))
    b = W.rhs_normal(A.n, 5)
    t = 2e-4
    for mode, k in [(K.TRUNC, 2), (K.RGS, 3), (K.CLASSICAL, 3)]:
        r = K.restarted(A, b, D.EXP_NEG, t, 3, k, 12, 2, 8, mode=mode, max_cycles=2)
        lam = np.linalg.eigvals(r.H).astype(complex)
        # divided differences of f(z) = exp(-t z) at the nodes
        dd = np.exp(-t * lam)
        for lev in range(1, len(lam)):
            dd[lev:] = (dd[lev:] - dd[lev - 1:-1]) / (lam[lev:] - lam[:-lev])
        Ad = A.to_dense().astype(complex)
        acc = dd[-1] * b.astype(complex)
        for i in range(len(lam) - 2, -1, -1):
            acc = dd[i] * b + (Ad @ acc - lam[i] * acc)
        assert np.abs(acc.imag).max() < 1e-9 * np.abs(acc).max()
        assert rel(acc.real, r.x) < 1e-9


def test_stopping_estimate_decreases():
    """Sec. 4: ||y|| of successive cycles decreases for the convergent case and
    the final update is below tol ||x||."""
    A = W.poisson2d(48)
    b = W.rhs_normal(A.n, 8, normalize=True)
    r = K.restarted(A, b, D.EXP_NEG, 1e-3, 20, 2, 60, 8, 3, mode=K.TRUNC, tol=1e-10, max_cycles=30)
    ys = [ci.update_norm for ci in r.info]
    assert ys[-1] <= 1e-10 * r.info[-1].x_norm
    assert all(ys[i + 1] < ys[i] for i in range(1, len(ys) - 1))


@pytest.mark.parametrize("mode", [K.TRUNC, K.RGS])
def test_restarted_phi1_converges_to_sine_modes(mode):
    """phi_1(-t A) b (the paper's phi function, Sec. 5) on the 5-point Laplacian
    for a mixture of eigenmodes: closed form phi_1(-t lambda) per mode."""
    N = 24
    A = W.poisson2d(N)
    b, c, p, q = W.sine_mode_mixture_2d(N, 6, 13)
    t = 2e-3
    r = K.restarted(A, b, D.PHI1_NEG, t, 10, 2 if mode == K.TRUNC else 10, 40, 8, 5, mode=mode, tol=1e-13,
                    max_cycles=40)
    assert rel(r.x, TR.sine_mode_phi1(N, c, p, q, t)) < 1e-10


@pytest.mark.parametrize("mode", [K.TRUNC, K.RGS])
def test_restarted_cos_converges_to_sine_modes(mode):
    """cos(t sqrt(A)) b (the membrane example, Sec. 5) on the 5-point Laplacian
    for a mixture of eigenmodes: closed form cos(t sqrt(lambda)) per mode."""
    N = 24
    A = W.poisson2d(N)
    b, c, p, q = W.sine_mode_mixture_2d(N, 6, 17)
    t = 0.02
    r = K.restarted(A, b, D.COS_SQRT, t, 12, 2 if mode == K.TRUNC else 12, 40, 8, 5, mode=mode, tol=1e-13,
                    max_cycles=60)
    assert rel(r.x, TR.sine_mode_cos(N, c, p, q, t)) < 1e-10


def test_rmat_laplacian_properties():
    """The graph stand-in: symmetric, zero row sums, diagonal = degree,
    off-diagonals -1, power-law rows (the longest far above the mean)."""
    L = W.rmat_laplacian(12, 16, 5)
    Dn = L.to_dense()
    assert np.array_equal(Dn, Dn.T)
    assert np.abs(Dn.sum(axis=1)).max() == 0.0
    off = Dn - np.diag(np.diag(Dn))
    assert set(np.unique(off)) <= {-1.0, 0.0}
    assert np.array_equal(np.diag(Dn), -off.sum(axis=1))
    deg = np.diff(L.row_ptr) - 1
    assert deg.max() > 256 and deg.max() > 20 * deg.mean()


def test_heat_kernel_on_graph_conserves_mass():
    """exp(-tL) x_0 with 1^T L = 0: the total probability stays 1 and the
    uniform vector is stationary (oracle, restarted, float64)."""
    L = W.rmat_laplacian(10, 8, 3)
    x0 = W.rhs_probability(L.n, 4)
    r = K.restarted(L, x0, D.EXP_NEG, 0.1, 20, 2, 60, 8, 3, mode=K.TRUNC, tol=1e-13, max_cycles=60)
    assert abs(r.x.sum() - 1.0) < 1e-12
    assert rel(r.x, TR.dense_fAb(L.to_dense(), x0, D.EXP_NEG, 0.1, symmetric=True)) < 1e-10
    ones = np.ones(L.n)
    r1 = K.restarted(L, ones, D.EXP_NEG, 0.1, 20, 2, 60, 8, 3, mode=K.TRUNC, tol=0.0, max_cycles=2)
    assert rel(r1.x, ones) < 1e-13


def test_rmat_laplacian_directed():
    """Directed variant: zero row sums (L 1 = 0), L[i, i] = out-degree, not
    symmetric; its uniform vector is stationary for the oracle's heat kernel."""
    L = W.rmat_laplacian(10, 8, 3, directed=True)
    Dn = L.to_dense()
    assert np.abs(Dn.sum(axis=1)).max() == 0.0
    assert not np.array_equal(Dn, Dn.T)
    ones = np.ones(L.n)
    r = K.restarted(L, ones, D.EXP_NEG, 0.1, 20, 20, 60, 8, 3, mode=K.RGS, tol=0.0, max_cycles=2)
    assert rel(r.x, ones) < 1e-13


# ---- reduced-precision storage of the basis (the precision form) ----------
def test_round_storage_bf16_matches_torch_conversion():
    """bfloat16 rounding (nearest, ties to even) against torch's float32 ->
    bfloat16 conversion, on random values and on exact halfway cases."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    v = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-30, 30, 4000),
                        [0.0, -0.0, 1.0, -2.5, 3.0e38]])
    f = v.astype(np.float32)
    # halfway cases: the dropped 16 bits are exactly 0x8000, upper half odd and even
    u = f.view(np.uint32)
    halves = ((u & np.uint32(0xFFFF0000)) | np.uint32(0x8000)).view(np.float32)
    f = np.concatenate([f, halves])
    want = torch.from_numpy(f).to(torch.bfloat16).to(torch.float64).numpy()
    got = K.round_storage(f.astype(np.float64), K.BF16)
    assert np.array_equal(got, want)


def test_round_storage_f32_and_f64():
    rng = np.random.default_rng(4)
    v = rng.standard_normal(1000) * 1e3
    assert np.array_equal(K.round_storage(v, K.F64), v)
    assert np.array_equal(K.round_storage(v, None), v)
    r = K.round_storage(v, K.F32)
    assert np.array_equal(r, v.astype(np.float32).astype(np.float64))
    assert np.all(np.abs(r - v) <= 2.0**-24 * np.abs(v))
    with pytest.raises(ValueError):
        K.round_storage(v, "f16")


@pytest.mark.parametrize("store,u", [(K.F32, 2.0**-24), (K.BF16, 2.0**-8)])
def test_stored_basis_is_representable_and_relation_holds_to_storage_rounding(store, u):
    """With a reduced-precision basis every stored column is exactly
    representable in the storage format, and the Arnoldi-like relation
    A W_m = W_{m+1} R_m (Eq. 5) holds for the stored vectors up to the storage
    rounding of each new column: column j's residual is at most
    u r_{j+1,j} ||w_{j+1}|| (u the unit roundoff of the format), while with
    FP64 storage it is at the FP64 rounding level."""
    A = W.convdiff(14, 2, (30.0, 10.0))
    b = W.rhs_normal(A.n, 8)
    m, k = 12, 2
    r = K.restarted(A, b, D.EXP_NEG, 1e-3, m, k, 40, 8, 9, mode=K.TRUNC, max_cycles=2, keep=True, store=store)
    r64 = K.restarted(A, b, D.EXP_NEG, 1e-3, m, k, 40, 8, 9, mode=K.TRUNC, max_cycles=2, keep=True)
    for ci, c64 in zip(r.info, r64.info):
        Wst, R = ci.W, ci.R
        assert np.array_equal(Wst, K.round_storage(Wst, store))
        AW = np.column_stack([K.csr_matvec(A, Wst[:, j]) for j in range(m)])
        res = np.linalg.norm(AW - Wst @ R, axis=0)
        bound = u * np.abs(np.diag(R, -1)) * np.linalg.norm(Wst[:, 1:], axis=0)
        assert np.all(res <= 1.01 * bound + 1e-12 * np.linalg.norm(AW, axis=0))
        # the storage rounding is what the relation misses: not FP64-level
        assert res.max() > 1e3 * 2.0**-53 * np.abs(np.diag(R, -1)).max()
        AW64 = np.column_stack([K.csr_matvec(A, c64.W[:, j]) for j in range(m)])
        res64 = np.linalg.norm(AW64 - c64.W @ c64.R, axis=0)
        assert np.all(res64 <= 1e-13 * np.linalg.norm(AW64, axis=0))


def test_store_rounds_the_start_vector():
    """A = c I: every vector is an eigenvector, so the cycle breaks down after
    one column and x = eta exp(-t c) w_1 exactly, with w_1 the STORED start
    vector round(b / eta); with FP64 storage that is exp(-t c) b.  The
    reduced-precision result differs from the FP64 one by exactly the storage
    rounding of b / eta."""
    n, c, t = 64, 3.7, 0.3
    A = W.Csr(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.full(n, c))
    b = W.rhs_normal(n, 6)
    eta = np.linalg.norm(b)
    r64 = K.restarted(A, b, D.EXP_NEG, t, 4, 2, 20, 8, 3, mode=K.TRUNC, max_cycles=1)
    assert r64.breakdown
    np.testing.assert_allclose(r64.x, np.exp(-t * c) * b, rtol=1e-14)
    for store in (K.F32, K.BF16):
        r = K.restarted(A, b, D.EXP_NEG, t, 4, 2, 20, 8, 3, mode=K.TRUNC, max_cycles=1, store=store)
        assert r.breakdown
        w1 = K.round_storage(b / eta, store)
        np.testing.assert_allclose(r.x, eta * np.exp(-t * c) * w1, rtol=1e-14)
        assert not np.allclose(r.x, r64.x, rtol=1e-3 * (2.0**-24 if store == K.F32 else 2.0**-8), atol=0)
    with pytest.raises(ValueError):
        K.restarted(A, b, D.EXP_NEG, t, 4, 2, 20, 8, 3, mode=K.RGS, max_cycles=1, store=K.F32)
