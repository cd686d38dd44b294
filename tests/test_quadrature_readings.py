"""The quadratures the GPU evaluates f of the projected matrix with, checked on
CPU against dense references (numpy / scipy), independent of the library.

* z^{-1/2} (the Stieltjes form z^{-1/2} = (2/pi) int_R e^u (z + e^{2u})^{-1} du,
  trapezoidal rule in u with step 0.2 on [0.5 ln(1e-18 a) - 38,
  0.5 ln(1e4 a) + 38], a = ||A||_inf): geometric accuracy off the negative
  real axis, tails below e^-38 relative for spectra in [1e-18 a, 1e4 a].
* exp(-t z) as a resolvent integral on the midpoint rule of the parabolic and
  hyperbolic contours of Trefethen, Weideman and Schmelzer (BIT 46, 2006),
  N = 32 points, the 16 with Im > 0 used through conjugate symmetry, after the
  shift sigma = (-ln ||exp(-tH) e_1|| - 2) / t.  The two contours disagree
  when one of them encloses a Ritz value the other misses (the solver's
  per-cycle self-check), but agree when both miss it, which only the
  comparison with scaling and squaring detects.
* The block forward substitution that gives the first column of
  (H + s I)^{-1} for the block lower-bidiagonal matrix of Algorithm 2 one
  block at a time, carrying one number per shift from block to block.
"""
import numpy as np
import pytest
import scipy.linalg as sla

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# --------------------------------------------------------------- z^{-1/2} --
def invsqrt_nodes(alpha):
    h = 0.2
    u_lo = 0.5 * np.log(alpha * 1e-18) - 38.0
    u_hi = 0.5 * np.log(alpha * 1e4) + 38.0
    n = int(np.ceil((u_hi - u_lo) / h)) + 1
    return u_lo + h * np.arange(n), h


def invsqrt_first_column(A):
    alpha = np.abs(A).sum(axis=1).max()
    u, h = invsqrt_nodes(alpha)
    e1 = np.zeros(A.shape[0])
    e1[0] = 1.0
    acc = np.zeros(A.shape[0])
    I = np.eye(A.shape[0])
    for ui in u:
        acc += (2.0 / np.pi) * h * np.exp(ui) * np.linalg.solve(A + np.exp(2.0 * ui) * I, e1)
    return acc


def test_invsqrt_node_count_does_not_depend_on_the_norm():
    """The interval is 0.5 ln(1e22) + 76 long whatever ||A||_inf: 508 nodes."""
    for alpha in (1e-3, 1.0, 40.0, 3.7e5):
        u, h = invsqrt_nodes(alpha)
        assert h == 0.2 and len(u) == 508


def invsqrt_scalar(z, alpha):
    u, h = invsqrt_nodes(alpha)
    return (2.0 / np.pi) * h * np.sum(np.exp(u) / (z + np.exp(2.0 * u)))


def test_invsqrt_rule_on_scalars_meets_its_tail_and_step_bounds():
    """On [1e-18 a, 1e4 a] the tails and the step leave only rounding; off
    the axis the error is the trapezoidal rule's geometric term, about
    2 exp(-2 pi d / h) with d = (pi - |arg z|) / 2 (~4e-11 at |arg z| = pi/2)."""
    alpha = 37.0
    for k in range(-18, 5):
        z = alpha * 10.0 ** k
        assert abs(invsqrt_scalar(z, alpha) - z ** -0.5) <= 1e-15 * z ** -0.5
    for frac in (0.25, 0.5, 0.75):
        bound = 2.5 * np.exp(-2.0 * np.pi * (np.pi - np.pi * frac) / 2.0 / 0.2) + 1e-15
        for r in (1e-12, 1.0, 1e3):
            z = alpha * r * np.exp(1j * np.pi * frac)
            assert abs(invsqrt_scalar(z, alpha) - z ** -0.5) <= bound * abs(z ** -0.5)


@pytest.mark.parametrize("cond", [1e2, 1e4])
def test_invsqrt_quadrature_matches_eigendecomposition_spd(cond):
    """Against the eigendecomposition of the same (rounded) matrix; a larger
    condition number measures the matrix's own sensitivity, not the rule."""
    rng = np.random.default_rng(11)
    n = 30
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.geomspace(1.0 / cond, 1.0, n) * 3.7e3
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    w, V = np.linalg.eigh(A)
    ref = (V * w ** -0.5) @ V[0]
    got = invsqrt_first_column(A)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_invsqrt_quadrature_nonsymmetric_convection_diffusion():
    """An upwind convection-diffusion matrix (non-normal, real positive
    spectrum): against the inverse of scipy's sqrtm."""
    nx = 12
    h = 1.0 / (nx + 1)
    T = (np.diag(np.full(nx, 2.0)) - np.diag(np.ones(nx - 1), 1) - np.diag(np.ones(nx - 1), -1)) / h ** 2
    C = (np.diag(np.ones(nx)) - np.diag(np.ones(nx - 1), -1)) * (30.0 / h)
    I = np.eye(nx)
    A = np.kron(I, T + C) + np.kron(T, I)
    ref = np.linalg.solve(np.real(sla.sqrtm(A)), np.eye(A.shape[0])[:, 0])
    got = invsqrt_first_column(A)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


# ---------------------------------------------------------- exp(-t z) --
EQ_N = 32


def contour_points(c):
    hq = 2.0 * np.pi / EQ_N
    th = (np.arange(EQ_N // 2) + 0.5) * hq
    if c == 0:  # parabolic
        z = EQ_N * (0.1309 - 0.1194 * th ** 2 + 0.25j * th)
        dz = EQ_N * (-2.0 * 0.1194 * th + 0.25j)
    else:  # hyperbolic
        A = 2.246 * EQ_N
        z = A * (1.0 - np.sin(1.1721 - 0.3443j * th))
        dz = A * 0.3443j * np.cos(1.1721 - 0.3443j * th)
    return z, dz, hq


def exp_w_times(W, v, c):
    """e^W v by the midpoint rule on contour c (real W and v)."""
    z, dz, hq = contour_points(c)
    I = np.eye(W.shape[0])
    acc = np.zeros(W.shape[0])
    for zk, dk in zip(z, dz):
        acc += np.imag(np.exp(zk) * dk * np.linalg.solve(zk * I - W, v.astype(complex)))
    return (hq / np.pi) * acc


def shifted_exp_first_column(H, t):
    e1 = np.zeros(H.shape[0])
    e1[0] = 1.0
    f1 = sla.expm(-t * H) @ e1
    sigma = (-np.log(np.linalg.norm(f1)) - 2.0) / t
    W = -t * (H - sigma * np.eye(H.shape[0]))
    return f1, [np.exp(-t * sigma) * exp_w_times(W, e1, c) for c in (0, 1)]


def nonnormal_real_spectrum(rng, n, lo, hi):
    D = np.diag(np.concatenate([[lo, 1.3 * lo + 1.0], rng.uniform(lo, hi, n - 2)]))
    N = np.triu(rng.standard_normal((n, n)), 1) * 0.05 * hi / n
    Q = np.eye(n) + 0.1 * rng.standard_normal((n, n))
    return Q @ (D + N) @ np.linalg.inv(Q)


@pytest.mark.parametrize("seed,t", [(1, 1e-2), (2, 1e-3), (3, 5e-2)])
def test_exp_contours_match_expm_on_nonnormal_matrices(seed, t):
    rng = np.random.default_rng(seed)
    H = nonnormal_real_spectrum(rng, 40, 3.0, 1e4)
    f1, (fp, fh) = shifted_exp_first_column(H, t)
    scale = np.abs(f1).max()
    assert np.abs(fp - f1).max() <= 1e-12 * scale
    assert np.abs(fh - f1).max() <= 1e-12 * scale
    assert np.abs(fp - fh).max() <= 1e-12 * scale


def complex_pairs(seed, t, im_lo, im_hi, n=20):
    """Eigenvalues re +- i im, re in [50, 500], t im in [im_lo, im_hi]."""
    rng = np.random.default_rng(seed)
    blocks = [np.array([[re, im], [-im, re]])
              for re, im in zip(rng.uniform(50.0, 500.0, n // 2), rng.uniform(im_lo / t, im_hi / t, n // 2))]
    Q = np.eye(n) + 0.1 * rng.standard_normal((n, n))
    return Q @ sla.block_diag(*blocks) @ np.linalg.inv(Q)


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_exp_contours_disagree_when_one_encloses_a_ritz_value_the_other_misses(seed):
    """Ritz values off the negative axis that the contours enclose
    differently (t |Im| up to 20): the two sums differ far beyond the 1e-12
    the solver accepts."""
    t = 1e-2
    for lo, hi in ((0.0, 3.0), (8.0, 20.0)):
        f1, (fp, fh) = shifted_exp_first_column(complex_pairs(seed, t, lo, hi), t)
        assert np.abs(fp - fh).max() > 1e-9 * np.abs(f1).max()


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_exp_contours_agree_but_both_miss_ritz_values_far_off_the_axis(seed):
    """Ritz values far outside both contours (t |Im| of 60 to 180, the range
    of the convection-diffusion operator's): both sums leave out their
    components alike, so the two agree to ~1e-14 while both are wrong.  The
    agreement of the contours cannot see this; the comparison with scaling
    and squaring in the cycles evaluated both ways does."""
    t = 1e-2
    f1, (fp, fh) = shifted_exp_first_column(complex_pairs(seed, t, 60.0, 180.0), t)
    scale = np.abs(f1).max()
    assert np.abs(fp - fh).max() <= 1e-12 * scale
    assert np.abs(fp - f1).max() >= 0.5 * scale and np.abs(fh - f1).max() >= 0.5 * scale


# ----------------------------------------------- block forward substitution --
def block_bidiagonal(rng, c, m):
    """Algorithm 2's H after c cycles: blocks X_a on the diagonal, gamma_{a-1}
    at row a m, column a m - 1 (the first row of block a, the last column of
    block a - 1)."""
    X = [rng.standard_normal((m, m)) + 4.0 * m * np.eye(m) for _ in range(c)]
    gam = rng.standard_normal(c - 1)
    H = np.zeros((c * m, c * m))
    for a in range(c):
        H[a * m:(a + 1) * m, a * m:(a + 1) * m] = X[a]
        if a > 0:
            H[a * m, a * m - 1] = gam[a - 1]
    return H, X, gam


def test_block_forward_substitution_gives_the_first_column_of_the_resolvent():
    rng = np.random.default_rng(7)
    c, m = 5, 6
    H, X, gam = block_bidiagonal(rng, c, m)
    for s in (0.0, 0.37, 2.0 + 1.5j):
        ref = np.linalg.solve(H + s * np.eye(c * m), np.eye(c * m)[:, 0].astype(complex))
        carry = None
        for a in range(c):
            rhs = np.zeros(m, dtype=complex)
            rhs[0] = 1.0 if a == 0 else -gam[a - 1] * carry
            y = np.linalg.solve(X[a] + s * np.eye(m), rhs)
            assert np.abs(y - ref[a * m:(a + 1) * m]).max() <= 1e-13 * np.abs(ref).max()
            carry = y[-1]
