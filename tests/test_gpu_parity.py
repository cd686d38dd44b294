"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (relative 2-norm of the result): 1e-10 with a float64 basis,
1e-5 with a float32 basis, 1e-3 with a bfloat16 basis; sketch rows and signs
bit-exact.  Parity runs use a fixed number of cycles (tol = 0) on both sides so
that no early-exit decision can differ.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dense as D
from oracle import krylov as K
from oracle import sketch as OS
from oracle import truth as TR

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-5, 2: 1e-3, 3: 1e-10}


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _gpu(A, b, fkind, t, m, k, s, zeta, seed, cycles, basis=0, adjoint=False, tol=0.0):
    import torch

    from paper_2503_22631_gb300 import Krylov

    kr = Krylov(A.row_ptr, A.col_idx, A.val, f=fkind, t=t, m=m, k=k, s=s, seed=seed, zeta=zeta, basis=basis)
    x = kr.apply(torch.from_numpy(b).cuda(), tol=tol, max_cycles=cycles, adjoint=adjoint)
    torch.cuda.synchronize()
    return x.cpu().numpy(), kr


@pytest.mark.parametrize("n,s,zeta,col0", [(5000, 60, 8, 0), (3000, 160, 8, 1 << 20), (2000, 17, 4, 7),
                                           (1000, 40, 32, 0), (4097, 200, 1, 123456), (3000, 255, 8, 99),
                                           (3000, 256, 8, 5), (2000, 1000, 16, 0), (500, 8, 8, 0)])
def test_sketch_columns_bit_exact(lib, cuda, n, s, zeta, col0):
    from paper_2503_22631_gb300 import sketch_columns

    seed = 0x1234_5678_9ABC_DEF0
    rows, signs = sketch_columns(col0 + n, s, zeta, seed, col0=col0, count=n)
    orows, osigns = OS.sketch_columns(col0 + n, s, zeta, seed, cols=np.arange(col0, col0 + n))
    assert np.array_equal(rows, orows)
    assert np.array_equal(signs.astype(np.float64), osigns)


@pytest.mark.parametrize("basis", [0, 3])
@pytest.mark.parametrize("cycles", [1, 2, 3])
def test_poisson2d_fp64_parity(lib, cuda, cycles, basis):
    A = W.poisson2d(64)
    b = W.rhs_normal(A.n, W.SEED, normalize=True)
    args = (D.EXP_NEG, 1e-3, 30, 2, 60, 8, 99)
    ref = K.restarted(A, b, *args, mode=K.TRUNC, tol=0.0, max_cycles=cycles)
    x, _ = _gpu(A, b, *args, cycles, basis=basis)
    assert _rel(x, ref.x) <= TOL[basis]


def test_poisson2d_converges_to_closed_form(lib, cuda):
    N = 64
    A = W.poisson2d(N)
    b, c, p, q = W.sine_mode_mixture_2d(N, 24, 3)
    x, kr = _gpu(A, b, D.EXP_NEG, 1e-3, 30, 2, 60, 8, 5, cycles=20, tol=1e-12)
    exact = TR.sine_mode_exp(N, c, p, q, 1e-3)
    assert _rel(x, exact) <= 1e-10


@pytest.mark.parametrize("basis", [1, 2])
def test_reduced_precision_basis(lib, cuda, basis):
    A = W.convdiff3d(24, (50.0, 50.0, 50.0))
    b = W.rhs_uniform(A.n, 4)
    args = (D.EXP_NEG, 2e-4, 24, 2, 96, 8, 17)
    ref = K.restarted(A, b, *args, mode=K.TRUNC, tol=0.0, max_cycles=3)
    x, _ = _gpu(A, b, *args, 3, basis=basis)
    assert _rel(x, ref.x) <= TOL[basis]


@pytest.mark.parametrize("basis", [0, 3])
def test_convdiff_fp64_parity_cycles(lib, cuda, basis):
    A = W.convdiff3d(20, (50.0, 50.0, 50.0))
    b = W.rhs_uniform(A.n, 8)
    args = (D.EXP_NEG, 1e-3, 20, 2, 80, 8, 23)
    ref = K.restarted(A, b, *args, mode=K.TRUNC, tol=0.0, max_cycles=4)
    x, _ = _gpu(A, b, *args, 4, basis=basis)
    assert _rel(x, ref.x) <= TOL[basis]


@pytest.mark.parametrize("basis", [0, 3])
def test_non_float32_values_and_generic_sketch(lib, cuda, basis):
    """Matrix values that do not round-trip through float32 (float-float value
    pairs), sketch with s > 255 (generic generator), window k = 3."""
    A = W.convdiff(40, 2, (7.3, 1.1))
    A = W.Csr(A.n, A.row_ptr, A.col_idx, A.val * (1.0 + 1e-9 * np.arange(A.nnz) / A.nnz))
    b = W.rhs_normal(A.n, 9)
    args = (D.EXP_NEG, 3e-4, 24, 3, 300, 12, 5)
    ref = K.restarted(A, b, *args, mode=K.TRUNC, tol=0.0, max_cycles=3)
    x, _ = _gpu(A, b, *args, 3, basis=basis)
    assert _rel(x, ref.x) <= TOL[basis]


@pytest.mark.parametrize("basis", [0, 3])
def test_inverse_function(lib, cuda, basis):
    A = W.convdiff(24, 2, (10.0, 5.0))
    b = W.rhs_normal(A.n, 2)
    args = (D.INV, 1.0, 30, 2, 90, 8, 3)
    ref = K.restarted(A, b, *args, mode=K.TRUNC, tol=0.0, max_cycles=3)
    x, _ = _gpu(A, b, *args, 3, basis=basis)
    assert _rel(x, ref.x) <= TOL[basis]


@pytest.mark.parametrize("basis", [0, 3])
def test_breakdown_single_mode(lib, cuda, basis):
    N = 32
    A = W.poisson2d(N)
    b, c, p, q = W.sine_mode_mixture_2d(N, 1, 9)
    x, kr = _gpu(A, b, D.EXP_NEG, 1e-3, 10, 2, 30, 8, 1, cycles=5, basis=basis)
    assert kr.stats["breakdown"] == 1
    assert _rel(x, TR.sine_mode_exp(N, c, p, q, 1e-3)) <= 1e-12


@pytest.mark.parametrize("basis", [0, 1, 3])
def test_adjoint_matches_oracle_on_transpose(lib, cuda, basis):
    A = W.convdiff3d(16, (20.0, 0.0, 0.0))
    b = W.rhs_normal(A.n, 5)
    args = (D.EXP_NEG, 2e-3, 20, 2, 80, 8, 41)
    ref = K.restarted(A.transpose(), b, *args, mode=K.TRUNC, tol=0.0, max_cycles=3)
    x, _ = _gpu(A, b, *args, 3, adjoint=True, basis=basis)
    assert _rel(x, ref.x) <= TOL[basis]


def test_small_problem_matches_oracle(lib, cuda):
    A = W.poisson2d(40)
    b = W.rhs_normal(A.n, 6, normalize=True)
    args = (D.EXP_NEG, 1e-3, 16, 2, 40, 8, 77)
    ref = K.restarted(A, b, *args, mode=K.TRUNC, tol=0.0, max_cycles=1, keep=True)
    x, kr = _gpu(A, b, *args, 1)
    T, X, z, me = kr.last_cycle()
    ci = ref.info[0]
    assert me == ci.m_eff
    assert np.allclose(T, ci.T, rtol=1e-11, atol=1e-11 * np.abs(ci.T).max())
    assert _rel(X, ci.X) <= 1e-10
    assert _rel(z, ci.z) <= 1e-10


@pytest.mark.parametrize("basis", [0, 3])
@pytest.mark.parametrize("N", [1, 2])
def test_tiny_exact_when_m_reaches_n(lib, cuda, N, basis):
    """One cycle with m = n <= k (full orthogonalization) spans the whole
    space: the result is f(A)b.  (With a truncated window and m = n the basis
    itself becomes numerically dependent, cond(T_m) ~ 1e16, so that case is
    not a well-posed exactness check.)"""
    A = W.poisson2d(N)
    b = W.rhs_normal(A.n, 1)
    m = A.n
    x, kr = _gpu(A, b, D.EXP_NEG, 1e-2, m, min(m, 4), m + 8, 4, 2, cycles=1, basis=basis)
    exact = TR.dense_fAb(A.to_dense(), b, D.EXP_NEG, 1e-2, symmetric=True)
    assert _rel(x, exact) <= 1e-10


@pytest.mark.parametrize("basis,tol", [(0, 1e-13), (1, 1e-6), (3, 1e-13)])
@pytest.mark.parametrize("s,zeta", [(60, 8), (300, 12)])
def test_sketch_table_equals_regeneration(lib, cuda, basis, tol, s, zeta):
    """S read from the device table and S regenerated inside the step kernels
    are the same matrix: results agree to rounding (atomic order only)."""
    import torch

    from paper_2503_22631_gb300 import Krylov

    A = W.convdiff3d(14, (50.0, 50.0, 50.0))
    b = torch.from_numpy(W.rhs_uniform(A.n, 2)).cuda()
    out = []
    for regen in (False, True):
        kr = Krylov(A.row_ptr, A.col_idx, A.val, f=D.EXP_NEG, t=1e-3, m=20, k=2, s=s, seed=3, zeta=zeta,
                    basis=basis, sketch_regenerate=regen)
        out.append(kr.apply(b, max_cycles=3).cpu().numpy())
    assert _rel(out[1], out[0]) <= tol


def test_product_kernel_variants_agree_bitwise(lib, cuda):
    """Float-float basis: the product kernel that stages the pieces of w_j in
    shared memory (autotune off: always when a segment plan exists) and the
    autotuned choice sum every row in the same order: identical results."""
    import torch

    from paper_2503_22631_gb300 import BASIS_DF64, F_EXP_NEG, Krylov

    A = W.convdiff3d(20, (50.0, 50.0, 50.0))
    b = torch.from_numpy(W.rhs_uniform(A.n, 3)).cuda()
    xs = []
    for autotune in (False, True):
        kr = Krylov(A.row_ptr, A.col_idx, A.val, f=F_EXP_NEG, t=2e-3, m=20, k=2, s=60, seed=5, zeta=8,
                    basis=BASIS_DF64, autotune=autotune)
        xs.append(kr.apply(b, tol=0.0, max_cycles=3).cpu().numpy())
    assert np.array_equal(xs[0], xs[1])


def test_random_sparse_matrix_gather_path(lib, cuda):
    """Columns spread over the whole range (no segment plan fits): the
    gather kernel, against the oracle."""
    rng = np.random.default_rng(17)
    n, per = 6000, 9
    cols = np.sort(rng.choice(n, size=(n, per - 1), replace=True), axis=1)
    rows = []
    for i in range(n):
        c = np.unique(np.concatenate([[i], cols[i]]))
        rows.append(c)
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(c) for c in rows])
    ci = np.concatenate(rows).astype(np.int32)
    val = rng.standard_normal(ci.size) * 0.1
    diag = rp[:-1] + np.array([np.searchsorted(c, i) for i, c in enumerate(rows)])
    val[diag] = 4.0 + np.abs(val[diag])
    A = W.Csr(n, rp.astype(np.int32), ci, val)
    b = W.rhs_normal(n, 4)
    args = (D.EXP_NEG, 0.1, 20, 2, 60, 8, 21)
    ref = K.restarted(A, b, *args, mode=K.TRUNC, tol=0.0, max_cycles=2)
    x, _ = _gpu(A, b, *args, 2, basis=3)
    assert _rel(x, ref.x) <= 1e-10


@pytest.mark.parametrize("adjoint", [False, True])
def test_wide_band_operator_parity(lib, cuda, adjoint):
    """A 2D Poisson matrix (bandwidth 200) with two couplings 39,999 rows apart:
    the bandwidth is at least 2^15, so the staged product kernel reads 4-byte
    column indices (a narrower band gets 2-byte offsets col - row); the
    operator and its transpose against the oracle."""
    import scipy.sparse as sp

    P = W.poisson2d(200)
    n = P.n
    Ps = sp.csr_matrix((P.val, P.col_idx, P.row_ptr), shape=(n, n))
    far = sp.csr_matrix((np.array([-2048.0, -1024.0]), (np.array([0, n - 1]), np.array([n - 1, 0]))), shape=(n, n))
    Aw = (Ps + far).tocsr()
    Aw.sort_indices()
    A = W.Csr(n, Aw.indptr.astype(np.int32), Aw.indices.astype(np.int32), Aw.data.astype(np.float64))
    assert np.abs(np.repeat(np.arange(n), np.diff(A.row_ptr)) - A.col_idx).max() >= 2**15
    b = W.rhs_normal(n, 6, normalize=True)
    args = (D.EXP_NEG, 1e-5, 20, 2, 60, 8, 9)
    ref = K.restarted(A.transpose() if adjoint else A, b, *args, mode=K.TRUNC, tol=0.0, max_cycles=2)
    x, _ = _gpu(A, b, *args, 2, basis=3, adjoint=adjoint)
    assert _rel(x, ref.x) <= 1e-10


def _odd_matrix(n, seed, long_row=False):
    """Random rows of 0..8 nonzeros (unaligned row starts), every 7th row
    empty, random normal values (not float32-exact); long_row adds ~300
    entries to the middle row."""
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(n):
        ln = int(rng.integers(0, 9))
        if i % 7 == 3:
            ln = 0
        cols = np.unique(rng.integers(0, n, size=ln)) if ln else np.zeros(0, dtype=np.int64)
        if long_row and i == n // 2:
            cols = np.unique(np.concatenate([cols, rng.choice(n, size=min(n, 300), replace=False)]))
        rows.append(cols)
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(c) for c in rows])
    ci = np.concatenate(rows).astype(np.int32)
    return W.Csr(n, rp.astype(np.int32), ci, rng.standard_normal(ci.size))


@pytest.mark.parametrize("basis", [0, 3])
@pytest.mark.parametrize("n", [1, 31, 32, 33, 4097])
def test_odd_shapes_empty_rows(lib, cuda, n, basis):
    """Sizes around a warp and a tile (n = 1, 31, 32, 33, 4097), empty rows,
    unaligned row starts, and at n = 4097 a row of ~300 nonzeros (the
    float-float product's long-row path): 3 cycles against the oracle (n = 1
    breaks down exactly in its first cycle)."""
    A = _odd_matrix(n, n, long_row=(n == 4097))
    b = W.rhs_normal(n, 5)
    m = min(10, n)
    s = max(m + 1, 16)
    args = (D.EXP_NEG, 0.3, m, min(2, m), s, min(4, s), 3)
    ref = K.restarted(A, b, *args, mode=K.TRUNC, tol=0.0, max_cycles=3)
    x, kr = _gpu(A, b, *args, 3, basis=basis)
    assert kr.stats["cycles"] == ref.cycles
    assert _rel(x, ref.x) <= 1e-10
