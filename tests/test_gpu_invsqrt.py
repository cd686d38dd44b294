"""f(z) = z^{-1/2} (and the breakdown path of f(z) = 1/z) through the CUDA path.

The GPU evaluates the first column of H^{-1/2} for the block lower-bidiagonal
projected matrix by a trapezoidal quadrature of the Stieltjes integral (shifted
block forward substitution per node); the oracle uses dense Denman-Beavers on
the whole H.  Both are accurate to ~1e-14 on these spectra, so the parity
tolerances are those of the basis precision.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dense as D
from oracle import krylov as K
from oracle import truth as TR

pytestmark = pytest.mark.gpu

# Stated tolerances per basis (float64, float32, bfloat16, float-float).  For
# the reduced-precision bases the method itself moves by the storage rounding
# of its basis (the Arnoldi-like relation of Eq. 5 holds only for the stored
# vectors), by an amount that depends on the operator: the tolerance is then
# max(stated, C_STORE * delta_store), where delta_store is the relative change
# of the FP64 oracle's own result when its stored basis is rounded to that
# format (oracle.krylov.restarted(..., store=...), all other arithmetic FP64).
# The GPU rounds once more in its float32 arithmetic, so C_STORE = 4.
STATED = {0: 1e-10, 1: 1e-5, 2: 1e-3, 3: 1e-10}
STORE = {1: K.F32, 2: K.BF16}
C_STORE = 4.0


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _tol(basis, A, b, args, cycles, ref_x):
    """The parity tolerance of `basis` on this problem (see STATED)."""
    if basis not in STORE:
        return STATED[basis]
    r = K.restarted(A, b, *args, mode=K.TRUNC, tol=0.0, max_cycles=cycles, store=STORE[basis])
    return max(STATED[basis], C_STORE * _rel(r.x, ref_x))


def _gpu(A, b, fkind, m, k, s, zeta, seed, cycles, basis=0, tol=0.0, adjoint=False):
    import torch

    from paper_2503_22631_gb300 import Krylov

    kr = Krylov(A.row_ptr, A.col_idx, A.val, f=fkind, t=1.0, m=m, k=k, s=s, seed=seed, zeta=zeta, basis=basis)
    x = kr.apply(torch.from_numpy(b).cuda(), tol=tol, max_cycles=cycles, adjoint=adjoint)
    torch.cuda.synchronize()
    return x.cpu().numpy(), kr


@pytest.mark.parametrize("basis", [0, 1, 2, 3])
@pytest.mark.parametrize("cycles", [1, 3])
def test_invsqrt_fem_parity(lib, cuda, basis, cycles):
    """Kuhn P1 stiffness with log-normal coefficients (the A^{-1/2} workload's
    matrix family, 11^3 unknowns), window k = 4 as in that workload."""
    A = W.fem_p1_kuhn(12, 1.0, W.SEED)
    b = W.rhs_normal(A.n, W.SEED)
    args = (D.INVSQRT, 1.0, 20, 4, 60, 8, 5)
    ref = K.restarted(A, b, *args, mode=K.TRUNC, tol=0.0, max_cycles=cycles)
    x, _ = _gpu(A, b, D.INVSQRT, 20, 4, 60, 8, 5, cycles, basis=basis)
    assert _rel(x, ref.x) <= _tol(basis, A, b, args, cycles, ref.x)


@pytest.mark.parametrize("basis", [0, 3])
def test_invsqrt_nonsymmetric_parity(lib, cuda, basis):
    A = W.convdiff(20, 2, (30.0, 10.0))
    b = W.rhs_normal(A.n, 3)
    ref = K.restarted(A, b, D.INVSQRT, 1.0, 25, 2, 80, 8, 11, mode=K.TRUNC, tol=0.0, max_cycles=4)
    x, _ = _gpu(A, b, D.INVSQRT, 25, 2, 80, 8, 11, 4, basis=basis)
    assert _rel(x, ref.x) <= STATED[basis]


def test_invsqrt_adjoint_parity(lib, cuda):
    A = W.convdiff(16, 2, (30.0, 10.0))
    b = W.rhs_normal(A.n, 4)
    ref = K.restarted(A.transpose(), b, D.INVSQRT, 1.0, 20, 2, 60, 8, 12, mode=K.TRUNC, tol=0.0, max_cycles=3)
    x, _ = _gpu(A, b, D.INVSQRT, 20, 2, 60, 8, 12, 3, adjoint=True)
    assert _rel(x, ref.x) <= 1e-10


def test_invsqrt_converges_to_eigendecomposition(lib, cuda):
    """SPD matrix: Q Lambda^{-1/2} Q^T b from a dense symmetric eigensolver."""
    A = W.fem_p1_kuhn(10, 1.0, 3)
    b = W.rhs_normal(A.n, 5)
    exact = TR.dense_fAb(A.to_dense(), b, D.INVSQRT, symmetric=True)
    x, kr = _gpu(A, b, D.INVSQRT, 30, 4, 90, 8, 6, 200, basis=3, tol=1e-12)
    assert kr.stats["cycles"] < 200
    assert _rel(x, exact) <= 1e-8


@pytest.mark.parametrize("fkind", [D.INVSQRT, D.INV])
def test_single_mode_breakdown(lib, cuda, fkind):
    """b an eigenvector: breakdown after one column, x = f(lambda) b exactly
    (exercises the shortened last block, m_eff = 1 < m)."""
    N = 32
    A = W.poisson2d(N)
    b, c, p, q = W.sine_mode_mixture_2d(N, 1, 9)
    h = 1.0 / (N + 1)
    lam = (4.0 / h**2) * (np.sin(p[0] * np.pi * h / 2) ** 2 + np.sin(q[0] * np.pi * h / 2) ** 2)
    x, kr = _gpu(A, b, fkind, 10, 2, 30, 8, 1, 5, basis=0)
    assert kr.stats["breakdown"] == 1
    fl = lam**-0.5 if fkind == D.INVSQRT else 1.0 / lam
    assert _rel(x, fl * b) <= 1e-12


@pytest.fixture(scope="module")
def fem160():
    cfg = W.CONFIGS["fem_kuhn_160"]
    A = cfg["matrix"]()
    b = cfg["rhs"](A.n)
    args = (D.INVSQRT, 1.0, cfg["m"], cfg["k"], cfg["s"], cfg["zeta"], W.SEED)
    ref = K.restarted(A, b, *args, mode=K.TRUNC, tol=0.0, max_cycles=1)
    return A, b, cfg, ref


@pytest.mark.slow
@pytest.mark.parametrize("basis", [0, 3, 1, 2])
def test_invsqrt_full_size_first_cycle(lib, cuda, fem160, basis):
    """The A^{-1/2} workload at full size (Kuhn P1, 160^3 cells, n = 4,019,679,
    nnz = 59,690,347; m = 50, k = 4, s = 200): one cycle against the oracle,
    for every basis.

    The FP64-class bases meet 1e-10.  The truncated basis of this matrix is
    nearly dependent (kappa(T) ~ 2e5 in the first cycle), so rounding the
    stored basis to float32 or bfloat16 moves the result by ~1e-2: the oracle
    itself moves that much with its stored basis rounded to those formats
    (tests/golden/store_sensitivity.json, written by the committed script
    beside it from oracle/ alone).  The reduced-precision bases are held to
    C_STORE times that sensitivity, and the measured error is reported."""
    import json
    import os

    A, b, cfg, ref = fem160
    x, _ = _gpu(A, b, D.INVSQRT, cfg["m"], cfg["k"], cfg["s"], cfg["zeta"], W.SEED, 1, basis=basis)
    err = _rel(x, ref.x)
    if basis in STORE:
        gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "store_sensitivity.json")))
        delta = gold["fem_kuhn_160"]["cycles_1"][STORE[basis]]
        tol = max(STATED[basis], C_STORE * delta)
    else:
        tol = STATED[basis]
    print(f"fem_kuhn_160 basis {basis}: relative error vs the FP64 oracle {err:.3e} (tolerance {tol:.3e})")
    assert err <= tol
