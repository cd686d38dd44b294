"""The randomized Gram-Schmidt cycle (Algorithm 1 inside Algorithm 2) on the GPU.

Parity with the oracle's `rgs` mode on the same seeded inputs and sketch,
with a window of k sketches (k < m) and with the full window (k = m: the
paper's randomized restart), for the float64 and float-float bases; then the
closed forms (Kronecker exponential, single-mode breakdown) and the status for
the bases the mode does not run with.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dense as D
from oracle import krylov as K
from oracle import truth as TR

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _gpu(A, b, fkind, t, m, k, s, zeta, seed, cycles, basis=0, tol=0.0):
    import torch

    from paper_2503_22631_gb300 import ORTHO_RGS, Krylov

    kr = Krylov(A.row_ptr, A.col_idx, A.val, f=fkind, t=t, m=m, k=k, s=s, seed=seed, zeta=zeta, basis=basis,
                ortho=ORTHO_RGS)
    x = kr.apply(torch.from_numpy(b).cuda(), tol=tol, max_cycles=cycles)
    torch.cuda.synchronize()
    return x.cpu().numpy(), kr


@pytest.mark.parametrize("basis", [0, 3])
@pytest.mark.parametrize("k", [2, 20])
@pytest.mark.parametrize("cycles", [1, 3])
def test_rgs_exp_parity(lib, cuda, basis, k, cycles):
    A = W.poisson2d(32)
    b = W.rhs_normal(A.n, 3, normalize=True)
    args = (D.EXP_NEG, 2e-3, 20, k, 60, 8, 17)
    ref = K.restarted(A, b, *args, mode=K.RGS, tol=0.0, max_cycles=cycles)
    x, kr = _gpu(A, b, *args, cycles, basis=basis)
    assert kr.stats["cycles"] == cycles
    assert _rel(x, ref.x) <= 1e-10


@pytest.mark.parametrize("fkind", [D.INV, D.INVSQRT])
def test_rgs_stieltjes_parity(lib, cuda, fkind):
    A = W.convdiff(24, 2, (10.0, 5.0))
    b = W.rhs_normal(A.n, 2)
    args = (fkind, 1.0, 25, 25, 80, 8, 3)
    ref = K.restarted(A, b, *args, mode=K.RGS, tol=0.0, max_cycles=3)
    x, _ = _gpu(A, b, *args, 3, basis=3)
    assert _rel(x, ref.x) <= 1e-10


def test_rgs_convdiff3d_window_and_sketch_table_sizes(lib, cuda):
    """s > 255 (16-bit sketch table) and zeta = 12, window k = 3."""
    A = W.convdiff3d(14, (50.0, 50.0, 50.0))
    b = W.rhs_uniform(A.n, 5)
    args = (D.EXP_NEG, 1e-3, 24, 3, 300, 12, 5)
    ref = K.restarted(A, b, *args, mode=K.RGS, tol=0.0, max_cycles=2)
    x, _ = _gpu(A, b, *args, 2, basis=0)
    assert _rel(x, ref.x) <= 1e-10


def test_rgs_full_window_converges_to_kronecker(lib, cuda):
    N = 12
    A = W.convdiff3d(N, (50.0, 50.0, 50.0))
    b = W.rhs_uniform(A.n, 7)
    t = 2e-2
    exact = TR.kron_expm_apply(N, 3, (50.0, 50.0, 50.0), t, b)
    x, kr = _gpu(A, b, D.EXP_NEG, t, 30, 30, 90, 8, 9, 60, basis=3, tol=1e-13)
    assert kr.stats["cycles"] < 60
    assert _rel(x, exact) <= 1e-9


def test_rgs_single_mode_breaks_down_exactly(lib, cuda):
    N = 32
    A = W.poisson2d(N)
    b, c, p, q = W.sine_mode_mixture_2d(N, 1, 9)
    x, kr = _gpu(A, b, D.EXP_NEG, 1e-3, 10, 10, 30, 8, 1, 5, basis=0)
    assert kr.stats["breakdown"] == 1 and kr.stats["cycles"] == 1
    assert _rel(x, TR.sine_mode_exp(N, c, p, q, 1e-3)) <= 1e-12


@pytest.mark.parametrize("basis", [1, 2])
def test_rgs_reduced_bases_are_unsupported(lib, cuda, basis):
    from paper_2503_22631_gb300 import KrylovError

    A = W.poisson2d(8)
    with pytest.raises(KrylovError) as e:
        _gpu(A, np.ones(A.n), D.EXP_NEG, 1e-3, 10, 10, 30, 8, 1, 1, basis=basis)
    assert e.value.status == -6
