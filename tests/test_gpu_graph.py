"""The graph-Laplacian heat kernel exp(-tL) x_0 on the GPU (Sec. 5, the
out-degree Laplacian of a network; an undirected R-MAT graph stands in for the
paper's networks).

Power-law rows: the float-float product runs the operator with its rows longer
than 48 nonzeros emptied through the usual kernels, then a long-row kernel
(a CTA per row above 1024 nonzeros, a warp per row below) completes those rows
and reduces.  The method runs as in the
paper's graph example: sketch-space orthogonalization of the whole cycle
(randomized Gram-Schmidt, k = m = 40, s = 320); a window of k = 2 vectors
loses the basis on these stiff operators (kappa(T) reaches 1e16 on the oracle
as well).  Checked: parity with the oracle on a small graph that has long
rows (truncated and randomized modes, float64 and float-float bases, and the
adjoint, which for this symmetric L equals the forward result and exercises
the transpose's long rows); at scale 20 (1M nodes, 32M nonzeros, rows up to
65,000 entries) mass conservation, the stationary uniform vector, and the
convergence the bench counts on (4 cycles to 1e-8).
"""
import numpy as np
import pytest

import workloads as W
from oracle import dense as D
from oracle import krylov as K

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _kr(L, t, m, k, s, basis, seed=3, ortho=0):
    from paper_2503_22631_gb300 import F_EXP_NEG, Krylov

    return Krylov(L.row_ptr, L.col_idx, L.val, f=F_EXP_NEG, t=t, m=m, k=k, s=s, seed=seed, zeta=8, basis=basis,
                  ortho=ortho)


@pytest.mark.parametrize("basis", [0, 3])
@pytest.mark.parametrize("mode", ["trunc", "rgs"])
def test_graph_heat_kernel_parity(lib, cuda, basis, mode):
    import torch

    L = W.rmat_laplacian(12, 16, 5)
    deg = np.diff(L.row_ptr)
    assert (deg > 1024).sum() >= 1 and ((deg > 48) & (deg <= 1024)).sum() > 100  # both long-row paths run
    x0 = W.rhs_probability(L.n, 6)
    if mode == "trunc":
        m, k, s, kmode, ortho = 20, 2, 60, K.TRUNC, 0
    else:
        m, k, s, kmode, ortho = 20, 20, 80, K.RGS, 1
    ref = K.restarted(L, x0, D.EXP_NEG, 0.1, m, k, s, 8, 3, mode=kmode, tol=0.0, max_cycles=3)
    kr = _kr(L, 0.1, m, k, s, basis, ortho=ortho)
    x = kr.apply(torch.from_numpy(x0).cuda(), tol=0.0, max_cycles=3).cpu().numpy()
    assert _rel(x, ref.x) <= 1e-10
    xa = kr.apply(torch.from_numpy(x0).cuda(), tol=0.0, max_cycles=3, adjoint=True).cpu().numpy()
    assert _rel(xa, ref.x) <= 1e-10


@pytest.mark.parametrize("basis", [0, 3])
def test_directed_graph_parity(lib, cuda, basis):
    """A directed R-MAT graph (the paper's uk-2002 is directed): L is not
    symmetric, so the adjoint is checked against the oracle on L^T; both
    directions have long rows (out- and in-degrees are power laws)."""
    import torch

    L = W.rmat_laplacian(12, 16, 9, directed=True)
    assert np.diff(L.row_ptr).max() > 48 and np.diff(L.transpose().row_ptr).max() > 48
    x0 = W.rhs_probability(L.n, 2)
    args = (D.EXP_NEG, 0.1, 20, 20, 80, 8, 3)
    ref = K.restarted(L, x0, *args, mode=K.RGS, tol=0.0, max_cycles=3)
    ref_t = K.restarted(L.transpose(), x0, *args, mode=K.RGS, tol=0.0, max_cycles=3)
    kr = _kr(L, 0.1, 20, 20, 80, basis, ortho=1)
    x = kr.apply(torch.from_numpy(x0).cuda(), tol=0.0, max_cycles=3).cpu().numpy()
    xa = kr.apply(torch.from_numpy(x0).cuda(), tol=0.0, max_cycles=3, adjoint=True).cpu().numpy()
    assert _rel(x, ref.x) <= 1e-10
    assert _rel(xa, ref_t.x) <= 1e-10
    assert _rel(xa, ref.x) > 1e-6  # the two directions differ


@pytest.mark.slow
def test_graph_heat_kernel_full_size(lib, cuda):
    import torch

    L = W.rmat_laplacian(20, 16, W.SEED)
    assert np.diff(L.row_ptr).max() > 60000
    x0 = W.rhs_probability(L.n, W.SEED)
    kr = _kr(L, 0.1, 40, 40, 320, 3, ortho=1)
    x8 = kr.apply(torch.from_numpy(x0).cuda(), tol=0.0, max_cycles=8).cpu().numpy()
    x4 = kr.apply(torch.from_numpy(x0).cuda(), tol=0.0, max_cycles=4).cpu().numpy()
    assert abs(x8.sum() - 1.0) < 1e-11
    assert _rel(x4, x8) <= 1e-8
    ones = kr.apply(torch.ones(L.n, dtype=torch.float64, device="cuda"), tol=0.0, max_cycles=2).cpu().numpy()
    # the float-float basis's floor u t ||L||_inf (u = 2^-48; ||L||_inf = 2 max degree = 1.3e5): 4.6e-11
    lnorm = 2.0 * (np.diff(L.row_ptr).max() - 1)
    assert np.abs(ones - 1.0).max() <= 2.0**-48 * 0.1 * lnorm
