"""exp(-t z) over many restart cycles: the contour-quadrature evaluation of the
projected exponential, whose cost per cycle does not grow with the cycle
count (Sec. 4 notes that f of the growing block matrix becomes expensive
after many restarts).

For exp(-t z) with t > 0 the library evaluates block a of exp(-t H) e_1 by a
resolvent quadrature on two contours (one complex m x m solve per point and
cycle, one complex number per point carried to the next cycle); the first 16
cycles are also evaluated by scaling and squaring, and the quadrature is used
alone afterwards only while it matched the squaring there and its two
contours agree.  Where the contours cannot enclose the spectrum (a rotation
generator: eigenvalues +-i w with w t up to 50) the check fails and scaling
and squaring carries the whole run.
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


def _gpu(A, b, t, m, k, s, seed, cycles, basis):
    import torch

    from paper_2503_22631_gb300 import F_EXP_NEG, Krylov

    kr = Krylov(A.row_ptr, A.col_idx, A.val, f=F_EXP_NEG, t=t, m=m, k=k, s=s, seed=seed, zeta=8, basis=basis)
    x = kr.apply(torch.from_numpy(b).cuda(), tol=0.0, max_cycles=cycles)
    torch.cuda.synchronize()
    return x.cpu().numpy(), kr.stats


@pytest.mark.parametrize("basis", [0, 3])
def test_48_cycles_match_oracle_with_quadrature(lib, cuda, basis):
    """2D Laplacian 32^2, t = 0.1 (t lambda_max ~ 870), m = 8: the restarted
    method needs about 20 cycles; 48 cycles run, the last 32 on the quadrature."""
    A = W.poisson2d(32)
    b = W.rhs_normal(A.n, 31)
    t, m, k, s, seed, cycles = 0.1, 8, 2, 24, 3, 48
    ref = K.restarted(A, b, D.EXP_NEG, t, m, k, s, 8, seed, mode=K.TRUNC, tol=0.0, max_cycles=cycles)
    x, st = _gpu(A, b, t, m, k, s, seed, cycles, basis)
    assert st["fquad_cycles"] == cycles - 16
    assert _rel(x, ref.x) <= 1e-10
    truth = TR.dense_fAb(A.to_dense(), b, D.EXP_NEG, t=t, symmetric=True)
    assert _rel(x, truth) <= 1e-10


def _rotation(n):
    """2 x 2 rotation generators [[0, w], [-w, 0]], w from 10 to 50."""
    w = np.linspace(10.0, 50.0, n // 2)
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.array([i + 1 if i % 2 == 0 else i - 1 for i in range(n)], dtype=np.int32)
    val = np.array([w[i // 2] if i % 2 == 0 else -w[i // 2] for i in range(n)])
    return W.Csr(n, rp, ci, val)


def test_quadrature_check_falls_back_to_squaring(lib, cuda):
    A = _rotation(200)
    b = W.rhs_normal(A.n, 5)
    t, m, k, s, seed, cycles = 1.0, 8, 2, 30, 3, 24
    ref = K.restarted(A, b, D.EXP_NEG, t, m, k, s, 8, seed, mode=K.TRUNC, tol=0.0, max_cycles=cycles)
    x, st = _gpu(A, b, t, m, k, s, seed, cycles, 0)
    assert st["fquad_cycles"] == 0
    assert _rel(x, ref.x) <= 1e-10
