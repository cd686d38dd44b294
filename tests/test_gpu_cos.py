"""cos(t sqrt(A)) b on the GPU (the membrane example of Sec. 5: the wave
equation u'' = -L u).

The projected matrix's cos(t sqrt(H)) uses the block-row machinery of the
exponential with the Taylor series of cos(sqrt(A)) in Horner form and the
double-angle step C(4A) = 2 C(A)^2 - I in place of a squaring: parity with the
oracle (which evaluates the propagator exp(t [[0, I], [-H, 0]]) densely) for
the truncated and randomized Gram-Schmidt modes, the float64 and float-float
bases, a mid-run rise of the number of double-angle steps, and convergence to
the sine-mode closed form cos(t sqrt(lambda)).
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


def _gpu(A, b, t, m, k, s, zeta, seed, cycles, basis, ortho=0, tol=0.0):
    import torch

    from paper_2503_22631_gb300 import F_COS_SQRT, Krylov

    kr = Krylov(A.row_ptr, A.col_idx, A.val, f=F_COS_SQRT, t=t, m=m, k=k, s=s, seed=seed, zeta=zeta, basis=basis,
                ortho=ortho)
    x = kr.apply(torch.from_numpy(b).cuda(), tol=tol, max_cycles=cycles)
    torch.cuda.synchronize()
    return x.cpu().numpy(), kr


@pytest.mark.parametrize("basis", [0, 3])
@pytest.mark.parametrize("cycles", [1, 3])
def test_cos_parity_truncated(lib, cuda, basis, cycles):
    A = W.convdiff(24, 2, (10.0, 5.0))
    b = W.rhs_normal(A.n, 3, normalize=True)
    ref = K.restarted(A, b, D.COS_SQRT, 0.05, 12, 2, 40, 8, 17, mode=K.TRUNC, tol=0.0, max_cycles=cycles)
    x, kr = _gpu(A, b, 0.05, 12, 2, 40, 8, 17, cycles, basis)
    assert kr.stats["cycles"] == cycles
    assert _rel(x, ref.x) <= 1e-10


@pytest.mark.parametrize("basis", [0, 3])
def test_cos_parity_rgs_full_window(lib, cuda, basis):
    A = W.poisson2d(32)
    b = W.rhs_normal(A.n, 5, normalize=True)
    ref = K.restarted(A, b, D.COS_SQRT, 0.05, 16, 16, 50, 8, 7, mode=K.RGS, tol=0.0, max_cycles=3)
    x, _ = _gpu(A, b, 0.05, 16, 16, 50, 8, 7, 3, basis, ortho=1)
    assert _rel(x, ref.x) <= 1e-10


def test_cos_double_angle_steps_rise_mid_run(lib, cuda):
    """t = 0.5 on a 3D operator with m = 6: the second cycle needs one more
    double-angle step than the first (5 -> 6, from the oracle's projected
    blocks), so block row 1 is redone at the new scale; 10 cycles converge."""
    A = W.convdiff3d(14, (50.0, 50.0, 50.0))
    b = W.rhs_normal(A.n, 2)
    ref = K.restarted(A, b, D.COS_SQRT, 0.5, 6, 2, 24, 8, 3, mode=K.TRUNC, tol=0.0, max_cycles=10)
    x, kr = _gpu(A, b, 0.5, 6, 2, 24, 8, 3, 10, 3)
    assert _rel(x, ref.x) <= 1e-10
    _, kr1 = _gpu(A, b, 0.5, 6, 2, 24, 8, 3, 1, 3)
    _, kr2 = _gpu(A, b, 0.5, 6, 2, 24, 8, 3, 2, 3)
    _, kr3 = _gpu(A, b, 0.5, 6, 2, 24, 8, 3, 3, 3)
    per_cycle = [kr1.stats["launches"], kr2.stats["launches"] - kr1.stats["launches"],
                 kr3.stats["launches"] - kr2.stats["launches"]]
    assert per_cycle[1] > per_cycle[2]  # the redone block row


def test_cos_converges_to_sine_modes(lib, cuda):
    N = 48
    A = W.poisson2d(N)
    b, c, p, q = W.sine_mode_mixture_2d(N, 8, 23)
    x, kr = _gpu(A, b, 0.3, 8, 2, 30, 8, 5, 60, 3, tol=1e-13)
    assert kr.stats["cycles"] < 60
    assert _rel(x, TR.sine_mode_cos(N, c, p, q, 0.3)) <= 1e-9


@pytest.mark.slow
def test_cos_full_size_double_angle(lib, cuda):
    """The membrane stand-in at full size (2D 5-point Laplacian, 1448^2 =
    2.1M unknowns, m = 40, k = 2, s = 160): GPU solves satisfy
    cos(2t sqrt(A)) b = 2 cos(t sqrt(A)) (cos(t sqrt(A)) b) - b, and the bench's
    4 cycles at t = 0.05 agree with a 12-cycle solve to 1e-8."""
    import torch

    from paper_2503_22631_gb300 import F_COS_SQRT, Krylov

    A = W.poisson2d(1448)
    b = torch.from_numpy(W.rhs_uniform(A.n, W.SEED)).cuda()

    def cosm(t, v, cycles):
        kr = Krylov(A.row_ptr, A.col_idx, A.val, f=F_COS_SQRT, t=t, m=40, k=2, s=160, seed=W.SEED, zeta=8, basis=3)
        return kr.apply(v, tol=0.0, max_cycles=cycles)

    y1 = cosm(0.025, b, 12)
    y2 = cosm(0.025, y1, 12)
    c2 = cosm(0.05, b, 12)
    c4 = cosm(0.05, b, 4)
    torch.cuda.synchronize()
    assert _rel((2.0 * y2 - b).cpu().numpy(), c2.cpu().numpy()) <= 1e-9
    assert _rel(c4.cpu().numpy(), c2.cpu().numpy()) <= 1e-8
