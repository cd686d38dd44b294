"""phi_1(-t A) b on the GPU (the phi function of Sec. 5: u(t) = u_0 + t phi_1(-L t) b).

The projected matrix's phi_1 rides on the exponential of the augmented matrix
[[-tH, e_1], [0, 0]]: parity with the oracle (which evaluates the same
augmented exponential densely) for the truncated and randomized Gram-Schmidt
modes, the float64 and float-float bases, including cycles that raise the
number of squarings; convergence to the sine-mode closed form; and at full
size (the 128^3 convection-diffusion operator) the identity
t A phi_1(-t A) b = b - exp(-t A) b against the Kronecker closed form of the
exponential.
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

    from paper_2503_22631_gb300 import F_PHI1_NEG, Krylov

    kr = Krylov(A.row_ptr, A.col_idx, A.val, f=F_PHI1_NEG, t=t, m=m, k=k, s=s, seed=seed, zeta=zeta, basis=basis,
                ortho=ortho)
    x = kr.apply(torch.from_numpy(b).cuda(), tol=tol, max_cycles=cycles)
    torch.cuda.synchronize()
    return x.cpu().numpy(), kr


@pytest.mark.parametrize("basis", [0, 3])
@pytest.mark.parametrize("cycles", [1, 4])
def test_phi1_parity_truncated(lib, cuda, basis, cycles):
    A = W.convdiff(24, 2, (10.0, 5.0))
    b = W.rhs_normal(A.n, 3, normalize=True)
    args = (D.PHI1_NEG, 2e-3, 20, 2, 60, 8, 17)
    ref = K.restarted(A, b, *args, mode=K.TRUNC, tol=0.0, max_cycles=cycles)
    x, kr = _gpu(A, b, 2e-3, 20, 2, 60, 8, 17, cycles, basis)
    assert kr.stats["cycles"] == cycles
    assert _rel(x, ref.x) <= 1e-10


@pytest.mark.parametrize("basis", [0, 3])
def test_phi1_parity_rgs_full_window(lib, cuda, basis):
    A = W.poisson2d(32)
    b = W.rhs_normal(A.n, 5, normalize=True)
    args = (D.PHI1_NEG, 1e-3, 20, 20, 60, 8, 7)
    ref = K.restarted(A, b, *args, mode=K.RGS, tol=0.0, max_cycles=3)
    x, _ = _gpu(A, b, 1e-3, 20, 20, 60, 8, 7, 3, basis, ortho=1)
    assert _rel(x, ref.x) <= 1e-10


def test_phi1_scale_levels_rise_mid_run(lib, cuda):
    """A stiff 3D operator with m = 8: ||t X|| of the second cycle needs one
    more squaring than the first (5 -> 6, from the oracle's projected blocks),
    so cycle 2 redoes block row 1 and its phi_1 vector at the new scale; the
    launch count shows it."""
    A = W.convdiff3d(14, (50.0, 50.0, 50.0))
    b = W.rhs_uniform(A.n, 2)
    args = (D.PHI1_NEG, 5e-3, 8, 2, 30, 8, 3)
    ref = K.restarted(A, b, *args, mode=K.TRUNC, tol=0.0, max_cycles=6)
    x, kr = _gpu(A, b, 5e-3, 8, 2, 30, 8, 3, 6, 3)
    assert _rel(x, ref.x) <= 1e-10
    _, kr1 = _gpu(A, b, 5e-3, 8, 2, 30, 8, 3, 1, 3)
    _, kr2 = _gpu(A, b, 5e-3, 8, 2, 30, 8, 3, 2, 3)
    _, kr3 = _gpu(A, b, 5e-3, 8, 2, 30, 8, 3, 3, 3)
    per_cycle = [kr1.stats["launches"], kr2.stats["launches"] - kr1.stats["launches"],
                 kr3.stats["launches"] - kr2.stats["launches"]]
    assert per_cycle[1] > per_cycle[2]  # the redone block row


def test_phi1_converges_to_sine_modes(lib, cuda):
    N = 32
    A = W.poisson2d(N)
    b, c, p, q = W.sine_mode_mixture_2d(N, 6, 21)
    x, kr = _gpu(A, b, 2e-3, 12, 2, 40, 8, 5, 60, 3, tol=1e-13)
    assert kr.stats["cycles"] < 60
    assert _rel(x, TR.sine_mode_phi1(N, c, p, q, 2e-3)) <= 1e-10


@pytest.mark.slow
def test_phi1_full_size_identity(lib, cuda):
    """128^3 convection-diffusion, t = 1e-2, m = 40, k = 2, s = 160 (the phi_1
    bench workload): a 20-cycle solve satisfies t A x = b - exp(-tA) b (the
    exponential from the Kronecker closed form) to 1e-10 relative, and 9 cycles
    (the bench's count) are within 1e-8 of it."""
    import torch

    from paper_2503_22631_gb300 import F_PHI1_NEG, Krylov

    N, t = 128, 1e-2
    A = W.convdiff3d(N)
    b = W.rhs_uniform(A.n, W.SEED)
    kr = Krylov(A.row_ptr, A.col_idx, A.val, f=F_PHI1_NEG, t=t, m=40, k=2, s=160, seed=W.SEED, zeta=8, basis=3)
    bd = torch.from_numpy(b).cuda()
    x20 = kr.apply(bd, tol=0.0, max_cycles=20)
    ax = kr.spmv(x20)
    x9 = kr.apply(bd, tol=0.0, max_cycles=9)
    torch.cuda.synchronize()
    rhs = b - TR.kron_expm_apply(N, 3, (50.0, 50.0, 50.0), t, b)
    assert _rel(t * ax.cpu().numpy(), rhs) <= 1e-10
    assert _rel(x9.cpu().numpy(), x20.cpu().numpy()) <= 1e-8
