"""KrylovExpm: gradients of L = ||exp(-tA) b - y||^2 through the CUDA path.

* small parity: the autograd gradients equal the oracle's (same cycles, same
  sketch) to the basis tolerance;
* exact references: the Kronecker closed form of the grid exponential gives the
  forward value, the adjoint (grad_b = 2 E^T (f - y)) and grad_t = -2 (f - y)^T A f
  on a 16^3 copy of the adjoint workload and at its full 96^3 size;
* central differences in t (FP64, h = 1e-6) of the GPU's own loss.
"""
import numpy as np
import pytest

import workloads as W
from oracle import grad as G
from oracle import krylov as K
from oracle import truth as TR

pytestmark = pytest.mark.gpu

BETA = (20.0, 0.0, 0.0)
T = 5e-3


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _handle(A, basis, m=40, k=2, s=160, zeta=8, seed=7, t=T):
    from paper_2503_22631_gb300 import F_EXP_NEG, Krylov

    return Krylov(A.row_ptr, A.col_idx, A.val, f=F_EXP_NEG, t=t, m=m, k=k, s=s, seed=seed, zeta=zeta, basis=basis)


def _loss_and_grads(kr, b_np, y_np, t, tol, cycles):
    import torch

    from paper_2503_22631_gb300 import krylov_expm

    b = torch.from_numpy(b_np).cuda().requires_grad_(True)
    tt = torch.tensor(t, dtype=torch.float64, requires_grad=True)
    y = torch.from_numpy(y_np).cuda()
    x = krylov_expm(b, tt, kr, tol, cycles)
    loss = ((x - y) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    return float(loss.detach()), x.detach().cpu().numpy(), b.grad.cpu().numpy(), float(tt.grad)


@pytest.mark.parametrize("basis", [0, 3])
def test_autograd_matches_oracle_gradients(lib, cuda, basis):
    A = W.convdiff3d(8, BETA)
    b = W.rhs_normal(A.n, 1)
    y = W.rhs_normal(A.n, 2)
    m, k, s, zeta, seed, cycles = 12, 2, 40, 8, 3, 3
    ref = G.expm_loss_grad(A, b, y, T, m, k, s, zeta, seed, mode=K.TRUNC, tol=0.0, max_cycles=cycles)
    kr = _handle(A, basis, m=m, k=k, s=s, zeta=zeta, seed=seed)
    loss, x, gb, gt = _loss_and_grads(kr, b, y, T, 0.0, cycles)
    assert _rel(x, ref.x) <= 1e-10
    assert _rel(gb, ref.grad_b) <= 1e-10
    assert abs(gt - ref.grad_t) <= 1e-10 * abs(ref.grad_t)
    assert abs(loss - ref.loss) <= 1e-10 * ref.loss


def _exact(N, b, y, t):
    A = W.convdiff3d(N, BETA)
    f = TR.kron_expm_apply(N, 3, BETA, t, b)
    gb = 2.0 * TR.kron_expm_apply(N, 3, BETA, t, f - y, transpose=True)
    gt = -2.0 * float(np.dot(f - y, K.csr_matvec(A, f)))
    return A, f, gb, gt


def test_autograd_16cube_matches_kronecker_and_differences(lib, cuda):
    import torch

    N = 16
    b = W.rhs_normal(N**3, W.SEED)
    y = W.rhs_normal(N**3, W.SEED + 1)
    A, f, gb_ref, gt_ref = _exact(N, b, y, T)
    kr = _handle(A, 3)
    loss, x, gb, gt = _loss_and_grads(kr, b, y, T, 1e-13, 60)
    assert _rel(x, f) <= 1e-11
    assert _rel(gb, gb_ref) <= 1e-10
    assert abs(gt - gt_ref) <= 1e-9 * abs(gt_ref)

    def L(t):
        kr.set_param(t)
        xt = kr.apply(torch.from_numpy(b).cuda(), tol=1e-14, max_cycles=80).cpu().numpy()
        return float(np.dot(xt - y, xt - y))

    h = 1e-6
    fd = (L(T + h) - L(T - h)) / (2 * h)
    assert abs(gt - fd) <= 1e-6 * abs(fd)


@pytest.mark.parametrize("basis,tol", [(1, 1e-4), (3, 1e-9)])
def test_autograd_full_size_96cube(lib, cuda, basis, tol):
    """The adjoint workload at full size (n = 884,736): float32 basis (floor
    ~1e-5) and float-float basis against the Kronecker closed forms."""
    cfg = W.CONFIGS["convdiff3d_96_adjoint"]
    N = 96
    b = cfg["rhs"](N**3)
    y = W.rhs_normal(N**3, W.SEED + 1)
    A, f, gb_ref, gt_ref = _exact(N, b, y, cfg["t"])
    kr = _handle(A, basis, m=cfg["m"], k=cfg["k"], s=cfg["s"], zeta=cfg["zeta"], seed=W.SEED, t=cfg["t"])
    loss, x, gb, gt = _loss_and_grads(kr, b, y, cfg["t"], 1e-11, 40)
    assert _rel(x, f) <= tol
    assert _rel(gb, gb_ref) <= tol
    assert abs(gt - gt_ref) <= tol * abs(gt_ref)


def test_autograd_without_t_gradient(lib, cuda):
    """t given as a float: only grad_b flows."""
    import torch

    from paper_2503_22631_gb300 import krylov_expm

    A = W.convdiff3d(6, BETA)
    kr = _handle(A, 0, m=10, k=2, s=30)
    b = torch.from_numpy(W.rhs_normal(A.n, 4)).cuda().requires_grad_(True)
    x = krylov_expm(b, T, kr, 1e-13, 40)
    x.sum().backward()
    ref = TR.kron_expm_apply(6, 3, BETA, T, np.ones(A.n), transpose=True)
    assert _rel(b.grad.cpu().numpy(), ref) <= 1e-10
