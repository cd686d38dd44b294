"""Degenerate inputs through the C ABI: a zero right-hand side, non-finite
right-hand sides, and invalid CSR structure at create.

* b = 0: f(A) 0 = 0; the call returns KRYLOV_OK after no cycle, x = 0 exactly.
* NaN or Inf in b: ||b|| is not finite, the call returns KRYLOV_ENONFINITE
  before the first cycle; the handle stays usable.
* Invalid CSR (a decreasing row_ptr, row_ptr[n] != nnz, a column index
  outside [0, n)): krylov_create copies the arrays and checks them on the
  device before anything else reads them, and returns KRYLOV_EINVAL.

After each failure a solve on the same device still matches the oracle.  The
file is collected last so that a failure here never hides the other tests.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dense as D
from oracle import krylov as K

pytestmark = pytest.mark.gpu

ARGS = (D.EXP_NEG, 1e-3, 30, 2, 60, 8, 99)  # f, t, m, k, s, zeta, seed (the 2D Laplacian parity case)


def _handle(A, basis=0):
    from paper_2503_22631_gb300 import Krylov

    f, t, m, k, s, zeta, seed = ARGS
    return Krylov(A.row_ptr, A.col_idx, A.val, f=f, t=t, m=m, k=k, s=s, zeta=zeta, seed=seed, basis=basis)


def _still_matches_oracle(kr, A):
    import torch

    b = W.rhs_normal(A.n, W.SEED, normalize=True)
    ref = K.restarted(A, b, *ARGS, mode=K.TRUNC, tol=0.0, max_cycles=2)
    x = kr.apply(torch.from_numpy(b).cuda(), tol=0.0, max_cycles=2).cpu().numpy()
    return np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)


@pytest.mark.parametrize("basis", [0, 3])
def test_zero_rhs_gives_zero_without_a_cycle(lib, cuda, basis):
    import torch

    A = W.poisson2d(64)
    kr = _handle(A, basis)
    out = torch.full((A.n,), 7.0, dtype=torch.float64, device="cuda")
    x = kr.apply(torch.zeros(A.n, dtype=torch.float64, device="cuda"), tol=1e-8, max_cycles=5, out=out)
    assert kr.status == 0 and kr.stats["cycles"] == 0
    assert torch.count_nonzero(x).item() == 0
    assert _still_matches_oracle(kr, A) <= 1e-10


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
def test_non_finite_rhs_is_reported(lib, cuda, bad):
    import torch

    from paper_2503_22631_gb300 import _lib

    A = W.poisson2d(64)
    kr = _handle(A)
    b = torch.from_numpy(W.rhs_normal(A.n, 3)).cuda()
    b[A.n // 3] = bad
    with pytest.raises(_lib.KrylovError) as e:
        kr.apply(b, tol=0.0, max_cycles=2)
    assert e.value.status == -4  # KRYLOV_ENONFINITE
    assert _still_matches_oracle(kr, A) <= 1e-10


def test_invalid_csr_is_rejected_at_create(lib, cuda):
    from paper_2503_22631_gb300 import Krylov, _lib

    A = W.poisson2d(64)
    f, t, m, k, s, zeta, seed = ARGS
    cases = []
    rp = A.row_ptr.copy()
    rp[10], rp[11] = rp[11], rp[10]  # decreasing row_ptr (same nnz)
    cases.append((rp, A.col_idx, A.val))
    rp = A.row_ptr.copy()
    rp[-1] -= 1  # row_ptr[n] != nnz
    cases.append((rp, A.col_idx, A.val))
    ci = A.col_idx.copy()
    ci[len(ci) // 2] = A.n  # column index out of range
    cases.append((A.row_ptr, ci, A.val))
    ci = A.col_idx.copy()
    ci[5] = -1
    cases.append((A.row_ptr, ci, A.val))
    for rp, ci, val in cases:
        with pytest.raises(_lib.KrylovError) as e:
            Krylov(rp, ci, val, f=f, t=t, m=m, k=k, s=s, zeta=zeta, seed=seed)
        assert e.value.status == -1  # KRYLOV_EINVAL
    assert _still_matches_oracle(_handle(A), A) <= 1e-10
