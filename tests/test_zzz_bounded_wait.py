"""Failure detection without a fault: the bounded device wait gives up and says so.

The staged kernels wait for their bulk copies with a bounded mbarrier wait;
when a wait gives up, the kernel sets a timeout flag, drains its own copies
and returns, and the call reports KRYLOV_ETIMEOUT instead of hanging.  The
library's probe runs that same wait on a barrier phase that completes and on
one that never does (transaction bytes announced, no copy issued: a flag that
nothing sets).  This test checks the two outcomes, the duration of the
failing wait against its bound, and that the device still computes correct
results afterwards.  It lives in a file that pytest collects last so that a
failure here never hides the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from oracle import dense as D
from oracle import krylov as K

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_device_stays_usable(lib, cuda):
    import torch

    from paper_2503_22631_gb300 import Krylov

    limit_ns = 2_000_000  # 2 ms
    timed_out = (C.c_int * 2)()
    wait_ns = (C.c_double * 2)()
    st = lib.krylov_probe_bounded_wait(limit_ns, C.cast(timed_out, C.c_void_p), C.cast(wait_ns, C.c_void_p))
    assert st == 0
    assert list(timed_out) == [0, 1]
    assert wait_ns[0] < limit_ns
    assert limit_ns <= wait_ns[1] < 1e9

    # the context is intact: a solve right after matches the oracle (the
    # configuration of the float64 parity test on the 2D Laplacian)
    A = W.poisson2d(64)
    b = W.rhs_normal(A.n, W.SEED, normalize=True)
    args = (D.EXP_NEG, 1e-3, 30, 2, 60, 8, 99)
    ref = K.restarted(A, b, *args, mode=K.TRUNC, tol=0.0, max_cycles=2)
    kr = Krylov(A.row_ptr, A.col_idx, A.val, f=args[0], t=args[1], m=args[2], k=args[3], s=args[4],
                zeta=args[5], seed=args[6])
    x = kr.apply(torch.from_numpy(b).cuda(), tol=0.0, max_cycles=2).cpu().numpy()
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-10
