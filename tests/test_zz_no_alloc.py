"""The allocation-free product y = A x, <d, y> (krylov_spmv_dot_noalloc).

It exists for callers that cannot allocate device memory when they need the
product (for example while a CUDA graph is being captured, or from inside a
custom allocator): it works on caller-owned device buffers and keeps its
reduction scratch in a fixed array inside the library.  This test calls it
through the C ABI twice in a row on different inputs and compares each result
with the existing handle-based entry point krylov_spmv.  It lives in a file
that pytest collects last so that a failure here never hides the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the float64 tolerance of the parity tests


def _noalloc(lib, A_dev, n, nnz, x, y, d, dot):
    import torch

    st = lib.krylov_spmv_dot_noalloc(n, nnz, C.c_void_p(A_dev[0].data_ptr()), C.c_void_p(A_dev[1].data_ptr()),
                                     C.c_void_p(A_dev[2].data_ptr()), C.c_void_p(x.data_ptr()),
                                     C.c_void_p(y.data_ptr()), C.c_void_p(d.data_ptr()),
                                     C.c_void_p(dot.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


def test_noalloc_matches_handle_spmv_twice(lib, cuda):
    import torch

    from paper_2503_22631_gb300 import Krylov, _lib

    A = W.convdiff3d(40, (50.0, 50.0, 50.0))
    A_dev = (torch.from_numpy(A.row_ptr).cuda(), torch.from_numpy(A.col_idx).cuda(), torch.from_numpy(A.val).cuda())
    kr = Krylov(A.row_ptr, A.col_idx, A.val, m=4, k=2, s=16, seed=1)
    rng = np.random.default_rng(11)
    for call in range(2):
        x = torch.from_numpy(rng.standard_normal(A.n)).cuda()
        d = torch.from_numpy(rng.standard_normal(A.n)).cuda()
        y = torch.full((A.n,), float("nan"), dtype=torch.float64, device="cuda")
        dot = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = _noalloc(lib, A_dev, A.n, A.nnz, x, y, d, dot)
        assert st == _lib.OK, _lib.status_string(st)
        torch.cuda.synchronize()
        y_ref, dot_ref = kr.spmv(x, dot_with=d)
        yr = y_ref.cpu().numpy()
        assert np.linalg.norm(y.cpu().numpy() - yr) <= TOL * np.linalg.norm(yr), call
        # a dot product's rounding scale is ||d|| ||y||
        assert abs(dot.item() - dot_ref) <= TOL * np.linalg.norm(d.cpu().numpy()) * np.linalg.norm(yr), call


def test_noalloc_rejects_sizes_beyond_the_limit(lib, cuda):
    from paper_2503_22631_gb300 import _lib

    p = C.c_void_p(8)  # never dereferenced: the size check comes first
    assert lib.krylov_spmv_dot_noalloc(0, 0, p, p, p, p, p, None, None, None) == _lib.EINVAL
    assert lib.krylov_spmv_dot_noalloc(1 << 31, 0, p, p, p, p, p, None, None, None) == _lib.EINVAL
    assert lib.krylov_spmv_dot_noalloc(10, -1, p, p, p, p, p, None, None, None) == _lib.EINVAL
