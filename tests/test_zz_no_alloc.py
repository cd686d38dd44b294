"""The allocation-free product y = A x, <d, y> (krylov_spmv_dot_noalloc).

It exists for callers that cannot allocate device memory when they need the
product: numerical code called back from inside a custom device allocator or
memory pool (a nested allocation would re-enter it) and real-time loops in
which cudaMalloc may block or synchronize the device.  It works on
caller-owned device buffers and keeps its reduction scratch in a fixed array
inside the library.

The tests call it through the C ABI, two calls in a row on different inputs,
and compare each result with a float64 CSR product formed on the host (scipy)
and with the library's handle-based entry point krylov_spmv.  One operator is
large enough that the grid is capped at 2048 CTAs and the last CTAs get no
rows.  The file is collected last so that a failure here never hides the
other tests.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the float64 tolerance of the parity tests


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _noalloc(lib, A_dev, n, nnz, x, y, d, dot):
    import torch

    return lib.krylov_spmv_dot_noalloc(n, nnz, _ptr(A_dev[0]), _ptr(A_dev[1]), _ptr(A_dev[2]), _ptr(x), _ptr(y),
                                       _ptr(d), _ptr(dot), C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _host_product(rp, ci, val, x, d):
    """y = A x and <d, y> in float64 on the host, with the error scale of each."""
    import scipy.sparse as sp

    n = rp.size - 1
    A = sp.csr_matrix((val, ci, rp), shape=(n, n))
    y = A @ x
    yscale = abs(A) @ np.abs(x)  # |A| |x|: the rounding scale of each entry
    return y, yscale, float(d @ y), float(np.abs(d) @ yscale)


def _banded_random(n, seed):
    """A random CSR with 1..9 entries per row inside a band of +-3000 columns."""
    rng = np.random.default_rng(seed)
    cnt = rng.integers(1, 10, size=n)
    rp = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(cnt, out=rp[1:])
    rows = np.repeat(np.arange(n), cnt)
    ci = np.clip(rows + rng.integers(-3000, 3001, size=rows.size), 0, n - 1).astype(np.int32)
    val = rng.standard_normal(rows.size)
    return rp, ci, val


def _check_two_calls(lib, rp, ci, val, seed, kr=None):
    import torch

    from paper_2503_22631_gb300 import _lib

    n, nnz = rp.size - 1, ci.size
    A_dev = (torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(), torch.from_numpy(val).cuda())
    rng = np.random.default_rng(seed)
    for call in range(2):
        x = rng.standard_normal(n)
        d = rng.standard_normal(n)
        xd, dd = torch.from_numpy(x).cuda(), torch.from_numpy(d).cuda()
        y = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        dot = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = _noalloc(lib, A_dev, n, nnz, xd, y, dd, dot)
        assert st == _lib.OK, _lib.status_string(st)
        torch.cuda.synchronize()
        y_host, yscale, dot_host, dscale = _host_product(rp, ci, val, x, d)
        yg = y.cpu().numpy()
        # every entry within a few roundings of its own |A| |x| scale
        assert np.all(np.abs(yg - y_host) <= 64 * 2.0**-52 * (yscale + 1e-300)), call
        assert np.linalg.norm(yg - y_host) <= TOL * np.linalg.norm(y_host), call
        assert abs(dot.item() - dot_host) <= TOL * dscale, call
        if kr is not None:  # the library's other product agrees as well
            y_ref, dot_ref = kr.spmv(xd, dot_with=dd)
            yr = y_ref.cpu().numpy()
            assert np.linalg.norm(yg - yr) <= TOL * np.linalg.norm(yr), call
            assert abs(dot.item() - dot_ref) <= TOL * dscale, call


def test_noalloc_matches_host_product_twice(lib, cuda):
    from paper_2503_22631_gb300 import Krylov

    A = W.convdiff3d(40, (50.0, 50.0, 50.0))
    kr = Krylov(A.row_ptr, A.col_idx, A.val, m=4, k=2, s=16, seed=1)
    _check_two_calls(lib, A.row_ptr, A.col_idx, A.val, seed=11, kr=kr)


def test_noalloc_capped_grid_with_empty_trailing_ctas(lib, cuda):
    # n = 2048 * 300 + 1: the grid is capped at 2048 CTAs of 301 rows, so the
    # last CTAs start past row n - 1 and contribute nothing but their arrival
    n = 2048 * 300 + 1
    assert (2047 * 301) >= n
    rp, ci, val = _banded_random(n, seed=5)
    _check_two_calls(lib, rp, ci, val, seed=12)


def test_noalloc_without_dot(lib, cuda):
    import torch

    from paper_2503_22631_gb300 import _lib

    A = W.convdiff3d(24, (50.0, 50.0, 50.0))
    A_dev = (torch.from_numpy(A.row_ptr).cuda(), torch.from_numpy(A.col_idx).cuda(), torch.from_numpy(A.val).cuda())
    x = np.random.default_rng(13).standard_normal(A.n)
    y = torch.full((A.n,), float("nan"), dtype=torch.float64, device="cuda")
    st = _noalloc(lib, A_dev, A.n, A.nnz, torch.from_numpy(x).cuda(), y, None, None)
    assert st == _lib.OK, _lib.status_string(st)
    torch.cuda.synchronize()
    y_host, yscale, _, _ = _host_product(A.row_ptr, A.col_idx, A.val, x, np.zeros(A.n))
    assert np.all(np.abs(y.cpu().numpy() - y_host) <= 64 * 2.0**-52 * (yscale + 1e-300))


def test_noalloc_rejects_sizes_beyond_the_limit(lib, cuda):
    from paper_2503_22631_gb300 import _lib

    p = C.c_void_p(8)  # never dereferenced: the size check comes first
    assert lib.krylov_spmv_dot_noalloc(0, 0, p, p, p, p, p, None, None, None) == _lib.EINVAL
    assert lib.krylov_spmv_dot_noalloc(1 << 31, 0, p, p, p, p, p, None, None, None) == _lib.EINVAL
    assert lib.krylov_spmv_dot_noalloc(10, -1, p, p, p, p, p, None, None, None) == _lib.EINVAL
    # a dot pointer without its output (or the reverse) is an argument error
    assert lib.krylov_spmv_dot_noalloc(10, 0, p, p, p, p, p, p, None, None) == _lib.EINVAL
