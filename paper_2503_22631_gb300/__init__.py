"""GB300-native randomized restarted Krylov method for f(A) b.

Python face of ``libkrylov.so`` (C ABI in ``include/krylov.h``).  The classes
below marshal arguments only; every step of the method runs in the library's
CUDA kernels for sm_103a.  PyTorch supplies device memory and streams.

    from paper_2503_22631_gb300 import Krylov, F_EXP_NEG
    K = Krylov(row_ptr, col_idx, val, f=F_EXP_NEG, t=1e-2, m=40, k=2, s=160, seed=1)
    x = K.apply(b)           # b: float64 CUDA tensor, x ~ exp(-t A) b
    x = krylov_expm(b, t, K) # differentiable in b and t (autograd)
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (BASIS_BF16, BASIS_DF64, BASIS_F32, BASIS_F64, BREAKDOWN_EXACT, F_COS_SQRT, F_EXP_NEG, F_INV, F_INVSQRT, F_PHI1_NEG,
                   NOT_CONVERGED, OK, ORTHO_RGS, ORTHO_TRUNC, KrylovError, status_string)

__all__ = ["Krylov", "KrylovExpm", "krylov_expm", "apply_batched", "sketch_columns", "KrylovError", "status_string", "F_COS_SQRT", "F_EXP_NEG", "F_INV", "F_INVSQRT", "F_PHI1_NEG",
           "BASIS_F64", "BASIS_F32", "BASIS_BF16", "BASIS_DF64", "ORTHO_TRUNC", "ORTHO_RGS", "OK", "NOT_CONVERGED",
           "BREAKDOWN_EXACT"]

_SUCCESS = (OK, NOT_CONVERGED, BREAKDOWN_EXACT)


def _torch():
    import torch

    return torch


def _as_int32_host(a):
    a = np.ascontiguousarray(np.asarray(a), dtype=np.int32)
    return a


class Krylov:
    """A handle: matrix A (CSR), f, restart length m, window k, sketch (s, zeta, seed)."""

    def __init__(self, row_ptr, col_idx, val, *, f=F_EXP_NEG, t=1.0, m=30, k=2, s=None, seed=0, zeta=8,
                 basis=BASIS_F64, narrow_values_if_exact=True, abs_tol=False, sketch_regenerate=False,
                 ortho=ORTHO_TRUNC, use_graph=True, autotune=True, block_rhs=True, stream=None):
        lib = _lib.load()
        torch = _torch()
        self._keep = []
        on_device = isinstance(row_ptr, torch.Tensor) and row_ptr.is_cuda
        if on_device:
            rp = row_ptr.to(torch.int32).contiguous()
            ci = col_idx.to(torch.int32).contiguous()
            vv = val.to(torch.float64).contiguous()
            self._keep += [rp, ci, vv]
            ptrs = (rp.data_ptr(), ci.data_ptr(), vv.data_ptr())
            n = rp.numel() - 1
            nnz = ci.numel()
        else:
            rp = _as_int32_host(row_ptr)
            ci = _as_int32_host(col_idx)
            vv = np.ascontiguousarray(np.asarray(val), dtype=np.float64)
            self._keep += [rp, ci, vv]
            ptrs = (rp.ctypes.data, ci.ctypes.data, vv.ctypes.data)
            n = rp.size - 1
            nnz = ci.size
        s = 2 * m if s is None else s
        csr = _lib.Csr(n, nnz, ptrs[0], ptrs[1], ptrs[2], 1 if on_device else 0)
        opt = _lib.Options()
        lib.krylov_options_default(C.byref(opt))
        opt.zeta = int(zeta)
        opt.basis_dtype = int(basis)
        opt.narrow_values_if_exact = 1 if narrow_values_if_exact else 0
        opt.abs_tol = 1 if abs_tol else 0
        opt.sketch_regenerate = 1 if sketch_regenerate else 0
        opt.ortho = int(ortho)
        opt.use_graph = 1 if use_graph else 0
        opt.autotune = 2 if autotune == "gather" else (1 if autotune else 0)
        opt.block_rhs = 1 if block_rhs else 0
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        opt.stream = C.c_void_p(int(stream.cuda_stream))
        h = C.c_void_p()
        st = lib.krylov_create(C.byref(csr), _lib.Func(int(f), float(t)), int(m), int(k), int(s),
                               C.c_uint64(int(seed)), C.byref(opt), C.byref(h))
        _lib.check(st, "krylov_create")
        self._h = h
        self.n, self.nnz, self.m, self.k, self.s, self.zeta = n, nnz, m, k, s, zeta
        self.f, self.t, self.basis, self.seed, self.ortho = f, t, basis, seed, ortho
        self.stats = None
        self._keep = []  # the library copied the matrix

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().krylov_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _vec(self, b):
        torch = _torch()
        if not (isinstance(b, torch.Tensor) and b.is_cuda and b.dtype == torch.float64 and b.numel() == self.n):
            raise ValueError(f"expected a float64 CUDA tensor with {self.n} entries")
        return b.contiguous()

    def apply(self, b, tol=0.0, max_cycles=1, out=None, adjoint=False):
        """x ~ f(A) b (or f(A)^T b); returns x (float64 CUDA tensor)."""
        torch = _torch()
        b = self._vec(b)
        x = torch.empty_like(b) if out is None else out
        stats = _lib.Stats()
        fn = _lib.load().krylov_apply_adjoint if adjoint else _lib.load().krylov_apply
        st = fn(self._h, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), float(tol), int(max_cycles),
                C.byref(stats))
        _lib.check(st, "krylov_apply_adjoint" if adjoint else "krylov_apply", ok=_SUCCESS)
        self.stats = stats.as_dict()
        self.status = st
        return x

    def apply_host(self, b, tol=0.0, max_cycles=1, out=None):
        """Same as apply with numpy (host) input and output; copies are part of the call."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        if b.size != self.n:
            raise ValueError("wrong size")
        x = np.empty_like(b) if out is None else out
        stats = _lib.Stats()
        st = _lib.load().krylov_apply_host(self._h, C.c_void_p(b.ctypes.data), C.c_void_p(x.ctypes.data),
                                           float(tol), int(max_cycles), C.byref(stats))
        _lib.check(st, "krylov_apply_host", ok=_SUCCESS)
        self.stats = stats.as_dict()
        self.status = st
        return x

    def set_param(self, t):
        _lib.check(_lib.load().krylov_set_param(self._h, float(t)), "krylov_set_param")
        self.t = t

    def spmv(self, x, transpose=False, dot_with=None):
        """y = A x (or A^T x); with dot_with also returns <dot_with, y>."""
        torch = _torch()
        x = self._vec(x)
        y = torch.empty_like(x)
        d = C.c_double(0.0)
        dw = C.c_void_p(self._vec(dot_with).data_ptr()) if dot_with is not None else None
        _lib.check(_lib.load().krylov_spmv(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                           1 if transpose else 0, dw, C.byref(d) if dot_with is not None else None),
                   "krylov_spmv")
        return (y, d.value) if dot_with is not None else y

    def last_cycle(self):
        """(T, X, z, m_eff) of the last cycle as numpy arrays (column-major data)."""
        m = self.m
        T = np.zeros((m + 1) * (m + 1))
        X = np.zeros(m * m)
        z = np.zeros(m)
        me = C.c_int(0)
        _lib.check(_lib.load().krylov_last_cycle(self._h, C.c_void_p(T.ctypes.data), T.size,
                                                 C.c_void_p(X.ctypes.data), X.size, C.c_void_p(z.ctypes.data),
                                                 z.size, C.byref(me)), "krylov_last_cycle")
        me = me.value
        nc = me + (0 if self.stats and self.stats["breakdown"] else 1)
        return (T[: nc * nc].reshape(nc, nc, order="F"), X[: me * me].reshape(me, me, order="F"), z[:me], me)


def apply_batched(handles, B, t=None, tol=0.0, max_cycles=1, raise_on_error=True):
    """Batched form: X[i][:, r] ~ f(A_i) B[i][:, r] for every handle i and column r.

    handles : distinct ``Krylov`` handles (one matrix each);
    B       : float64 CUDA tensors, B[i] of shape (n_i, n_rhs), row-major contiguous;
    t       : None or one t per handle (f(z) = exp(-t z));
    returns (X, stats): X[i] like B[i]; stats[i][r] the per-right-hand-side stats
    (with their own "status").  raise_on_error=False returns even when some
    right-hand side failed (its column of X is then unspecified).
    """
    torch = _torch()
    n_inst = len(handles)
    if n_inst == 0 or len(B) != n_inst:
        raise ValueError("one right-hand-side block per handle")
    n_rhs = B[0].shape[1]
    Bs, Xs = [], []
    for h, b in zip(handles, B):
        if not (isinstance(b, torch.Tensor) and b.is_cuda and b.dtype == torch.float64 and b.dim() == 2
                and b.shape[0] == h.n and b.shape[1] == n_rhs):
            raise ValueError("B[i] must be a float64 CUDA tensor of shape (n_i, n_rhs)")
        b = b.contiguous()
        Bs.append(b)
        Xs.append(torch.empty_like(b))
    hp = (C.c_void_p * n_inst)(*[h._h.value for h in handles])
    bp = (C.c_void_p * n_inst)(*[b.data_ptr() for b in Bs])
    xp = (C.c_void_p * n_inst)(*[x.data_ptr() for x in Xs])
    tp = None if t is None else (C.c_double * n_inst)(*[float(v) for v in t])
    stats = (_lib.Stats * (n_inst * n_rhs))()
    st = _lib.load().krylov_apply_batched(hp, n_inst, n_rhs, bp, xp, tp, float(tol), int(max_cycles), stats)
    if raise_on_error or st == _lib.EINVAL:
        _lib.check(st, "krylov_apply_batched", ok=_SUCCESS)
    out_stats = [[stats[i * n_rhs + r].as_dict() for r in range(n_rhs)] for i in range(n_inst)]
    return Xs, out_stats


def sketch_columns(n, s, zeta, seed, col0=0, count=None):
    """Rows (int32, count x zeta) and signs (int8) of sketch columns generated on the GPU."""
    count = n - col0 if count is None else count
    rows = np.zeros((count, zeta), dtype=np.int32)
    signs = np.zeros((count, zeta), dtype=np.int8)
    st = _lib.load().krylov_sketch_columns(int(n), int(s), int(zeta), C.c_uint64(int(seed)), int(col0), int(count),
                                           C.c_void_p(rows.ctypes.data), C.c_void_p(signs.ctypes.data))
    _lib.check(st, "krylov_sketch_columns")
    return rows, signs


from .autograd import KrylovExpm, krylov_expm  # noqa: E402  (needs the names above)
