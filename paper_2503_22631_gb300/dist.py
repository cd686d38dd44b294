"""Row-partitioned solve: one process per GPU, each owning a contiguous block of rows.

The method shards by rows.  Rank r owns rows [lo_r, hi_r) of A, b and x.
Per Arnoldi step the ranks exchange the halo of the current basis vector (the
entries of other ranks' rows that rank r's rows reference) and sum k + 2
scalars (||A w_j||^2 and the window dots of Algorithm 1's loop body, then
||w_{j+1}||^2); the sketch S w of a basis vector is the sum over ranks of
their rows' sketches, because S's columns are keyed by global row (Sec. 2.1,
Eq. 3 applied columnwise), and is summed once per cycle as exact integer
words.  Every rank solves the small projected problem (whitening, f of the
block matrix, z) from identical inputs; the solution update x += W z is local.

This module holds the host-side bookkeeping of that scheme -- the partition
plan (row blocks, local column numbering, halo and send lists) and the
collective callbacks, built on ``torch.distributed`` -- and passes both to
``krylov_create_partition``; every step of the method runs in the library's
kernels.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import BASIS_F64, F_EXP_NEG, ORTHO_TRUNC


def row_blocks(row_ptr, world: int):
    """Contiguous row blocks with about the same number of nonzeros each:
    block q is [bounds[q], bounds[q + 1])."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    n = rp.size - 1
    if world < 1 or world > n:
        raise ValueError("need 1 <= world <= n")
    targets = rp[-1] * np.arange(1, world) / world
    cuts = np.searchsorted(rp, targets, side="left")
    bounds = np.concatenate([[0], cuts, [n]]).astype(np.int64)
    for q in range(1, world + 1):  # every block keeps at least one row
        bounds[q] = min(max(bounds[q], bounds[q - 1] + 1), n - (world - q))
    return bounds


@dataclass
class PartitionPlan:
    """Rank `rank`'s share of a row partition of an n x n CSR matrix.

    row_ptr, col_idx, val: the rank's rows, columns renumbered so that
    [0, n_local) are its own rows and [n_local, n_local + n_halo) its halo
    columns (global indices `halo`, ascending, i.e. grouped by owner rank).
    recv_counts[q]: halo entries owned by rank q (in that order);
    send_idx: local rows whose entries the other ranks need, grouped by
    destination rank in rank order (send_counts[q] for rank q), ascending
    within a group -- the order in which rank q lists them in its halo."""

    rank: int
    world: int
    n_global: int
    lo: int
    hi: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray
    halo: np.ndarray
    recv_counts: np.ndarray
    send_idx: np.ndarray
    send_counts: np.ndarray

    @property
    def n_local(self) -> int:
        return self.hi - self.lo

    @property
    def n_halo(self) -> int:
        return int(self.halo.size)


def _halo_of(row_ptr, col_idx, lo, hi):
    cols = np.asarray(col_idx[row_ptr[lo]:row_ptr[hi]], dtype=np.int64)
    ext = cols[(cols < lo) | (cols >= hi)]
    return np.unique(ext)


def plan_partition(row_ptr, col_idx, val, world: int, rank: int, bounds=None) -> PartitionPlan:
    """The partition plan of `rank` (every rank computes every rank's halo from
    the global sparsity pattern, so no exchange is needed to build it)."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    ci = np.asarray(col_idx, dtype=np.int64)
    n = rp.size - 1
    if bounds is None:
        bounds = row_blocks(rp, world)
    lo, hi = int(bounds[rank]), int(bounds[rank + 1])
    halo = _halo_of(rp, ci, lo, hi)
    owner = np.searchsorted(bounds, halo, side="right") - 1
    recv_counts = np.bincount(owner, minlength=world).astype(np.int64)
    send_parts, send_counts = [], np.zeros(world, dtype=np.int64)
    for q in range(world):
        if q == rank:
            continue
        hq = _halo_of(rp, ci, int(bounds[q]), int(bounds[q + 1]))
        mine = hq[(hq >= lo) & (hq < hi)] - lo
        send_parts.append(mine)
        send_counts[q] = mine.size
    send_idx = np.concatenate(send_parts) if send_parts else np.zeros(0, dtype=np.int64)
    cols = ci[rp[lo]:rp[hi]]
    own = (cols >= lo) & (cols < hi)
    loc = np.where(own, cols - lo, (hi - lo) + np.searchsorted(halo, cols))
    return PartitionPlan(rank=rank, world=world, n_global=n, lo=lo, hi=hi,
                         row_ptr=(rp[lo:hi + 1] - rp[lo]).astype(np.int32), col_idx=loc.astype(np.int32),
                         val=np.ascontiguousarray(np.asarray(val)[rp[lo]:rp[hi]], dtype=np.float64),
                         halo=halo, recv_counts=recv_counts, send_idx=send_idx.astype(np.int32),
                         send_counts=send_counts)


class _DeviceArray:
    """A device buffer exposed through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr: int, count: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


class TorchComm:
    """The collective operations of a partitioned solve over a torch.distributed
    process group: sums and maxima of small buffers and the halo exchange.

    With NCCL the operations run on the solve's stream on device tensors; with
    gloo (CPU transport) the buffers are staged through host memory.  The
    tensor-level methods work on CPU tensors as well."""

    def __init__(self, plan: PartitionPlan, group=None):
        import torch.distributed as dist

        self.plan = plan
        self.group = group
        self.dist = dist
        self.nccl = dist.get_backend(group) == "nccl"
        self.error = None
        self._keep = []

    # ---- tensor-level operations (CPU or CUDA tensors) ----
    def allreduce(self, t, op: str):
        dist = self.dist
        o = dist.ReduceOp.SUM if op == "sum" else dist.ReduceOp.MAX
        if t.is_cuda and not self.nccl:
            h = t.cpu()
            dist.all_reduce(h, op=o, group=self.group)
            t.copy_(h)
        else:
            dist.all_reduce(t, op=o, group=self.group)

    def halo_exchange(self, send, recv):
        """send: the entries listed by plan.send_idx; recv: the halo entries."""
        dist = self.dist
        p = self.plan
        staged = send.is_cuda and not self.nccl
        s = send.cpu() if staged else send
        r = recv.new_empty(recv.shape, device="cpu") if staged else recv
        soff = np.concatenate([[0], np.cumsum(p.send_counts)])
        roff = np.concatenate([[0], np.cumsum(p.recv_counts)])
        ops = []
        for q in range(p.world):
            if q == p.rank:
                continue
            if p.send_counts[q] > 0:
                ops.append(dist.P2POp(dist.isend, s[int(soff[q]):int(soff[q + 1])], q, group=self.group))
            if p.recv_counts[q] > 0:
                ops.append(dist.P2POp(dist.irecv, r[int(roff[q]):int(roff[q + 1])], q, group=self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        if staged:
            recv.copy_(r)

    # ---- the library's callbacks (device pointers on the solve's stream) ----
    def _run(self, fn, stream):
        import torch

        try:
            ext = torch.cuda.ExternalStream(int(stream)) if stream else torch.cuda.default_stream()
            with torch.cuda.stream(ext):
                if not self.nccl:
                    ext.synchronize()
                fn()
                if not self.nccl:
                    ext.synchronize()
            return 0
        except Exception as e:  # reported by the library as a failed collective
            self.error = e
            return 1

    def _view(self, ptr, count, typestr):
        import torch

        return torch.as_tensor(_DeviceArray(ptr, count, typestr), device="cuda")

    def as_struct(self) -> _lib.Comm:
        def ar_f64(ctx, buf, count, stream):
            return self._run(lambda: self.allreduce(self._view(buf, count, "<f8"), "sum"), stream)

        def ar_i64(ctx, buf, count, stream):
            return self._run(lambda: self.allreduce(self._view(buf, count, "<i8"), "sum"), stream)

        def ar_max(ctx, buf, count, stream):
            return self._run(lambda: self.allreduce(self._view(buf, count, "<f8"), "max"), stream)

        def halo(ctx, send, recv, stream):
            p = self.plan
            return self._run(lambda: self.halo_exchange(self._view(send, p.send_idx.size, "<f8"),
                                                        self._view(recv, p.n_halo, "<f8")), stream)

        cbs = (_lib.ALLREDUCE_F64(ar_f64), _lib.ALLREDUCE_I64(ar_i64), _lib.ALLREDUCE_F64(ar_max),
               _lib.HALO_F64(halo))
        self._keep.append(cbs)  # the library keeps the function pointers
        return _lib.Comm(None, *cbs)


class PartitionedKrylov:
    """This rank's handle of a row-partitioned solve (float64 basis, truncated
    orthogonalization).  apply() is collective: every rank calls it with its
    rows of b and gets its rows of x."""

    def __init__(self, plan: PartitionPlan, comm: TorchComm, *, f=F_EXP_NEG, t=1.0, m=30, k=2, s=None, seed=0,
                 zeta=8, abs_tol=False, stream=None):
        import torch

        lib = _lib.load()
        self.plan, self.comm = plan, comm
        s = 2 * m if s is None else s
        rp, ci, vv = plan.row_ptr, plan.col_idx, plan.val
        csr = _lib.Csr(plan.n_local, ci.size, rp.ctypes.data, ci.ctypes.data, vv.ctypes.data, 0)
        opt = _lib.Options()
        lib.krylov_options_default(C.byref(opt))
        opt.zeta = int(zeta)
        opt.basis_dtype = BASIS_F64
        opt.ortho = ORTHO_TRUNC
        opt.abs_tol = 1 if abs_tol else 0
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        opt.stream = C.c_void_p(int(stream.cuda_stream))
        self._comm_struct = comm.as_struct()
        send = np.ascontiguousarray(plan.send_idx, dtype=np.int32)
        h = C.c_void_p()
        st = lib.krylov_create_partition(C.byref(csr), plan.n_halo, plan.lo, plan.n_global,
                                         C.c_void_p(send.ctypes.data), send.size, C.byref(self._comm_struct),
                                         _lib.Func(int(f), float(t)), int(m), int(k), int(s), C.c_uint64(int(seed)),
                                         C.byref(opt), C.byref(h))
        self._raise(st, "krylov_create_partition")
        self._h = h
        self.stats = None

    def _raise(self, st, where, ok=(_lib.OK,)):
        if st not in ok and self.comm.error is not None:
            raise RuntimeError(f"{where}: collective failed") from self.comm.error
        _lib.check(st, where, ok=ok)

    def apply(self, b_local, tol=0.0, max_cycles=1, out=None):
        import torch

        if not (isinstance(b_local, torch.Tensor) and b_local.is_cuda and b_local.dtype == torch.float64
                and b_local.numel() == self.plan.n_local):
            raise ValueError(f"expected a float64 CUDA tensor with {self.plan.n_local} entries")
        b_local = b_local.contiguous()
        x = torch.empty_like(b_local) if out is None else out
        stats = _lib.Stats()
        st = _lib.load().krylov_apply(self._h, C.c_void_p(b_local.data_ptr()), C.c_void_p(x.data_ptr()),
                                      float(tol), int(max_cycles), C.byref(stats))
        self._raise(st, "krylov_apply", ok=(_lib.OK, _lib.NOT_CONVERGED, _lib.BREAKDOWN_EXACT))
        self.stats = stats.as_dict()
        self.status = st
        return x

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().krylov_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
