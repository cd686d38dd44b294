"""Rank processes of the row-partitioned solve tests (started with the spawn
method by tests/test_partition.py and tests/test_gpu_partition.py).

Each rank joins a gloo process group on 127.0.0.1, builds its partition plan
from the global matrix and writes what it computed to `outdir` as
rank<r>_*.npy for the parent test to check."""
import os
import sys
from datetime import timedelta

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _init(rank, world, port):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                            timeout=timedelta(seconds=120))
    return dist


def problem(name):
    """The test problems, from the seeded generators."""
    import workloads as W

    if name == "convdiff2d":
        A = W.convdiff(24, 2, (30.0, 10.0))
        return A, W.rhs_normal(A.n, 21), dict(t=2e-3, m=12, k=2, s=40, zeta=8, seed=5, cycles=3)
    if name == "convdiff3d":
        A = W.convdiff3d(12, (50.0, 50.0, 50.0))
        return A, W.rhs_uniform(A.n, 22), dict(t=1e-3, m=16, k=2, s=48, zeta=8, seed=6, cycles=3)
    raise ValueError(name)


def _local_sketch(plan, s, zeta, seed):
    from oracle.sketch import sketch_columns

    rows, signs = sketch_columns(plan.n_global, s, zeta, seed)
    return rows[plan.lo:plan.hi], signs[plan.lo:plan.hi]


def distributed_trunc(plan, comm, b_loc, fkind, t, m, k, s, zeta, seed, cycles):
    """The truncated, whitened restarted method (the oracle's TRUNC mode) on one
    rank's rows, with every n-length sum taken over ranks by the plan's
    collectives: the partition scheme of the row-partitioned solve, in numpy."""
    import torch

    from oracle import dense as D

    def ar(v):
        t_ = torch.from_numpy(np.atleast_1d(np.asarray(v, dtype=np.float64)).copy())
        comm.allreduce(t_, "sum")
        return t_.numpy()

    def halo(w):
        send = torch.from_numpy(np.ascontiguousarray(w[plan.send_idx]))
        recv = torch.empty(plan.n_halo, dtype=torch.float64)
        comm.halo_exchange(send, recv)
        return recv.numpy()

    rows, signs = _local_sketch(plan, s, zeta, seed)
    rp, ci, val = plan.row_ptr, plan.col_idx, plan.val
    rid = np.repeat(np.arange(plan.n_local), np.diff(rp))

    def product(w):
        wext = np.concatenate([w, halo(w)])
        return np.bincount(rid, weights=val * wext[ci], minlength=plan.n_local)

    def sketch(V):
        sc = 1.0 / np.sqrt(zeta)
        out = np.zeros((s, V.shape[1]))
        for j in range(V.shape[1]):
            out[:, j] = np.bincount(rows.ravel(), weights=((signs * sc) * V[:, j][:, None]).ravel(), minlength=s)
        return ar(out.ravel()).reshape(s, V.shape[1])

    n = plan.n_local
    x = np.zeros(n)
    H = np.zeros((0, 0))
    start, coupling, beta = b_loc.copy(), 0.0, None
    for c in range(1, cycles + 1):
        if c == 1:
            eta = np.sqrt(ar(b_loc @ b_loc)[0])
            w1 = b_loc / eta
        else:
            w1 = start
        W = np.zeros((n, m + 1))
        R = np.zeros((m + 1, m))
        W[:, 0] = w1
        for j in range(m):
            p = product(W[:, j])
            win = list(range(max(0, j - k + 1), j + 1))
            sums = ar([W[:, i] @ p for i in win] + [W[:, i] @ W[:, i] for i in win])
            for q, i in enumerate(win):
                R[i, j] = sums[q] / sums[len(win) + q]
            for i in win:
                p = p - R[i, j] * W[:, i]
            R[j + 1, j] = np.sqrt(ar(p @ p)[0])
            W[:, j + 1] = p / R[j + 1, j]
        U = sketch(W)
        Q, T = D.qr_positive(U)
        Tm = T[:m, :m]
        Tm_inv = np.linalg.inv(Tm)
        X = Tm @ R[:m, :m] @ Tm_inv
        tvec, tau, r = T[:m, m], T[m, m], R[m, m - 1]
        X = X + (r / Tm[m - 1, m - 1]) * np.outer(tvec, np.eye(m)[m - 1])
        a = H.shape[0]
        Hn = np.zeros((a + m, a + m))
        Hn[:a, :a] = H
        Hn[a:, a:] = X
        if c == 1:
            beta = eta * T[0, 0]
        else:
            Hn[a, a - 1] = coupling * T[0, 0]
        H = Hn
        g = Tm_inv @ tvec
        start = (W[:, m] - W[:, :m] @ g) / tau
        coupling = r * tau / Tm[m - 1, m - 1]
        F = D.f_dense(fkind, H, t)
        z = beta * (Tm_inv @ F[a:, 0])
        x = x + W[:, :m] @ z
    return x


def run_cpu(rank, world, port, outdir, name):
    """Partition plan, halo exchange and the distributed method on CPU tensors."""
    import torch

    from oracle import dense as D
    from paper_2503_22631_gb300.dist import TorchComm, plan_partition

    _init(rank, world, port)
    A, b, cfg = problem(name)
    plan = plan_partition(A.row_ptr, A.col_idx, A.val, world, rank)
    comm = TorchComm(plan)
    # the halo exchange delivers exactly the global entries the plan lists
    v = np.sin(np.arange(A.n) * 0.37) + 0.01 * np.arange(A.n)
    recv = torch.empty(plan.n_halo, dtype=torch.float64)
    comm.halo_exchange(torch.from_numpy(np.ascontiguousarray(v[plan.lo:plan.hi][plan.send_idx])), recv)
    np.save(os.path.join(outdir, f"rank{rank}_halo.npy"), recv.numpy() - v[plan.halo])
    x = distributed_trunc(plan, comm, b[plan.lo:plan.hi], D.EXP_NEG, cfg["t"], cfg["m"], cfg["k"], cfg["s"],
                          cfg["zeta"], cfg["seed"], cfg["cycles"])
    np.save(os.path.join(outdir, f"rank{rank}_x.npy"), x)
    np.save(os.path.join(outdir, f"rank{rank}_range.npy"), np.array([plan.lo, plan.hi]))
    import torch.distributed as dist

    dist.destroy_process_group()


def run_gpu(rank, world, port, outdir, name):
    """The library's partitioned solve on cuda:0 (every rank on the same GPU;
    gloo carries the collectives through host memory, so no kernel waits on
    another rank's kernel)."""
    import torch

    from paper_2503_22631_gb300 import F_EXP_NEG, build
    from paper_2503_22631_gb300.dist import PartitionedKrylov, TorchComm, plan_partition

    build.build()
    torch.cuda.set_device(0)
    _init(rank, world, port)
    A, b, cfg = problem(name)
    plan = plan_partition(A.row_ptr, A.col_idx, A.val, world, rank)
    comm = TorchComm(plan)
    kr = PartitionedKrylov(plan, comm, f=F_EXP_NEG, t=cfg["t"], m=cfg["m"], k=cfg["k"], s=cfg["s"],
                           seed=cfg["seed"], zeta=cfg["zeta"])
    bl = torch.from_numpy(np.ascontiguousarray(b[plan.lo:plan.hi])).cuda()
    for rep in range(2):  # two calls: the handle's state is reset between calls
        x = kr.apply(bl, tol=0.0, max_cycles=cfg["cycles"])
        torch.cuda.synchronize()
        np.save(os.path.join(outdir, f"rank{rank}_x{rep}.npy"), x.cpu().numpy())
    np.save(os.path.join(outdir, f"rank{rank}_range.npy"), np.array([plan.lo, plan.hi]))
    np.save(os.path.join(outdir, f"rank{rank}_cycles.npy"), np.array([kr.stats["cycles"]]))
    kr.close()
    import torch.distributed as dist

    dist.destroy_process_group()
