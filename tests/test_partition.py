"""Row-partitioned solve on CPU: the partition plan, the halo exchange and the
reduction scheme, against the single-process oracle.

The plan (paper_2503_22631_gb300.dist) splits the rows into contiguous blocks,
renumbers each block's columns (own rows first, then the halo) and lists what
every rank sends to every other.  Two gloo ranks then exchange halos and run
the truncated, whitened restarted method with every n-length sum taken over
ranks (tests/partition_worker.py); their rows of x must equal the oracle's
single-process result.
"""
import multiprocessing as mp
import socket

import numpy as np
import pytest

import workloads as W
from oracle import dense as D
from oracle import krylov as K
from paper_2503_22631_gb300.dist import plan_partition, row_blocks


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _spawn(target, world, *args, timeout=300):
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port) + args) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout)
    for p in procs:
        if p.is_alive():
            p.kill()
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_plan_reproduces_the_global_product(world):
    """Each rank's rows of A x from its local CSR and the halo entries equal
    the rows of the global product; send lists match the receivers' halos."""
    A = W.convdiff3d(10, (50.0, 50.0, 50.0))
    x = np.random.default_rng(1).standard_normal(A.n)
    y = K.csr_matvec(A, x)
    bounds = row_blocks(A.row_ptr, world)
    assert bounds[0] == 0 and bounds[-1] == A.n and np.all(np.diff(bounds) >= 1)
    plans = [plan_partition(A.row_ptr, A.col_idx, A.val, world, r, bounds) for r in range(world)]
    for p in plans:
        rid = np.repeat(np.arange(p.n_local), np.diff(p.row_ptr))
        wext = np.concatenate([x[p.lo:p.hi], x[p.halo]])
        assert p.col_idx.max(initial=0) < p.n_local + p.n_halo
        yl = np.bincount(rid, weights=p.val * wext[p.col_idx], minlength=p.n_local)
        np.testing.assert_array_equal(yl, y[p.lo:p.hi])  # same products, same order
        assert np.all(np.diff(p.halo) > 0) and not np.any((p.halo >= p.lo) & (p.halo < p.hi))
        assert p.recv_counts.sum() == p.n_halo and p.recv_counts[p.rank] == 0
    for r, pr in enumerate(plans):  # what r sends to q is q's halo segment owned by r
        soff = np.concatenate([[0], np.cumsum(pr.send_counts)])
        for q, pq in enumerate(plans):
            if q == r:
                continue
            roff = np.concatenate([[0], np.cumsum(pq.recv_counts)])
            sent = pr.lo + pr.send_idx[soff[q]:soff[q + 1]]
            np.testing.assert_array_equal(sent, pq.halo[roff[r]:roff[r + 1]])


def test_row_blocks_balance_nonzeros():
    A = W.poisson2d(40)
    b = row_blocks(A.row_ptr, 4)
    nnz = np.diff(A.row_ptr[b])
    assert nnz.max() - nnz.min() <= 2 * np.diff(A.row_ptr).max()
    with pytest.raises(ValueError):
        row_blocks(A.row_ptr, A.n + 1)


@pytest.mark.parametrize("name", ["convdiff2d", "convdiff3d"])
def test_two_gloo_ranks_match_the_oracle(tmp_path, name):
    import partition_worker as PW

    _spawn(PW.run_cpu, 2, str(tmp_path), name)
    A, b, cfg = PW.problem(name)
    ref = K.restarted(A, b, D.EXP_NEG, cfg["t"], cfg["m"], cfg["k"], cfg["s"], cfg["zeta"], cfg["seed"],
                      mode=K.TRUNC, tol=0.0, max_cycles=cfg["cycles"])
    x = np.zeros(A.n)
    for r in range(2):
        assert np.all(np.load(tmp_path / f"rank{r}_halo.npy") == 0.0)
        lo, hi = np.load(tmp_path / f"rank{r}_range.npy")
        x[lo:hi] = np.load(tmp_path / f"rank{r}_x.npy")
    assert np.linalg.norm(x - ref.x) <= 1e-12 * np.linalg.norm(ref.x)
