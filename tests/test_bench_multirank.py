"""Host logic of bench.py for N > 1 ranks, on CPU with the gloo backend.

Every rank solves its own replica (no data-path collective); the timed region
is the slowest rank's, and the whole-job value counts every rank's solves.
"""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, world, rank)
        ms = 100.0 + 25.0 * rank  # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, world, torch.device("cpu"))
        q.put((rank, ms_max, bench.seconds_per_solve(ms_max, 5, world)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_and_count_all_solves():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    out = sorted(q.get(timeout=5) for _ in range(2))
    for rank, ms_max, sps in out:
        assert ms_max == pytest.approx(125.0)
        # 2 ranks x 5 solves in 125 ms
        assert sps == pytest.approx(0.125 / 10)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(42.0, 1, None) == 42.0
    assert bench.seconds_per_solve(42.0, 3, 1) == pytest.approx(0.014)
