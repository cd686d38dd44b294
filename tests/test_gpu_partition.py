"""Row-partitioned solve through the library (krylov_create_partition).

One, two and three ranks, each a process on cuda:0 with a gloo process group
(the collectives pass through host memory, so no rank's kernel waits on
another's).  The ranks' rows of x, put together, must match the single-process
oracle within the float64 tolerance, and two calls in a row must agree
exactly (the handle's cycle state is reset between calls).
"""
import numpy as np
import pytest

from oracle import dense as D
from oracle import krylov as K

pytestmark = pytest.mark.gpu

TOL = 1e-10  # float64 basis


@pytest.mark.parametrize("world,name", [(1, "convdiff2d"), (2, "convdiff2d"), (2, "convdiff3d"), (3, "convdiff3d")])
def test_partitioned_solve_matches_oracle(lib, cuda, tmp_path, world, name):
    import partition_worker as PW
    from test_partition import _spawn

    _spawn(PW.run_gpu, world, str(tmp_path), name, timeout=600)
    A, b, cfg = PW.problem(name)
    ref = K.restarted(A, b, D.EXP_NEG, cfg["t"], cfg["m"], cfg["k"], cfg["s"], cfg["zeta"], cfg["seed"],
                      mode=K.TRUNC, tol=0.0, max_cycles=cfg["cycles"])
    xs = [np.zeros(A.n), np.zeros(A.n)]
    for r in range(world):
        lo, hi = np.load(tmp_path / f"rank{r}_range.npy")
        assert int(np.load(tmp_path / f"rank{r}_cycles.npy")[0]) == cfg["cycles"]
        for rep in range(2):
            xs[rep][lo:hi] = np.load(tmp_path / f"rank{r}_x{rep}.npy")
    err = np.linalg.norm(xs[0] - ref.x) / np.linalg.norm(ref.x)
    print(f"{name}, {world} rank(s): relative error vs oracle {err:.2e}")
    assert err <= TOL
    np.testing.assert_array_equal(xs[0], xs[1])
