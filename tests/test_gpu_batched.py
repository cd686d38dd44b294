"""Batched form: many matrices of uneven size, many right-hand sides each.

* small batch: every sampled (instance, right-hand side) matches the oracle at
  the basis tolerance, per-instance t is honoured and restored, and the batched
  call equals one krylov_apply per right-hand side;
* the batched workload at full size (16 instances, n log-uniform in [1e4, 1e6],
  64 right-hand sides each, float32 basis, m = 30, k = 2, s = 120): the oracle on
  4 sampled right-hand sides per instance (one cycle, run in a spawned process
  pool), and the float-float basis against the Kronecker closed form to 1e-8.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import workloads as W
from oracle import dense as D
from oracle import krylov as K
from oracle import truth as TR

pytestmark = pytest.mark.gpu

M, KW, S, ZETA = 30, 2, 120, 8


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _rhs_block(n, n_rhs, seed):
    return W.rhs_normal(n * n_rhs, seed).reshape(n, n_rhs)


def _oracle_one(args):
    _, inst, col, seed, cycles = args
    A = W.batched_matrix(inst)
    b = _rhs_block(inst["n"], inst["n_rhs"], seed)[:, col].copy()
    r = K.restarted(A, b, D.EXP_NEG, inst["t"], M, KW, S, ZETA, W.SEED, mode=K.TRUNC, tol=0.0, max_cycles=cycles)
    return r.x


def _oracle_many(jobs):
    procs = max(1, min(len(jobs), os.cpu_count() or 1, 16))
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_oracle_one, jobs)


def _handles(insts, basis, block_rhs=True):
    from paper_2503_22631_gb300 import F_EXP_NEG, Krylov

    hs = []
    for inst in insts:
        A = W.batched_matrix(inst)
        hs.append(Krylov(A.row_ptr, A.col_idx, A.val, f=F_EXP_NEG, t=1.0, m=M, k=KW, s=S, seed=W.SEED, zeta=ZETA,
                         basis=basis, block_rhs=block_rhs))
    return hs


def _run(insts, n_rhs, basis, tol, cycles, raise_on_error=True, block_rhs=True):
    import torch

    from paper_2503_22631_gb300 import apply_batched

    hs = _handles(insts, basis, block_rhs)
    B = [torch.from_numpy(_rhs_block(inst["n"], n_rhs, 100 + i)).cuda() for i, inst in enumerate(insts)]
    X, st = apply_batched(hs, B, t=[inst["t"] for inst in insts], tol=tol, max_cycles=cycles,
                          raise_on_error=raise_on_error)
    torch.cuda.synchronize()
    return hs, B, [x.cpu().numpy() for x in X], st


SMALL = [dict(i, n_rhs=8) for i in W.batched_instances(4, 77, n_lo=1e3, n_hi=2e4)]


@pytest.mark.parametrize("basis,tol", [(0, 1e-10), (1, 1e-5), (3, 1e-10)])
def test_small_batch_matches_oracle(lib, cuda, basis, tol):
    """float64 runs one by one; float32 and float-float through the block
    kernels (8 right-hand sides of a matrix advanced together)."""
    hs, B, X, st = _run(SMALL, 8, basis, 0.0, 2)
    jobs = [(i, inst, col, 100 + i, 2) for i, inst in enumerate(SMALL) for col in (0, 3, 5, 7)]
    refs = _oracle_many(jobs)
    for (i, inst, col, seed, _), ref in zip(jobs, refs):
        assert _rel(X[i][:, col], ref) <= tol
        assert st[i][col]["cycles"] == 2 and st[i][col]["status"] == 1  # tol = 0: runs the fixed count


def test_batched_equals_single_applies(lib, cuda):
    """Same kernels, same inputs: with the block kernels switched off the
    batched call gives each right-hand side's single-call result (and the
    handle's t is back to its value afterwards)."""
    hs, B, X, st = _run(SMALL, 8, 1, 1e-6, 10, block_rhs=False)
    for i, (h, inst) in enumerate(zip(hs, SMALL)):
        h.set_param(inst["t"])
        for col in range(8):
            x = h.apply(B[i][:, col].contiguous(), tol=1e-6, max_cycles=10).cpu().numpy()
            assert _rel(X[i][:, col], x) <= 1e-14
            assert st[i][col]["cycles"] == h.stats["cycles"]


def test_float32_block_form_matches_one_by_one(lib, cuda):
    """The float32 block kernels (float-float arithmetic on float32 storage)
    against the float32 single-vector kernels: both are float32 methods, so
    they agree to the float32 tolerance, not bitwise."""
    _, _, Xb, stb = _run(SMALL, 8, 1, 0.0, 3)
    _, _, X1, st1 = _run(SMALL, 8, 1, 0.0, 3, block_rhs=False)
    for i in range(len(SMALL)):
        for col in range(8):
            assert _rel(Xb[i][:, col], X1[i][:, col]) <= 2e-5
            assert stb[i][col]["cycles"] == st1[i][col]["cycles"] == 3


def test_batched_rejects_repeated_handles(lib, cuda):
    import torch

    from paper_2503_22631_gb300 import KrylovError, apply_batched

    hs = _handles(SMALL[:1], 1)
    B = [torch.zeros(SMALL[0]["n"], 2, dtype=torch.float64, device="cuda")] * 2
    with pytest.raises(KrylovError):
        apply_batched([hs[0], hs[0]], B)


FULL = [dict(i, n_rhs=64) for i in W.batched_instances(16, W.SEED)]


def _stiffness(inst):
    """t * ||A||_inf, the scale of t A's spectrum."""
    A = W.batched_matrix(inst)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    return inst["t"] * np.bincount(rows, weights=np.abs(A.val), minlength=A.n).max()


@pytest.mark.slow
def test_full_batch_float32_matches_oracle(lib, cuda):
    """One cycle, 4 sampled right-hand sides per instance.  Tolerance
    max(1e-5, u32 t ||A||_inf): rounding the stored basis to float32 moves the
    Ritz values by about u32 ||A||, and exp(-t z) turns a shift d of z into a
    relative change t d, so for stiff instances (t ||A|| up to 8e4 here) the
    float32 result is only that accurate; the float64 basis meets 1e-10."""
    hs, B, X, st = _run(FULL, 64, 1, 0.0, 1)
    jobs = [(i, inst, col, 100 + i, 1) for i, inst in enumerate(FULL) for col in (0, 21, 42, 63)]
    refs = _oracle_many(jobs)
    for (i, inst, col, seed, _), ref in zip(jobs, refs):
        tol = max(1e-5, 2.0**-24 * _stiffness(inst))
        assert _rel(X[i][:, col], ref) <= tol


@pytest.mark.slow
def test_full_batch_float_float_reaches_1e8(lib, cuda):
    """Float-float basis, relative stop 1e-12, at most 60 cycles: every
    right-hand side of every instance with t ||A||_inf <= 4e4 is within
    1e-8 ||f(A) b|| + u t ||A||_inf ||b|| of the Kronecker closed form, u = 2^-48
    the unit roundoff of the float-float basis.  The second term is the
    attainable floor: a product A w formed with the basis rounded to u is the
    exact product of a matrix A + E with ||E|| <= u ||A||, and the Frechet
    derivative of exp(-tA) (a contraction for these M-matrices) maps E to at
    most t ||E|| ||b|| in the solution.  It matters where f(A) b is small next
    to b: the 3D instances whose f(A) b is 1e-18..1e-45 of ||b|| (strong
    convection with large t), where a relative error has no meaning, and the
    stiff 2D instance (t ||A||_inf = 3.5e4, ||b|| / ||f(A) b|| = 2.8e3) whose
    error stagnates at 1.2e-8 relative (2.9e-9 with the float64 basis, whose
    floor is u = 2^-53 in the same bound).  The one instance beyond the
    stiffness bound (2D, t ||A||_inf ~ 8e4) needs far more than 60 restarts
    of length 30 and is only required to return a status."""
    hs, B, X, st = _run(FULL, 64, 3, 1e-12, 60, raise_on_error=False)
    for i, inst in enumerate(FULL):
        dim = 2 if inst["kind"] == "2d" else 3
        stiff = _stiffness(inst)
        for col in (0, 21, 42, 63):
            status = st[i][col]["status"]
            if stiff > 4e4:
                assert status in (0, 1, 2, -4)
                continue
            assert status in (0, 1, 2)
            b = B[i][:, col].cpu().numpy()
            ref = TR.kron_expm_apply(inst["N"], dim, inst["beta"], inst["t"], b)
            err = np.linalg.norm(X[i][:, col] - ref)
            assert err <= 1e-8 * np.linalg.norm(ref) + 2.0**-48 * stiff * np.linalg.norm(b)


def _run_df64(insts, n_rhs, tol, cycles, block_rhs):
    import torch

    from paper_2503_22631_gb300 import BASIS_DF64, F_EXP_NEG, Krylov, apply_batched

    hs = []
    for inst in insts:
        A = W.batched_matrix(inst)
        hs.append(Krylov(A.row_ptr, A.col_idx, A.val, f=F_EXP_NEG, t=1.0, m=M, k=KW, s=S, seed=W.SEED, zeta=ZETA,
                         basis=BASIS_DF64, block_rhs=block_rhs))
    B = [torch.from_numpy(_rhs_block(inst["n"], n_rhs, 100 + i)).cuda() for i, inst in enumerate(insts)]
    X, st = apply_batched(hs, B, t=[inst["t"] for inst in insts], tol=tol, max_cycles=cycles)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in X], st


@pytest.mark.parametrize("n_rhs", [8, 40, 70])
def test_block_kernels_match_one_by_one(lib, cuda, n_rhs):
    """Float-float basis: the block kernels (right-hand sides advanced together,
    chunks of at most 64) agree with the single-vector kernels to rounding."""
    insts = SMALL[:2]
    Xb, stb = _run_df64(insts, n_rhs, 0.0, 3, True)
    Xs, sts = _run_df64(insts, n_rhs, 0.0, 3, False)
    for i in range(len(insts)):
        for col in range(n_rhs):
            assert _rel(Xb[i][:, col], Xs[i][:, col]) <= 1e-12
            assert stb[i][col]["cycles"] == sts[i][col]["cycles"] == 3


def test_block_kernels_match_oracle_and_stop_rule(lib, cuda):
    insts = SMALL[2:4]
    Xb, stb = _run_df64(insts, 16, 0.0, 2, True)
    jobs = [(i, dict(inst, n_rhs=16), col, 100 + i, 2) for i, inst in enumerate(insts) for col in (0, 7, 15)]
    refs = _oracle_many(jobs)
    for (i, inst, col, seed, _), ref in zip(jobs, refs):
        assert _rel(Xb[i][:, col], ref) <= 1e-10
    # relative stop: every right-hand side stops at its own cycle, as one by one
    Xb, stb = _run_df64(insts, 12, 1e-9, 16, True)
    Xs, sts = _run_df64(insts, 12, 1e-9, 16, False)
    for i in range(len(insts)):
        for col in range(12):
            assert stb[i][col]["cycles"] == sts[i][col]["cycles"]
            assert _rel(Xb[i][:, col], Xs[i][:, col]) <= 1e-10


def test_block_kernels_redo_breakdown_alone(lib, cuda):
    """A right-hand side that is an eigenvector breaks down in the first step:
    the block form hands it to the single-vector kernels (exact result)."""
    import torch

    from paper_2503_22631_gb300 import BASIS_DF64, F_EXP_NEG, Krylov, apply_batched

    N = 32
    A = W.poisson2d(N)
    mode, c, p, q = W.sine_mode_mixture_2d(N, 1, 9)
    Bn = _rhs_block(A.n, 6, 3)
    Bn[:, 2] = mode
    kr = Krylov(A.row_ptr, A.col_idx, A.val, f=F_EXP_NEG, t=1e-3, m=10, k=2, s=30, seed=1, zeta=8, basis=BASIS_DF64)
    X, st = apply_batched([kr], [torch.from_numpy(Bn).cuda()], t=[1e-3], tol=0.0, max_cycles=3)
    x = X[0].cpu().numpy()
    assert st[0][2]["breakdown"] == 1
    assert _rel(x[:, 2], TR.sine_mode_exp(N, c, p, q, 1e-3)) <= 1e-12
    kr1 = Krylov(A.row_ptr, A.col_idx, A.val, f=F_EXP_NEG, t=1e-3, m=10, k=2, s=30, seed=1, zeta=8, basis=BASIS_DF64)
    x0 = kr1.apply(torch.from_numpy(Bn[:, 0].copy()).cuda(), tol=0.0, max_cycles=3).cpu().numpy()
    assert _rel(x[:, 0], x0) <= 1e-12
