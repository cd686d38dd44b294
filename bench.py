#!/usr/bin/env python
"""Benchmark: seconds to 1e-8 relative error per f(A)b at n = 2.1M.

Workload: 3D convection-diffusion -Lap u + beta . grad u, 7-point upwind
stencil on a 128^3 interior grid (n = 2,097,152, nnz = 14,581,760,
beta = (50, 50, 50)), f(A) b = exp(-t A) b with t = 1e-2, b ~ U[0, 1) from the
fixed seed; restart length m = 40, window k = 2, sketch s = 160 rows with
zeta = 8 nonzeros per column.  One "step" is one complete f(A) b solve: all
restart cycles needed for 1e-8 relative error (every row of the hot path:
sparse products, truncated orthogonalization, sketches, whitening, f of the
projected matrix, solution updates).

Inputs are synthetic and resident in HBM before the timed region; the working
set (matrix 125 MB + float-float basis 688 MB) is larger than the 129 MB L2, so no flush
is needed between steps.  ``e2e`` repeats the measurement through the host
entry point (b copied in and x copied out inside the timed region).

--impl reference times the CPU oracle (plain FP64 numpy, one thread) on a
bounded sample of the same workload and extrapolates to one solve.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run every rank solves its own replica (no data-path
collective: independent problems), ``value`` is the job's solves per second
expressed as seconds per solve, and the max over ranks is taken.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

# restart cycles of phi_1(-tA) b on the headline operator for 1e-8 relative
# error: 9 cycles are within 2e-10 of a 20-cycle solve (8 cycles: 1e-7), whose
# identity residual t A x - (b - exp(-tA) b) against the Kronecker closed form
# is 1e-11 (tests/test_gpu_phi1.py checks both)
PHI1_CYCLES = 9
# restart cycles of cos(t sqrt(A)) b, 2D Laplacian 1448^2, t = 0.05, for 1e-8:
# 3 cycles are 9e-8 from a 30-cycle solve, 4 cycles equal it
# (tests/test_gpu_cos.py checks 4 cycles and the double-angle identity)
COS_CYCLES = 4

WORKLOAD = dict(
    workload="convdiff3d_128_exp",
    grid=128, beta=(50.0, 50.0, 50.0), t=1e-2, m=40, k=2, s=160, zeta=8,
)
# the Arnoldi-step pair timed by the roofline, per basis (the product kernel of
# the float-float and float32/bfloat16 bases is picked at create by timing; on
# the 7-point stencil it is the sliced-layout one)
STEP_KERNEL_LABEL = {
    "df64": "Arnoldi step: ff_mat_tma_kernel + ff_spmv_sell_kernel (materialize/sketch, sliced-layout SpMV/dots; "
            "tiles and row streams staged by bulk copies)",
    "f32": "Arnoldi step: s32_mat_tma_kernel + s32_spmv_sell_kernel (float32 basis, staged pair)",
    "bf16": "Arnoldi step: s32_mat_tma_kernel + s32_spmv_sell_kernel (bfloat16 basis, staged pair)",
    "f64": "Arnoldi step: step_kernel<double> (fused SpMV + truncated orthogonalization + sketch, float64 arithmetic)",
}
# Restart cycles that reach <= 1e-8 relative error against the closed-form
# Kronecker reference on this workload with the float64 basis (verified by
# tests/test_gpu_headline.py at this exact configuration).
CYCLES_TO_1E8 = {"df64": 10, "f64": 10, "f32": None, "bf16": None}
SEED = 20250331  # workloads.SEED
# The timed solves cycle over five right-hand sides b ~ U[0, 1) (seeds SEED ..
# SEED + 4); each runs the cycle count at which its relative error against the
# Kronecker closed form first reaches 1e-8, found by an instrumented run and
# checked per seed by tests/test_gpu_headline.py.
HEADLINE_SEEDS = tuple(SEED + q for q in range(5))
CYCLES_BY_SEED = {"df64": {SEED + q: c for q, c in enumerate((10, 9, 9, 9, 9))},
                  "f64": {SEED + q: c for q, c in enumerate((10, 9, 9, 9, 9))}}
METRIC = "seconds to 1e-8 rel err per f(A)b at n=2.1M"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--basis", default="df64", choices=["df64", "f64", "f32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain float64-basis solve timed beside the headline")
    ap.add_argument("--parallelism", default="replicas", choices=["replicas", "partition"],
                    help="N > 1: independent replicas of the headline solve (default), or one solve of the "
                         "headline problem row-partitioned over the N ranks (float64 basis)")
    ap.add_argument("--cycles", type=int, default=None, help="override the cycle count (profiling)")
    ap.add_argument("--workload", default="convdiff3d_128",
                    choices=["convdiff3d_128", "convdiff3d_128_rgs", "convdiff3d_128_phi1", "poisson2d_1448_cos",
                             "rmat20_heat", "fem_kuhn_160", "batched16", "convdiff3d_96_adjoint",
                             "convdiff3d_128_long", "poisson2d_1448_long"],
                    help="convdiff3d_128 is the headline; the others time the remaining configurations")
    ap.add_argument("--profile", action="store_true",
                    help="profiling run: no warm-up floor, no e2e, no CPU baseline, no clock sampling")
    ap.add_argument("--product", default="auto", choices=["auto", "gather"],
                    help="float-float product kernel: timed choice at create (default) or always the "
                         "gather kernel (a fixed launch sequence for ncu captures)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_inputs():
    import workloads as W

    A = W.convdiff3d(WORKLOAD["grid"], WORKLOAD["beta"])
    b = W.rhs_uniform(A.n, W.SEED)
    return A, b


def make_rhs(n, seed):
    import workloads as W

    return W.rhs_uniform(n, seed)


# ------------------------------------------------------------------ oracle --
def host_cpu():
    """Host core count and CPU model (for the baseline's description)."""
    model = ""
    try:
        for line in Path("/proc/cpuinfo").read_text().splitlines():
            k = line.split(":", 1)[0].strip().lower()
            if k in ("model name", "cpu model", "hardware") and ":" in line:
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if not model:
        import platform

        model = platform.processor() or platform.machine()
    return os.cpu_count() or 1, model


def _oracle_sample_child(out_path: str, cycles: int):
    """Child process: time `cycles` whole restart cycles of the oracle (m = 40
    Arnoldi steps, the sketch, the whitening QR, the dense exp of the block
    matrix and the update each) on the full headline workload."""
    import workloads as W
    from oracle import dense as D
    from oracle import krylov as K
    from oracle.sketch import SparseSign

    A, b = make_inputs()
    S = SparseSign(A.n, WORKLOAD["s"], WORKLOAD["zeta"], W.SEED)  # generated once per run
    t0 = time.perf_counter()
    K.restarted(A, b, D.EXP_NEG, WORKLOAD["t"], WORKLOAD["m"], WORKLOAD["k"], WORKLOAD["s"], WORKLOAD["zeta"],
                W.SEED, mode=K.TRUNC, tol=0.0, max_cycles=cycles, sketch=S)
    dt = time.perf_counter() - t0
    Path(out_path).write_text(json.dumps({"seconds": dt, "cycles": cycles}))


def oracle_seconds_per_solve(cycles: int, threads: int = 1, sample_cycles: int = 1):
    """Run `sample_cycles` whole oracle cycles in a fresh process with `threads`
    BLAS threads (the oracle's only multithreaded parts are its dense BLAS
    calls; its sparse product is one numpy pass); scale linearly in cycles."""
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t, CUDA_VISIBLE_DEVICES="")
    with tempfile.TemporaryDirectory() as td:
        out = Path(td) / "o.json"
        code = (f"import sys; sys.path.insert(0, {str(ROOT)!r}); import bench; "
                f"bench._oracle_sample_child({str(out)!r}, {sample_cycles})")
        subprocess.run([sys.executable, "-c", code], check=True, env=env, cwd=str(ROOT))
        r = json.loads(out.read_text())
    return r["seconds"] / r["cycles"] * cycles, r


def cpu_baseline_line(cycles: int):
    """The oracle timed on the host: one whole restart cycle at full size on one
    thread and on all host cores, scaled to `cycles` cycles."""
    ncpu, model = host_cpu()
    v1, r1 = oracle_seconds_per_solve(cycles, 1)
    vn, rn = oracle_seconds_per_solve(cycles, ncpu)
    best, cores = (vn, ncpu) if vn < v1 else (v1, 1)
    return {"value": best, "unit": "s", "cores": cores, "kind": "oracle",
            "host": {"nproc": ncpu, "cpu": model},
            "single_thread": {"value": v1, "cores": 1, "cycle_seconds": r1["seconds"]},
            "all_cores": {"value": vn, "cores": ncpu, "cycle_seconds": rn["seconds"]},
            "sample": (f"one whole oracle restart cycle (40 Arnoldi steps, sketch, whitening QR, dense exp, "
                       f"update) on the full workload, {r1['seconds']:.1f} s on 1 thread and "
                       f"{rn['seconds']:.1f} s with {ncpu} BLAS threads, scaled linearly to {cycles} cycles; "
                       f"value = the faster of the two")}


def reference_main(args, rank):
    if rank != 0:
        return
    cycles = CYCLES_TO_1E8["df64"]
    ncpu, model = host_cpu()
    vals = []
    sample = None
    for _ in range(args.warmup):
        oracle_seconds_per_solve(cycles, ncpu)
    for _ in range(args.steps):
        v, sample = oracle_seconds_per_solve(cycles, ncpu)
        vals.append(v)
    value = statistics.median(vals)
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": value * 1e3,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD["workload"], "n": 128**3, "m": 40, "k": 2, "s": 160, "zeta": 8,
                   "t": 1e-2, "cycles": cycles},
        "cpu_baseline": {"value": value, "unit": "s", "cores": ncpu, "kind": "oracle",
                         "host": {"nproc": ncpu, "cpu": model},
                         "sample": f"one whole oracle restart cycle at full size per bench step ({ncpu} BLAS "
                                   f"threads; last {sample['seconds']:.1f} s), scaled linearly to {cycles} "
                                   f"cycles; median of {args.steps}"},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def step_traffic():
    """DRAM bytes of one Arnoldi step from the committed ncu summary, or None
    when the step kernels changed since those counters were taken."""
    import hashlib

    tf = ROOT / "profiles" / "step_kernel_traffic.txt"
    csrc = ROOT / "paper_2503_22631_gb300" / "csrc"
    srcs = [csrc / "step_kernels.cu", csrc / "step_common.cuh", csrc / "kernels.cuh"]
    if not tf.exists() or not all(p.exists() for p in srcs):
        return None
    kv = dict(line.split("=", 1) for line in tf.read_text().splitlines()
              if "=" in line and not line.startswith("#"))
    digest = hashlib.sha256(b"".join(p.read_bytes() for p in srcs)).hexdigest()[:16]
    if kv.get("step_kernels_sha256_16") != digest:
        return None
    return float(kv["bytes_per_launch"])


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, enabled: bool = True):
        self.gpu = gpu_index
        self.enabled = enabled
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def __enter__(self):
        if not self.enabled:
            return self
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        self.tmp.flush()
        rows = []
        try:
            for line in Path(self.tmp.name).read_text().splitlines():
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        finally:
            os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------- aggregation --
def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's timed-region length (all ranks must call it)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def seconds_per_solve(ms_max: float, steps: int, world: int) -> float:
    """Whole-job seconds per f(A) b: every rank solves `steps` independent
    problems in the timed region, so the job does steps * world solves in
    ms_max milliseconds."""
    return ms_max / 1e3 / (steps * world)


# ------------------------------------------------------- other configurations --
def _timed(fn, steps, warmup, stream):
    """CUDA-event time of `steps` calls of fn() after `warmup` calls (ms)."""
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def secondary_main(args):
    """One JSON line for a non-headline configuration (one GPU; the config names
    what a step is)."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2503_22631_gb300 import (BASIS_BF16, BASIS_DF64, BASIS_F32, BASIS_F64, F_COS_SQRT, F_EXP_NEG,
                                        F_INVSQRT, F_PHI1_NEG, ORTHO_RGS, Krylov, apply_batched, build,
                                        krylov_expm)

    build.build()
    basis = {"df64": BASIS_DF64, "f64": BASIS_F64, "f32": BASIS_F32, "bf16": BASIS_BF16}[args.basis]
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    warmup = max(args.warmup, 3)
    wl = args.workload
    stats = []
    if wl == "convdiff3d_128_rgs":
        A, b = make_inputs()
        kr = Krylov(A.row_ptr, A.col_idx, A.val, f=F_EXP_NEG, t=WORKLOAD["t"], m=WORKLOAD["m"], k=WORKLOAD["m"],
                    s=WORKLOAD["s"], seed=SEED, zeta=WORKLOAD["zeta"], basis=basis, ortho=ORTHO_RGS)
        bd = torch.from_numpy(b).cuda()
        cycles = 10

        def fn():
            kr.apply(bd, tol=0.0, max_cycles=cycles)
            stats.append(dict(kr.stats))

        metric = "seconds to 1e-8 rel err per f(A)b at n=2.1M, randomized Gram-Schmidt with the full window"
        config = {"workload": wl, "n": A.n, "nnz": A.nnz, "m": 40, "k": 40, "s": 160, "zeta": 8, "t": 1e-2,
                  "cycles": cycles, "basis": args.basis, "ortho": "rgs"}
        units = 1
    elif wl in ("convdiff3d_128_long", "poisson2d_1448_long"):
        # 64 restart cycles: the projected exponential's cost per cycle, with
        # the contour quadrature alone after the first 16 cycles where its
        # checks pass (the 2D Laplacian's Ritz values lie near the real axis;
        # the convection operator's have t Im up to ~180, which no contour
        # around the negative real axis encloses, so scaling and squaring
        # carries that run)
        if wl == "convdiff3d_128_long":
            A, b = make_inputs()
            tt, mm, ss = WORKLOAD["t"], WORKLOAD["m"], WORKLOAD["s"]
        else:  # short cycles (m = 12) on a stiff operator: many restarts before convergence
            A = W.poisson2d(1448)
            b = W.rhs_uniform(A.n, SEED)
            tt, mm, ss = 3e-5, 12, 48
        kr = Krylov(A.row_ptr, A.col_idx, A.val, f=F_EXP_NEG, t=tt, m=mm, k=WORKLOAD["k"],
                    s=ss, seed=SEED, zeta=WORKLOAD["zeta"], basis=basis)
        bd = torch.from_numpy(b).cuda()
        cycles = 64
        kr.apply(bd, tol=0.0, max_cycles=16)
        kr.apply(bd, tol=0.0, max_cycles=16)
        small16 = kr.stats["ms_small"]

        def fn():
            kr.apply(bd, tol=0.0, max_cycles=cycles)
            stats.append(dict(kr.stats))

        metric = "seconds per 64 restart cycles of exp(-tA)b at n=2.1M"
        config = {"workload": wl, "n": A.n, "nnz": A.nnz, "m": mm, "k": 2, "s": ss, "zeta": 8, "t": tt,
                  "cycles": cycles, "basis": args.basis}
        units = 1
    elif wl == "convdiff3d_128_phi1":
        # phi_1(-tA) b (the phi function of Sec. 5) on the headline operator
        A, b = make_inputs()
        kr = Krylov(A.row_ptr, A.col_idx, A.val, f=F_PHI1_NEG, t=WORKLOAD["t"], m=WORKLOAD["m"], k=WORKLOAD["k"],
                    s=WORKLOAD["s"], seed=SEED, zeta=WORKLOAD["zeta"], basis=basis)
        bd = torch.from_numpy(b).cuda()
        cycles = PHI1_CYCLES

        def fn():
            kr.apply(bd, tol=0.0, max_cycles=cycles)
            stats.append(dict(kr.stats))

        metric = "seconds to 1e-8 rel err per phi_1(-tA)b at n=2.1M"
        config = {"workload": wl, "n": A.n, "nnz": A.nnz, "m": 40, "k": 2, "s": 160, "zeta": 8, "t": 1e-2,
                  "cycles": cycles, "basis": args.basis, "f": "phi1"}
        units = 1
    elif wl == "poisson2d_1448_cos":
        # cos(t sqrt(A)) b (the membrane example of Sec. 5) on a 2D 5-point
        # Laplacian of the headline's size, t sqrt(lambda_max) ~ 200
        A = W.poisson2d(1448)
        b = W.rhs_uniform(A.n, SEED)
        kr = Krylov(A.row_ptr, A.col_idx, A.val, f=F_COS_SQRT, t=0.05, m=40, k=2, s=160, seed=SEED, zeta=8,
                    basis=basis)
        bd = torch.from_numpy(b).cuda()
        cycles = COS_CYCLES

        def fn():
            kr.apply(bd, tol=0.0, max_cycles=cycles)
            stats.append(dict(kr.stats))

        metric = "seconds to 1e-8 rel err per cos(t sqrt(A))b at n=2.1M (2D Laplacian)"
        config = {"workload": wl, "n": A.n, "nnz": A.nnz, "m": 40, "k": 2, "s": 160, "zeta": 8, "t": 0.05,
                  "cycles": cycles, "basis": args.basis, "f": "cos_sqrt"}
        units = 1
    elif wl == "rmat20_heat":
        # the graph example of Sec. 5: heat kernel exp(-tL) x_0 on the out-degree
        # Laplacian, an undirected R-MAT graph (2^20 nodes, power-law rows) for
        # the paper's networks, in the paper's configuration for it
        # (randomized Gram-Schmidt over the whole cycle, m = k = 40, s = 320)
        A = W.rmat_laplacian(20, 16, SEED)
        b = W.rhs_probability(A.n, SEED)
        kr = Krylov(A.row_ptr, A.col_idx, A.val, f=F_EXP_NEG, t=0.1, m=40, k=40, s=320, seed=SEED, zeta=8,
                    basis=basis, ortho=ORTHO_RGS)
        bd = torch.from_numpy(b).cuda()
        cycles = 4  # 2e-12 from an 8-cycle solve (3 cycles: 4e-8); tests/test_gpu_graph.py checks it

        def fn():
            kr.apply(bd, tol=0.0, max_cycles=cycles)
            stats.append(dict(kr.stats))

        metric = "seconds to 1e-8 rel err per heat kernel exp(-tL)x_0 on a 1M-node R-MAT graph (32M nonzeros)"
        config = {"workload": wl, "n": A.n, "nnz": A.nnz, "max_row": int(np.diff(A.row_ptr).max()), "m": 40,
                  "k": 40, "s": 320, "zeta": 8, "t": 0.1, "cycles": cycles, "basis": args.basis, "ortho": "rgs"}
        units = 1
    elif wl == "fem_kuhn_160":
        cfg = W.CONFIGS["fem_kuhn_160"]
        A = cfg["matrix"]()
        b = cfg["rhs"](A.n)
        kr = Krylov(A.row_ptr, A.col_idx, A.val, f=F_INVSQRT, t=1.0, m=cfg["m"], k=cfg["k"], s=cfg["s"], seed=W.SEED,
                    zeta=cfg["zeta"], basis=basis)
        bd = torch.from_numpy(b).cuda()
        cycles = 20

        def fn():
            kr.apply(bd, tol=0.0, max_cycles=cycles)
            stats.append(dict(kr.stats))

        metric = "seconds per 20 restart cycles of A^{-1/2} b at n=4.0M (P1 FEM, k=4)"
        config = {"workload": wl, "n": A.n, "nnz": A.nnz, "m": cfg["m"], "k": cfg["k"], "s": cfg["s"],
                  "zeta": cfg["zeta"], "cycles": cycles, "basis": args.basis, "f": "invsqrt"}
        units = 1
    elif wl == "batched16":
        insts = W.batched_instances(16, W.SEED)
        hs, B = [], []
        for i, inst in enumerate(insts):
            Ai = W.batched_matrix(inst)
            hs.append(Krylov(Ai.row_ptr, Ai.col_idx, Ai.val, f=F_EXP_NEG, t=inst["t"], m=30, k=2, s=120, seed=W.SEED,
                             zeta=8, basis=basis))
            B.append(torch.from_numpy(W.rhs_normal(inst["n"] * 64, 100 + i).reshape(inst["n"], 64)).cuda())
        # every right-hand side runs to the relative stop ||y|| <= tol ||x|| of
        # its basis (the float32 floor 1e-5, else 1e-8) within the block form's
        # 16 cycles
        cycles = 16
        btol = 1e-5 if args.basis in ("f32", "bf16") else 1e-8
        ts = [inst["t"] for inst in insts]

        def fn():
            _, st = apply_batched(hs, B, t=ts, tol=btol, max_cycles=cycles, raise_on_error=False)
            stats.extend(x for row in st for x in row)

        metric = f"seconds per batched call: 16 matrices x 64 right-hand sides, each to a relative update of {btol:g}"
        config = {"workload": wl, "instances": 16, "rhs": 64, "n_total": int(sum(i["n"] for i in insts)),
                  "m": 30, "k": 2, "s": 120, "zeta": 8, "max_cycles": cycles, "tol": btol, "basis": args.basis}
        units = 1
    else:  # convdiff3d_96_adjoint
        cfg = W.CONFIGS["convdiff3d_96_adjoint"]
        A = cfg["matrix"]()
        kr = Krylov(A.row_ptr, A.col_idx, A.val, f=F_EXP_NEG, t=cfg["t"], m=cfg["m"], k=cfg["k"], s=cfg["s"],
                    seed=W.SEED, zeta=cfg["zeta"], basis=basis)
        b0 = torch.from_numpy(cfg["rhs"](A.n)).cuda()
        y = torch.from_numpy(W.rhs_normal(A.n, W.SEED + 1)).cuda()

        def fn():
            bb = b0.clone().requires_grad_(True)
            tt = torch.tensor(cfg["t"], dtype=torch.float64, requires_grad=True)
            x = krylov_expm(bb, tt, kr, 1e-10, 40)
            ((x - y) ** 2).sum().backward()
            stats.append(dict(kr.stats))

        metric = "seconds per loss gradient (grad_b and grad_t of ||exp(-tA)b - y||^2) at n=885K"
        config = {"workload": wl, "n": A.n, "nnz": A.nnz, "m": cfg["m"], "k": 2, "s": 160, "zeta": 8,
                  "t": cfg["t"], "tol": 1e-10, "basis": args.basis}
        units = 1
    with ClockSampler(0, enabled=not args.profile) as clk:
        ms = _timed(fn, args.steps, warmup, stream)
    per_call = max(1, len(stats) // (warmup + args.steps))
    stats = stats[-per_call * args.steps:]  # the timed calls only
    steps_ms = sum(x.get("ms_steps", 0.0) for x in stats)
    step_bytes = sum(x.get("step_bytes", 0.0) for x in stats)
    peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) if (ROOT / "MEASURED_PEAKS.json").exists() else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = step_bytes / (steps_ms / 1e3) / 1e9 if steps_ms > 0 else None
    value = ms / 1e3 / (args.steps * units)
    line = {
        "metric": metric, "value": value, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": args.basis, "data": "synthetic", "config": config,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": None,
                     "kernel": "Arnoldi-step phase (step kernels of every cycle)",
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in peaks else "fallback"},
        "cpu_baseline": None, "e2e": None,
        "gpu_launches": int(sum(x.get("launches", 0) for x in stats)),
        "clocks": clk.summary(),
    }
    if wl == "batched16":
        cyc = [x["cycles"] for x in stats]
        line["config"]["cycles_mean"] = float(np.mean(cyc)) if cyc else None
        line["config"]["cycles_max"] = int(max(cyc)) if cyc else None
    if wl in ("convdiff3d_128_long", "poisson2d_1448_long"):
        last = stats[-1]
        line["small_problem"] = {
            "ms_per_cycle_first_16": small16 / 16,
            "ms_per_cycle_after_16": (last["ms_small"] - small16) / max(1, last["cycles"] - 16),
            "quadrature_cycles": last["fquad_cycles"], "cycles_run": last["cycles"]}
    print(json.dumps(line), flush=True)


def plain_fp64_solve(A, bds, cyc, warmup, steps, stream, peak, barrier):
    """Time the same solves (right-hand sides bds, cycle counts cyc) with the
    float64 basis (float64 streaming arithmetic) on the same stream and GPU;
    returns its sub-object of the JSON line."""
    import torch

    from paper_2503_22631_gb300 import BASIS_F64, F_EXP_NEG, Krylov

    kr = Krylov(A.row_ptr, A.col_idx, A.val, f=F_EXP_NEG, t=WORKLOAD["t"], m=WORKLOAD["m"], k=WORKLOAD["k"],
                s=WORKLOAD["s"], seed=SEED, zeta=WORKLOAD["zeta"], basis=BASIS_F64, stream=stream)
    x = torch.empty_like(bds[0])
    cycles = cyc[0]
    for w in range(warmup):
        kr.apply(bds[w % len(bds)], tol=0.0, max_cycles=cyc[w % len(bds)], out=x)
    barrier()
    stats = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for q in range(steps):
        kr.apply(bds[q % len(bds)], tol=0.0, max_cycles=cyc[q % len(bds)], out=x)
        stats.append(dict(kr.stats))
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    steps_ms = sum(s["ms_steps"] for s in stats)
    achieved = sum(s["step_bytes"] for s in stats) / (steps_ms / 1e3) / 1e9
    del kr
    return {"basis": "f64", "value": ms / 1e3 / steps, "unit": "s", "ms_total": ms, "cycles": cycles,
            "ms_steps_per_solve": steps_ms / steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "kernel": "Arnoldi step: step_kernel<double> (fused SpMV + truncated orthogonalization + "
                                   "sketch, float64 arithmetic)"}}


def partition_main(args, rank, world, local):
    """One headline solve row-partitioned over the ranks (NCCL collectives,
    float64 basis): every timed step is one whole f(A) b of the full problem."""
    import torch

    from paper_2503_22631_gb300 import F_EXP_NEG, build
    from paper_2503_22631_gb300.dist import PartitionedKrylov, TorchComm, plan_partition

    build.build()
    cycles = args.cycles or CYCLES_TO_1E8["f64"]
    warmup = max(args.warmup, 3)
    A, b = make_inputs()
    plan = plan_partition(A.row_ptr, A.col_idx, A.val, world, rank)
    stream = torch.cuda.current_stream()
    kr = PartitionedKrylov(plan, TorchComm(plan), f=F_EXP_NEG, t=WORKLOAD["t"], m=WORKLOAD["m"], k=WORKLOAD["k"],
                           s=WORKLOAD["s"], seed=SEED, zeta=WORKLOAD["zeta"], stream=stream)
    bl = torch.from_numpy(b[plan.lo:plan.hi].copy()).cuda()
    x = torch.empty_like(bl)
    for _ in range(warmup):
        kr.apply(bl, tol=0.0, max_cycles=cycles, out=x)
    torch.cuda.synchronize()
    torch.distributed.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.distributed.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            kr.apply(bl, tol=0.0, max_cycles=cycles, out=x)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.distributed.barrier()
    ms_max = max_over_ranks(e0.elapsed_time(e1), world, torch.device("cuda", local))
    if rank != 0:
        return
    value = ms_max / 1e3 / args.steps  # one whole problem per step for the job
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": False, "scaling": "strong", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD["workload"], "n": A.n, "nnz": A.nnz, "m": WORKLOAD["m"], "k": WORKLOAD["k"],
                   "s": WORKLOAD["s"], "zeta": WORKLOAD["zeta"], "t": WORKLOAD["t"], "cycles": cycles,
                   "basis": "f64", "parallelism": f"row partition over {world} ranks (halo exchange + all-reduce "
                                                  f"per step)", "l2": "working set > L2 (no flush)"},
        "roofline": None, "cpu_baseline": None, "e2e": None,
        "gpu_launches": int(kr.stats["launches"]) * args.steps, "clocks": clk.summary()}), flush=True)


# ------------------------------------------------------------------- main ---
def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_main(args, rank)
        return
    if args.workload != "convdiff3d_128":
        if rank == 0:
            secondary_main(args)
        return

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        if args.parallelism == "partition":
            partition_main(args, rank, world, local)
            dist.destroy_process_group()
            return
    from paper_2503_22631_gb300 import BASIS_BF16, BASIS_DF64, BASIS_F32, BASIS_F64, F_EXP_NEG, Krylov, build

    build.build()
    basis = {"df64": BASIS_DF64, "f64": BASIS_F64, "f32": BASIS_F32, "bf16": BASIS_BF16}[args.basis]
    table = CYCLES_BY_SEED.get(args.basis, CYCLES_BY_SEED["df64"])
    seeds = HEADLINE_SEEDS
    cyc = [args.cycles or table[sd] for sd in seeds]  # per seed
    cycles = cyc[0]
    if args.profile:
        args.no_e2e = args.no_cpu_baseline = True
        seeds, cyc = seeds[:1], cyc[:1]  # one fixed launch sequence for profilers
    warmup = args.warmup if args.profile else max(args.warmup, 3)
    A, b = make_inputs()
    rhs = [b] + [make_rhs(A.n, sd) for sd in seeds[1:]]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        kr = Krylov(A.row_ptr, A.col_idx, A.val, f=F_EXP_NEG, t=WORKLOAD["t"], m=WORKLOAD["m"], k=WORKLOAD["k"],
                    s=WORKLOAD["s"], seed=SEED, zeta=WORKLOAD["zeta"], basis=basis, stream=stream,
                    autotune="gather" if args.product == "gather" else True)
        bds = [torch.from_numpy(v).cuda() for v in rhs]
        bd = bds[0]
        x = torch.empty_like(bd)
        stream.synchronize()

        def barrier():
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
                torch.cuda.synchronize()

        for w in range(warmup):
            kr.apply(bds[w % len(bds)], tol=0.0, max_cycles=cyc[w % len(bds)], out=x)
        barrier()
        stats = []
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(torch.cuda.current_device(), enabled=not args.profile) as clk:
            barrier()
            ev0.record(stream)
            for q in range(args.steps):  # step q solves right-hand side q mod 5
                kr.apply(bds[q % len(bds)], tol=0.0, max_cycles=cyc[q % len(bds)], out=x)
                stats.append(dict(kr.stats))
            ev1.record(stream)
            barrier()
        ms = ev0.elapsed_time(ev1)
        clocks = clk.summary()
        ms_max = max_over_ranks(ms, world, torch.device("cuda", local))
        sec_per_solve = seconds_per_solve(ms_max, args.steps, world)

        # dominant kernel: the fused step kernel (per launch averages)
        steps_ms = sum(s["ms_steps"] for s in stats)
        step_bytes = sum(s["step_bytes"] for s in stats)
        step_launches = sum(s["step_launches"] for s in stats)
        launches = stats[-1]["launches"]
        peaks = {}
        pk = ROOT / "MEASURED_PEAKS.json"
        if pk.exists():
            peaks = json.loads(pk.read_text())
        peak = peaks.get("hbm_gbs", 6800.0)
        achieved = step_bytes / (steps_ms / 1e3) / 1e9
        traffic = step_traffic()

        # end to end through the host entry point (pinned host buffers)
        e2e = None
        if not args.no_e2e:
            bhs = [torch.from_numpy(v).pin_memory() for v in rhs]
            xh = torch.empty_like(bhs[0]).pin_memory()
            kr.apply_host(bhs[0].numpy(), tol=0.0, max_cycles=cyc[0], out=xh.numpy())
            barrier()
            t0 = time.perf_counter()
            for q in range(args.steps):
                kr.apply_host(bhs[q % len(bhs)].numpy(), tol=0.0, max_cycles=cyc[q % len(bhs)], out=xh.numpy())
            barrier()
            e2e_s = (time.perf_counter() - t0) / (args.steps * world)
            e2e = {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 8 * A.n, "d2h_bytes_per_step": 8 * A.n}

        # the plain float64 form on the same GPU and workload (same cycles, same
        # timing protocol): the mixed-precision comparison point
        fp64 = None
        if not args.no_fp64 and not args.profile and args.basis != "f64":
            fp64 = plain_fp64_solve(A, bds, [CYCLES_BY_SEED["f64"][sd] for sd in seeds], warmup, args.steps, stream,
                                    peak, barrier)
            if world > 1:
                fp64["value"] = seconds_per_solve(max_over_ranks(fp64["ms_total"], world,
                                                                 torch.device("cuda", local)), args.steps, world)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_line(cycles)
    line = {
        "metric": METRIC,
        "value": sec_per_solve,
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": warmup,
        "ms_per_step": ms_max / args.steps,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": args.basis,
        "data": "synthetic",
        "config": {"workload": WORKLOAD["workload"], "n": A.n, "nnz": A.nnz, "m": WORKLOAD["m"],
                   "k": WORKLOAD["k"], "s": WORKLOAD["s"], "zeta": WORKLOAD["zeta"], "t": WORKLOAD["t"],
                   "cycles": cycles, "seeds": list(seeds), "cycles_by_seed": cyc,
                   "basis": args.basis, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "working set > L2 (no flush)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic if args.basis == "df64" else None,
                     "kernel": STEP_KERNEL_LABEL[args.basis],
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in peaks else "fallback"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches * args.steps,
        "clocks": clocks,
        "fp64": fp64,
        "solve": {"cycles": stats[-1]["cycles"], "step_launches_per_solve": step_launches // args.steps,
                  "ms_steps_per_solve": steps_ms / args.steps, "last_update_rel": stats[-1]["last_update_norm"] /
                  max(stats[-1]["x_norm"], 1e-300)},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
