"""Write store_sensitivity.json: how far the oracle's own result moves when its
stored basis is rounded to float32 or bfloat16, for the workloads whose
reduced-precision GPU results are compared at full size.

For each case the FP64 oracle (oracle.krylov.restarted, TRUNC mode) is run
twice on the same seeded inputs -- once with FP64 storage and once with the
stored basis rounded to the format (``store``), every other operation in FP64
-- and the relative 2-norm difference of the two results is recorded.  That
number is the method's own sensitivity to the storage precision (the
Arnoldi-like relation of Sec. 2.2, Eq. 5, then holds only for the stored
vectors); a GPU run with that storage format is compared with the FP64 oracle
at a tolerance derived from it.  Only oracle/ and the input generators are
used.

Usage: python tests/golden/make_store_sensitivity.py  (about 10-20 minutes on
one core: one FP64 and two reduced-storage oracle runs of the 4.0M-unknown FEM
workload per cycle count)
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import dense as D  # noqa: E402
from oracle import krylov as K  # noqa: E402
from oracle.sketch import SparseSign  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "store_sensitivity.json")


def fem_kuhn_160(cycles):
    cfg = W.CONFIGS["fem_kuhn_160"]
    A = cfg["matrix"]()
    b = cfg["rhs"](A.n)
    S = SparseSign(A.n, cfg["s"], cfg["zeta"], W.SEED)
    args = (D.INVSQRT, 1.0, cfg["m"], cfg["k"], cfg["s"], cfg["zeta"], W.SEED)
    out = {}
    ref = K.restarted(A, b, *args, mode=K.TRUNC, tol=0.0, max_cycles=cycles, sketch=S)
    nref = np.linalg.norm(ref.x)
    for store in (K.F32, K.BF16):
        r = K.restarted(A, b, *args, mode=K.TRUNC, tol=0.0, max_cycles=cycles, sketch=S, store=store)
        out[store] = float(np.linalg.norm(r.x - ref.x) / nref)
    out["kappa_T_f64"] = [float(c.kappa_T) for c in ref.info]
    return out


def main():
    t0 = time.time()
    res = {"_about": "relative 2-norm change of the FP64 oracle's result when its stored basis is rounded "
                     "to float32 / bfloat16 (all other arithmetic FP64); written by make_store_sensitivity.py",
           "fem_kuhn_160": {}}
    for cycles in (1,):
        res["fem_kuhn_160"][f"cycles_{cycles}"] = fem_kuhn_160(cycles)
        print(cycles, res["fem_kuhn_160"][f"cycles_{cycles}"], f"{time.time() - t0:.0f} s", flush=True)
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
