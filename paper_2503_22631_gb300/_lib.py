"""ctypes binding of ``libkrylov.so`` (the C ABI declared in ``include/krylov.h``).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Tensors are passed as raw device pointers (``tensor.data_ptr()``);
PyTorch provides device memory and the stream.  If the shared library is
missing the import fails loudly; there is no host fallback.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

LIB_PATH = Path(__file__).resolve().parent / "libkrylov.so"

# krylov_status
OK = 0
NOT_CONVERGED = 1
BREAKDOWN_EXACT = 2
EINVAL = -1
ENOMEM = -2
ECUDA = -3
ENONFINITE = -4
ETIMEOUT = -5
EUNSUPPORTED = -6

# krylov_fkind
ORTHO_TRUNC = 0
ORTHO_RGS = 1

F_EXP_NEG = 0
F_INVSQRT = 1
F_INV = 2
F_PHI1_NEG = 3
F_COS_SQRT = 4

# krylov_basis
BASIS_F64 = 0
BASIS_F32 = 1
BASIS_BF16 = 2
BASIS_DF64 = 3

EXPORTED = [
    "krylov_options_default",
    "krylov_create",
    "krylov_apply",
    "krylov_apply_host",
    "krylov_apply_adjoint",
    "krylov_set_param",
    "krylov_spmv",
    "krylov_size",
    "krylov_destroy",
    "krylov_status_string",
    "krylov_sketch_columns",
    "krylov_last_cycle",
    "krylov_spmv_dot_noalloc",
    "krylov_apply_batched",
    "krylov_probe_bounded_wait",
    "krylov_create_partition",
]


class Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p),
                ("val", C.c_void_p), ("on_device", C.c_int)]


class Func(C.Structure):
    _fields_ = [("kind", C.c_int), ("t", C.c_double)]


class Options(C.Structure):
    _fields_ = [("zeta", C.c_int), ("basis_dtype", C.c_int), ("ortho", C.c_int),
                ("narrow_values_if_exact", C.c_int), ("use_graph", C.c_int), ("abs_tol", C.c_int),
                ("sketch_regenerate", C.c_int), ("stream", C.c_void_p), ("autotune", C.c_int),
                ("block_rhs", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("breakdown", C.c_int), ("steps", C.c_int),
                ("last_update_norm", C.c_double), ("x_norm", C.c_double), ("kappa_T_max", C.c_double),
                ("ms_total", C.c_double), ("bytes_moved", C.c_double), ("launches", C.c_int),
                ("step_launches", C.c_int), ("ms_steps", C.c_double), ("step_bytes", C.c_double),
                ("status", C.c_int), ("fquad_cycles", C.c_int), ("ms_small", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# collective callbacks of a row-partitioned solve (krylov_comm)
ALLREDUCE_F64 = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p)
ALLREDUCE_I64 = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p)
HALO_F64 = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p)


class Comm(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("allreduce_sum_f64", ALLREDUCE_F64), ("allreduce_sum_i64", ALLREDUCE_I64),
                ("allreduce_max_f64", ALLREDUCE_F64), ("halo_exchange_f64", HALO_F64)]


class KrylovError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {status_string(status)} ({status})")
        self.status = status


_lib = None


def load() -> C.CDLL:
    """Load the shared library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2503_22631_gb300.build.build()")
    lib = C.CDLL(str(LIB_PATH))
    P = C.c_void_p
    lib.krylov_options_default.argtypes = [C.POINTER(Options)]
    lib.krylov_options_default.restype = None
    lib.krylov_create.argtypes = [C.POINTER(Csr), Func, C.c_int, C.c_int, C.c_int, C.c_uint64,
                                  C.POINTER(Options), C.POINTER(P)]
    lib.krylov_create.restype = C.c_int
    for name in ("krylov_apply", "krylov_apply_host", "krylov_apply_adjoint"):
        fn = getattr(lib, name)
        fn.argtypes = [P, P, P, C.c_double, C.c_int, C.POINTER(Stats)]
        fn.restype = C.c_int
    lib.krylov_set_param.argtypes = [P, C.c_double]
    lib.krylov_set_param.restype = C.c_int
    lib.krylov_spmv.argtypes = [P, P, P, C.c_int, P, C.POINTER(C.c_double)]
    lib.krylov_spmv.restype = C.c_int
    lib.krylov_size.argtypes = [P]
    lib.krylov_size.restype = C.c_int64
    lib.krylov_destroy.argtypes = [P]
    lib.krylov_destroy.restype = None
    lib.krylov_status_string.argtypes = [C.c_int]
    lib.krylov_status_string.restype = C.c_char_p
    lib.krylov_sketch_columns.argtypes = [C.c_int64, C.c_int, C.c_int, C.c_uint64, C.c_int64, C.c_int64, P, P]
    lib.krylov_sketch_columns.restype = C.c_int
    lib.krylov_last_cycle.argtypes = [P, P, C.c_int64, P, C.c_int64, P, C.c_int64, C.POINTER(C.c_int)]
    lib.krylov_last_cycle.restype = C.c_int
    lib.krylov_spmv_dot_noalloc.argtypes = [C.c_int64, C.c_int64, P, P, P, P, P, P, P, P]
    lib.krylov_spmv_dot_noalloc.restype = C.c_int
    lib.krylov_apply_batched.argtypes = [P, C.c_int, C.c_int, P, P, P, C.c_double, C.c_int, C.POINTER(Stats)]
    lib.krylov_apply_batched.restype = C.c_int
    lib.krylov_probe_bounded_wait.argtypes = [C.c_uint64, P, P]
    lib.krylov_probe_bounded_wait.restype = C.c_int
    lib.krylov_create_partition.argtypes = [C.POINTER(Csr), C.c_int64, C.c_int64, C.c_int64, P, C.c_int64,
                                            C.POINTER(Comm), Func, C.c_int, C.c_int, C.c_int, C.c_uint64,
                                            C.POINTER(Options), C.POINTER(P)]
    lib.krylov_create_partition.restype = C.c_int
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().krylov_status_string(int(status)).decode()


def check(status: int, where: str, ok=(OK,)) -> int:
    if status not in ok:
        raise KrylovError(status, where)
    return status
