"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/*.h declares (no compute calls)."""
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w \*]*?\b(krylov_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("krylov_create", "krylov_apply", "krylov_apply_adjoint", "krylov_destroy",
                     "krylov_set_param", "krylov_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2503_22631_gb300 import _lib

    names = declared_functions()
    assert names == set(_lib.EXPORTED)
    for name in sorted(names):
        assert getattr(lib, name) is not None


def test_status_strings_without_gpu(lib):
    from paper_2503_22631_gb300 import _lib

    assert _lib.status_string(0) == "ok"
    assert "invalid" in _lib.status_string(-1)


def test_product_path_does_not_import_the_oracle():
    """The package and its C sources never reference the test oracle."""
    pkg = ROOT / "paper_2503_22631_gb300"
    for f in list(pkg.rglob("*.py")) + list(pkg.rglob("*.cu")) + list(pkg.rglob("*.cuh")) + list(pkg.rglob("*.h")):
        text = f.read_text()
        assert not re.search(r"\boracle\b", text), f


def test_options_layout_matches_header(lib):
    """krylov_options: the ctypes mirror lists the header's fields in order, and
    krylov_options_default (no GPU needed) writes exactly sizeof(Options)
    bytes with the documented defaults: a field added on one side only
    shows up as a wrong default or as bytes written past the mirror's end."""
    import ctypes as C
    import re

    from paper_2503_22631_gb300 import _lib

    hdr = (ROOT / "include" / "krylov.h").read_text()
    end = hdr.index("} krylov_options;")
    body = hdr[hdr.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"(?:int|void\*)\s+(\w+)\s*;", body)
    assert names == [f[0] for f in _lib.Options._fields_]
    pad = 64
    buf = (C.c_ubyte * (C.sizeof(_lib.Options) + pad))()
    C.memset(buf, 0x5A, C.sizeof(buf))
    opt = _lib.Options.from_buffer(buf)
    lib.krylov_options_default(C.byref(opt))
    assert bytes(buf[C.sizeof(_lib.Options):]) == b"\x5a" * pad
    assert (opt.zeta, opt.basis_dtype, opt.ortho, opt.narrow_values_if_exact, opt.use_graph, opt.abs_tol,
            opt.sketch_regenerate, opt.autotune, opt.block_rhs) == (8, 0, 0, 1, 1, 0, 0, 1, 1)
    assert not opt.stream


def test_struct_mirrors_list_the_header_fields():
    """krylov_stats, krylov_csr and krylov_func: the ctypes mirrors name the
    header's fields in the header's order."""
    from paper_2503_22631_gb300 import _lib

    hdr = (ROOT / "include" / "krylov.h").read_text()
    for cname, mirror in (("krylov_stats", _lib.Stats), ("krylov_csr", _lib.Csr), ("krylov_func", _lib.Func)):
        end = hdr.index("} %s;" % cname)
        body = hdr[hdr.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        names = re.findall(r"(?:int|int64_t|double|void\*|const int32_t\*|const double\*|const void\*)\s+(\w+)\s*;",
                           body)
        assert names == [f[0] for f in mirror._fields_], cname


def _host_csr():
    """A 4 x 4 tridiagonal matrix in host memory, plus the arrays that keep it alive."""
    import ctypes as C

    import numpy as np

    from paper_2503_22631_gb300 import _lib

    rp = np.array([0, 2, 5, 8, 10], dtype=np.int32)
    ci = np.array([0, 1, 0, 1, 2, 1, 2, 3, 2, 3], dtype=np.int32)
    val = np.array([2.0, -1, -1, 2, -1, -1, 2, -1, -1, 2])
    csr = _lib.Csr(n=4, nnz=10, row_ptr=rp.ctypes.data_as(C.c_void_p), col_idx=ci.ctypes.data_as(C.c_void_p),
                   val=val.ctypes.data_as(C.c_void_p), on_device=0)
    return csr, (rp, ci, val)


def test_create_validates_arguments_before_any_device_call(lib):
    """krylov_create checks every argument on the host before its first CUDA
    call: each invalid choice returns KRYLOV_EINVAL (the randomized
    Gram-Schmidt cycle with a float32 basis KRYLOV_EUNSUPPORTED) and leaves
    *out NULL, with or without a GPU."""
    import ctypes as C

    from paper_2503_22631_gb300 import _lib

    csr, keep = _host_csr()
    EINVAL, EUNSUP = -1, -6

    def create(A=csr, kind=0, t=1.0, m=2, k=2, s=8, opt=None, out=True):
        h = C.c_void_p(0x1234)
        st = lib.krylov_create(C.byref(A) if A is not None else None, _lib.Func(kind, t), m, k, s, 7,
                               C.byref(opt) if opt is not None else None, C.byref(h) if out else None)
        return st, h

    def options(**kw):
        o = _lib.Options()
        lib.krylov_options_default(C.byref(o))
        for key, v in kw.items():
            setattr(o, key, v)
        return o

    def bad_csr(**kw):
        c = _lib.Csr()
        C.memmove(C.byref(c), C.byref(csr), C.sizeof(c))
        for key, v in kw.items():
            setattr(c, key, v)
        return c

    cases = [
        dict(A=None), dict(out=False),
        dict(A=bad_csr(n=0)), dict(A=bad_csr(n=1 << 31)), dict(A=bad_csr(nnz=-1)),
        dict(A=bad_csr(nnz=1 << 31)), dict(A=bad_csr(row_ptr=None)), dict(A=bad_csr(col_idx=None)),
        dict(A=bad_csr(val=None)),
        dict(m=0), dict(m=257, s=300), dict(k=0), dict(s=2), dict(s=1025), dict(k=5, m=8, s=16),
        dict(opt=options(zeta=0)), dict(opt=options(zeta=9)), dict(opt=options(zeta=33), s=64),
        dict(opt=options(basis_dtype=4)), dict(opt=options(basis_dtype=-1)), dict(opt=options(ortho=2)),
        dict(opt=options(autotune=3)), dict(opt=options(ortho=1), k=3),
        dict(kind=5), dict(kind=-1), dict(t=float("inf")), dict(t=float("nan")),
    ]
    for kw in cases:
        st, h = create(**kw)
        assert st == EINVAL, kw
        if kw.get("out", True) and kw.get("A", csr) is not None:
            assert h.value is None, kw
    for basis in (1, 2):  # float32 / bfloat16 bases under randomized Gram-Schmidt
        st, h = create(opt=options(ortho=1, basis_dtype=basis))
        assert st == EUNSUP and h.value is None
    # valid arguments with no device: the first CUDA call fails and the status
    # says so (there is no host fallback)
    import torch

    if not torch.cuda.is_available():
        st, h = create()
        assert st == -3 and h.value is None


def test_calls_on_a_null_handle_are_rejected(lib):
    """Every entry point that takes a handle answers a NULL one with
    KRYLOV_EINVAL (no device call), and krylov_destroy(NULL) is a no-op."""
    import ctypes as C

    from paper_2503_22631_gb300 import _lib

    buf = (C.c_double * 4)()
    p = C.cast(buf, C.c_void_p)
    st = _lib.Stats()
    assert lib.krylov_apply(None, p, p, 1e-8, 3, C.byref(st)) == -1
    assert st.status == -1
    assert lib.krylov_apply_adjoint(None, p, p, 1e-8, 3, None) == -1
    assert lib.krylov_apply_host(None, p, p, 1e-8, 3, None) == -1
    assert lib.krylov_set_param(None, 0.5) == -1
    assert lib.krylov_spmv(None, p, p, 0, None, None) == -1
    assert lib.krylov_size(None) == 0
    assert lib.krylov_last_cycle(None, None, 0, None, 0, None, 0, None) == -1
    lib.krylov_destroy(None)
    hs = (C.c_void_p * 1)(None)
    assert lib.krylov_apply_batched(C.cast(hs, C.c_void_p), 1, 1, p, p, None, 1e-8, 3, None) == -1
    assert lib.krylov_apply_batched(None, 1, 1, p, p, None, 1e-8, 3, None) == -1
    # sketch generator arguments out of range
    rows = (C.c_int32 * 8)()
    signs = (C.c_int8 * 8)()
    r, s_ = C.cast(rows, C.c_void_p), C.cast(signs, C.c_void_p)
    for args in [(0, 8, 1, 0, 0, 1), (8, 0, 1, 0, 0, 1), (8, 40000, 1, 0, 0, 1), (8, 8, 9, 0, 0, 1),
                 (8, 64, 33, 0, 0, 1), (8, 8, 1, 0, -1, 1), (8, 8, 1, 0, 4, 5), (8, 8, 1, 0, 0, -1)]:
        assert lib.krylov_sketch_columns(*args, r, s_) == -1, args
    assert lib.krylov_sketch_columns(8, 8, 1, 0, 0, 0, r, s_) == 0  # nothing to generate
    # bounded-wait probe: bound out of range or missing outputs
    to = (C.c_int * 2)()
    ns = (C.c_double * 2)()
    pto, pns = C.cast(to, C.c_void_p), C.cast(ns, C.c_void_p)
    for args in [(0, pto, pns), (10**10 + 1, pto, pns), (1000, None, pns), (1000, pto, None)]:
        assert lib.krylov_probe_bounded_wait(*args) == -1, args


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "krylov.h"

int main(void) {
  krylov_options opt;
  krylov_options_default(&opt);
  if (opt.zeta != 8 || opt.basis_dtype != KRYLOV_BASIS_F64 || opt.ortho != KRYLOV_ORTHO_TRUNC) return 10;
  if (strcmp(krylov_status_string(KRYLOV_OK), "ok") != 0) return 11;
  opt.zeta = 1; /* one nonzero per sketch column (s = 3 rows below) */
  /* 2 x 2 diagonal matrix in host memory */
  const int32_t rp[3] = {0, 1, 2};
  const int32_t ci[2] = {0, 1};
  const double val[2] = {1.0, 2.0};
  krylov_csr A = {2, 2, rp, ci, val, 0};
  krylov_func f = {KRYLOV_F_EXP_NEG, 1.0};
  krylov_handle* h = (krylov_handle*)&A; /* must be reset to NULL on failure */
  if (krylov_create(&A, f, 1, 1, 1, 7, &opt, &h) != KRYLOV_EINVAL || h != NULL) return 12; /* s < m + 1 */
  h = (krylov_handle*)&A;
  krylov_status st = krylov_create(&A, f, 2, 2, 3, 7, &opt, &h);
  printf("%d\n", (int)st);
  if (st == KRYLOV_OK) {
    double b[2] = {1.0, 1.0}, x[2] = {0.0, 0.0};
    krylov_stats s;
    st = krylov_apply_host(h, b, x, 0.0, 1, &s);
    printf("%d %.17g %.17g\n", (int)st, x[0], x[1]);
    krylov_destroy(h);
  } else if (h != NULL) {
    return 13;
  }
  return 0;
}
"""


def test_header_compiles_as_c99_and_links(lib, tmp_path):
    """include/krylov.h is plain C: a C99 program that includes it builds with
    warnings as errors, links against the library and runs.  Without a GPU its
    create call reports KRYLOV_ECUDA; with one, exp(-A) b for the 2 x 2
    diagonal matrix is exact after one cycle of m = 2 (the whole space: a
    happy breakdown)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest

        pytest.skip("no C compiler")
    src = tmp_path / "use_krylov.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "use_krylov"
    libdir = ROOT / "paper_2503_22631_gb300"
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", str(ROOT / "include"), str(src),
                    "-L", str(libdir), "-lkrylov", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    lines = r.stdout.split("\n")
    import torch

    if torch.cuda.is_available():
        import math

        assert lines[0] == "0"
        st, x0, x1 = lines[1].split()
        assert int(st) >= 0
        assert abs(float(x0) - math.exp(-1.0)) < 1e-14 and abs(float(x1) - math.exp(-2.0)) < 1e-14
    else:
        assert lines[0] == "-3"  # KRYLOV_ECUDA: no device
