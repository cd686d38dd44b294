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
