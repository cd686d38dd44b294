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
