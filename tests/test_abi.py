"""The C-ABI library loads without a GPU and exports every function declared in include/*.h."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(arbgpu_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("arbgpu_dot", "arbgpu_approx_dot", "arbgpu_mat_mul", "arbgpu_create",
                     "arbgpu_get_status",
                     "arbgpu_int_mat_mul"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build()
    from paper_1901_04289_gb300 import _lib
    L = _lib.lib()
    missing = [n for n in sorted(declared_functions()) if not hasattr(L, n)]
    assert not missing, missing
    assert set(_lib.exported_symbols()) <= declared_functions()
    assert L.arbgpu_version() >= 100


def test_status_strings_without_gpu():
    from paper_1901_04289_gb300 import _lib
    assert _lib.status_string(0) == "ok"
    assert "unsupported" in _lib.status_string(2)
