"""The C ABI library loads and exports every entry point include/relax.h declares
(no GPU needed: nothing here calls into CUDA)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*([a-z_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("relax_create", "relax_solve", "relax_destroy", "prox_persp", "relax_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2603_01306_gb300 as relax
    if not os.path.exists(relax.lib_path()):
        pytest.skip("library not built")
    lib = relax.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(relax.exported_symbols()) == sorted(set(relax.binding.EXPORTS))


def test_strerror_is_host_only():
    import paper_2603_01306_gb300 as relax
    if not os.path.exists(relax.lib_path()):
        pytest.skip("library not built")
    assert relax.relax_strerror(0) == "ok"
    assert "invalid" in relax.relax_strerror(1)
    assert relax.relax_strerror(999) == "unknown status"
