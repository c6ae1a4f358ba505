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


def test_handle_rejects_mistyped_buffers():
    """The C ABI takes bare pointers; the binding checks element type, length
    and contiguity before handing a buffer over (an FP64 warm start given to
    an FP32 handle would otherwise be read as FP32 words)."""
    torch = pytest.importorskip("torch")
    from paper_2603_01306_gb300.binding import Handle
    h = object.__new__(Handle)
    h.h, h.p, h.dtype = None, 5, torch.float32
    h._vec(torch.zeros(5, dtype=torch.float32), "warm_start")
    h._vec(torch.zeros((3, 5), dtype=torch.int8), "fixings", rows=3, dtype=torch.int8)
    with pytest.raises(TypeError):
        h._vec(torch.zeros(5, dtype=torch.float64), "warm_start")
    with pytest.raises(TypeError):
        h._vec(torch.zeros(5, dtype=torch.int32), "fixings", dtype=torch.int8)
    with pytest.raises(ValueError):
        h._vec(torch.zeros(6, dtype=torch.float32), "beta_out")
    with pytest.raises(ValueError):
        h._vec(torch.zeros((2, 5), dtype=torch.float32), "warm_start", rows=3)
    with pytest.raises(ValueError):
        h._vec(torch.zeros((5, 2), dtype=torch.float32)[:, 0], "beta")
