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


def _c_struct_fields(src, name):
    """(type, field) pairs of `typedef struct { ... } name;` in a header."""
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + ";", src).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        m = re.match(r"([A-Za-z0-9_]+)\s+([A-Za-z0-9_]+)(\[(\d+)\])?$", decl)
        assert m, decl
        out.append((m.group(1), m.group(2), int(m.group(4)) if m.group(4) else None))
    return out


def test_ctypes_mirrors_match_the_header_structs():
    """relax_options and relax_result as the binding mirrors them: same fields,
    same order, same C types (a drift here would shift every later field)."""
    import ctypes
    from paper_2603_01306_gb300.binding import Options, Result
    src = open(os.path.join(ROOT, "include", "relax.h")).read()
    ctype = {"double": ctypes.c_double, "int32_t": ctypes.c_int32}
    for cls, name in ((Options, "relax_options"), (Result, "relax_result")):
        fields = _c_struct_fields(src, name)
        assert [f for _, f, _ in fields] == [f for f, _ in cls._fields_], name
        for (ct, f, n), (pf, pt) in zip(fields, cls._fields_):
            want = ctype[ct] * n if n else ctype[ct]
            assert ctypes.sizeof(pt) == ctypes.sizeof(want) and getattr(pt, "_type_", pt) == getattr(want, "_type_", want), f


def test_constants_match_the_headers():
    """Status codes, loss and dtype codes, and the warm-start parameter sizes
    as the binding spells them."""
    from paper_2603_01306_gb300 import binding as B
    src = open(os.path.join(ROOT, "include", "relax.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    enum = dict((k, int(v)) for k, v in re.findall(r"\b(RELAX_[A-Z0-9_]+)\s*=\s*(\d+)", src))
    for code, name in B.STATUS.items():
        assert enum[name] == code, name
    assert (enum["RELAX_LS"], enum["RELAX_LOGISTIC"]) == (B.RELAX_LS, B.RELAX_LOGISTIC)
    assert (enum["RELAX_F64"], enum["RELAX_F32"], enum["RELAX_BF16"], enum["RELAX_FP8E4M3"]) == \
        (B.RELAX_F64, B.RELAX_F32, B.RELAX_BF16, B.RELAX_FP8E4M3)
    ws = open(os.path.join(ROOT, "include", "warmstart.h")).read()
    defs = dict((k, int(v)) for k, v in re.findall(r"#define (RELAX_MLP_[A-Z]+) (\d+)", ws))
    assert (defs["RELAX_MLP_NTRAIN"], defs["RELAX_MLP_NPARAM"]) == (B.MLP_NTRAIN, B.MLP_NPARAM)
