"""Argument checks of the C ABI (include/relax.h): every entry point rejects
invalid arguments with RELAX_EINVAL before it touches the GPU, so these run on
the CPU through the raw ctypes functions (the binding's own type checks are
bypassed on purpose).  Pointers passed here are never dereferenced: each call
fails its argument validation first."""
import ctypes
import math
import os

import pytest

import paper_2603_01306_gb300 as relax
from paper_2603_01306_gb300 import binding as B

EINVAL = 1

pytestmark = pytest.mark.skipif(not os.path.exists(relax.lib_path()), reason="library not built")

FAKE = ctypes.c_void_p(0x1000)      # a non-null pointer that validation never follows


def _create(**kw):
    a = dict(out=True, X=FAKE, y=FAKE, n=10, p=20, ldx=20, dtype=B.RELAX_F32, loss=B.RELAX_LS, k=3,
             lambda2=0.5, opt=None)
    a.update(kw)
    h = ctypes.c_void_p()
    opt = ctypes.byref(a["opt"]) if a["opt"] is not None else None
    return relax.load().relax_create(ctypes.byref(h) if a["out"] else None, a["X"], a["y"], a["n"], a["p"],
                                     a["ldx"], a["dtype"], a["loss"], a["k"], a["lambda2"], opt, None)


@pytest.mark.parametrize("bad", [
    dict(out=False), dict(X=None), dict(y=None), dict(n=0), dict(p=-1), dict(ldx=19), dict(k=0),
    dict(lambda2=0.0), dict(lambda2=-1.0), dict(lambda2=math.nan), dict(dtype=7), dict(dtype=B.RELAX_BF16),
    dict(loss=2),
])
def test_create_rejects_invalid_arguments(bad):
    assert _create(**bad) == EINVAL


@pytest.mark.parametrize("field,value", [("M", -1.0), ("M", math.nan), ("eta", -2.0), ("lipschitz", -1.0),
                                         ("max_iters", -5), ("watchdog_ms", -1), ("chunk", -3), ("method", 2),
                                         ("method", -1), ("restart", 3), ("step_rule", 2), ("step_rule", -1)])
def test_create_rejects_invalid_options(field, value):
    o = B.make_options()
    setattr(o, field, value)
    assert _create(opt=o) == EINVAL


def test_create_rejects_low_precision_of_f64_data():
    # BF16 / FP8 loop storage is a quantized copy of FP32 data only
    o = B.make_options(precision=B.RELAX_BF16)
    assert _create(dtype=B.RELAX_F64, opt=o) == EINVAL
    o = B.make_options(precision=B.RELAX_FP8E4M3)
    assert _create(dtype=B.RELAX_F64, opt=o) == EINVAL


def test_solve_and_batch_reject_invalid_arguments():
    lib = relax.load()
    res = B.Result()
    res_arr = (B.Result * 2)()
    assert lib.relax_solve(None, None, None, 1e-6, FAKE, ctypes.byref(res)) == EINVAL        # no handle
    assert lib.relax_solve(FAKE, None, None, 0.0, FAKE, ctypes.byref(res)) == EINVAL         # gap_tol <= 0
    assert lib.relax_solve(FAKE, None, None, -1.0, FAKE, ctypes.byref(res)) == EINVAL
    assert lib.relax_solve(FAKE, None, None, math.nan, FAKE, ctypes.byref(res)) == EINVAL
    assert lib.relax_solve(FAKE, None, None, 1e-6, None, ctypes.byref(res)) == EINVAL        # no beta_out
    assert lib.relax_solve(FAKE, None, None, 1e-6, FAKE, None) == EINVAL                     # no result
    assert lib.relax_solve_batch(None, 2, None, None, 1e-6, FAKE, res_arr) == EINVAL
    assert lib.relax_solve_batch(FAKE, 0, None, None, 1e-6, FAKE, res_arr) == EINVAL         # nb <= 0
    assert lib.relax_solve_batch(FAKE, 2, None, None, 0.0, FAKE, res_arr) == EINVAL
    assert lib.relax_solve_batch(FAKE, 2, None, None, 1e-6, None, res_arr) == EINVAL
    assert lib.relax_solve_batch(FAKE, 2, None, None, 1e-6, FAKE, None) == EINVAL
    assert lib.relax_batch_xpass(None, 2, FAKE, FAKE, FAKE, None) == EINVAL
    assert lib.relax_batch_xpass(FAKE, 0, FAKE, FAKE, FAKE, None) == EINVAL
    assert lib.relax_batch_xpass(FAKE, 2, None, FAKE, FAKE, None) == EINVAL
    assert lib.relax_batch_xpass(FAKE, 2, FAKE, None, FAKE, None) == EINVAL
    assert lib.relax_batch_xpass(FAKE, 2, FAKE, FAKE, None, None) == EINVAL
    assert lib.relax_set_cutoff(None, 1.0) == EINVAL
    assert lib.relax_set_cutoff(FAKE, math.nan) == EINVAL
    assert lib.relax_xpass(None, FAKE, None, FAKE, None) == EINVAL
    assert lib.relax_xpass(FAKE, None, None, FAKE, None) == EINVAL
    out2 = (ctypes.c_double * 2)()
    assert lib.relax_certify(FAKE, None, None, FAKE, out2) == EINVAL
    assert lib.relax_certify(FAKE, None, FAKE, FAKE, None) == EINVAL
    assert lib.relax_destroy(None) == EINVAL
    waited = ctypes.c_double()
    assert lib.relax_watchdog_probe(0, ctypes.byref(waited), None) == EINVAL
    assert lib.relax_watchdog_probe(60001, ctypes.byref(waited), None) == EINVAL


@pytest.mark.parametrize("fn", ["prox_persp", "prox_persp_noalloc"])
def test_prox_rejects_invalid_arguments(fn):
    f = getattr(relax.load(), fn)
    F64 = B.RELAX_F64
    good = dict(vin=FAKE, vout=FAKE, p=100, step=0.1, k=5, lam2=1.0, M=2.0, fix=None, dtype=F64, counts=None)

    def call(**kw):
        a = dict(good)
        a.update(kw)
        return f(a["vin"], a["vout"], a["p"], a["step"], a["k"], a["lam2"], a["M"], a["fix"], a["dtype"],
                 a["counts"], None)
    for bad in (dict(vin=None), dict(vout=None), dict(p=0), dict(p=-3), dict(step=0.0), dict(step=math.nan),
                dict(k=-1), dict(lam2=0.0), dict(M=0.0), dict(M=-1.0), dict(M=math.nan), dict(dtype=B.RELAX_BF16),
                dict(dtype=9)):
        assert call(**bad) == EINVAL, bad


def test_regularizer_values_reject_invalid_arguments():
    lib = relax.load()
    out = ctypes.c_double()
    F64 = B.RELAX_F64
    assert lib.gval_persp(FAKE, 10, 2, 1.0, None, F64, None, None) == EINVAL       # no output
    assert lib.gval_persp(None, 10, 2, 1.0, None, F64, ctypes.byref(out), None) == EINVAL
    assert lib.gval_persp(FAKE, 0, 2, 1.0, None, F64, ctypes.byref(out), None) == EINVAL
    assert lib.gval_persp(FAKE, 10, 2, 0.0, None, F64, ctypes.byref(out), None) == EINVAL
    assert lib.gstar_persp(FAKE, 10, -1, 1.0, None, F64, ctypes.byref(out), None) == EINVAL
    assert lib.gstar_persp(FAKE, 10, 2, 1.0, None, 5, ctypes.byref(out), None) == EINVAL
