"""ctypes marshalling for the C ABI of ``include/relax.h``.

Only argument marshalling lives here: tensors become device pointers, the
current torch stream becomes the ``void* stream`` argument, C structs are
mirrored with ctypes.  Status codes other than RELAX_OK raise ``RelaxError``
(except where noted, where the code is returned with the result).
"""
from __future__ import annotations

import ctypes
import os

RELAX_LS, RELAX_LOGISTIC = 0, 1
RELAX_F64, RELAX_F32, RELAX_BF16, RELAX_FP8E4M3 = 0, 1, 2, 3
STATUS = {0: "RELAX_OK", 1: "RELAX_EINVAL", 2: "RELAX_ENOMEM", 3: "RELAX_ECUDA", 4: "RELAX_ENOTCONV",
          5: "RELAX_ETIMEOUT", 6: "RELAX_ENUMERIC", 7: "RELAX_EINVALID_BOUND", 8: "RELAX_ENOTSUP"}

EXPORTS = ["relax_create", "relax_solve", "relax_solve_batch", "relax_set_cutoff", "relax_xpass", "relax_batch_xpass",
           "relax_certify",
           "relax_certify_batch",
           "relax_destroy", "relax_watchdog_probe",
           "prox_persp", "prox_persp_noalloc", "gval_persp", "gstar_persp",
           "relax_mlp_features", "relax_mlp_forward", "relax_mlp_grad", "relax_mlp_adam",
           "relax_strerror", "relax_error_detail"]

# learned warm start (include/warmstart.h)
MLP_NTRAIN = 4609
MLP_NPARAM = 4619


class RelaxError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("M", ctypes.c_double), ("eta", ctypes.c_double), ("lipschitz", ctypes.c_double),
                ("max_iters", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("watchdog_ms", ctypes.c_int32), ("no_certify", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("timing", ctypes.c_int32),
                ("stall_window", ctypes.c_int32), ("method", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("step_rule", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class Result(ctypes.Structure):
    _fields_ = [("primal", ctypes.c_double), ("dual_bound", ctypes.c_double), ("gap", ctypes.c_double),
                ("rel_gap", ctypes.c_double), ("primal_loop", ctypes.c_double),
                ("dual_loop", ctypes.c_double), ("lipschitz", ctypes.c_double),
                ("iters", ctypes.c_int32), ("restarts", ctypes.c_int32), ("status", ctypes.c_int32),
                ("n_nz", ctypes.c_int32), ("launches", ctypes.c_int32), ("xpass_count", ctypes.c_int32),
                ("xpass_ms", ctypes.c_double), ("pphase_ms", ctypes.c_double),
                ("stalled", ctypes.c_int32), ("polish_iters", ctypes.c_int32),
                ("cutoff_rule", ctypes.c_int32), ("backtracks", ctypes.c_int32), ("ladder", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_LIB = None


def lib_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "librelax.so")


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    lib.relax_create.argtypes = [ctypes.POINTER(vp), vp, vp, i64, i64, i64, i32, i32, i32, dbl,
                                 ctypes.POINTER(Options), vp]
    lib.relax_solve.argtypes = [vp, vp, vp, dbl, vp, ctypes.POINTER(Result)]
    lib.relax_xpass.argtypes = [vp, vp, vp, vp, ctypes.POINTER(dbl)]
    lib.relax_batch_xpass.argtypes = [vp, i32, vp, vp, vp, ctypes.POINTER(dbl)]
    lib.relax_set_cutoff.argtypes = [vp, dbl]
    lib.relax_watchdog_probe.argtypes = [i32, ctypes.POINTER(dbl), vp]
    lib.relax_solve_batch.argtypes = [vp, i32, vp, vp, dbl, vp, vp]
    lib.relax_certify.argtypes = [vp, vp, vp, vp, ctypes.POINTER(dbl)]
    lib.relax_certify_batch.argtypes = [vp, i32, vp, vp, ctypes.POINTER(dbl)]
    lib.relax_certify_batch.restype = i32
    lib.relax_destroy.argtypes = [vp]
    lib.prox_persp.argtypes = [vp, vp, i64, dbl, i32, dbl, dbl, vp, i32, vp, vp]
    lib.prox_persp_noalloc.argtypes = [vp, vp, i64, dbl, i32, dbl, dbl, vp, i32, vp, vp]
    lib.gval_persp.argtypes = [vp, i64, i32, dbl, vp, i32, ctypes.POINTER(dbl), vp]
    lib.gstar_persp.argtypes = [vp, i64, i32, dbl, vp, i32, ctypes.POINTER(dbl), vp]
    lib.relax_mlp_features.argtypes = [vp, vp, vp, vp]
    lib.relax_mlp_forward.argtypes = [vp, i32, vp, vp, i64, vp, vp]
    lib.relax_mlp_grad.argtypes = [vp, i32, vp, vp, vp, i64, vp, vp, vp]
    lib.relax_mlp_adam.argtypes = [vp, vp, vp, vp, i32, dbl, dbl, dbl, dbl, vp]
    lib.relax_strerror.argtypes = [ctypes.c_int]
    lib.relax_strerror.restype = ctypes.c_char_p
    lib.relax_error_detail.argtypes = []
    lib.relax_error_detail.restype = ctypes.c_char_p
    for name in EXPORTS[:-2]:
        getattr(lib, name).restype = ctypes.c_int
    _LIB = lib
    return lib


def exported_symbols() -> list[str]:
    """Names of the C entry points present in the shared library."""
    lib = load()
    return [n for n in EXPORTS if hasattr(lib, n)]


def relax_strerror(code: int) -> str:
    return load().relax_strerror(code).decode()


def relax_error_detail() -> str:
    return load().relax_error_detail().decode()


def _check(code: int, what: str):
    if code != 0:
        detail = relax_error_detail()
        raise RelaxError(code, f"{what} ({detail})" if detail else what)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device=None):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dtype_code(t):
    import torch
    if t.dtype == torch.float64:
        return RELAX_F64
    if t.dtype == torch.float32:
        return RELAX_F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("tensors must live on the GPU")


METHODS = {"fista": 0, "pgd": 1}
RESTARTS = {"gap": 0, "function": 1, "none": 2}
STEP_RULES = {"fixed": 0, "backtracking": 1}


def make_options(M=2.0, eta=0.0, lipschitz=0.0, max_iters=0, precision=0, watchdog_ms=0,
                 certify=True, chunk=0, timing=False, stall_window=0, method="fista", restart="gap",
                 step="fixed") -> Options:
    o = Options()
    o.M = float(M)
    o.eta = float(eta)
    o.lipschitz = float(lipschitz)
    o.max_iters = int(max_iters)
    o.precision = int(precision)
    o.watchdog_ms = int(watchdog_ms)
    o.no_certify = 0 if certify else 1
    o.chunk = int(chunk)
    o.timing = 1 if timing else 0
    o.stall_window = int(stall_window)
    o.method = METHODS[method] if isinstance(method, str) else int(method)
    o.restart = RESTARTS[restart] if isinstance(restart, str) else int(restart)
    o.step_rule = STEP_RULES[step] if isinstance(step, str) else int(step)
    return o


def relax_create(X, y, loss, k, lambda2, options: Options | None = None):
    """relax_create: X (n x p, row-major, ldx = X.stride(0)) and y on the GPU."""
    _need_cuda(X, y)
    if X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be a row-major 2-D tensor")
    h = ctypes.c_void_p()
    lib = load()
    code = lib.relax_create(ctypes.byref(h), _ptr(X), _ptr(y), X.shape[0], X.shape[1], X.stride(0),
                            _dtype_code(X), int(loss), int(k), float(lambda2),
                            ctypes.byref(options) if options is not None else None, _stream(X.device))
    _check(code, "relax_create")
    return h


def relax_solve(h, fixings, warm_start, gap_tol, beta_out):
    """relax_solve; returns (status_code, Result) -- ENOTCONV etc. are not raised."""
    _need_cuda(fixings, warm_start, beta_out)
    res = Result()
    code = load().relax_solve(h, _ptr(fixings), _ptr(warm_start), float(gap_tol), _ptr(beta_out),
                              ctypes.byref(res))
    if code in (1, 2, 3, 8):
        _check(code, "relax_solve")
    return code, res


def relax_xpass(h, beta, z_out, g_out):
    _need_cuda(beta, z_out, g_out)
    loss = (ctypes.c_double * 2)()
    _check(load().relax_xpass(h, _ptr(beta), _ptr(z_out), _ptr(g_out), loss), "relax_xpass")
    return float(loss[0]), float(loss[1])


def relax_certify(h, fixings, beta_primal, beta_dual):
    _need_cuda(fixings, beta_primal, beta_dual)
    out = (ctypes.c_double * 2)()
    _check(load().relax_certify(h, _ptr(fixings), _ptr(beta_primal), _ptr(beta_dual), out),
           "relax_certify")
    return float(out[0]), float(out[1])


def relax_mlp_forward(theta, feat, out, base=None, bf16=True):
    """out = base + f(feat) (f alone when base is None); float32 device tensors."""
    _need_cuda(theta, feat, base, out)
    _f32(theta, feat, base, out)
    rows = feat.shape[0]
    _check(load().relax_mlp_forward(_ptr(theta), 1 if bf16 else 0, _ptr(feat), _ptr(base), int(rows), _ptr(out),
                                    _stream(feat.device)), "relax_mlp_forward")
    return out


def relax_mlp_grad(theta, feat, base, target, grad, loss=None, bf16=True):
    """grad (and loss, a 1-element tensor) of mean (base + f(feat) - target)^2."""
    _need_cuda(theta, feat, base, target, grad, loss)
    _f32(theta, feat, base, target, grad, loss)
    _check(load().relax_mlp_grad(_ptr(theta), 1 if bf16 else 0, _ptr(feat), _ptr(base), _ptr(target),
                                 int(feat.shape[0]), _ptr(grad), _ptr(loss), _stream(feat.device)),
           "relax_mlp_grad")
    return grad


def relax_mlp_adam(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _need_cuda(theta, grad, m, v)
    _f32(theta, grad, m, v)
    _check(load().relax_mlp_adam(_ptr(theta), _ptr(grad), _ptr(m), _ptr(v), int(t), float(lr), float(beta1),
                                 float(beta2), float(eps), _stream(theta.device)), "relax_mlp_adam")


def _f32(*ts):
    import torch
    for t in ts:
        if t is not None and (t.dtype != torch.float32 or not t.is_contiguous()):
            raise TypeError("warm-start network buffers are contiguous float32 tensors")


def relax_watchdog_probe(watchdog_ms):
    """(status code, device ms waited) of the bounded-wait diagnostic."""
    waited = ctypes.c_double(0.0)
    code = load().relax_watchdog_probe(int(watchdog_ms), ctypes.byref(waited), _stream())
    if code not in (0, 5):
        _check(code, "relax_watchdog_probe")
    return code, waited.value


def relax_destroy(h):
    _check(load().relax_destroy(h), "relax_destroy")


def prox_persp(beta_in, beta_out, step, k, lambda2, M, fixings=None, counts_out=None):
    _need_cuda(beta_in, beta_out, fixings, counts_out)
    code = load().prox_persp(_ptr(beta_in), _ptr(beta_out), beta_in.numel(), float(step), int(k),
                             float(lambda2), float(M), _ptr(fixings), _dtype_code(beta_in),
                             _ptr(counts_out), _stream(beta_in.device))
    _check(code, "prox_persp")


def prox_persp_noalloc(beta_in, beta_out, step, k, lambda2, M, fixings=None, counts_out=None):
    """prox_persp with its scratch in the library's fixed device array (no allocation)."""
    _need_cuda(beta_in, beta_out, fixings, counts_out)
    code = load().prox_persp_noalloc(_ptr(beta_in), _ptr(beta_out), beta_in.numel(), float(step), int(k),
                                     float(lambda2), float(M), _ptr(fixings), _dtype_code(beta_in),
                                     _ptr(counts_out), _stream(beta_in.device))
    _check(code, "prox_persp_noalloc")


def gval_persp(beta, k, M, fixings=None) -> float:
    _need_cuda(beta, fixings)
    out = ctypes.c_double()
    _check(load().gval_persp(_ptr(beta), beta.numel(), int(k), float(M), _ptr(fixings),
                             _dtype_code(beta), ctypes.byref(out), _stream(beta.device)),
           "gval_persp")
    return out.value


def gstar_persp(alpha, k, M, fixings=None) -> float:
    _need_cuda(alpha, fixings)
    out = ctypes.c_double()
    _check(load().gstar_persp(_ptr(alpha), alpha.numel(), int(k), float(M), _ptr(fixings),
                              _dtype_code(alpha), ctypes.byref(out), _stream(alpha.device)),
           "gstar_persp")
    return out.value


class Handle:
    """Owns a relax_handle; X and y must outlive it."""

    def __init__(self, X, y, loss="ls", k=10, lambda2=1.0, M=2.0, eta=0.0, lipschitz=0.0,
                 max_iters=0, precision=0, certify=True, chunk=0, watchdog_ms=0, timing=False,
                 stall_window=0, method="fista", restart="gap", step="fixed"):
        self.loss = {"ls": RELAX_LS, "logistic": RELAX_LOGISTIC}[loss] if isinstance(loss, str) else loss
        self.X, self.y = X, y
        self.n, self.p = X.shape
        self.dtype = X.dtype
        self.opts = make_options(M=M, eta=eta, lipschitz=lipschitz, max_iters=max_iters,
                                 precision=precision, watchdog_ms=watchdog_ms, certify=certify,
                                 chunk=chunk, timing=timing, stall_window=stall_window, method=method,
                                 restart=restart, step=step)
        self.h = relax_create(X, y, self.loss, k, lambda2, self.opts)

    def _vec(self, t, what, rows=None, dtype=None):
        """The C ABI takes bare pointers: check what it cannot (element type,
        length, contiguity) before a buffer is handed over."""
        if t is None:
            return
        import torch
        want = self.dtype if dtype is None else dtype
        shape = (self.p,) if rows is None else (rows, self.p)
        if t.dtype != want:
            raise TypeError(f"{what}: dtype {t.dtype}, expected {want}")
        if tuple(t.shape) != shape and not (rows is None and t.numel() == self.p):
            raise ValueError(f"{what}: shape {tuple(t.shape)}, expected {shape}")
        if not t.is_contiguous():
            raise ValueError(f"{what}: must be contiguous")

    def solve(self, fixings=None, warm_start=None, gap_tol=1e-6, beta_out=None):
        import torch
        if beta_out is None:
            beta_out = torch.empty(self.p, dtype=self.dtype, device=self.X.device)
        self._vec(fixings, "fixings", dtype=torch.int8)
        self._vec(warm_start, "warm_start")
        self._vec(beta_out, "beta_out")
        code, res = relax_solve(self.h, fixings, warm_start, gap_tol, beta_out)
        return beta_out, res, code

    def solve_batch(self, nb, fixings=None, warm_start=None, gap_tol=1e-6, beta_out=None):
        """relax_solve_batch: nb node relaxations sharing X.  fixings: (nb, p)
        int8 device tensor or None; warm_start: (nb, p) or None.  Returns
        (beta (nb, p), [Result per node], status code)."""
        import torch
        _need_cuda(fixings, warm_start)
        if beta_out is None:
            beta_out = torch.empty((nb, self.p), dtype=self.dtype, device=self.X.device)
        self._vec(fixings, "fixings", rows=nb, dtype=torch.int8)
        self._vec(warm_start, "warm_start", rows=nb)
        self._vec(beta_out, "beta_out", rows=nb)
        res = (Result * nb)()
        code = load().relax_solve_batch(self.h, int(nb), _ptr(fixings), _ptr(warm_start), float(gap_tol),
                                        _ptr(beta_out), res)
        if code not in (0, 4):
            _check(code, "relax_solve_batch")
        return beta_out, list(res), code

    def xpass(self, beta):
        import torch
        self._vec(beta, "beta")
        z = torch.empty(self.n, dtype=self.dtype, device=self.X.device)
        g = torch.empty(self.p, dtype=self.dtype, device=self.X.device)
        loss = relax_xpass(self.h, beta, z, g)
        return z, g, loss

    def batch_xpass(self, points, timing=False):
        """relax_batch_xpass: (z, g) = (X b_s, X' X b_s) for the rows b_s of
        `points` (nb x p, the handle's dtype), as FP64 device tensors; with
        timing also the device ms of the two tensor-core launches."""
        import torch
        nb = points.shape[0]
        self._vec(points, "points", rows=nb)
        z = torch.empty((nb, self.n), dtype=torch.float64, device=self.X.device)
        g = torch.empty((nb, self.p), dtype=torch.float64, device=self.X.device)
        ms = (ctypes.c_double * 2)()
        _check(load().relax_batch_xpass(self.h, int(nb), _ptr(points), _ptr(z), _ptr(g), ms if timing else None),
               "relax_batch_xpass")
        return (z, g, (ms[0], ms[1])) if timing else (z, g)

    def set_cutoff(self, cutoff=float("inf")):
        """Dynamic termination against the incumbent's objective (inf: off)."""
        _check(load().relax_set_cutoff(self.h, float(cutoff)), "relax_set_cutoff")

    def mlp_features(self, beta_parent, fixings=None, out=None):
        """(p, 5) float32 features of a child node (include/warmstart.h)."""
        import torch
        self._vec(beta_parent, "beta_parent")
        self._vec(fixings, "fixings", dtype=torch.int8)
        if out is None:
            out = torch.empty((self.p, 5), dtype=torch.float32, device=self.X.device)
        _f32(out)
        _check(load().relax_mlp_features(self.h, _ptr(beta_parent), _ptr(fixings), _ptr(out)), "relax_mlp_features")
        return out

    def certify(self, beta_primal, beta_dual=None, fixings=None):
        import torch
        self._vec(beta_primal, "beta_primal")
        self._vec(beta_dual, "beta_dual")
        self._vec(fixings, "fixings", dtype=torch.int8)
        return relax_certify(self.h, fixings, beta_primal,
                             beta_primal if beta_dual is None else beta_dual)

    def certify_batch(self, points, fixings=None):
        """relax_certify_batch: (nb, 2) float64 numpy array {Phi(b_s), Psi(-grad F(X b_s))}
        for the rows b_s of points (nb x p, handle dtype); fixings (nb, p) int8 or None."""
        import numpy as np
        import torch
        nb = int(points.shape[0])
        self._vec(points, "points", rows=nb)
        self._vec(fixings, "fixings", rows=nb, dtype=torch.int8)
        out = (ctypes.c_double * (2 * nb))()
        _check(load().relax_certify_batch(self.h, nb, _ptr(fixings), _ptr(points), out), "relax_certify_batch")
        return np.frombuffer(out, dtype=np.float64).reshape(nb, 2).copy()

    def close(self):
        if self.h is not None:
            relax_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

