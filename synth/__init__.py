"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds no arithmetic of the relaxation method itself: it only draws
random numbers and shapes them into the data the paper's experiments describe
(Sec. 5.2: correlated Gaussian design, k equally spaced unit coefficients,
Gaussian noise at a given SNR; logistic labels are signs of a noisy linear
score).  The paper's own generator lives in its missing appendix, so the recipe
below is this project's reading of it (correlation Sigma_ij = rho^|i-j|, drawn
as an AR(1) recursion along each row).

Random numbers come from Philox4x64-10 (Salmon et al., "Parallel random numbers:
as easy as 1, 2, 3", SC'11) in numpy's stream layout: raw value r of a stream
with key (k0, k1) is lane r % 4 of the block computed from counter
(r // 4 + 1, 0, 0, 0).  Normals are Box-Muller pairs of consecutive raw values.
A CUDA implementation of the same definition (``synth/gen.cu``) produces the
multi-GB designs directly in device memory; it agrees with the numpy path up to
the last-ulp differences of the two platforms' log/sin/cos.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

# stream ids (second Philox key word)
STREAM_X = 1
STREAM_NOISE = 2
STREAM_PROX = 3
STREAM_FIX = 4
STREAM_WARM = 5


def raw_stream(seed: int, stream: int, count: int) -> np.ndarray:
    """First ``count`` raw uint64 values of the Philox4x64-10 stream (seed, stream)."""
    bg = np.random.Philox(key=np.array([seed, stream], dtype=np.uint64))
    return bg.random_raw(count).astype(np.uint64)


def normals(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` standard normals (float64) by Box-Muller on raw pairs.

    Normal 2s uses r*cos, normal 2s+1 uses r*sin of the pair (raw[2s], raw[2s+1]),
    with u1 = ((raw >> 11) + 1) * 2^-53 in (0, 1] and u2 = (raw >> 11) * 2^-53.
    """
    npairs = (count + 1) // 2
    raw = raw_stream(seed, stream, 2 * npairs)
    u1 = ((raw[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (raw[1::2] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * math.pi * u2
    out = np.empty(2 * npairs, dtype=np.float64)
    out[0::2] = r * np.cos(t)
    out[1::2] = r * np.sin(t)
    return out[:count]


def uniforms(seed: int, stream: int, count: int) -> np.ndarray:
    raw = raw_stream(seed, stream, count)
    return (raw >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def ar1_design(n: int, p: int, rho: float, seed: int, dtype=np.float64) -> np.ndarray:
    """Rows ~ N(0, Sigma), Sigma_ij = rho^|i-j|, via x_{i,0}=e_{i,0},
    x_{i,j} = rho x_{i,j-1} + sqrt(1-rho^2) e_{i,j} (FP64, then cast).

    e_{i,j} is normal number i*p + j of stream (seed, STREAM_X).
    """
    e = normals(seed, STREAM_X, n * p).reshape(n, p)
    c = math.sqrt(1.0 - rho * rho)
    x = np.empty((n, p), dtype=np.float64)
    x[:, 0] = e[:, 0]
    for j in range(1, p):
        x[:, j] = rho * x[:, j - 1] + c * e[:, j]
    return x.astype(dtype)


def support(p: int, k: int) -> np.ndarray:
    """Indices of the true nonzeros: floor(i*p/k), i = 0..k-1 (equally spaced)."""
    return np.array([(i * p) // k for i in range(k)], dtype=np.int64)


def response(signal: np.ndarray, loss: str, snr: float, seed: int) -> np.ndarray:
    """y from the noiseless score s = X beta* (beta* = 1 on the support).

    least squares: y = s + sigma e, sigma^2 = ||s||^2 / (n * snr);
    logistic: y = sign(s + 0.5 e) in {-1, +1}.
    """
    n = signal.shape[0]
    e = normals(seed, STREAM_NOISE, n)
    if loss == "ls":
        sigma = math.sqrt(float(np.dot(signal, signal)) / (n * snr))
        return signal + sigma * e
    if loss == "logistic":
        return np.where(signal + 0.5 * e >= 0.0, 1.0, -1.0)
    raise ValueError(loss)


def signal_from_design(X: np.ndarray, k: int) -> np.ndarray:
    """s_i = sum over the support of X[i, j] in increasing j (FP64)."""
    s = np.zeros(X.shape[0], dtype=np.float64)
    for j in support(X.shape[1], k):
        s += X[:, j].astype(np.float64)
    return s


def node_fixings(p: int, seed: int, node: int, j0_max: int, j1_max: int,
                 k: int | None = None) -> np.ndarray:
    """Random branch-and-bound node: |J0| ~ U{0..j0_max}, |J1| ~ U{0..j1_max}
    (J1 capped at k), on distinct coordinates.  -1 = J0, 0 = free, +1 = J1."""
    u = uniforms(seed + 1000003 * (node + 1), STREAM_FIX, p + 2)
    n0 = int(u[0] * (j0_max + 1))
    n1 = int(u[1] * (j1_max + 1))
    if k is not None:
        n1 = min(n1, k)
    order = np.argsort(u[2:], kind="stable")
    fix = np.zeros(p, dtype=np.int8)
    fix[order[:n0]] = -1
    fix[order[n0:n0 + n1]] = 1
    return fix


def prox_input(p: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """gamma ~ N(0, I_p) (the prox micro-benchmark recipe of Sec. 5.1)."""
    return scale * normals(seed, STREAM_PROX, p)


# ---------------------------------------------------------------------------
# problem configurations (the five synthetic workloads)
# ---------------------------------------------------------------------------
@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    p: int
    rho: float
    k: int
    lambda2: float
    loss: str = "ls"
    snr: float = 5.0
    M: float = 2.0
    dtype: str = "f32"
    gap_tol: float = 1e-6
    seed: int = 0
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    "ls_500x1000_f64": Workload("ls_500x1000_f64", 500, 1000, 0.5, 10, 1.0, "ls", 5.0,
                                dtype="f64", gap_tol=1e-8),
    "ls_20000x50000_f32": Workload("ls_20000x50000_f32", 20000, 50000, 0.9, 50, 0.1,
                                   "ls", 3.0),
    "logistic_20000x50000_f32": Workload("logistic_20000x50000_f32", 20000, 50000, 0.9,
                                         50, 0.1, "logistic", 3.0),
    # the same recipe on a fifth of the rows (800 MB of X, still far larger than
    # L2): the case counter captures of the fused pass run on
    "ls_4000x50000_f32": Workload("ls_4000x50000_f32", 4000, 50000, 0.9, 50, 0.1, "ls", 3.0),
    "batch256_5000x10000_f32": Workload("batch256_5000x10000_f32", 5000, 10000, 0.7, 20,
                                        0.5, "ls", 5.0,
                                        extra={"nodes": 256, "j0_max": 40, "j1_max": 19}),
    "logistic_100000x20000_lowp": Workload("logistic_100000x20000_lowp", 100000, 20000,
                                           0.5, 30, 0.1, "logistic", 5.0),
    # the same recipe on a quarter of the rows (2 GB of FP32 X, 1 GB as BF16):
    # the case counter captures of the quantized passes run on
    "logistic_25000x20000_lowp": Workload("logistic_25000x20000_lowp", 25000, 20000,
                                          0.5, 30, 0.1, "logistic", 5.0),
    "bnb_2000x5000_f32": Workload("bnb_2000x5000_f32", 2000, 5000, 0.8, 15, 0.2, "ls",
                                  5.0),
}
# The root-relaxation sweep of Sec. 5.2: n = p in {1000, ..., 16000}, rho 0.5,
# k 10, M 2, lambda2 1, SNR 5 (least squares and logistic), FP32 data.
for _p in (1000, 2000, 4000, 8000, 16000):
    for _loss in ("ls", "logistic"):
        _name = f"paper_{_loss}_{_p}x{_p}_f32"
        WORKLOADS[_name] = Workload(_name, _p, _p, 0.5, 10, 1.0, _loss, 5.0)


def make_problem_cpu(w: Workload, n: int | None = None, p: int | None = None,
                     dtype=None):
    """(X, y) on the host with the workload's recipe, optionally at a reduced size."""
    n = w.n if n is None else n
    p = w.p if p is None else p
    if dtype is None:
        dtype = np.float64 if w.dtype == "f64" else np.float32
    X = ar1_design(n, p, w.rho, w.seed, dtype)
    s = signal_from_design(X, w.k)
    y = response(s, w.loss, w.snr, w.seed).astype(dtype)
    return X, y


# ---------------------------------------------------------------------------
# device-side generator (large designs); loaded lazily, built by build()
# ---------------------------------------------------------------------------
_LIB = None


def _lib_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libsynth.so")


def load_gpu_lib():
    global _LIB
    if _LIB is None:
        path = _lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"synthetic-input GPU generator not built: {path}")
        lib = ctypes.CDLL(path)
        lib.synth_ar1_design.restype = ctypes.c_int
        lib.synth_ar1_design.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.c_double, ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
        lib.synth_signal.restype = ctypes.c_int
        lib.synth_signal.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_int64, ctypes.c_int, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_void_p]
        _LIB = lib
    return _LIB


def make_problem_gpu(w: Workload, device="cuda:0", n: int | None = None,
                     p: int | None = None, storage=None):
    """(X, y) built on the device (X row-major, leading dimension p).

    Returns torch tensors.  y is finished on the host from the device-computed
    signal (same FP64 summation order as the host recipe).
    """
    import torch
    n = w.n if n is None else n
    p = w.p if p is None else p
    tdt = torch.float64 if w.dtype == "f64" else torch.float32
    if storage is not None:
        tdt = storage
    lib = load_gpu_lib()
    X = torch.empty((n, p), dtype=tdt, device=device)
    stream = torch.cuda.current_stream(X.device).cuda_stream
    code = {torch.float64: 0, torch.float32: 1}[tdt]
    rc = lib.synth_ar1_design(ctypes.c_void_p(X.data_ptr()), n, p, p, float(w.rho),
                              w.seed, STREAM_X, code, ctypes.c_void_p(stream))
    if rc != 0:
        raise RuntimeError(f"synth_ar1_design failed: {rc}")
    sup = torch.tensor(support(p, w.k), dtype=torch.int64, device=device)
    s = torch.empty(n, dtype=torch.float64, device=device)
    rc = lib.synth_signal(ctypes.c_void_p(X.data_ptr()), n, p, p, code, w.k,
                          ctypes.c_void_p(sup.data_ptr()), ctypes.c_void_p(s.data_ptr()))
    if rc != 0:
        raise RuntimeError(f"synth_signal failed: {rc}")
    torch.cuda.synchronize(X.device)
    y = response(s.cpu().numpy(), w.loss, w.snr, w.seed)
    return X, torch.tensor(y, dtype=tdt, device=device)
