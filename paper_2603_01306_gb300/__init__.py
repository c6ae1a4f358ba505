"""GB300 node lower bounds for k-sparse GLMs (arxiv 2603.01306).

Thin ctypes binding of the C ABI in ``include/relax.h``: same entry-point
names, argument marshalling only.  Every step of the hot path runs in the CUDA
library ``_lib/librelax.so``; torch tensors supply device memory and streams.
There is no CPU fallback: calls fail when the library is not built.
"""
from .binding import (  # noqa: F401
    RELAX_F32, RELAX_F64, RELAX_BF16, RELAX_FP8E4M3, RELAX_LS, RELAX_LOGISTIC,
    RelaxError, Options, Result, Handle, load, lib_path, exported_symbols,
    relax_create, relax_solve, relax_xpass, relax_certify, relax_destroy,
    prox_persp, prox_persp_noalloc, gval_persp, gstar_persp, relax_strerror, relax_error_detail, STATUS,
    relax_mlp_forward, relax_mlp_grad, relax_mlp_adam, MLP_NTRAIN, MLP_NPARAM, relax_watchdog_probe,
)
