"""GLM losses F(z) = f(z, y), their gradients and Fenchel conjugates (FP64 oracle).

The paper's per-loss formulas are in its missing appendix; this oracle reads them
as (Sec. 2.3 problem (1) pairs f with lambda2 ||beta||^2, no intercept):
  least squares  F(z) = ||y - z||^2,            F*(w) = w'y + ||w||^2 / 4;
  logistic       F(z) = sum log(1 + exp(-y_i z_i)), y_i in {-1, +1},
                 F*(w) = sum [u log u + (1-u) log(1-u)], u_i = -y_i w_i in [0, 1].
"""
from __future__ import annotations

import numpy as np


def F(z, y, loss):
    z = np.asarray(z, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if loss == "ls":
        r = y - z
        return float(np.dot(r, r))
    if loss == "logistic":
        return float(np.sum(np.logaddexp(0.0, -y * z)))
    raise ValueError(loss)


def grad_F(z, y, loss):
    z = np.asarray(z, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if loss == "ls":
        return 2.0 * (z - y)
    if loss == "logistic":
        # d/dz log(1 + exp(-y z)) = -y / (1 + exp(y z))
        return -y * np.exp(-np.logaddexp(0.0, y * z))
    raise ValueError(loss)


def _xlogx(u):
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    m = u > 0
    out[m] = u[m] * np.log(u[m])
    return out


def F_conj(w, y, loss):
    """F*(w) = sup_z w'z - F(z); +inf outside its domain (logistic)."""
    w = np.asarray(w, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if loss == "ls":
        return float(np.dot(w, y) + 0.25 * np.dot(w, w))
    if loss == "logistic":
        u = -y * w
        if np.any(u < 0) or np.any(u > 1):
            return float("inf")
        return float(np.sum(_xlogx(u) + _xlogx(1.0 - u)))
    raise ValueError(loss)


def lipschitz_factor(loss):
    """Curvature bound of f in z: 2 for least squares, 1/4 for logistic."""
    return {"ls": 2.0, "logistic": 0.25}[loss]
