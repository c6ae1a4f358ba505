"""Exact references for tiny instances (FP64 oracle).

* ``ridge``: problem (1) with k >= p and M = inf is ridge regression; with
  F = ||y - X beta||^2 its minimizer solves (X'X + lambda2 I) beta = X'y.
* ``ksparse_opt``: the true optimum of problem (1) at a node (J1 in the support,
  J0 out of it) by enumerating every support S with |S| <= k and solving the
  box-constrained restricted problem on S.  The relaxation's bound can never
  exceed it.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from scipy.optimize import minimize

from . import losses


def ridge(X, y, lambda2):
    X = np.asarray(X, dtype=np.float64)
    p = X.shape[1]
    return np.linalg.solve(X.T @ X + lambda2 * np.eye(p), X.T @ np.asarray(y, np.float64))


def restricted_opt(X, y, loss, lambda2, M, S):
    """min over beta_S of F(X_S beta_S) + lambda2 ||beta_S||^2, |beta_S| <= M."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    S = list(S)
    if not S:
        return losses.F(np.zeros(X.shape[0]), y, loss), np.zeros(0)
    XS = X[:, S]

    def fun(b):
        z = XS @ b
        val = losses.F(z, y, loss) + lambda2 * float(b @ b)
        grad = XS.T @ losses.grad_F(z, y, loss) + 2.0 * lambda2 * b
        return val, grad

    bounds = None if math.isinf(M) else [(-M, M)] * len(S)
    res = minimize(fun, np.zeros(len(S)), jac=True, method="L-BFGS-B", bounds=bounds,
                   options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 10000})
    return float(res.fun), res.x


def ksparse_opt(X, y, loss, k, lambda2, M, fix=None):
    p = np.asarray(X).shape[1]
    fix = np.zeros(p, dtype=np.int8) if fix is None else np.asarray(fix, dtype=np.int8)
    J1 = [j for j in range(p) if fix[j] > 0]
    Jf = [j for j in range(p) if fix[j] == 0]
    best = math.inf
    for extra in range(0, max(0, k - len(J1)) + 1):
        for comb in itertools.combinations(Jf, extra):
            val, _ = restricted_opt(X, y, loss, lambda2, M, sorted(J1 + list(comb)))
            best = min(best, val)
    return best
