"""FISTA with duality-gap restarts for the node perspective relaxation (FP64 oracle).

Primal (Eq. 6):  Phi(beta) = F(X beta) + G(beta),  G = 2*lambda2*g_N.
Dual   (Eq. 7):  Psi(zeta) = -F*(-zeta) - G*(X' zeta),  G*(w) = 2*lambda2*g_N*(w / (2*lambda2)).
Induced dual point (Sec. 3.3): zeta = -grad F(X beta).
FISTA (Beck 2017, Sec. 10.7) with fixed step s = 1/L, L = c_f * ||X||_2^2
(c_f = 2 least squares, 1/4 logistic).  Gap-based restart (Sec. 3.4): restart
when Phi(beta^t) - Psi(zeta^t) <= (Phi(beta^0) - Psi(zeta^0)) / eta, where
beta^0 is the epoch's starting point; eta = e^3 by default (Sec. 5.2).  Stop when
the best certified gap (min Phi - max Psi) is <= gap_tol * max(1, |min Phi|).

Every quantity is computed by separate plain matrix-vector products; nothing
is fused or reordered.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import losses, regularizer


def spectral_norm_sq(X, iters=200, seed=12345):
    """||X||_2^2 by power iteration on X'X (FP64); exact SVD for small X."""
    X = np.asarray(X, dtype=np.float64)
    if X.shape[0] * X.shape[1] <= 4_000_000:
        return float(np.linalg.norm(X, 2) ** 2)
    v = np.random.default_rng(seed).standard_normal(X.shape[1])
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = X.T @ (X @ v)
        lam_new = float(np.linalg.norm(w))
        v = w / lam_new
        if abs(lam_new - lam) <= 1e-12 * lam_new:
            lam = lam_new
            break
        lam = lam_new
    return lam


def lipschitz(X, loss):
    return losses.lipschitz_factor(loss) * spectral_norm_sq(X)


def primal(beta, X, y, loss, fix, k, M, lambda2):
    """Phi(beta) = F(X beta) + 2 lambda2 g_N(beta) (Eq. 6)."""
    z = np.asarray(X, dtype=np.float64) @ beta
    return losses.F(z, y, loss) + 2.0 * lambda2 * regularizer.g_alg1(beta, fix, k, M)


def dual(zeta, X, y, loss, fix, k, M, lambda2):
    """Psi(zeta) = -F*(-zeta) - 2 lambda2 g_N*(X' zeta / (2 lambda2)) (Eq. 7)."""
    w = np.asarray(X, dtype=np.float64).T @ zeta
    return (-losses.F_conj(-zeta, y, loss)
            - 2.0 * lambda2 * regularizer.gstar(w / (2.0 * lambda2), fix, k, M))


def induced_dual(beta, X, y, loss):
    """zeta = -grad F(X beta) (Sec. 3.3)."""
    return -losses.grad_F(np.asarray(X, dtype=np.float64) @ beta, y, loss)


@dataclass
class Result:
    beta: np.ndarray            # primal point with the smallest Phi seen
    primal: float               # min Phi
    dual_bound: float           # max Psi (a valid lower bound by weak duality)
    gap: float                  # primal - dual_bound
    rel_gap: float
    iters: int
    restarts: int
    converged: bool
    history: list = field(default_factory=list)   # (t, Phi_t, Psi_t, restart)
    beta_last: np.ndarray | None = None


def solve(X, y, loss, k, lambda2, M=2.0, fix=None, warm=None, gap_tol=1e-6,
          eta=math.e ** 3, L=None, max_iters=100000, record=False):
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n, p = X.shape
    fix = np.zeros(p, dtype=np.int8) if fix is None else np.asarray(fix, dtype=np.int8)
    if L is None:
        L = lipschitz(X, loss)
    s = 1.0 / L
    rho = 2.0 * lambda2 * s                  # prox of s*G = prox of rho*g_N

    def evaluate(b):
        phi = primal(b, X, y, loss, fix, k, M, lambda2)
        psi = dual(induced_dual(b, X, y, loss), X, y, loss, fix, k, M, lambda2)
        return phi, psi

    x0 = np.zeros(p) if warm is None else np.asarray(warm, dtype=np.float64).copy()
    phi, psi = evaluate(x0)
    best_phi, best_psi, best_beta = phi, psi, x0.copy()
    gap_ref = phi - psi                       # +inf when the start is outside dom g
    hist = [(0, phi, psi, False)] if record else []

    def done():
        return (math.isfinite(best_phi)
                and best_phi - best_psi <= gap_tol * max(1.0, abs(best_phi)))

    x_prev = x0
    yk = x0
    t = 1.0
    it = 0
    restarts = 0
    converged = done()
    while not converged and it < max_iters:
        it += 1
        grad = X.T @ losses.grad_F(X @ yk, y, loss)
        x = regularizer.prox_g(yk - s * grad, rho, fix, k, M)
        phi, psi = evaluate(x)
        if phi < best_phi:
            best_phi, best_beta = phi, x.copy()
        best_psi = max(best_psi, psi)
        gap = phi - psi
        if not math.isfinite(gap_ref):
            gap_ref = gap
            restart = False
        else:
            restart = gap <= gap_ref / eta
        if record:
            hist.append((it, phi, psi, restart))
        t_next = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
        if restart:
            restarts += 1
            gap_ref = gap
            yk = x
            t = 1.0
        else:
            yk = x + ((t - 1.0) / t_next) * (x - x_prev)
            t = t_next
        x_prev = x
        converged = done()
    gap = best_phi - best_psi
    return Result(best_beta, best_phi, best_psi, gap, gap / max(1.0, abs(best_phi)), it,
                  restarts, converged, hist, x_prev)
