"""The methods of the paper's convergence study (Sec. 5.2, "How much can our
restart scheme accelerate convergence?"), FP64, for the same node relaxation
as solver.solve (test infrastructure).

* method "fista": FISTA (Beck 2017, Sec. 10.7); "pgd": the proximal gradient
  method (Beck 2017, Sec. 10.2).
* step "fixed": s = 1/L with L = c_F ||X||_2^2; "backtracking": Beck 2017,
  Sec. 10.4.2 / 10.7.3 -- from the previous L_k, multiply by 2 until the point
  x = prox_{(1/L) G}(y - grad F(y) / L) satisfies
  F(x) <= F(y) + grad F(y)'(x - y) + (L / 2) ||x - y||^2 (up to an FP64
  rounding slack of 1e-12 |F(y)|), and keep that L.
* restart "gap": the duality-gap restart of Sec. 3.4 (restart when the gap has
  fallen by the factor eta since the epoch began); "function": the heuristic
  of O'Donoghue and Candes (2015), restart when Phi(x^k) > Phi(x^{k-1});
  "none": plain FISTA.  Restarts reset t = 1 and the extrapolation point.

The defaults (fista, fixed, gap, eta = e^3) take the same steps as
solver.solve.  The AC-FGM variant of the study is not included.
"""
from __future__ import annotations

import math

import numpy as np

from . import losses, regularizer
from .solver import Result, dual, induced_dual, lipschitz, primal


def solve(X, y, loss, k, lambda2, M=2.0, fix=None, warm=None, gap_tol=1e-6, method="fista", step="fixed",
          restart="gap", eta=math.e ** 3, L=None, max_iters=100000, record=False, cutoff=None):
    """Returns solver.Result; with record, history rows are
    (t, Phi_t, Psi_t, restarted, L_t).  cutoff (the incumbent's objective)
    adds the dynamic termination of Sec. 5.3: stop once Phi(beta^t) <= cutoff
    (the node will be branched) or Psi(zeta^t) >= cutoff (it is pruned); the
    rule that fired is returned as result.cutoff_rule (1 or 2, 0 none)."""
    if method not in ("fista", "pgd") or step not in ("fixed", "backtracking") or \
            restart not in ("gap", "function", "none"):
        raise ValueError("unknown method, step rule or restart")
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    p = X.shape[1]
    fix = np.zeros(p, dtype=np.int8) if fix is None else np.asarray(fix, dtype=np.int8)
    L_glob = lipschitz(X, loss) if L is None else L
    # backtracking starts below the global constant and only grows
    Lk = L_glob if step == "fixed" else L_glob / 64.0

    def evaluate(b):
        return (primal(b, X, y, loss, fix, k, M, lambda2),
                dual(induced_dual(b, X, y, loss), X, y, loss, fix, k, M, lambda2))

    def F_and_grad(b):
        z = X @ b
        return losses.F(z, y, loss), X.T @ losses.grad_F(z, y, loss)

    def prox_step(yk, Lval, grad):
        s = 1.0 / Lval                       # the solver's arithmetic: y - s grad, rho = 2 lambda2 s
        return regularizer.prox_g(yk - s * grad, 2.0 * lambda2 * s, fix, k, M)

    x0 = np.zeros(p) if warm is None else np.asarray(warm, dtype=np.float64).copy()
    phi, psi = evaluate(x0)
    best_phi, best_psi, best_beta = phi, psi, x0.copy()
    gap_ref = phi - psi
    phi_prev = phi
    hist = [(0, phi, psi, False, Lk)] if record else []

    def done():
        return math.isfinite(best_phi) and best_phi - best_psi <= gap_tol * max(1.0, abs(best_phi))

    x_prev, yk, t = x0, x0, 1.0
    it = restarts = 0
    cut_rule = 0
    converged = done()
    while not converged and not cut_rule and it < max_iters:
        it += 1
        Fy, grad = F_and_grad(yk)
        if step == "fixed":
            x = prox_step(yk, Lk, grad)
        else:
            while True:
                x = prox_step(yk, Lk, grad)
                d = x - yk
                # the test in FP64 with a rounding slack: near the optimum
                # F(x) and F(y) agree to more digits than FP64 resolves, and a
                # test without slack would double L on rounding noise alone
                if losses.F(X @ x, y, loss) <= Fy + grad @ d + 0.5 * Lk * (d @ d) + 1e-12 * max(1.0, abs(Fy)):
                    break
                Lk *= 2.0
        phi, psi = evaluate(x)
        if phi < best_phi:
            best_phi, best_beta = phi, x.copy()
        best_psi = max(best_psi, psi)
        gap = phi - psi
        do_restart = False
        if method == "fista":
            if restart == "gap":
                if not math.isfinite(gap_ref):
                    gap_ref = gap
                else:
                    do_restart = gap <= gap_ref / eta
            elif restart == "function":
                do_restart = it > 1 and phi > phi_prev
        if record:
            hist.append((it, phi, psi, do_restart, Lk))
        if method == "pgd":
            yk = x
        elif do_restart:
            restarts += 1
            gap_ref = gap
            yk, t = x, 1.0
        else:
            t_next = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
            yk = x + ((t - 1.0) / t_next) * (x - x_prev)
            t = t_next
        x_prev = x
        phi_prev = phi
        converged = done()
        if cutoff is not None:
            if phi <= cutoff:
                cut_rule = 1
            if psi >= cutoff:
                cut_rule = 2
    gap = best_phi - best_psi
    res = Result(best_beta, best_phi, best_psi, gap, gap / max(1.0, abs(best_phi)), it, restarts, converged,
                 hist, x_prev)
    res.cutoff_rule = cut_rule
    return res
