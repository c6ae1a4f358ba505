"""Pins of oracle/variants.py, the methods of the convergence study (Sec.
5.2): agreement with the pinned solver at its own settings, one optimum for
every method, the textbook properties of PGD and of backtracking, and the
restart rules firing only where they should."""
import math

import numpy as np
import pytest

import synth
from oracle import losses, regularizer, solver, variants


def _problem(loss, seed=0):
    # lambda2 = 2 keeps the unrestarted and first-order methods within seconds
    w = synth.Workload("var", 40, 80, 0.5, 5, 2.0, loss, seed=seed)
    X, y = synth.make_problem_cpu(w, dtype=np.float64)
    return w, X, y


@pytest.mark.parametrize("loss", ["ls", "logistic"])
def test_defaults_take_the_solvers_steps(loss):
    w, X, y = _problem(loss)
    L = solver.lipschitz(X, loss)
    a = solver.solve(X, y, loss, w.k, w.lambda2, w.M, gap_tol=1e-9, L=L, record=True)
    b = variants.solve(X, y, loss, w.k, w.lambda2, w.M, gap_tol=1e-9, L=L, record=True)
    assert a.iters == b.iters and a.restarts == b.restarts
    np.testing.assert_array_equal(a.beta, b.beta)
    assert [h[:4] for h in a.history] == [h[:4] for h in b.history]


@pytest.mark.parametrize("loss", ["ls", "logistic"])
def test_every_method_reaches_the_same_bound(loss):
    w, X, y = _problem(loss, seed=1)
    ref = solver.solve(X, y, loss, w.k, w.lambda2, w.M, gap_tol=1e-11, max_iters=200000)
    for method, step, restart in [("fista", "fixed", "none"), ("fista", "fixed", "function"),
                                  ("fista", "backtracking", "gap"), ("fista", "backtracking", "function"),
                                  ("pgd", "fixed", "none"), ("pgd", "backtracking", "none")]:
        r = variants.solve(X, y, loss, w.k, w.lambda2, w.M, gap_tol=1e-8, method=method, step=step,
                           restart=restart, max_iters=50000)
        assert r.converged, (method, step, restart)
        assert r.dual_bound <= ref.primal + 1e-12 * abs(ref.primal)            # valid
        assert r.dual_bound == pytest.approx(ref.dual_bound, rel=1e-7), (method, step, restart)


def test_pgd_decreases_phi_monotonically():
    # sufficient decrease of the proximal gradient step (Beck 2017, Lemma 10.4)
    w, X, y = _problem("ls", seed=2)
    for step in ("fixed", "backtracking"):
        r = variants.solve(X, y, "ls", w.k, w.lambda2, w.M, gap_tol=1e-8, method="pgd", step=step,
                           record=True, max_iters=100000)
        phis = [h[1] for h in r.history[1:]]
        assert all(b <= a + 1e-12 * abs(a) for a, b in zip(phis, phis[1:])), step


def test_backtracking_constants_grow_and_stay_below_twice_the_global_one():
    w, X, y = _problem("logistic", seed=3)
    L = solver.lipschitz(X, "logistic")
    r = variants.solve(X, y, "logistic", w.k, w.lambda2, w.M, gap_tol=1e-8, step="backtracking", record=True)
    Ls = [h[4] for h in r.history]
    assert all(b >= a for a, b in zip(Ls, Ls[1:]))      # L_k never decreases
    assert Ls[-1] <= 2.0 * L                             # Beck 2017: L_k <= max(2 L_f, L_0)
    assert Ls[0] < Ls[-1]                                # the start L_f / 64 was too small and grew


def test_restart_rules():
    w, X, y = _problem("ls", seed=4)
    fn = variants.solve(X, y, "ls", w.k, w.lambda2, w.M, gap_tol=1e-9, restart="function", record=True)
    h = fn.history
    for i in range(2, len(h)):
        if h[i][3]:
            assert h[i][1] > h[i - 1][1]             # only where Phi went up
    assert fn.restarts == sum(1 for r in h if r[3])
    none = variants.solve(X, y, "ls", w.k, w.lambda2, w.M, gap_tol=1e-9, restart="none", max_iters=50000)
    gap = variants.solve(X, y, "ls", w.k, w.lambda2, w.M, gap_tol=1e-9)
    assert none.restarts == 0 and gap.restarts > 0
    assert gap.iters < none.iters                  # restarts make the method linear (Sec. 3.4)
    # a smaller restart factor restarts more often (eta in {e, e^2, e^3})
    r1 = variants.solve(X, y, "ls", w.k, w.lambda2, w.M, gap_tol=1e-9, eta=math.e)
    r3 = variants.solve(X, y, "ls", w.k, w.lambda2, w.M, gap_tol=1e-9, eta=math.e ** 3)
    assert r1.restarts > r3.restarts


def test_unknown_options_are_rejected():
    w, X, y = _problem("ls")
    with pytest.raises(ValueError):
        variants.solve(X, y, "ls", w.k, w.lambda2, w.M, method="acfgm")


def test_dynamic_termination_rules_of_the_oracle():
    """Sec. 5.3: above the optimum the loop stops at the first iterate whose
    Phi is at most the cutoff; below it, at the first whose Psi reaches it,
    with that Psi as a bound proving the pruning.  Both stop before the full
    solve does."""
    w, X, y = _problem("ls", seed=5)
    full = variants.solve(X, y, "ls", w.k, w.lambda2, w.M, gap_tol=1e-10, record=True)
    opt = full.dual_bound
    up = variants.solve(X, y, "ls", w.k, w.lambda2, w.M, gap_tol=1e-10, cutoff=1.05 * opt, record=True)
    assert up.cutoff_rule == 1 and up.iters < full.iters
    first = next(h[0] for h in full.history if h[1] <= 1.05 * opt)     # same iterates until the stop
    assert up.iters == first
    down = variants.solve(X, y, "ls", w.k, w.lambda2, w.M, gap_tol=1e-10, cutoff=0.95 * opt, record=True)
    assert down.cutoff_rule == 2 and down.iters < full.iters
    assert 0.95 * opt <= down.dual_bound <= opt * (1 + 1e-12)
    assert variants.solve(X, y, "ls", w.k, w.lambda2, w.M, gap_tol=1e-10).cutoff_rule == 0
