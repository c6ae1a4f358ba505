"""The methods of the convergence study (Sec. 5.2) on the device against the
FP64 oracle's (oracle/variants.py) at the same L, FP64 data and a fixed
number of accepted steps K: FISTA or PGD (Beck 2017 Sec. 10.7 / 10.2), fixed
step or backtracking (Sec. 10.4.2), duality-gap (Sec. 3.4), function-value
(O'Donoghue and Candes) or no restart.  The same best iterate, restart count
and final L (backtracking) to rounding, as for the default method's
trajectory test."""
import math

import numpy as np
import pytest

import synth
from oracle import solver, variants

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

VARIANTS = [
    # (method, step, restart)
    ("fista", "fixed", "function"),
    ("fista", "fixed", "none"),
    ("pgd", "fixed", "gap"),
    ("fista", "backtracking", "gap"),
    ("fista", "backtracking", "function"),
    ("pgd", "backtracking", "gap"),
]


@pytest.mark.parametrize("loss", ["ls", "logistic"])
@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_trajectory_is_the_oracles(lib, loss, variant):
    method, step, restart = variant
    w = synth.Workload("var", 120, 260, 0.6, 6, 0.3, loss)
    X, y = synth.make_problem_cpu(w, dtype=np.float64)
    L = solver.lipschitz(X, loss)
    fix = synth.node_fixings(260, 2, 0, 12, 2, k=6)
    Xd, yd = torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda")
    fx = torch.tensor(fix, device="cuda")
    for K in (1, 4, 33, 120):
        ref = variants.solve(X, y, loss, w.k, w.lambda2, w.M, fix=fix, gap_tol=1e-300, method=method, step=step,
                             restart=restart, L=L, max_iters=K, record=True)
        h = lib.Handle(Xd, yd, loss=loss, k=w.k, lambda2=w.lambda2, M=w.M, lipschitz=L, max_iters=K, certify=False,
                       chunk=5, method=method, restart=restart, step=step, stall_window=-1)
        beta, res, code = h.solve(fixings=fx, gap_tol=1e-300)
        h.close()
        assert code == 4, lib.STATUS[code]          # RELAX_ENOTCONV: stopped by max_iters
        assert res.iters == ref.iters == K
        assert res.restarts == ref.restarts
        if step == "backtracking":
            L_ref = ref.history[-1][4]
            assert res.lipschitz == pytest.approx(L_ref, rel=1e-12)
            assert res.backtracks == round(math.log2(L_ref / (L / 64.0)))
        else:
            assert res.backtracks == 0 and res.lipschitz == L
        np.testing.assert_allclose(beta.cpu().numpy(), ref.beta, rtol=1e-9, atol=1e-11)
        assert res.primal_loop == pytest.approx(ref.primal, rel=1e-10)
        assert res.dual_loop == pytest.approx(ref.dual_bound, rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("variant", [("fista", "backtracking", "gap"), ("pgd", "fixed", "gap")])
def test_variant_certifies_the_same_bound(lib, variant):
    """Run to the gap: every method reaches the same certified bound (the
    relaxation's optimum) within the bars of the default solve."""
    method, step, restart = variant
    w = synth.Workload("varc", 200, 400, 0.5, 8, 0.5, "ls")
    X, y = synth.make_problem_cpu(w, dtype=np.float64)
    L = solver.lipschitz(X, "ls")
    opt = solver.solve(X, y, "ls", w.k, w.lambda2, w.M, gap_tol=1e-12, L=L, max_iters=200000).dual_bound
    h = lib.Handle(torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda"), k=w.k, lambda2=w.lambda2,
                   M=w.M, lipschitz=L, method=method, restart=restart, step=step, max_iters=200000)
    _, res, code = h.solve(gap_tol=1e-8)
    h.close()
    assert code == 0, lib.STATUS[code]
    assert res.dual_bound == pytest.approx(opt, rel=1e-6)
    assert res.dual_bound <= opt + 1e-12 * abs(opt)
