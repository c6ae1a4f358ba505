"""Whole-solve parity: relax_solve (fused X-pass + p-phase on the GPU, FP64
certification) against the FP64 oracle's FISTA with gap restarts (Sec. 3.4,
5.2) on the same seeded inputs and the same step 1/L.

Bars (from the method's specification): dual bounds within 1e-6 relative at
gap 1e-8 (FP64), beta within 1e-5 relative (norm-wise) where the solve is run
tight enough for beta to be determined to that accuracy, every reported bound
valid (<= the oracle's optimum), and the trajectory itself identical for FP64
(same iterate after the same number of steps, to rounding).
"""
import math

import numpy as np
import pytest

import synth
from oracle import brute, solver

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def problem(w, n=None, p=None, dtype=np.float64):
    X, y = synth.make_problem_cpu(w, n=n, p=p, dtype=dtype)
    return X, y


def gpu_solve(lib, X, y, loss, k, lam2, M, L, fix=None, warm=None, tol=1e-8, max_iters=0,
              certify=True, chunk=0):
    dt = torch.float64 if X.dtype == np.float64 else torch.float32
    Xd = torch.tensor(X, device="cuda")
    yd = torch.tensor(y, device="cuda")
    h = lib.Handle(Xd, yd, loss=loss, k=k, lambda2=lam2, M=M, lipschitz=L, max_iters=max_iters,
                   certify=certify, chunk=chunk)
    fx = None if fix is None else torch.tensor(fix, dtype=torch.int8, device="cuda")
    ws = None if warm is None else torch.tensor(warm, dtype=dt, device="cuda")
    beta, res, code = h.solve(fixings=fx, warm_start=ws, gap_tol=tol)
    out = beta.double().cpu().numpy()
    h.close()
    return out, res, code


def test_config0_ls_f64_parity(lib):
    """X 500x1000 FP64, rho=0.5, k=10, lambda2=1, SNR 5, gap 1e-8."""
    w = synth.WORKLOADS["ls_500x1000_f64"]
    X, y = problem(w)
    L = solver.lipschitz(X, "ls")
    ref = solver.solve(X, y, "ls", w.k, w.lambda2, w.M, gap_tol=1e-8, L=L)
    tight = solver.solve(X, y, "ls", w.k, w.lambda2, w.M, gap_tol=1e-12, L=L, max_iters=200000)
    beta, res, code = gpu_solve(lib, X, y, "ls", w.k, w.lambda2, w.M, L, tol=1e-8)
    assert code == 0, lib.STATUS[code]
    assert res.rel_gap <= 1e-8 * 1.0001
    opt = tight.dual_bound
    assert res.dual_bound == pytest.approx(ref.dual_bound, rel=1e-6)
    assert res.dual_bound <= opt + 1e-12 * abs(opt)                  # a valid bound
    assert res.primal >= opt - 1e-12 * abs(opt)
    assert abs(res.iters - ref.iters) <= max(3, 0.02 * ref.iters), (res.iters, ref.iters)
    # beta of the tight solves agree to 1e-5 relative
    b2, r2, c2 = gpu_solve(lib, X, y, "ls", w.k, w.lambda2, w.M, L, tol=1e-12, max_iters=200000)
    assert c2 == 0
    assert np.linalg.norm(b2 - tight.beta) <= 1e-5 * np.linalg.norm(tight.beta)


@pytest.mark.parametrize("loss", ["ls", "logistic"])
def test_trajectory_is_the_oracles(lib, loss):
    """Same L, FP64, fixed iteration count: the same best iterate (restarts and
    momentum resets included), to rounding."""
    w = synth.Workload("traj", 120, 300, 0.6, 6, 0.3, loss)
    X, y = problem(w)
    L = solver.lipschitz(X, loss)
    rng = np.random.default_rng(1)
    fix = np.zeros(300, dtype=np.int8)
    perm = rng.permutation(300)
    fix[perm[:10]] = -1
    fix[perm[10:12]] = 1
    for K in (1, 2, 37, 150):
        ref = solver.solve(X, y, loss, w.k, w.lambda2, w.M, fix=fix, gap_tol=1e-300, L=L,
                           max_iters=K)
        beta, res, code = gpu_solve(lib, X, y, loss, w.k, w.lambda2, w.M, L, fix=fix, tol=1e-300,
                                    max_iters=K, chunk=7)
        assert code == 4      # RELAX_ENOTCONV: stopped by max_iters
        assert res.iters == ref.iters == K
        assert res.restarts == ref.restarts
        np.testing.assert_allclose(beta, ref.beta, rtol=1e-9, atol=1e-11)
        assert res.primal_loop == pytest.approx(ref.primal, rel=1e-10)
        assert res.dual_loop == pytest.approx(ref.dual_bound, rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("loss", ["ls", "logistic"])
def test_f32_trajectory_is_the_oracles(lib, loss):
    """FP32 storage of X: after the same K steps from the same L, the iterate
    matches the FP64 oracle's on the same FP32-rounded X element by element
    within 1e-5 relative (the FP32 bar), each coordinate against the iterate's
    largest magnitude as its floor.  The device keeps the loop vectors in FP64
    and forms the products from FP32 X, so the differences are the products'
    FP32 rounding carried through K steps."""
    w = synth.Workload("traj32", 160, 400, 0.6, 8, 0.3, loss)
    X, y = problem(w, dtype=np.float32)
    X64, y64 = X.astype(np.float64), y.astype(np.float64)
    L = solver.lipschitz(X64, loss)
    fix = synth.node_fixings(400, 7, 0, 20, 3, k=8)
    for K in (1, 3, 40, 120):
        ref = solver.solve(X64, y64, loss, w.k, w.lambda2, w.M, fix=fix, gap_tol=1e-300, L=L,
                           max_iters=K)
        beta, res, code = gpu_solve(lib, X, y, loss, w.k, w.lambda2, w.M, L, fix=fix, tol=1e-300,
                                    max_iters=K, certify=False)
        assert code == 4      # RELAX_ENOTCONV: stopped by max_iters
        assert res.iters == ref.iters == K
        assert res.restarts == ref.restarts
        scale = float(np.max(np.abs(ref.beta)))
        np.testing.assert_allclose(beta, ref.beta, rtol=1e-5, atol=1e-5 * scale)
        # the same support: a coordinate is zero on one side only where the
        # other side is below the floor
        flip = (beta != 0) != (ref.beta != 0)
        assert np.all(np.abs(beta[flip]) + np.abs(ref.beta[flip]) <= 1e-5 * scale)
        assert res.primal_loop == pytest.approx(ref.primal, rel=1e-6)


@pytest.mark.parametrize("loss", ["ls", "logistic"])
def test_node_fixings_and_warm_start(lib, loss):
    w = synth.Workload("node", 200, 400, 0.7, 8, 0.5, loss)
    X, y = problem(w)
    L = solver.lipschitz(X, loss)
    fix = synth.node_fixings(400, 3, 0, 40, 5, k=8)
    ref = solver.solve(X, y, loss, w.k, w.lambda2, w.M, fix=fix, gap_tol=1e-10, L=L)
    # warm start outside dom g (nonzero on J0): accepted, same optimum
    warm = synth.prox_input(400, 9, scale=0.5)
    beta, res, code = gpu_solve(lib, X, y, loss, w.k, w.lambda2, w.M, L, fix=fix, warm=warm, tol=1e-8)
    assert code == 0
    assert res.dual_bound == pytest.approx(ref.dual_bound, rel=1e-6)
    assert res.dual_bound <= ref.primal + 1e-12 * abs(ref.primal)
    assert np.all(beta[fix < 0] == 0.0)


@pytest.mark.parametrize("loss", ["ls", "logistic"])
def test_f32_bounds_and_beta(lib, loss):
    w = synth.Workload("f32", 400, 900, 0.7, 10, 0.5, loss)
    X, y = problem(w, dtype=np.float32)
    X64, y64 = X.astype(np.float64), y.astype(np.float64)
    L = solver.lipschitz(X64, loss)
    tight = solver.solve(X64, y64, loss, w.k, w.lambda2, w.M, gap_tol=1e-12, L=L, max_iters=200000)
    beta, res, code = gpu_solve(lib, X, y, loss, w.k, w.lambda2, w.M, L, tol=1e-6)
    assert code == 0, lib.STATUS[code]
    opt = tight.dual_bound
    assert res.rel_gap <= 1e-6
    assert res.dual_bound <= opt + 1e-12 * abs(opt)                    # valid, certified in FP64
    assert res.dual_bound == pytest.approx(opt, rel=1e-6)
    # quadratic growth: |beta - beta*| <= sqrt(2 gap / alpha); report and bound it
    rel = np.linalg.norm(beta - tight.beta) / np.linalg.norm(tight.beta)
    assert rel <= 1e-3, rel


def test_ridge_closed_form_on_device(lib):
    w = synth.Workload("ridge", 80, 30, 0.5, 30, 0.7, "ls")
    X, y = problem(w)
    L = solver.lipschitz(X, "ls")
    beta, res, code = gpu_solve(lib, X, y, "ls", 30, 0.7, math.inf, L, tol=1e-13, max_iters=100000)
    b = brute.ridge(X, y, 0.7)
    opt = float(np.sum((y - X @ b) ** 2) + 0.7 * b @ b)
    assert res.dual_bound == pytest.approx(opt, rel=1e-11)
    np.testing.assert_allclose(beta, b, rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("loss", ["ls", "logistic"])
def test_bound_below_bruteforce(lib, loss):
    rng = np.random.default_rng(5)
    for trial in range(3):
        w = synth.Workload("bf", 30, 8, 0.5, 2, 0.5, loss, seed=trial)
        X, y = problem(w)
        fix = np.zeros(8, dtype=np.int8)
        fix[rng.integers(0, 8)] = -1
        k = 3
        L = solver.lipschitz(X, loss)
        beta, res, code = gpu_solve(lib, X, y, loss, k, 0.5, 1.5, L, fix=fix, tol=1e-9)
        assert code == 0
        opt = brute.ksparse_opt(X, y, loss, k, 0.5, 1.5, fix)
        assert res.dual_bound <= opt + 1e-9 * max(1, abs(opt))


def test_all_fixed_node(lib):
    w = synth.Workload("fixed", 30, 7, 0.5, 3, 0.3, "ls")
    X, y = problem(w)
    fix = np.array([1, -1, 1, -1, -1, 1, -1], dtype=np.int8)
    L = solver.lipschitz(X, "ls")
    beta, res, code = gpu_solve(lib, X, y, "ls", 3, 0.3, 1.0, L, fix=fix, tol=1e-11, max_iters=100000)
    opt, _ = brute.restricted_opt(X, y, "ls", 0.3, 1.0, [0, 2, 5])
    assert res.dual_bound == pytest.approx(opt, rel=1e-7)


def test_invalid_node_rejected(lib):
    w = synth.Workload("bad", 20, 6, 0.5, 1, 0.3, "ls")
    X, y = problem(w)
    fix = np.array([1, 1, 0, 0, 0, 0], dtype=np.int8)     # |J1| = 2 > k = 1
    with pytest.raises(lib.RelaxError):
        gpu_solve(lib, X, y, "ls", 1, 0.3, 1.0, 1.0, fix=fix)


def test_solve_is_deterministic(lib):
    """Two handles on the same data (L estimated on the device each time) give
    bit-identical L, iteration counts, bounds and beta: every reduction on the
    path sums in a fixed order."""
    w = synth.Workload("det", 600, 3000, 0.8, 12, 0.3, "ls")
    X, y = problem(w, dtype=np.float32)
    Xd = torch.tensor(X, device="cuda")
    yd = torch.tensor(y, device="cuda")
    runs = []
    for _ in range(2):
        h = lib.Handle(Xd, yd, loss="ls", k=w.k, lambda2=w.lambda2, M=w.M)
        beta, res, code = h.solve(gap_tol=1e-6)
        runs.append((beta.cpu().numpy().copy(), res, code))
        h.close()
    (b0, r0, c0), (b1, r1, c1) = runs
    assert c0 == c1 == 0
    assert r0.lipschitz == r1.lipschitz
    assert r0.iters == r1.iters and r0.restarts == r1.restarts
    assert r0.dual_bound == r1.dual_bound and r0.primal == r1.primal
    assert np.array_equal(b0, b1)
    # the Lanczos estimate is within its 1% margin above ||X||^2 (times 2 for LS)
    lam = np.linalg.norm(X.astype(np.float64), 2) ** 2
    assert 2 * lam * 0.999 <= r0.lipschitz <= 2 * lam * 1.0101


@pytest.mark.parametrize("loss", ["ls", "logistic"])
def test_stall_rule_ends_a_solve_below_the_fp32_floor(lib, loss):
    """A gap target that FP32 data cannot resolve (1e-13): the loop's best gap
    stops falling, the stall rule ends the solve long before max_iters, the
    status says the target was missed, and the certified bound stays valid and
    as close to the optimum as the FP32 bar."""
    w = synth.Workload("stall", 400, 900, 0.7, 10, 0.5, loss)
    X, y = problem(w, dtype=np.float32)
    X64, y64 = X.astype(np.float64), y.astype(np.float64)
    L = solver.lipschitz(X64, loss)
    opt = solver.solve(X64, y64, loss, w.k, w.lambda2, w.M, gap_tol=1e-12, L=L, max_iters=200000).dual_bound
    beta, res, code = gpu_solve(lib, X, y, loss, w.k, w.lambda2, w.M, L, tol=1e-13, max_iters=100000)
    assert code == 4, lib.STATUS[code]
    assert res.iters < 20000, (res.iters, res.stalled)
    assert res.dual_bound <= opt + 1e-12 * abs(opt)
    assert res.dual_bound == pytest.approx(opt, rel=1e-6)


def test_dynamic_termination_rules(lib):
    """Sec. 5.3's dynamic termination against an incumbent's objective: above
    the node's optimum the loop stops once Phi falls to it (rule 1, branch);
    below the optimum it stops once Psi reaches it (rule 2, prune), and the
    certified bound then proves the pruning.  Off again, the solve is the
    plain one.  In a batch every node follows the same rules."""
    w = synth.Workload("cut", 300, 700, 0.7, 8, 0.5, "ls")
    X, y = problem(w)
    L = solver.lipschitz(X, "ls")
    opt = solver.solve(X, y, "ls", w.k, w.lambda2, w.M, gap_tol=1e-12, L=L, max_iters=200000).dual_bound
    h = lib.Handle(torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda"), loss="ls", k=w.k,
                   lambda2=w.lambda2, M=w.M, lipschitz=L)
    _, r0, c0 = h.solve(gap_tol=1e-10)
    assert c0 == 0 and r0.cutoff_rule == 0
    h.set_cutoff(1.05 * opt)
    _, r1, c1 = h.solve(gap_tol=1e-10)
    assert c1 == 0 and r1.cutoff_rule == 1 and r1.iters < r0.iters
    assert r1.primal <= 1.05 * opt * (1 + 1e-9) and r1.dual_bound <= opt + 1e-12 * abs(opt)
    h.set_cutoff(0.95 * opt)
    _, r2, c2 = h.solve(gap_tol=1e-10)
    assert c2 == 0 and r2.cutoff_rule == 2 and r2.iters < r0.iters
    assert 0.95 * opt * (1 - 1e-9) <= r2.dual_bound <= opt + 1e-12 * abs(opt)
    nb = 4
    fix = np.stack([synth.node_fixings(w.p, 7, j, 40, 5, k=w.k) for j in range(nb)])
    _, rb, cb = h.solve_batch(nb, fixings=torch.tensor(fix, device="cuda"), gap_tol=1e-10)
    assert cb == 0
    for r in rb:                      # every node's optimum is at least the root's
        assert r.cutoff_rule == 2 and r.dual_bound >= 0.95 * opt * (1 - 1e-9)
    h.set_cutoff()
    _, r3, c3 = h.solve(gap_tol=1e-10)
    assert c3 == 0 and r3.cutoff_rule == 0 and r3.iters == r0.iters
    h.close()


@pytest.mark.parametrize("loss", ["ls", "logistic"])
@pytest.mark.parametrize("factor,rule", [(1.02, 1), (0.98, 2)])
def test_cutoff_stop_is_the_oracles(lib, loss, factor, rule):
    """The dynamic termination of Sec. 5.3 stops the device loop at the same
    iterate as the oracle's (oracle.variants.solve with the same cutoff, FP64,
    same L): the first iterate whose Phi falls to the cutoff (rule 1) or
    whose Psi reaches it (rule 2), with the same best point and values."""
    from oracle import variants
    w = synth.Workload("cutpar", 150, 320, 0.6, 6, 0.4, loss)
    X, y = problem(w)
    L = solver.lipschitz(X, loss)
    fix = synth.node_fixings(320, 5, 1, 15, 2, k=6)
    opt = solver.solve(X, y, loss, w.k, w.lambda2, w.M, fix=fix, gap_tol=1e-12, L=L,
                       max_iters=200000).dual_bound
    cut = factor * opt
    ref = variants.solve(X, y, loss, w.k, w.lambda2, w.M, fix=fix, gap_tol=1e-300, L=L, cutoff=cut)
    assert ref.cutoff_rule == rule
    h = lib.Handle(torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda"), loss=loss, k=w.k,
                   lambda2=w.lambda2, M=w.M, lipschitz=L, certify=False)
    h.set_cutoff(cut)
    beta, res, code = h.solve(fixings=torch.tensor(fix, device="cuda"), gap_tol=1e-300)
    h.close()
    assert code == 0 and res.cutoff_rule == rule
    assert res.iters == ref.iters and res.restarts == ref.restarts
    np.testing.assert_allclose(beta.cpu().numpy(), ref.beta, rtol=1e-9, atol=1e-11)
    assert res.primal_loop == pytest.approx(ref.primal, rel=1e-10)
    assert res.dual_loop == pytest.approx(ref.dual_bound, rel=1e-9, abs=1e-9)


def test_watchdog_probe_times_out_and_the_context_survives(lib):
    """Failure detection without a fault: a wait on a partner that never
    arrives ends by its bound with RELAX_ETIMEOUT, and the GPU context serves
    a solve afterwards."""
    code, ms = lib.relax_watchdog_probe(50)
    assert code == 5, lib.STATUS[code]                # RELAX_ETIMEOUT
    assert 50.0 <= ms < 2000.0, ms
    w = synth.Workload("wd", 60, 120, 0.5, 4, 0.5, "ls")
    X, y = problem(w)
    L = solver.lipschitz(X, "ls")
    _, res, c = gpu_solve(lib, X, y, "ls", w.k, w.lambda2, w.M, L, tol=1e-8)
    assert c == 0
