"""Pins for the FP64 oracle: each check ties it to something other than itself
(the paper's worked examples, closed forms, Fenchel-Young equalities, generic
numerical solves of the defining problems, brute force over supports)."""
import json
import math
import os

import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import brute, losses, regularizer as R, solver
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rand_fix(rng, p, n0, n1):
    fix = np.zeros(p, dtype=np.int8)
    perm = rng.permutation(p)
    fix[perm[:n0]] = -1
    fix[perm[n0:n0 + n1]] = 1
    return fix


def rand_dom(rng, fix, k, M, scale=1.0):
    """A random point of dom g_N (Eq. 4): zero on J0, |b| <= M, sum_Jf |b| <= M kbar."""
    p = fix.size
    b = rng.standard_normal(p) * scale
    b[fix < 0] = 0.0
    b = np.clip(b, -M, M)
    Jf = fix == 0
    kbar = k - int(np.sum(fix > 0))
    s = np.sum(np.abs(b[Jf]))
    if s > M * kbar:
        b[Jf] *= (M * kbar) / s * 0.999
    return b


# ---------------------------------------------------------------- Algorithm 1
def test_alg1_worked_examples():
    cases = json.load(open(os.path.join(GOLD, "majorization_examples.json")))["cases"]
    for c in cases:
        b = np.array(c["beta"])
        want = 0.5 * float(np.sum(np.array(c["omega"]) ** 2))
        assert R.g_alg1(b, None, c["k"], c["M"]) == pytest.approx(want, rel=1e-15)
        assert R.g_bisect(b, None, c["k"], c["M"]) == pytest.approx(want, rel=1e-12)
    # the two published values: 2.0 and 2.25
    assert R.g_alg1(np.array([1.4, 0.6]), None, 1, 2.0) == pytest.approx(2.0)
    assert R.g_alg1(np.array([0.6, 1.2, 1.2]), None, 2, 1.5) == pytest.approx(2.25)


def test_g_k1_root_closed_form():
    # root node, k = 1: g = 0.5 ||b||_1^2 on ||b||_1 <= M (figure caption, Sec. 4.1)
    rng = np.random.default_rng(0)
    for _ in range(50):
        p = rng.integers(1, 9)
        b = rng.standard_normal(p)
        M = float(np.sum(np.abs(b))) * rng.uniform(1.0, 2.0)
        assert R.g_alg1(b, None, 1, M) == pytest.approx(0.5 * np.sum(np.abs(b)) ** 2, rel=1e-13)
        # on the boundary ||b||_1 = M the value is M^2 / 2
        bb = b * (M / np.sum(np.abs(b)))
        assert R.g_alg1(bb, None, 1, M) == pytest.approx(0.5 * M * M, rel=1e-12)
    assert math.isinf(R.g_alg1(np.array([1.0, 1.0]), None, 1, 1.5))


def test_gstar_k1_root_closed_form():
    # k = 1 root: g* = H_M(||a||_inf) (figure caption, Sec. 4.1); g* = M^2/2 at max|a| = M
    rng = np.random.default_rng(1)
    for _ in range(50):
        a = rng.standard_normal(rng.integers(1, 9)) * 2
        M = rng.uniform(0.3, 3.0)
        want = float(R.huber(np.max(np.abs(a)), M))
        assert R.gstar(a, None, 1, M) == pytest.approx(want, rel=1e-14)
    assert R.gstar(np.array([1.0, -0.5]), None, 1, 1.0) == pytest.approx(0.5)


def test_huber_closed_form():
    M = 1.5
    assert R.huber(1.0, M) == pytest.approx(0.5)
    assert R.huber(-3.0, M) == pytest.approx(1.5 * 3.0 - 0.5 * 2.25)
    assert R.huber(1.5, M) == pytest.approx(1.125)
    x, tau = 4.0, 0.5           # |x| > M(1+tau) = 2.25 -> x - tau M
    assert R.prox_huber(x, tau, M) == pytest.approx(4.0 - 0.75)
    assert R.prox_huber(1.0, tau, M) == pytest.approx(1.0 / 1.5)


def test_g_full_cardinality_is_half_square():
    rng = np.random.default_rng(2)
    for _ in range(30):
        p = rng.integers(1, 12)
        fix = rand_fix(rng, p, rng.integers(0, p // 2 + 1), 0)
        k = p
        b = rand_dom(rng, fix, k, 2.0)
        assert R.g_alg1(b, fix, k, 2.0) == pytest.approx(0.5 * np.sum(b ** 2), rel=1e-13)
        assert R.gstar(b, fix, k, 2.0) == pytest.approx(
            float(np.sum(R.huber(b[fix >= 0], 2.0))), rel=1e-13)


def test_alg1_matches_definition_bisection():
    rng = np.random.default_rng(3)
    for trial in range(300):
        p = int(rng.integers(1, 40))
        n0 = int(rng.integers(0, p // 3 + 1))
        n1 = int(rng.integers(0, (p - n0) // 3 + 1))
        fix = rand_fix(rng, p, n0, n1)
        k = n1 + int(rng.integers(0, p - n0 - n1 + 2))
        M = float(rng.choice([0.5, 1.0, 2.0, math.inf]))
        b = rand_dom(rng, fix, k, M if math.isfinite(M) else 10.0, scale=rng.uniform(0.1, 2))
        ga, gb = R.g_alg1(b, fix, k, M), R.g_bisect(b, fix, k, M)
        assert ga == pytest.approx(gb, rel=1e-9, abs=1e-12), (trial, ga, gb)


def test_g_outside_domain_is_inf():
    fix = np.array([-1, 0, 0], dtype=np.int8)
    assert math.isinf(R.g_alg1(np.array([0.1, 0.0, 0.0]), fix, 1, 2.0))   # J0 nonzero
    assert math.isinf(R.g_alg1(np.array([0.0, 2.5, 0.0]), fix, 2, 2.0))   # box
    assert math.isinf(R.g_alg1(np.array([0.0, 1.5, 1.5]), fix, 1, 2.0))   # l1 cap M*kbar


# ------------------------------------------------------------ conjugate g*
def _gstar_numeric(a, fix, k, M):
    """sup_beta a'beta - g(beta) via the joint (beta, z) concave program of Eq. 5."""
    p = a.size
    J0 = fix < 0
    J1 = fix > 0
    Jf = fix == 0
    kbar = k - int(J1.sum())
    best = -math.inf
    rng = np.random.default_rng(0)
    for start in range(4):
        x0 = np.concatenate([rng.standard_normal(p) * 0.1, np.full(p, 0.5)])

        def negobj(v):
            b, z = v[:p], np.maximum(v[p:], 1e-12)
            return -(a @ b - 0.5 * np.sum(b * b / z))

        cons = [{"type": "ineq", "fun": lambda v: kbar - np.sum(v[p:][Jf])}]
        cons += [{"type": "ineq", "fun": (lambda v, j=j: M * v[p + j] - v[j])} for j in range(p)]
        cons += [{"type": "ineq", "fun": (lambda v, j=j: M * v[p + j] + v[j])} for j in range(p)]
        bounds = []
        for j in range(p):
            bounds.append((0.0, 0.0) if J0[j] else (None, None))
        for j in range(p):
            bounds.append((1e-9, 1e-9) if J0[j] else ((1.0, 1.0) if J1[j] else (1e-9, 1.0)))
        res = minimize(negobj, x0, method="SLSQP", bounds=bounds, constraints=cons,
                       options={"ftol": 1e-13, "maxiter": 2000})
        best = max(best, -res.fun)
    return best


def test_gstar_matches_numerical_conjugate():
    rng = np.random.default_rng(4)
    for _ in range(12):
        p = int(rng.integers(2, 5))
        fix = rand_fix(rng, p, int(rng.integers(0, 2)), int(rng.integers(0, 2)))
        k = int(np.sum(fix > 0)) + int(rng.integers(1, 3))
        M = float(rng.choice([0.7, 1.5]))
        a = rng.standard_normal(p) * 1.5
        assert R.gstar(a, fix, k, M) == pytest.approx(_gstar_numeric(a, fix, k, M),
                                                     rel=1e-5, abs=1e-6)


# ------------------------------------------------------------------- prox
def test_prox_full_cardinality_and_fixed_closed_form():
    rng = np.random.default_rng(5)
    for _ in range(50):
        p = int(rng.integers(1, 30))
        fix = rand_fix(rng, p, int(rng.integers(0, p // 2 + 1)), int(rng.integers(0, 3)))
        v = rng.standard_normal(p) * 3
        rho = rng.uniform(0.05, 3)
        M = 1.3
        u = R.prox_g(v, rho, fix, p, M)          # kbar >= pbar: no cardinality coupling
        want = np.clip(v / (1 + rho), -M, M)
        want[fix < 0] = 0.0
        np.testing.assert_allclose(u, want, rtol=1e-13, atol=1e-15)
        # J1 / J0 coordinates follow the same closed form at any k
        k = int(np.sum(fix > 0)) + 1
        u2 = R.prox_g(v, rho, fix, k, M)
        np.testing.assert_allclose(u2[fix > 0], np.clip(v[fix > 0] / (1 + rho), -M, M), rtol=1e-13)
        assert np.all(u2[fix < 0] == 0.0)


def test_prox_fenchel_young_and_subgradient():
    """u = prox_{rho g}(v) iff a = (v-u)/rho in dg(u) iff g(u) + g*(a) = u'a."""
    rng = np.random.default_rng(6)
    for trial in range(300):
        p = int(rng.integers(1, 60))
        n0 = int(rng.integers(0, p // 4 + 1))
        n1 = int(rng.integers(0, (p - n0) // 4 + 1))
        fix = rand_fix(rng, p, n0, n1)
        k = n1 + int(rng.integers(0, max(1, (p - n0 - n1) // 2) + 1))
        M = float(rng.choice([0.5, 1.0, 2.0, math.inf]))
        rho = float(10 ** rng.uniform(-3, 1))
        v = rng.standard_normal(p) * float(10 ** rng.uniform(-1, 1))
        u = R.prox_g(v, rho, fix, k, M)
        assert R.in_domain(u, fix, k, M, rtol=1e-12)
        a = (v - u) / rho
        gu, ga = R.g_alg1(u, fix, k, M), R.gstar(a, fix, k, M)
        scale = max(1.0, abs(gu) + abs(ga))
        assert gu + ga - float(u @ a) == pytest.approx(0.0, abs=1e-10 * scale), trial
        assert np.all(u * v >= 0)
        for _ in range(5):      # subgradient inequality at random points of the domain
            w = rand_dom(rng, fix, k, M if math.isfinite(M) else 5.0)
            gw = R.g_alg1(w, fix, k, M)
            assert gw >= gu + float(a @ (w - u)) - 1e-9 * max(1.0, abs(gw)), trial


def _prox_numeric(v, rho, fix, k, M):
    """min_u 0.5||u - v||^2 + (rho/2) sum u^2/z over (u, z) in D (Eq. 4, 5)."""
    p = v.size
    J0, J1, Jf = fix < 0, fix > 0, fix == 0
    kbar = k - int(J1.sum())

    def obj(x):
        u, z = x[:p], np.maximum(x[p:], 1e-12)
        return 0.5 * np.sum((u - v) ** 2) + 0.5 * rho * np.sum(u * u / z)

    cons = [{"type": "ineq", "fun": lambda x: kbar - np.sum(x[p:][Jf])}]
    cons += [{"type": "ineq", "fun": (lambda x, j=j: M * x[p + j] - x[j])} for j in range(p)]
    cons += [{"type": "ineq", "fun": (lambda x, j=j: M * x[p + j] + x[j])} for j in range(p)]
    bounds = [(0.0, 0.0) if J0[j] else (None, None) for j in range(p)]
    bounds += [(1e-9, 1e-9) if J0[j] else ((1.0, 1.0) if J1[j] else (1e-9, 1.0))
               for j in range(p)]
    x0 = np.concatenate([v * 0.5, np.full(p, 0.5)])
    res = minimize(obj, x0, method="SLSQP", bounds=bounds, constraints=cons,
                   options={"ftol": 1e-14, "maxiter": 3000})
    return res.x[:p]


def test_prox_matches_generic_convex_solve():
    rng = np.random.default_rng(7)
    for _ in range(15):
        p = int(rng.integers(2, 6))
        fix = rand_fix(rng, p, int(rng.integers(0, 2)), int(rng.integers(0, 2)))
        k = int(np.sum(fix > 0)) + 1
        M = float(rng.choice([0.8, 1.6]))
        rho = float(rng.uniform(0.2, 2.0))
        v = rng.standard_normal(p) * 1.5
        np.testing.assert_allclose(R.prox_g(v, rho, fix, k, M),
                                   _prox_numeric(v, rho, fix, k, M), atol=2e-4)


def test_prox_threshold_info():
    # tie-free example where the pooled block straddles kbar: counts are consistent
    rng = np.random.default_rng(8)
    v = rng.standard_normal(200)
    u, (n_top, n_nz) = R.prox_g(v, 0.05, None, 10, 2.0, return_info=True)
    assert n_nz == np.count_nonzero(u)
    assert 0 <= n_top <= 10 <= n_nz


# ----------------------------------------------------------------- losses
@pytest.mark.parametrize("loss", ["ls", "logistic"])
def test_loss_conjugate_fenchel_young(loss):
    rng = np.random.default_rng(9)
    n = 50
    y = rng.standard_normal(n) if loss == "ls" else np.where(rng.random(n) < 0.5, -1.0, 1.0)
    z = rng.standard_normal(n) * 2
    zeta = -losses.grad_F(z, y, loss)
    # equality F(z) + F*(-zeta) = -zeta'z at zeta = -grad F(z)
    assert losses.F(z, y, loss) + losses.F_conj(-zeta, y, loss) == pytest.approx(
        float(-zeta @ z), abs=1e-10 * n)
    # inequality at other points
    for _ in range(20):
        z2 = rng.standard_normal(n) * 2
        assert losses.F_conj(-zeta, y, loss) >= float(-zeta @ z2) - losses.F(z2, y, loss) - 1e-9
    # gradient by central differences
    e = np.zeros(n); e[3] = 1e-6
    fd = (losses.F(z + e, y, loss) - losses.F(z - e, y, loss)) / 2e-6
    assert losses.grad_F(z, y, loss)[3] == pytest.approx(fd, rel=1e-6)


def test_logistic_conjugate_scalar_sup():
    # 1-D check of F*(w) = sup_z wz - log(1 + exp(-y z)) by a dense grid
    zs = np.linspace(-40, 40, 400001)
    for y in (-1.0, 1.0):
        for u in (0.1, 0.5, 0.93):
            w = -y * u
            sup = np.max(w * zs - np.logaddexp(0, -y * zs))
            assert losses.F_conj(np.array([w]), np.array([y]), "logistic") == pytest.approx(sup, abs=1e-6)


# ------------------------------------------------------------ whole solve
def small_problem(loss, n=40, p=8, seed=0, rho=0.5):
    X = synth.ar1_design(n, p, rho, seed)
    s = synth.signal_from_design(X, 2)
    y = synth.response(s, loss, 5.0, seed)
    return X, y


def test_ridge_closed_form_k_equals_p():
    X, y = small_problem("ls", n=60, p=10)
    lam2 = 0.7
    res = solver.solve(X, y, "ls", k=10, lambda2=lam2, M=math.inf, gap_tol=1e-12,
                       max_iters=20000)
    b = brute.ridge(X, y, lam2)
    # |beta - beta*| ~ sqrt(gap / lambda2): the objective pins below are the tight ones
    np.testing.assert_allclose(res.beta, b, rtol=1e-4, atol=1e-6)
    opt = float(np.sum((y - X @ b) ** 2) + lam2 * b @ b)
    assert res.dual_bound == pytest.approx(opt, rel=1e-10)
    assert res.primal == pytest.approx(opt, rel=1e-10)


@pytest.mark.parametrize("loss", ["ls", "logistic"])
def test_relaxation_below_bruteforce(loss):
    rng = np.random.default_rng(10)
    for trial in range(4):
        p = 8
        X, y = small_problem(loss, n=30, p=p, seed=trial)
        fix = rand_fix(rng, p, int(rng.integers(0, 2)), int(rng.integers(0, 2)))
        k = int(np.sum(fix > 0)) + 2
        lam2, M = 0.5, 1.5
        res = solver.solve(X, y, loss, k, lam2, M, fix=fix, gap_tol=1e-9, max_iters=50000)
        assert res.converged
        opt = brute.ksparse_opt(X, y, loss, k, lam2, M, fix)
        assert res.dual_bound <= opt + 1e-9 * max(1, abs(opt))
        assert res.primal <= opt + 1e-7 * max(1, abs(opt))


@pytest.mark.parametrize("loss", ["ls", "logistic"])
def test_relaxation_exact_without_cardinality(loss):
    # k >= p: z = 1 is optimal, the relaxation IS problem (1) (perspective term exact)
    X, y = small_problem(loss, n=30, p=6, seed=3)
    lam2, M = 0.4, 1.2
    res = solver.solve(X, y, loss, 6, lam2, M, gap_tol=1e-11, max_iters=50000)
    opt, _ = brute.restricted_opt(X, y, loss, lam2, M, range(6))
    assert res.dual_bound == pytest.approx(opt, rel=1e-7)


def test_all_fixed_node_is_restricted_problem():
    X, y = small_problem("ls", n=30, p=7, seed=4)
    fix = np.array([1, -1, 1, -1, -1, 1, -1], dtype=np.int8)
    lam2, M = 0.3, 1.0
    res = solver.solve(X, y, "ls", 3, lam2, M, fix=fix, gap_tol=1e-11, max_iters=50000)
    opt, _ = brute.restricted_opt(X, y, "ls", lam2, M, [0, 2, 5])
    assert res.dual_bound == pytest.approx(opt, rel=1e-7)


@pytest.mark.parametrize("loss", ["ls", "logistic"])
def test_weak_duality_and_restart_contraction(loss):
    X, y = small_problem(loss, n=80, p=40, seed=5, rho=0.7)
    res = solver.solve(X, y, loss, 4, 0.3, 2.0, gap_tol=1e-9, record=True, max_iters=20000)
    assert res.converged
    phis = [h[1] for h in res.history]
    psis = [h[2] for h in res.history]
    assert max(psis) <= min(phis) + 1e-10 * max(1, abs(min(phis)))
    # every restart happens only after the gap has contracted by eta
    eta = math.e ** 3
    ref = phis[0] - psis[0]
    for (t, phi, psi, rs) in res.history[1:]:
        if rs:
            assert phi - psi <= ref / eta * (1 + 1e-12)
            ref = phi - psi
    assert res.restarts >= 2


def test_restart_beats_plain_fista():
    X, y = small_problem("ls", n=120, p=60, seed=6, rho=0.8)
    L = solver.lipschitz(X, "ls")
    a = solver.solve(X, y, "ls", 5, 0.05, 2.0, gap_tol=1e-10, L=L, max_iters=4000)
    b = solver.solve(X, y, "ls", 5, 0.05, 2.0, gap_tol=1e-10, L=L, max_iters=4000,
                     eta=math.inf)
    assert a.converged
    assert a.iters < b.iters or not b.converged


def test_spectral_norm_power_iteration_matches_svd():
    X = synth.ar1_design(300, 400, 0.6, 1)
    want = float(np.linalg.norm(X, 2) ** 2)
    # force the power-iteration branch
    Xb = np.tile(X, (12, 10))
    got = solver.spectral_norm_sq(Xb, iters=2000)
    assert got == pytest.approx(float(np.linalg.norm(Xb, 2) ** 2), rel=1e-8)
    assert want > 0
