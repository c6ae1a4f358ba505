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


def _kkt_threshold(m, rho, kbar, M):
    """The multiplier c >= 0 of the budget sum_Jf z_j <= kbar in the joint
    problem min_{u,z} 1/2 ||u - v||^2 + rho/2 sum u_j^2 / z_j (Eq. 5 inside the
    prox), found by bisection.  For fixed c each free coordinate decouples:
    minimising over z_j gives an l1 weight c on u_j while z_j < 1, so
    u_j = |v_j| - c and z_j = (|v_j| - c) / w(c) with w(c) = min(c / rho, M)
    (the box |u_j| <= M z_j binds once c > rho M); z_j = 1 gives the J1 prox
    min(|v_j| / (1 + rho), M).  sum_j z_j(c) falls in c; the root is c."""
    if kbar <= 0:
        return math.inf
    if np.count_nonzero(m) <= kbar:
        return 0.0

    def zsum(c):
        w = min(c / rho, M)
        return float(np.sum(np.minimum(np.maximum(m - c, 0.0) / w, 1.0)))

    # sum z(c) = kbar can hold on a whole interval (the box binds and the
    # kbar-th and next |v_j| lie more than M apart): every c there is a
    # multiplier and the prox is the same; take the interval's midpoint
    lo, hi = 0.0, float(np.max(m))
    for _ in range(200):                 # smallest root
        mid = 0.5 * (lo + hi)
        if zsum(mid) > kbar:
            lo = mid
        else:
            hi = mid
    c_lo = hi
    lo, hi = c_lo, float(np.max(m))
    for _ in range(200):                 # largest root
        mid = 0.5 * (lo + hi)
        if zsum(mid) >= kbar:
            lo = mid
        else:
            hi = mid
    return 0.5 * (c_lo + lo)


def _threshold_cases():
    """Tie-free prox inputs with J0/J1 fixings, a slack budget, thresholds on
    both sides of rho M (box inactive / active) and M = inf."""
    rng = np.random.default_rng(21)
    cases = []
    for t in range(40):
        p = int(rng.integers(30, 400))
        k = int(rng.integers(1, 12))
        n1 = int(rng.integers(0, min(k, 4) + 1))
        n0 = int(rng.integers(0, p // 5))
        fix = rand_fix(rng, p, n0, n1)
        scale = [0.3, 1.0, 3.0, 10.0][t % 4]
        v = rng.standard_normal(p) * scale
        rho = float([0.02, 0.3, 1.0, 4.0][(t // 4) % 4])
        M = [2.0, 0.5, math.inf, 1.0][(t // 16) % 4] if t % 7 else 0.2
        cases.append((v, rho, fix, k, M))
    # a slack budget: fewer nonzero free inputs than kbar
    v = np.zeros(50)
    v[[3, 17, 40]] = [1.5, -0.7, 2.5]
    cases.append((v, 0.5, None, 5, 2.0))
    return cases


def test_prox_threshold_counts_from_independent_definitions():
    """(n_top, n_nz) of prox_g against two definitions that share nothing with
    its block scan of Algorithm 2: (i) read off the prox output alone, a free
    coordinate is before the pooled block exactly when its output is the J1
    prox min(|v_j| / (1 + rho), M) (pooled coordinates get |v_j| - c, which is
    strictly smaller); (ii) from the KKT threshold c found by bisection,
    n_top = #{|v_j| >= c + w(c)} and n_nz = #{|v_j| > c} over Jf."""
    seen_box, seen_free, seen_slack = False, False, False
    for v, rho, fix, k, M in _threshold_cases():
        p = v.size
        fixa = np.zeros(p, dtype=np.int8) if fix is None else fix
        Jf = fixa == 0
        kbar = k - int(np.sum(fixa > 0))
        u, (n_top, n_nz) = R.prox_g(v, rho, fix, k, M, return_info=True)
        m, uf = np.abs(v[Jf]), np.abs(u[Jf])
        # (i) output classification
        j1_like = np.minimum(m / (1.0 + rho), M)
        top_i = (uf > 0) & np.isclose(uf, j1_like, rtol=1e-12, atol=0.0)
        assert n_nz == int(np.count_nonzero(uf))
        assert n_top == int(np.count_nonzero(top_i)), (n_top, int(np.count_nonzero(top_i)))
        # (ii) KKT threshold
        c = _kkt_threshold(m, rho, kbar, M)
        if math.isinf(c):
            assert n_top == n_nz == 0
            continue
        if c == 0.0:
            seen_slack = True
            assert n_top == n_nz == int(np.count_nonzero(m))
            continue
        w = min(c / rho, M)
        T = c + w
        # tie-free: no free input sits within 1e-9 of a breakpoint
        assert np.all(np.abs(m - T) > 1e-9 * T) and np.all(np.abs(m - c) > 1e-9 * c)
        assert n_top == int(np.count_nonzero(m >= T))
        assert n_nz == int(np.count_nonzero(m > c))
        # the pooled coordinates' outputs are |v_j| - c (Algorithm 2's block value)
        mid = (m > c) & (m < T)
        np.testing.assert_allclose(uf[mid], m[mid] - c, rtol=1e-9, atol=1e-12)
        seen_box |= c > rho * M
        seen_free |= c < rho * M
    assert seen_box and seen_free and seen_slack


def test_prox_threshold_counts_catch_block_scan_mistakes():
    """The pin above is sensitive to the plausible mistakes of a block scan:
    counting the pooled block's end instead of its start, a start off by one,
    or the block that holds sorted position kbar (0-based) instead of the one
    straddling kbar - 1 and kbar.  Each mutant disagrees with the KKT count on
    some of the same inputs."""
    mutants = {"end": 0, "start-1": 0, "start+1": 0, "pos-kbar": 0}
    for v, rho, fix, k, M in _threshold_cases():
        p = v.size
        fixa = np.zeros(p, dtype=np.int8) if fix is None else fix
        kbar = k - int(np.sum(fixa > 0))
        Jf = fixa == 0
        m = np.abs(v[Jf])
        c = _kkt_threshold(m, rho, kbar, M)
        if not (0.0 < c < math.inf):
            continue
        truth = int(np.count_nonzero(m >= c + min(c / rho, M)))
        _, (n_top, n_nz) = R.prox_g(v, rho, fix, k, M, return_info=True)
        assert n_top == truth
        _, blocks = R.prox_gstar(v / rho, 1.0 / rho, fix, k, M, return_blocks=True)

        def scan(pick, pos_lo, pos_hi):
            for s_, e_ in blocks:
                if s_ <= pos_lo <= e_ and e_ >= pos_hi:
                    return max(0, min(pick(s_, e_), n_nz))
            return n_nz
        mutants["end"] += scan(lambda s_, e_: e_ + 1, kbar - 1, kbar) != truth
        mutants["start-1"] += scan(lambda s_, e_: s_ - 1, kbar - 1, kbar) != truth
        mutants["start+1"] += scan(lambda s_, e_: s_ + 1, kbar - 1, kbar) != truth
        mutants["pos-kbar"] += scan(lambda s_, e_: s_, kbar, kbar + 1) != truth
    assert all(v > 0 for v in mutants.values()), mutants
