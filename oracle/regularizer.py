"""Implicit perspective regularizer g_N, its conjugate and prox (FP64 oracle).

Node N is given by ``fix``: -1 marks J0 (z_j = 0), +1 marks J1 (z_j = 1), 0 marks
Jf (z_j in [0, 1]).  k is the cardinality bound, M the box bound (M may be inf).
Notation follows the paper: kbar = k - |J1|, pbar = |Jf|.
"""
from __future__ import annotations

import math

import numpy as np


def _sets(fix, p):
    fix = np.zeros(p, dtype=np.int8) if fix is None else np.asarray(fix, dtype=np.int8)
    return fix, np.flatnonzero(fix < 0), np.flatnonzero(fix > 0), np.flatnonzero(fix == 0)


def huber(alpha, M):
    """H_M(a) = a^2/2 if |a| <= M else M|a| - M^2/2 (Eq. huber_loss_in_bnb, Sec. 4.1)."""
    a = np.abs(np.asarray(alpha, dtype=np.float64))
    if math.isinf(M):
        return 0.5 * a * a
    return np.where(a <= M, 0.5 * a * a, M * a - 0.5 * M * M)


def prox_huber(x, tau, M):
    """prox of tau*H_M at x (tau >= 0): the a with a + tau*H_M'(a) = x.

    |x| <= M(1+tau): a = x/(1+tau); otherwise a = x - tau*M*sign(x).
    """
    x = np.asarray(x, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64)
    inner = x / (1.0 + tau)
    if math.isinf(M):
        return inner
    return np.where(np.abs(x) <= M * (1.0 + tau), inner, x - tau * M * np.sign(x))


def in_domain(beta, fix, k, M, rtol=0.0):
    """beta in dom g_N: beta_J0 = 0, |beta| <= M, sum_Jf |beta| <= M*kbar (from Eq. 4)."""
    beta = np.asarray(beta, dtype=np.float64)
    fix, J0, J1, Jf = _sets(fix, beta.size)
    kbar = k - J1.size
    if kbar < 0:
        return False
    if np.any(beta[J0] != 0.0):
        return False
    if math.isinf(M):
        return bool(kbar > 0 or np.all(beta[Jf] == 0.0))
    if np.any(np.abs(beta) > M * (1.0 + rtol)):
        return False
    return bool(np.sum(np.abs(beta[Jf])) <= M * kbar * (1.0 + rtol))


DOMAIN_RTOL = 1e-12


def g_alg1(beta, fix, k, M, domain_rtol=DOMAIN_RTOL):
    """g_N(beta) by Algorithm 1 (Thm 4.4); +inf outside dom g_N.

    Points within domain_rtol (relative) of the box or l1 boundary count as on
    it, so that rounding of a boundary point does not make g infinite.
    """
    beta = np.asarray(beta, dtype=np.float64)
    fix, J0, J1, Jf = _sets(fix, beta.size)
    if not in_domain(beta, fix, k, M, rtol=domain_rtol):
        return math.inf
    kbar = k - J1.size
    pbar = Jf.size
    val = 0.5 * float(np.sum(beta[J1] ** 2))
    if kbar == 0 or pbar == 0:
        return val
    b = np.sort(np.abs(beta[Jf]))[::-1]          # |b_(1)| >= ... >= |b_(pbar)|
    theta = float(np.sum(b))
    omega = np.zeros(kbar)
    for j in range(1, kbar + 1):                  # j = 1..kbar
        bj = b[j - 1] if j <= pbar else 0.0
        tbar = theta / (kbar - j + 1)
        if tbar >= bj:
            omega[j - 1:] = tbar
            break
        omega[j - 1] = bj
        theta -= bj
    return val + 0.5 * float(np.sum(omega ** 2))


def g_bisect(beta, fix, k, M, iters=200):
    """g_N(beta) straight from its definition (Eq. 5), independent of Algorithm 1.

    For fixed beta the infimum over z separates: z_j = 1 on J1, z_j = 0 on J0,
    and on Jf minimize (1/2) sum beta_j^2 / z_j subject to sum z_j <= kbar,
    |beta_j|/M <= z_j <= 1.  Its KKT point is z_j = clip(s |beta_j|, |beta_j|/M, 1)
    for a scalar s >= 0 fixed by sum z_j = kbar (when that bound is active); s is
    found by bisection.
    """
    beta = np.asarray(beta, dtype=np.float64)
    fix, J0, J1, Jf = _sets(fix, beta.size)
    if not in_domain(beta, fix, k, M, rtol=DOMAIN_RTOL):
        return math.inf
    kbar = k - J1.size
    val = 0.5 * float(np.sum(beta[J1] ** 2))
    b = np.abs(beta[Jf])
    b = b[b > 0]
    if b.size == 0:
        return val
    lo_z = (b / M) if not math.isinf(M) else np.zeros_like(b)
    if b.size <= kbar:                            # z = 1 everywhere is feasible and optimal
        return val + 0.5 * float(np.sum(b ** 2))

    def zsum(s):
        return float(np.sum(np.clip(s * b, lo_z, 1.0)))

    lo, hi = 0.0, 1.0
    while zsum(hi) < kbar:
        hi *= 2.0
        if hi > 1e300:
            break
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if zsum(mid) < kbar:
            lo = mid
        else:
            hi = mid
    z = np.clip(hi * b, lo_z, 1.0)
    return val + 0.5 * float(np.sum(b * b / z))


def gstar(alpha, fix, k, M):
    """g_N*(alpha) = sum_J1 H_M(alpha_j) + TopSum_{kbar}(H_M(alpha_Jf)) (Lemma 4.2)."""
    alpha = np.asarray(alpha, dtype=np.float64)
    fix, J0, J1, Jf = _sets(fix, alpha.size)
    kbar = k - J1.size
    if kbar < 0:
        raise ValueError("k < |J1|")
    h = np.sort(huber(alpha[Jf], M))[::-1]
    return float(np.sum(huber(alpha[J1], M))) + float(np.sum(h[:kbar]))


def prox_gstar(beta, rho, fix, k, M, return_blocks=False):
    """prox of rho*g_N* at beta by Algorithm 2 (sort + pool adjacent violators).

    The pooled quantities are the magnitudes |beta_pi(j)| (the sign is re-applied
    at the end).  PAVA is the textbook stack form (each new position is pushed as
    its own block and merged backwards while the fit is increasing), not the
    paper's block up-and-down search, which lives in its missing appendix.
    """
    beta = np.asarray(beta, dtype=np.float64)
    p = beta.size
    fix, J0, J1, Jf = _sets(fix, p)
    kbar = k - J1.size
    if kbar < 0:
        raise ValueError("k < |J1|")
    pbar = Jf.size
    alpha = np.empty(p, dtype=np.float64)
    alpha[J0] = beta[J0]
    alpha[J1] = prox_huber(beta[J1], rho, M)
    blocks = []
    if pbar > 0:
        bbar = beta[Jf]
        mag = np.abs(bbar)
        pi = np.lexsort((np.arange(pbar), -mag))   # |.| descending, ties by index
        w = np.where(np.arange(pbar) < kbar, rho, 0.0)
        # stack of blocks: [start, end, sum_w, sum_x, value]
        for j in range(pbar):
            x = mag[pi[j]]
            blocks.append([j, j, w[j], x, float(prox_huber(x, w[j], M))])
            while len(blocks) > 1 and blocks[-2][4] < blocks[-1][4]:
                b2 = blocks.pop()
                b1 = blocks.pop()
                cnt = b2[1] - b1[0] + 1
                sw = b1[2] + b2[2]
                sx = b1[3] + b2[3]
                blocks.append([b1[0], b2[1], sw, sx, float(prox_huber(sx / cnt, sw / cnt, M))])
        ahat = np.empty(pbar)
        for b in blocks:
            ahat[b[0]:b[1] + 1] = b[4]
        out = np.empty(pbar)
        out[pi] = ahat
        alpha[Jf] = np.sign(bbar) * out
    if return_blocks:
        return alpha, [(b[0], b[1]) for b in blocks]
    return alpha


def prox_g(v, rho, fix, k, M, return_info=False):
    """prox of rho*g_N at v by the extended Moreau decomposition (Eq. prox:gN):
    prox_{rho g}(v) = v - rho * prox_{rho^{-1} g*}(v / rho).

    On free positions that Algorithm 2 leaves as unpooled singletons of weight 0
    (sorted position > kbar) the conjugate prox returns v/rho itself, so the
    primal output is exactly 0; it is set to 0 there rather than left as the
    +-1 ulp residue of v - rho*(v/rho).

    With ``return_info`` also returns (n_top, n_nz): the number of free
    coordinates placed before the pooled block that straddles sorted positions
    kbar and kbar+1 (all nonzero free coordinates when nothing is pooled there),
    and the number of nonzero free outputs.
    """
    v = np.asarray(v, dtype=np.float64)
    fix, J0, J1, Jf = _sets(fix, v.size)
    kbar = k - J1.size
    alpha, blocks = prox_gstar(v / rho, 1.0 / rho, fix, k, M, return_blocks=True)
    u = v - rho * alpha
    u[J0] = 0.0
    if Jf.size > 0:
        mag = np.abs(v[Jf])
        pi = np.lexsort((np.arange(Jf.size), -mag))
        uf = u[Jf]
        for s, e in blocks:
            if s == e and s >= kbar:
                uf[pi[s]] = 0.0
        u[Jf] = uf
    if not return_info:
        return u
    n_nz = int(np.count_nonzero(u[Jf]))
    n_top = n_nz
    if 0 < kbar < Jf.size:
        for s, e in blocks:
            if s <= kbar - 1 <= e and e >= kbar:      # 0-based positions kbar-1, kbar
                n_top = min(s, n_nz)
                break
    return u, (n_top, n_nz)
