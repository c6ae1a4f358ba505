"""Batched node relaxations (relax_solve_batch): the nodes of one branch-and-
bound tree share X, so their matrix-vector products become X B and X' R
GEMMs, while every node keeps its own FISTA state with gap restarts (Sec. 3.4)
and its own prox / g / g* (Algorithms 1-2) over its node sets (Sec. 2.3).

Each node's result is checked against the FP64 oracle solved on the same node:
the certified bound is valid (never above the oracle's optimum) and within the
bars of the single-node parity tests (FP64: 1e-6 relative at gap 1e-8; FP32:
1e-6 relative at gap 1e-6).  The nodes converge after uneven iteration counts.
"""
import numpy as np
import pytest

import synth
from oracle import solver

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _nodes(p, nb, k, j0_max, j1_max, seed):
    return np.stack([synth.node_fixings(p, seed, j, j0_max, j1_max, k=k) for j in range(nb)])


@pytest.mark.parametrize("loss", ["ls", "logistic"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_batch_matches_oracle_per_node(lib, loss, dtype):
    w = synth.Workload("bt", 300, 700, 0.7, 8, 0.5, loss)
    X, y = synth.make_problem_cpu(w, dtype=dtype)
    X64, y64 = X.astype(np.float64), y.astype(np.float64)
    nb = 6
    fix = _nodes(w.p, nb, w.k, 40, 5, seed=3)
    L = solver.lipschitz(X64, loss)
    tol = 1e-8 if dtype == np.float64 else 1e-6
    h = lib.Handle(torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda"), loss=loss, k=w.k,
                   lambda2=w.lambda2, M=w.M, lipschitz=L)
    beta, res, code = h.solve_batch(nb, fixings=torch.tensor(fix, device="cuda"), gap_tol=tol)
    h.close()
    assert code == 0, lib.STATUS[code]
    iters = []
    for j in range(nb):
        ref = solver.solve(X64, y64, loss, w.k, w.lambda2, w.M, fix=fix[j], gap_tol=1e-12, L=L,
                           max_iters=200000)
        opt = ref.dual_bound
        r = res[j]
        assert r.status == 0 and r.rel_gap <= tol
        assert r.dual_bound <= opt + 1e-12 * abs(opt)          # valid
        assert r.dual_bound == pytest.approx(opt, rel=1e-6)
        b = beta[j].double().cpu().numpy()
        assert np.all(b[fix[j] < 0] == 0.0)                    # J0 stays at zero
        iters.append(r.iters)
    assert len(set(iters)) > 1, iters                          # uneven convergence


def test_batch_agrees_with_single_solves(lib):
    """Same handle, same nodes: the batch's certified bounds agree with
    relax_solve's node by node (different product arithmetic, same method)."""
    w = synth.Workload("bs", 500, 1200, 0.7, 12, 0.5, "ls")
    X, y = synth.make_problem_cpu(w, dtype=np.float32)
    nb = 5
    fix = _nodes(w.p, nb, w.k, 40, 19, seed=11)
    Xd, yd = torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda")
    h = lib.Handle(Xd, yd, loss="ls", k=w.k, lambda2=w.lambda2, M=w.M)
    fixd = torch.tensor(fix, device="cuda")
    _, res, code = h.solve_batch(nb, fixings=fixd, gap_tol=1e-6)
    assert code == 0, lib.STATUS[code]
    for j in range(nb):
        _, r1, c1 = h.solve(fixings=fixd[j].contiguous(), gap_tol=1e-6)
        assert c1 == 0
        assert res[j].dual_bound == pytest.approx(r1.dual_bound, rel=2e-6)
    h.close()


def test_batch_root_with_warm_starts(lib):
    """fixings = NULL (every node the root) with per-node warm starts outside
    dom g: every node reaches the same root bound."""
    w = synth.Workload("bw", 200, 400, 0.6, 6, 0.5, "ls")
    X, y = synth.make_problem_cpu(w, dtype=np.float64)
    L = solver.lipschitz(X, "ls")
    ref = solver.solve(X, y, "ls", w.k, w.lambda2, w.M, gap_tol=1e-12, L=L, max_iters=200000)
    nb = 3
    warm = np.stack([synth.prox_input(w.p, 20 + j, scale=0.5) for j in range(nb)])
    h = lib.Handle(torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda"), loss="ls", k=w.k,
                   lambda2=w.lambda2, M=w.M, lipschitz=L)
    _, res, code = h.solve_batch(nb, warm_start=torch.tensor(warm, device="cuda"), gap_tol=1e-8)
    h.close()
    assert code == 0, lib.STATUS[code]
    for r in res:
        assert r.dual_bound <= ref.dual_bound + 1e-12 * abs(ref.dual_bound)
        assert r.dual_bound == pytest.approx(ref.dual_bound, rel=1e-6)
