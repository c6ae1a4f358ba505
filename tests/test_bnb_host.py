"""Host logic of the branch-and-bound driver and of the warm-start parameter
block (no GPU): branching choice, incumbent support, parameter layout."""
import numpy as np
import pytest

from oracle import mlp


def test_branch_variable_is_the_largest_free_coordinate():
    from paper_2603_01306_gb300.bnb import _branch_var
    beta = np.array([0.5, -3.0, 2.0, 0.0, -2.5])
    fix = np.array([0, -1, 1, 0, 0], dtype=np.int8)    # |beta_1| is largest but in J0; beta_2 is in J1
    assert _branch_var(beta, fix) == 4
    assert _branch_var(np.array([0.0, 1.0]), np.array([0, 1], dtype=np.int8)) == -1   # nothing free and nonzero


def test_incumbent_support_keeps_j1_and_fills_by_magnitude():
    from paper_2603_01306_gb300.bnb import _incumbent_fix
    beta = np.array([0.1, -0.9, 0.05, 0.7, 0.0, -0.3])
    fix = np.array([1, 0, 0, 0, 0, -1], dtype=np.int8)
    f = _incumbent_fix(beta, fix, k=3)
    assert list(np.flatnonzero(f == 1)) == [0, 1, 3]   # J1 first, then |beta| descending
    assert np.all(f[[2, 4, 5]] == -1)                  # everything else fixed to zero
    # fewer free nonzeros than k: the support stays smaller, zeros are never added
    f2 = _incumbent_fix(np.array([0.0, 0.2, 0.0]), np.zeros(3, dtype=np.int8), k=3)
    assert list(np.flatnonzero(f2 == 1)) == [1]


def test_parameter_block_layout_and_initial_network():
    from paper_2603_01306_gb300.binding import MLP_NPARAM, MLP_NTRAIN
    from paper_2603_01306_gb300.warmstart import init_params
    assert (MLP_NTRAIN, MLP_NPARAM) == (mlp.N_TRAIN, mlp.N_PARAM)
    th = init_params(seed=3)
    assert th.shape == (MLP_NPARAM,)
    W1, b1, W2, b2, w3, b3, shift, scale = mlp.unpack(th)
    assert np.all(w3 == 0) and b3 == 0                 # the untrained network is the parent start
    assert np.all(shift == 0) and np.all(scale == 1)
    assert W1.std() == pytest.approx(np.sqrt(2 / 5), rel=0.2)
    assert W2.std() == pytest.approx(np.sqrt(2 / 64), rel=0.1)
    F = np.random.default_rng(0).standard_normal((9, 5))
    out, _ = mlp.forward(th, F)
    assert np.all(out == 0)


class _OracleHandle:
    """A stand-in for the device handle with the same methods the driver
    calls, solving each node with the FP64 oracle on the CPU (test
    infrastructure only).  `fail` lists fixings (as bytes) whose solve
    returns RELAX_ECUDA, a failure injected on the host."""

    def __init__(self, X, y, k, lam2, M, fail=()):
        import torch
        self.X = torch.tensor(X)
        self.Xn, self.y, self.k, self.lam2, self.M = X, y, k, lam2, M
        self.p = X.shape[1]
        self.dtype = torch.float64
        self.cut = float("inf")
        self.fail = set(fail)
        self.cut_calls = []

    def set_cutoff(self, c=float("inf")):
        self.cut = c
        self.cut_calls.append(c)

    def solve(self, fixings=None, warm_start=None, gap_tol=1e-6, beta_out=None):
        import types
        import torch
        from oracle import variants
        fix = fixings.cpu().numpy()
        warm = None if warm_start is None else warm_start.double().cpu().numpy()
        cut = None if self.cut == float("inf") else self.cut
        r = variants.solve(self.Xn, self.y, "ls", self.k, self.lam2, self.M, fix=fix, warm=warm,
                           gap_tol=gap_tol, cutoff=cut)
        code = 0 if (r.converged or r.cutoff_rule) else 4
        if fix.tobytes() in self.fail:
            code = 3
        res = types.SimpleNamespace(primal=r.primal, dual_bound=r.dual_bound, iters=r.iters,
                                    cutoff_rule=r.cutoff_rule, polish_iters=0, status=code)
        return torch.tensor(r.beta), res, code


def _tiny(seed=0):
    import synth
    X = synth.ar1_design(30, 7, 0.5, seed)
    y = synth.response(synth.signal_from_design(X, 2), "ls", 4.0, seed)
    return X, y


def test_bnb_reaches_the_bruteforce_optimum_with_cutoffs():
    """With every solve exact (oracle) the queue empties, the run is
    certified and its incumbent is the k-sparse optimum by support
    enumeration; children are solved with the incumbent as cutoff."""
    from oracle import brute
    from paper_2603_01306_gb300 import bnb
    X, y = _tiny()
    k, lam2, M = 2, 0.3, 2.0
    h = _OracleHandle(X, y, k, lam2, M)
    st = bnb.run(h, k, max_nodes=200, gap_tol=1e-9)
    opt = brute.ksparse_opt(X, y, "ls", k, lam2, M)
    assert st.certified and not st.dropped
    assert st.incumbent == pytest.approx(opt, rel=1e-7)
    assert st.best_bound == st.incumbent
    assert any(c != float("inf") for c in h.cut_calls)     # children ran with the incumbent cutoff
    assert h.cut == float("inf")                            # and the handle is left without one
    st2 = bnb.run(_OracleHandle(X, y, k, lam2, M), k, max_nodes=200, gap_tol=1e-9, cutoff=False)
    assert st2.certified and st2.incumbent == pytest.approx(opt, rel=1e-7)
    assert st.cut_branch + st.cut_prune > 0 and st2.cut_branch + st2.cut_prune == 0


def test_bnb_is_not_certified_when_a_child_solve_fails():
    from paper_2603_01306_gb300 import bnb
    X, y = _tiny(1)
    k, lam2, M = 2, 0.3, 2.0
    # find the first child the driver will solve: the root's branching coordinate to J0
    probe = _OracleHandle(X, y, k, lam2, M)
    import torch
    b0, r0, _ = probe.solve(torch.zeros(7, dtype=torch.int8), gap_tol=1e-9)
    j = bnb._branch_var(b0.numpy(), np.zeros(7, dtype=np.int8))
    f0 = np.zeros(7, dtype=np.int8)
    f0[j] = -1
    h = _OracleHandle(X, y, k, lam2, M, fail=[f0.tobytes()])
    st = bnb.run(h, k, max_nodes=200, gap_tol=1e-9)
    assert not st.certified
    assert st.dropped == [pytest.approx(r0.dual_bound)]     # the root's bound covers the lost subtree
    assert st.best_bound <= r0.dual_bound


@pytest.mark.parametrize("batch", [1, 4])
def test_bnb_is_not_certified_when_the_node_budget_runs_out(batch):
    from paper_2603_01306_gb300 import bnb
    X, y = _tiny(2)
    k, lam2, M = 3, 0.2, 2.0
    h = _OracleHandle(X, y, k, lam2, M)
    h.solve_batch = None   # the batched path is exercised below through a list of single solves

    def solve_batch(nb, fixings=None, warm_start=None, gap_tol=1e-6, beta_out=None):
        import torch
        outs = [h.solve(fixings[i], warm_start[i], gap_tol) for i in range(nb)]
        return torch.stack([o[0] for o in outs]), [o[1] for o in outs], 0
    h.solve_batch = solve_batch
    st = bnb.run(h, k, max_nodes=3, gap_tol=1e-9, batch=batch)
    assert st.nodes <= 3
    assert not st.certified
    assert st.best_bound <= st.incumbent


def test_batched_bnb_reaches_the_optimum_and_solves_each_support_once():
    """The batched driver (children of several open nodes per call) reaches
    the brute-force k-sparse optimum, certified; its incumbent heuristic
    solves every candidate support once (later candidates with a support
    already solved reuse its objective)."""
    import torch
    from oracle import brute
    from paper_2603_01306_gb300 import bnb
    import synth
    # a weak signal (SNR 1) on 30 x 12, k = 3: 37 nodes, and candidate
    # supports that repeat across the tree
    X = synth.ar1_design(30, 12, 0.5, 1)
    y = synth.response(synth.signal_from_design(X, 3), "ls", 1.0, 1)
    k, lam2, M = 3, 0.05, 2.0
    h = _OracleHandle(X, y, k, lam2, M)
    incumbent_supports = []
    candidates = []
    fix_of = bnb._incumbent_fix

    def solve_batch(nb, fixings=None, warm_start=None, gap_tol=1e-6, beta_out=None):
        if h.cut == float("inf"):   # the incumbent heuristic's solves run without a cutoff
            incumbent_supports.extend(np.flatnonzero(fixings[i].cpu().numpy() > 0).tobytes() for i in range(nb))
        outs = [h.solve(fixings[i], None if warm_start is None else warm_start[i], gap_tol) for i in range(nb)]
        return torch.stack([o[0] for o in outs]), [o[1] for o in outs], 0
    h.solve_batch = solve_batch

    def counting_fix(beta, fix, kk):
        f = fix_of(beta, fix, kk)
        candidates.append(np.flatnonzero(f > 0).tobytes())
        return f
    bnb._incumbent_fix = counting_fix
    try:
        st = bnb.run(h, k, max_nodes=400, gap_tol=1e-9, batch=4)
    finally:
        bnb._incumbent_fix = fix_of
    opt = brute.ksparse_opt(X, y, "ls", k, lam2, M)
    assert st.certified and not st.dropped
    assert st.incumbent == pytest.approx(opt, rel=1e-7)
    assert st.best_bound == st.incumbent
    assert len(incumbent_supports) == len(set(incumbent_supports))   # no support solved twice
    assert st.incumbent_solves == len(incumbent_supports) + 1         # + the root's, solved alone
    assert len(incumbent_supports) >= 5
    # every distinct candidate support was solved exactly once (the root's alone)
    assert set(incumbent_supports) <= set(candidates)
    assert len(set(candidates)) == len(incumbent_supports) + 1
