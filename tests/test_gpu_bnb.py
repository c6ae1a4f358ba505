"""The branch-and-bound driver on the GPU: children solved one at a time and
children of up to 16 open nodes solved together in one batched call.  A
child's feasible set is inside its parent's, so its relaxation bound is at
least the parent's (up to the certified gap of the two solves); every
incumbent is a feasible value, so no open bound exceeds it by more than the
same tolerance."""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_sequential_and_batched_bnb(lib):
    """With and without the dynamic termination of Sec. 5.3: children solved
    to the gap have bounds at least their parent's; children stopped by
    rule 1 carry an earlier (valid, looser) bound; rule 2 prunes."""
    from paper_2603_01306_gb300 import bnb
    w = synth.Workload("bb", 800, 2000, 0.8, 15, 0.2, "ls")
    X, y = synth.make_problem_cpu(w)
    h = lib.Handle(torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda"), loss="ls", k=w.k,
                   lambda2=w.lambda2, M=w.M)
    runs = {}
    for batch in (1, 16):
        for cutoff in (False, True):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = bnb.run(h, w.k, max_nodes=97, gap_tol=1e-6, batch=batch, cutoff=cutoff)
            torch.cuda.synchronize()
            runs[batch, cutoff] = (st, time.perf_counter() - t0)
    h.close()
    for (batch, cutoff), (st, secs) in runs.items():
        assert st.nodes == 97
        assert len(st.bounds) == st.nodes - 1                  # every child, not the root
        for pb, cb, rule in st.bounds:
            if rule == 0:
                assert cb >= pb - 2e-6 * max(1.0, abs(pb)), (batch, pb, cb)
            else:
                assert cutoff
        assert st.best_bound <= st.incumbent * (1 + 2e-6)
        if not cutoff:
            assert st.cut_branch == st.cut_prune == 0
        print(f"batch {batch} cutoff {cutoff}: {st.nodes} nodes in {secs:.2f} s ({st.nodes / secs:.1f} nodes/s), "
              f"iterations {st.iters} (rule 1: {st.cut_branch}, rule 2: {st.cut_prune}), "
              f"incumbent {st.incumbent:.6f}, best open bound {st.best_bound:.6f}")
    # the early stops save iterations
    assert runs[1, True][0].cut_branch + runs[1, True][0].cut_prune > 0


def test_certify_batch_matches_single_certify(lib):
    """relax_certify_batch: the same {Phi, Psi} as relax_certify point by
    point (same passes, enqueued together), with and without fixings; +inf
    Phi for a point outside dom g (a nonzero on a J0 coordinate)."""
    w = synth.Workload("cb", 300, 700, 0.6, 8, 0.5, "ls")
    X, y = synth.make_problem_cpu(w)
    Xd, yd = torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda")
    h = lib.Handle(Xd, yd, loss="ls", k=w.k, lambda2=w.lambda2, M=w.M)
    rng = np.random.default_rng(5)
    nb = 6
    pts = np.zeros((nb, w.p), dtype=np.float32)
    for s in range(nb):
        idx = rng.choice(w.p, 6, replace=False)
        pts[s, idx] = rng.uniform(-1.5, 1.5, 6)
    fix = np.zeros((nb, w.p), dtype=np.int8)
    fix[1, 3:9] = -1
    fix[2, np.flatnonzero(pts[2])[:2]] = 1
    fix[3, np.flatnonzero(pts[3])[0]] = -1        # a nonzero in J0: outside dom g
    pd = torch.tensor(pts, device="cuda")
    fd = torch.tensor(fix, device="cuda")
    got = h.certify_batch(pd, fd)
    for s in range(nb):
        ref = h.certify(pd[s].contiguous(), fixings=fd[s].contiguous())
        assert got[s, 0] == ref[0] or (np.isinf(got[s, 0]) and np.isinf(ref[0]))
        assert got[s, 1] == ref[1]
    assert np.isinf(got[3, 0])
    free = h.certify_batch(pd)
    for s in range(nb):
        ref = h.certify(pd[s].contiguous())
        assert free[s, 0] == ref[0] and free[s, 1] == ref[1]
    bad = fix.copy()
    bad[0, :w.k + 1] = 1                           # more than k in J1
    with pytest.raises(lib.RelaxError):
        h.certify_batch(pd, torch.tensor(bad, device="cuda"))
    h.close()
