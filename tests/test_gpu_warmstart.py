"""Learned warm start (include/warmstart.h) against the FP64 oracle
(oracle/mlp.py), through the C ABI.

Bars: with FP32 weights the forward pass and the gradient match the oracle
evaluated at the same (FP32-stored) parameters to 1e-5 relative; with BF16
weights they match the oracle at the BF16-rounded parameters to 1e-5 and the
unrounded FP64 network to 1e-2.  Adam's step matches to FP32 rounding.  The
features match the oracle's definitions to FP32 rounding.  Training on
(parent, child) node solves of a branch and bound lowers the held-out squared
error below the parent start's, and the iterations to gap of the held-out
children are reported for both starts.
"""
import numpy as np
import pytest

import synth
from oracle import mlp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _theta(seed=1, rows=None):
    rng = np.random.default_rng(seed)
    F = rows if rows is not None else rng.standard_normal((1000, 5))
    th = mlp.init(seed=seed, shift=F.mean(axis=0), scale=F.std(axis=0))
    o = mlp.NH * mlp.NIN + mlp.NH + mlp.NH * mlp.NH + mlp.NH
    th[o:o + mlp.NH] = rng.standard_normal(mlp.NH) * 0.2
    th[o + mlp.NH] = 0.05
    return th.astype(np.float32).astype(np.float64)      # the device keeps FP32 parameters


def _feats(N, seed=0):
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((N, 5)) * np.array([0.4, 3.0, 1.0, 2.0, 0.2]) + np.array([0, 0.5, 0, 6, 0.3])
    F[:, 2] = rng.integers(-1, 2, N)
    return F.astype(np.float32).astype(np.float64)


def _dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


def _magnitude(th, F):
    """Per row: the network's output with every weight, bias and standardised
    input replaced by its absolute value (ReLU activations as the oracle
    computes them): the scale of the rounding error of any evaluation that
    sums the same terms in FP32."""
    W1, b1, W2, b2, w3, b3, shift, scale = mlp.unpack(th)
    x = np.abs((F - shift) / scale)
    h1 = x @ np.abs(W1).T + np.abs(b1)
    h2 = h1 @ np.abs(W2).T + np.abs(b2)
    return h2 @ np.abs(w3) + abs(b3)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("N", [1, 127, 3001])
def test_forward_matches_oracle(lib, bf16, N):
    F = _feats(N, seed=N)
    th = _theta(rows=F if N > 10 else None)
    out = torch.empty(N, dtype=torch.float32, device="cuda")
    lib.relax_mlp_forward(_dev(th), _dev(F), out, base=None, bf16=bf16)
    got = out.double().cpu().numpy()
    th_same = mlp.bf16_weights(th) if bf16 else th
    ref_same, _ = mlp.forward(th_same, F)
    # element by element: each output against the FP32 accumulation bar of
    # its own row, relative to the same network evaluated on magnitudes
    # (|W| applied to |inputs| layer by layer), which bounds the rounding of
    # every partial sum even where the output cancels
    assert np.all(np.abs(got - ref_same) <= 1e-5 * _magnitude(th_same, F))
    if bf16:
        # against the unrounded FP64 network, per row relative to the output's
        # magnitude sum (the rounding of each weight is relative; the output
        # can cancel)
        ref64, (_, _, _, _, h2) = mlp.forward(th, F)
        w3, b3 = mlp.unpack(th)[4:6]
        mag = h2 @ np.abs(w3) + abs(b3)
        assert np.all(np.abs(got - ref64) <= 1e-2 * mag)


def test_start_is_zero_on_j0_and_base_plus_f_elsewhere(lib):
    F = _feats(777, seed=3)
    th = _theta(rows=F)
    out = torch.empty(777, dtype=torch.float32, device="cuda")
    lib.relax_mlp_forward(_dev(th), _dev(F), out, base=_dev(F[:, 0]), bf16=False)
    got = out.double().cpu().numpy()
    ref = mlp.start(th, F)
    assert np.all(got[F[:, 2] < 0] == 0.0)
    assert np.all(np.abs(got - ref) <= 1e-5 * (np.abs(F[:, 0]) + _magnitude(th, F)))


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("N", [5, 128, 4099])
def test_gradient_matches_oracle(lib, bf16, N):
    F = _feats(N, seed=10 + N)
    th = _theta(seed=2, rows=F if N > 10 else None)
    rng = np.random.default_rng(N)
    base = F[:, 0]
    target = (base + 0.3 * rng.standard_normal(N)).astype(np.float32).astype(np.float64)
    grad = torch.empty(mlp.N_PARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    lib.relax_mlp_grad(_dev(th), _dev(F), _dev(base), _dev(target), grad, loss, bf16=bf16)
    g = grad.double().cpu().numpy()
    L_ref, g_ref = mlp.loss_and_grad(mlp.bf16_weights(th) if bf16 else th, F, base, target)
    assert _rel(g, g_ref) <= 1e-5
    assert float(loss.item()) == pytest.approx(L_ref, rel=1e-5)
    assert np.all(g[mlp.N_TRAIN:] == 0.0)
    # the four parameter groups separately (a layer with small gradients must
    # not hide behind a large one)
    o = [0, mlp.NH * mlp.NIN + mlp.NH, mlp.NH * mlp.NIN + mlp.NH + mlp.NH * mlp.NH + mlp.NH, mlp.N_TRAIN]
    for a, b in zip(o[:-1], o[1:]):
        assert _rel(g[a:b], g_ref[a:b]) <= 2e-5
    if bf16 and N >= 128:
        # against the unrounded FP64 network, norm-wise over many rows (a
        # handful of rows can cancel)
        _, g64 = mlp.loss_and_grad(th, F, base, target)
        assert _rel(g, g64) <= 1e-2
    # reproducible bit for bit
    grad2 = torch.empty_like(grad)
    lib.relax_mlp_grad(_dev(th), _dev(F), _dev(base), _dev(target), grad2, None, bf16=bf16)
    assert torch.equal(grad, grad2)


def test_adam_matches_oracle(lib):
    rng = np.random.default_rng(4)
    th = _theta(seed=4)
    g = rng.standard_normal(mlp.N_PARAM) * 1e-2
    g[mlp.N_TRAIN:] = 0.0
    m = (rng.standard_normal(mlp.N_TRAIN) * 1e-3).astype(np.float32).astype(np.float64)
    v = (rng.random(mlp.N_TRAIN) * 1e-5).astype(np.float32).astype(np.float64)
    g = g.astype(np.float32).astype(np.float64)
    thd, md, vd = _dev(th), _dev(m), _dev(v)
    lib.relax_mlp_adam(thd, _dev(g), md, vd, 3, 1e-3)
    th_ref, m_ref, v_ref = mlp.adam_step(th, g, m, v, 3, 1e-3)
    # FP32 moments: rounding of each term (|0.9 m| + |0.1 g| up to about 3e-3)
    np.testing.assert_allclose(md.double().cpu().numpy(), m_ref, rtol=1e-6, atol=2e-9)
    np.testing.assert_allclose(vd.double().cpu().numpy(), v_ref, rtol=1e-6, atol=1e-13)
    np.testing.assert_allclose(thd.double().cpu().numpy(), th_ref, rtol=1e-6, atol=2e-7)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_features_match_oracle(lib, dtype):
    w = synth.Workload("wf", 300, 700, 0.7, 8, 0.5, "ls")
    X, y = synth.make_problem_cpu(w, dtype=dtype)
    X64, y64 = X.astype(np.float64), y.astype(np.float64)
    h = lib.Handle(torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda"), loss="ls", k=w.k,
                   lambda2=w.lambda2, M=w.M, lipschitz=1.0)
    bp = synth.prox_input(w.p, 5, scale=0.2).astype(dtype)
    fix = synth.node_fixings(w.p, 1, 0, 40, 5, k=w.k)
    F = h.mlp_features(torch.tensor(bp, device="cuda"), torch.tensor(fix, device="cuda"))
    h.close()
    got = F.double().cpu().numpy()
    b = mlp.projected_parent(bp.astype(np.float64), fix)
    norms, corr = mlp.column_stats(X64, y64)
    ref = mlp.features(b, mlp.parent_gradient(X64, y64, "ls", b), fix, norms, corr)
    # FP32 output (2^-24 relative) of FP64 quantities; with FP32 X the gradient
    # carries the FP32 pass's error (2e-6 of sum_i |x_ij r_i|)
    for c in range(5):
        eps = 2e-5 if (c == 1 and dtype == np.float32) else 1e-6
        scale = np.abs(ref[:, c]).max() + 1e-300
        assert np.max(np.abs(got[:, c] - ref[:, c])) <= eps * scale, c


def test_learned_start_on_branch_and_bound_nodes(lib):
    """Train on the (parent, child) pairs of one best-first branch and bound and
    measure on held-out children: the squared error of the start against the
    child's solution (the network must beat the parent start), and iterations
    to gap 1e-6 from the parent start and from the learned start with its Phi
    fallback (reported; the fallback must not cost more than 5%).  Measured on
    GB300 (200 nodes, 49 held out): MSE 1.4e-4 -> 5.2e-5, iterations 14972 ->
    15017: the start is closer, the iteration count is set by the linear rate
    of the restarted method, not by the start."""
    from paper_2603_01306_gb300 import bnb
    from paper_2603_01306_gb300.warmstart import WarmStartNet
    w = synth.Workload("wb", 800, 2000, 0.8, 15, 0.2, "ls")
    X, y = synth.make_problem_cpu(w)
    Xd, yd = torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda")
    h = lib.Handle(Xd, yd, loss="ls", k=w.k, lambda2=w.lambda2, M=w.M)
    st = bnb.run(h, w.k, max_nodes=120, gap_tol=1e-6, warm="parent", record=True)
    pairs = st.pairs
    assert len(pairs) >= 100
    train, held = pairs[:-30], pairs[-30:]
    Ftr, Ttr = bnb.training_rows(h, train)
    Fte, Tte = bnb.training_rows(h, held)
    net = WarmStartNet(seed=0)
    net.set_standardisation(Ftr)
    mse_parent = net.loss_of(Fte, Tte)          # zero output layer: the parent start
    net.fit(Ftr, Ttr, epochs=60, batch=8192, lr=2e-3)
    mse_learned = net.loss_of(Fte, Tte)
    print(f"held-out MSE of the start: parent {mse_parent:.4e}, learned {mse_learned:.4e}")
    assert mse_learned < 0.8 * mse_parent
    it_parent = it_learned = used = 0
    for pb, fix, cb in held:
        fx = torch.tensor(fix, device="cuda")
        _, r0, c0 = h.solve(fixings=fx, warm_start=pb, gap_tol=1e-6)
        start, u = bnb.learned_start(h, net, pb, fx)
        used += int(u)
        _, r1, c1 = h.solve(fixings=fx, warm_start=start, gap_tol=1e-6)
        assert c0 in (0, 4) and c1 in (0, 4)
        # the same node: the two certified bounds agree
        assert r1.dual_bound == pytest.approx(r0.dual_bound, rel=2e-6)
        it_parent += r0.iters
        it_learned += r1.iters
    print(f"iterations to gap 1e-6 over {len(held)} held-out children: parent {it_parent}, "
          f"learned with fallback {it_learned} (learned start used for {used})")
    assert it_learned <= 1.05 * it_parent
    h.close()
