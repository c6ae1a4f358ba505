"""The certificate on the device against the oracle: Phi(beta) = F(X beta) +
2 lambda2 g_N(beta) (Eq. 6) and Psi(zeta) at the induced dual point zeta =
-grad F(X beta_d) (Eq. 7, Sec. 3.3).

Three device paths are covered:
* relax_certify with two different vectors: two forward products in one pass
  (Phi at beta_p, the dual point from X beta_d);
* relax_certify / relax_certify_batch with one vector: one product;
* the solve's certificate: one pass with two right-hand sides, Psi at the
  loop's dual point and at -grad F(X beta_best), the better one reported.
FP64 data takes FP64 passes; FP32 data float-float passes on the FP32 X,
whose values the oracle takes exactly (in FP64)."""
import numpy as np
import pytest

import synth
from oracle import solver

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _points(rng, p, k, M, count):
    """Sparse points inside dom g: at most k nonzeros of magnitude <= M."""
    pts = np.zeros((count, p))
    for s in range(count):
        idx = rng.choice(p, k - 1, replace=False)
        pts[s, idx] = rng.uniform(-0.9 * M, 0.9 * M, k - 1)
    return pts


def _tol(dtype):
    # FP64 passes: fixed-point z and FP64 sums; FP32 data: float-float
    # products and sums (about 48 bits) -- both far below this bar
    return 1e-10 if dtype == np.float64 else 1e-9


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("loss", ["ls", "logistic"])
def test_certify_is_the_oracles(lib, loss, dtype):
    w = synth.Workload("cert", 400, 900, 0.6, 8, 0.5, loss)
    X, y = synth.make_problem_cpu(w, dtype=dtype)
    X64, y64 = X.astype(np.float64), y.astype(np.float64)
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    h = lib.Handle(torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda"), loss=loss, k=w.k,
                   lambda2=w.lambda2, M=w.M)
    rng = np.random.default_rng(11)
    pts = _points(rng, w.p, w.k, w.M, 4).astype(dtype)
    fix = np.zeros((4, w.p), dtype=np.int8)
    fix[1, np.flatnonzero(pts[1])[:2]] = 1                  # J1 on two of the support
    zero = np.flatnonzero(pts[2] == 0)[:30]
    fix[2, zero] = -1                                       # J0 on coordinates that are zero
    tol = _tol(dtype)
    for s in range(4):
        bp = pts[s]
        bd = pts[(s + 1) % 4]
        fx = fix[s] if fix[s].any() else None
        fxd = None if fx is None else torch.tensor(fx, device="cuda")
        fo = np.zeros(w.p, dtype=np.int8) if fx is None else fx
        phi = solver.primal(bp.astype(np.float64), X64, y64, loss, fo, w.k, w.M, w.lambda2)
        for dual_vec in (bd, bp):
            zeta = solver.induced_dual(dual_vec.astype(np.float64), X64, y64, loss)
            psi = solver.dual(zeta, X64, y64, loss, fo, w.k, w.M, w.lambda2)
            bpt = torch.tensor(bp, dtype=tdt, device="cuda")
            if dual_vec is bp:
                got = h.certify(bpt, fixings=fxd)                          # one product
            else:
                got = h.certify(bpt, torch.tensor(bd, dtype=tdt, device="cuda"), fixings=fxd)
            assert abs(got[0] - phi) <= tol * max(1.0, abs(phi)), (s, got[0], phi)
            assert abs(got[1] - psi) <= tol * max(1.0, abs(psi)), (s, got[1], psi)
    # the batched entry point, one product per point
    got = h.certify_batch(torch.tensor(pts, device="cuda"), torch.tensor(fix, device="cuda"))
    for s in range(4):
        zeta = solver.induced_dual(pts[s].astype(np.float64), X64, y64, loss)
        psi = solver.dual(zeta, X64, y64, loss, fix[s], w.k, w.M, w.lambda2)
        phi = solver.primal(pts[s].astype(np.float64), X64, y64, loss, fix[s], w.k, w.M, w.lambda2)
        assert abs(got[s, 0] - phi) <= tol * max(1.0, abs(phi))
        assert abs(got[s, 1] - psi) <= tol * max(1.0, abs(psi))
    h.close()


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("loss", ["ls", "logistic"])
def test_solve_certificate_is_the_oracles(lib, loss, dtype):
    """The solve's certified values at its returned beta: Phi equal to the
    oracle's Phi(beta); the bound at least the oracle's Psi at -grad F(X
    beta) (the better of that and the loop's dual point is kept) and at most
    Phi (weak duality)."""
    w = synth.Workload("cert", 400, 900, 0.6, 8, 0.5, loss)
    X, y = synth.make_problem_cpu(w, dtype=dtype)
    X64, y64 = X.astype(np.float64), y.astype(np.float64)
    h = lib.Handle(torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda"), loss=loss, k=w.k,
                   lambda2=w.lambda2, M=w.M)
    beta, res, code = h.solve(gap_tol=1e-6)
    h.close()
    assert code == 0
    b = beta.double().cpu().numpy()
    fo = np.zeros(w.p, dtype=np.int8)
    phi = solver.primal(b, X64, y64, loss, fo, w.k, w.M, w.lambda2)
    psi_self = solver.dual(solver.induced_dual(b, X64, y64, loss), X64, y64, loss, fo, w.k, w.M, w.lambda2)
    # FP32 data: the returned beta is the certified FP64 beta_best rounded to
    # FP32, which moves Phi and Psi by about its rounding
    tol = _tol(dtype) if dtype == np.float64 else 1e-6
    assert abs(res.primal - phi) <= tol * max(1.0, abs(phi)), (res.primal, phi)
    assert res.dual_bound >= psi_self - tol * max(1.0, abs(psi_self)), (res.dual_bound, psi_self)
    assert res.dual_bound <= phi + tol * max(1.0, abs(phi))
    assert res.rel_gap <= 1e-6
