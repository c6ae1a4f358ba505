"""Parity at the benchmark's full size: LS, X 20000 x 50000 FP32 (rho 0.9,
k 50, lambda2 0.1, SNR 3), in the launch configuration bench.py times.  The
FP64 oracle cannot run the whole solve in a test's time at this size, so it
checks what it can compute exactly:

* the fused pass at a dense point: z_i for 64 sampled rows and
  g_j = (X' grad F(z))_j for 64 sampled columns, against FP64 products over
  all rows, at the FP32 bar of the pass tests;
* the solve: the oracle's Phi (Eq. 6) and Psi at zeta = -grad F(X beta)
  (Eq. 7), evaluated in FP64 from its own loss and regularizer functions at the
  returned beta.  The library's certified primal is that Phi, up to the
  rounding of beta to FP32 on output.  Its bound is at least that Psi, and at
  most Phi (weak duality).  The certified relative gap is within 1e-6.
"""
import numpy as np
import pytest

import synth
from oracle import losses, regularizer

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CHUNK = 2000


def _xv(Xh, v):
    """X v in FP64, row chunks of the FP32 host copy."""
    out = np.empty(Xh.shape[0])
    for i in range(0, Xh.shape[0], CHUNK):
        out[i:i + CHUNK] = Xh[i:i + CHUNK].astype(np.float64) @ v
    return out


def _xtv(Xh, u):
    """X' u in FP64."""
    out = np.zeros(Xh.shape[1])
    for i in range(0, Xh.shape[0], CHUNK):
        out += Xh[i:i + CHUNK].astype(np.float64).T @ u[i:i + CHUNK]
    return out


def test_full_size_pass_and_certificate(lib):
    w = synth.WORKLOADS["ls_20000x50000_f32"]
    X, y = synth.make_problem_gpu(w)
    h = lib.Handle(X, y, loss=w.loss, k=w.k, lambda2=w.lambda2, M=w.M)
    Xh = X.cpu().numpy()
    yh = y.double().cpu().numpy()
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(w.n, 64, replace=False))
    cols = np.sort(rng.choice(w.p, 64, replace=False))

    # ---- the fused pass at a dense point
    beta = torch.tensor(synth.prox_input(w.p, 5, scale=0.01), dtype=torch.float32, device="cuda")
    z, g, _ = h.xpass(beta)
    torch.cuda.synchronize()
    b64 = beta.double().cpu().numpy()
    z_ref = _xv(Xh, b64)
    Xa = np.abs(Xh[rows]).astype(np.float64)
    zmag_rows = Xa @ np.abs(b64)
    zg = z.double().cpu().numpy()
    tol = 2e-6
    assert np.all(np.abs(zg[rows] - z_ref[rows]) <= tol * zmag_rows), \
        np.max(np.abs(zg[rows] - z_ref[rows]) / zmag_rows)
    r_ref = losses.grad_F(z_ref, yh, w.loss)
    Xc = Xh[:, cols].astype(np.float64)
    g_ref = Xc.T @ r_ref
    zmag_all = np.empty(w.n)
    for i in range(0, w.n, CHUNK):
        zmag_all[i:i + CHUNK] = np.abs(Xh[i:i + CHUNK]).astype(np.float64) @ np.abs(b64)
    gmag = np.abs(Xc).T @ np.abs(r_ref)
    gbound = tol * gmag + 2.0 * (np.abs(Xc).T @ (tol * zmag_all))     # r = 2 (z - y) carries z's error
    gg = g.double().cpu().numpy()
    assert np.all(np.abs(gg[cols] - g_ref) <= 1.5 * gbound), np.max(np.abs(gg[cols] - g_ref) / gbound)

    # ---- the solve to relative gap 1e-6 and its certificate
    beta_out, res, code = h.solve(gap_tol=1e-6)
    torch.cuda.synchronize()
    h.close()
    assert code == 0, lib.STATUS[code]
    assert res.rel_gap <= 1e-6
    b = beta_out.double().cpu().numpy()
    zb = _xv(Xh, b)
    # beta comes back rounded to FP32: allow that rounding in the domain test
    phi = losses.F(zb, yh, w.loss) + 2.0 * w.lambda2 * regularizer.g_alg1(b, None, w.k, w.M, domain_rtol=1e-6)
    zeta = -losses.grad_F(zb, yh, w.loss)
    wv = _xtv(Xh, zeta)
    psi = -losses.F_conj(-zeta, yh, w.loss) - 2.0 * w.lambda2 * regularizer.gstar(wv / (2.0 * w.lambda2), None,
                                                                                   w.k, w.M)
    print(f"full size: certified primal {res.primal:.10g} (oracle Phi {phi:.10g}), bound {res.dual_bound:.10g} "
          f"(oracle Psi {psi:.10g}), rel gap {res.rel_gap:.3e}, iterations {res.iters}")
    assert np.isfinite(phi) and np.isfinite(psi)
    assert res.primal == pytest.approx(phi, rel=1e-6)
    assert res.dual_bound >= psi - 1e-6 * abs(psi)
    assert res.dual_bound <= phi + 1e-9 * abs(phi)


def test_full_size_batch_certificates(lib):
    """256 nodes sharing X 5000 x 10000 (the batched configuration): every node
    certifies rel. gap 1e-6, and for 6 sampled nodes the oracle's Phi and Psi
    at the returned beta under that node's fixings bracket the bound."""
    w = synth.WORKLOADS["batch256_5000x10000_f32"]
    nb = w.extra["nodes"]
    X, y = synth.make_problem_gpu(w)
    fix = np.stack([synth.node_fixings(w.p, 0, j, w.extra["j0_max"], w.extra["j1_max"], k=w.k) for j in range(nb)])
    h = lib.Handle(X, y, loss=w.loss, k=w.k, lambda2=w.lambda2, M=w.M)
    betas, res, code = h.solve_batch(nb, fixings=torch.tensor(fix, device="cuda"), gap_tol=1e-6)
    torch.cuda.synchronize()
    h.close()
    assert code == 0, lib.STATUS[code]
    assert all(r.status == 0 and r.rel_gap <= 1e-6 for r in res)
    Xh = X.cpu().numpy()
    yh = y.double().cpu().numpy()
    for j in (0, 1, 57, 128, 200, 255):
        b = betas[j].double().cpu().numpy()
        assert np.all(b[fix[j] < 0] == 0.0)
        zb = _xv(Xh, b)
        phi = losses.F(zb, yh, w.loss) + 2.0 * w.lambda2 * regularizer.g_alg1(b, fix[j], w.k, w.M, domain_rtol=1e-6)
        zeta = -losses.grad_F(zb, yh, w.loss)
        wv = _xtv(Xh, zeta)
        psi = (-losses.F_conj(-zeta, yh, w.loss)
               - 2.0 * w.lambda2 * regularizer.gstar(wv / (2.0 * w.lambda2), fix[j], w.k, w.M))
        r = res[j]
        assert np.isfinite(phi) and np.isfinite(psi), j
        assert r.primal == pytest.approx(phi, rel=1e-6), j
        assert psi - 1e-6 * abs(psi) <= r.dual_bound <= phi + 1e-9 * abs(phi), (j, psi, r.dual_bound, phi)
