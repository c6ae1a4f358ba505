"""Parity of the fused X-pass (relax_xpass through the C ABI) with plain FP64
matrix-vector products: z = X beta, r = grad F(z), g = X' r, and the loss
sums F(z), -F*(-zeta) at zeta = -r (Sec. 2.4, Eq. 6-7).

Tolerance: FP64 -> 1e-12 relative to the magnitude sums sum_j |X_ij b_j| (and
sum_i |X_ij r_i| for g); FP32 (FP32 accumulation over at most p terms, tree
reduced) -> 2e-6 relative to the same magnitude sums.
"""
import numpy as np
import pytest

import synth
from oracle import losses

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = [(1, 1), (5, 3), (37, 1001), (513, 2049), (300, 50000), (2000, 5000), (1024, 12345),
          (9, 20001), (4099, 257)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("loss", ["ls", "logistic"])
def test_xpass_matches_matvec(lib, shape, dtype, loss):
    n, p = shape
    w = synth.Workload("t", n, p, 0.6, max(1, min(5, p)), 0.5, loss)
    X, y = synth.make_problem_cpu(w, dtype=np.float64)
    npdt = np.float64 if dtype == torch.float64 else np.float32
    X = X.astype(npdt)
    y = y.astype(npdt)
    beta = synth.prox_input(p, 3, scale=0.3).astype(npdt)
    Xd = torch.tensor(X, device="cuda")
    yd = torch.tensor(y, device="cuda")
    h = lib.Handle(Xd, yd, loss=loss, k=1, lambda2=0.5, lipschitz=1.0)
    z, g, (F, D) = h.xpass(torch.tensor(beta, device="cuda"))
    torch.cuda.synchronize()
    X64, b64, y64 = X.astype(np.float64), beta.astype(np.float64), y.astype(np.float64)
    z_ref = X64 @ b64
    r_ref = losses.grad_F(z_ref, y64, loss)
    g_ref = X64.T @ r_ref
    tol = 1e-12 if dtype == torch.float64 else 2e-6
    zmag = np.abs(X64) @ np.abs(b64) + 1e-300
    gmag = np.abs(X64).T @ np.abs(r_ref) + 1e-300
    zg = z.double().cpu().numpy()
    gg = g.double().cpu().numpy()
    assert np.all(np.abs(zg - z_ref) <= tol * zmag + 1e-300), np.max(np.abs(zg - z_ref) / zmag)
    # g also carries the error of r = grad F(z); bound it through |X|'|dr| with |dr| <= c |dz|
    c = 2.0 if loss == "ls" else 0.25
    gbound = tol * gmag + c * (np.abs(X64).T @ (tol * zmag))
    assert np.all(np.abs(gg - g_ref) <= gbound * 1.5), np.max(np.abs(gg - g_ref) / gbound)
    F_ref = losses.F(z_ref, y64, loss)
    D_ref = -losses.F_conj(r_ref, y64, loss)     # -F*(-zeta), zeta = -r
    ftol = 1e-10 if dtype == torch.float64 else 1e-5
    assert F == pytest.approx(F_ref, rel=ftol, abs=ftol)
    assert D == pytest.approx(D_ref, rel=ftol, abs=ftol)
    h.close()


def test_xpass_unaligned_leading_dimension(lib):
    # ldx * 4 bytes not a multiple of 16: the handle keeps an aligned copy
    n, p = 64, 103
    base = torch.tensor(synth.ar1_design(n, p + 2, 0.5, 1), dtype=torch.float32, device="cuda")
    X = base[:, :p]
    assert X.stride(0) == p + 2
    y = torch.tensor(synth.prox_input(n, 2), dtype=torch.float32, device="cuda")
    h = lib.Handle(X, y, k=1, lambda2=1.0, lipschitz=1.0)
    beta = torch.tensor(synth.prox_input(p, 4), dtype=torch.float32, device="cuda")
    z, g, _ = h.xpass(beta)
    Xn = X.double().cpu().numpy()
    z_ref = Xn @ beta.double().cpu().numpy()
    np.testing.assert_allclose(z.double().cpu().numpy(), z_ref, rtol=1e-5, atol=1e-5)
    h.close()
