"""The batched products (relax_batch_xpass: z_s = X b_s, g_s = X' z_s) against
FP64 matrix products on the same values, through the C ABI.

FP32 X runs the library's tcgen05 kernel on BF16 planes (the FP32 values split
exactly into three BF16 parts, six plane products per pair, FP32 sums in
tensor memory over a K chunk, FP64 sums over the chunks).  Bars, per output
element, relative to the sum of the magnitudes of its terms (|X| |b|):
  * worst case: the FP32 summation bound over the whole reduction length K
    plus the dropped plane products (<= 2^-23 each), with a factor 2 margin;
  * typical: the RMS of that relative error <= 2e-7, which a product left
    out (x1 b3, ~2^-16 per term) or a plane laid out wrong would exceed.
The shapes span several M, N and K tiles with ragged tails, one N-tile and
two, N = 1, and a long K over few tiles (a tile summed from 16 pieces).  FP64 X uses FP64 products (1e-12 relative)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = [
    # (n, p, nb)
    (300, 200, 5),
    (129, 129, 17),
    (1000, 777, 37),
    (257, 1030, 256),     # one full N tile of 256
    (130, 64, 1),
    (700, 1500, 300),     # two N tiles (balanced: 2 x 160)
    (4000, 3000, 64),
    (200, 20000, 8),      # 2 tiles of 625 K blocks: each cut into 15-16 pieces of the CTAs' ranges
]


def _points(nb, p, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((nb, p)) * np.exp(rng.uniform(-3, 3, (nb, 1)))   # points of unequal scale
    B[rng.random((nb, p)) < 0.7] = 0.0                                      # sparse, like prox outputs
    return B


def _check(got, want, mag, K):
    u = 2.0 ** -24
    bound = 2.0 * ((K + 4) * u + 2.0 ** -23) * mag + 1e-300
    err = np.abs(got - want)
    assert np.all(err <= bound), float(np.max(err / bound))
    rel = err / np.maximum(mag, 1e-300)
    rms = float(np.sqrt(np.mean(rel ** 2)))
    assert rms <= 2e-7, rms
    return rms


@pytest.mark.parametrize("shape", SHAPES)
def test_batch_products_f32_match_fp64(lib, shape):
    n, p, nb = shape
    w = synth.Workload("bg", n, p, 0.6, 5, 0.5, "ls", seed=n + p)
    X, y = synth.make_problem_cpu(w, dtype=np.float32)
    X64 = X.astype(np.float64)
    B = _points(nb, p, nb).astype(np.float32)
    B64 = B.astype(np.float64)
    Xd, yd = torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda")
    h = lib.Handle(Xd, yd, k=w.k, lambda2=w.lambda2, lipschitz=1.0)
    z, g = h.batch_xpass(torch.tensor(B, device="cuda"))
    z, g = z.cpu().numpy(), g.cpu().numpy()
    z_ref = B64 @ X64.T                          # [nb][n]
    rz = _check(z, z_ref, np.abs(B64) @ np.abs(X64).T, p)
    # the second product is taken of the device's own z (FP64 values, split
    # to 24 bits): compare with X' applied to that z
    g_ref = z @ X64
    rg = _check(g, g_ref, np.abs(z) @ np.abs(X64), n)
    print(f"shape {shape}: RMS relative error z {rz:.2e}, g {rg:.2e}")
    # deterministic: a fixed split and fixed-order FP64 sums
    z2, g2 = h.batch_xpass(torch.tensor(B, device="cuda"))
    assert np.array_equal(z2.cpu().numpy(), z) and np.array_equal(g2.cpu().numpy(), g)
    h.close()


def test_batch_products_f64_match_fp64(lib):
    n, p, nb = 333, 517, 21
    w = synth.Workload("bg64", n, p, 0.6, 5, 0.5, "ls", seed=3)
    X, y = synth.make_problem_cpu(w, dtype=np.float64)
    B = _points(nb, p, 9)
    h = lib.Handle(torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda"), k=w.k, lambda2=w.lambda2,
                   lipschitz=1.0)
    z, g = h.batch_xpass(torch.tensor(B, device="cuda"))
    h.close()
    z, g = z.cpu().numpy(), g.cpu().numpy()
    np.testing.assert_allclose(z, B @ X.T, rtol=1e-12, atol=1e-12 * np.abs(z).max())
    np.testing.assert_allclose(g, z @ X, rtol=1e-12, atol=1e-12 * np.abs(g).max())
