"""Parity of the device regularizer kernels (prox_persp, gval_persp, gstar_persp)
with the FP64 oracle (Algorithm 1, Algorithm 2 + Eq. prox:gN, Lemma 4.2).

Tolerances.  FP64 inputs: outputs agree to 1e-12 relative (both sides are exact
algorithms; only rounding order differs) and the threshold counts (n_top, n_nz)
are bit-exact on tie-free inputs.  FP32 inputs: the device takes every
threshold decision in FP64 on the exact FP32 values (the same decisions as the
FP64 oracle on the same values), so the counts are still bit-exact; values
differ by the final rounding to FP32 (<= 1 ulp, checked at 2^-22 relative).
"""
import math

import numpy as np
import pytest

import synth
from oracle import regularizer as R

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(a, dtype):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def rand_fix(rng, p, n0, n1):
    f = np.zeros(p, dtype=np.int8)
    perm = rng.permutation(p)
    f[perm[:n0]] = -1
    f[perm[n0:n0 + n1]] = 1
    return f


CASES = [
    # (p, k, rho, M, n0, n1)
    (1, 1, 0.5, 2.0, 0, 0),
    (7, 2, 0.3, 1.0, 1, 1),
    (100, 10, 1.0, 1.0, 0, 0),            # the prox micro-benchmark recipe (Sec. 5.1)
    (1000, 10, 0.5, 2.0, 37, 4),
    (1001, 50, 1e-3, 2.0, 0, 0),
    (4097, 5, 2e-7, 2.0, 20, 3),          # tiny rho: the regime of FISTA steps 1/L
    (50000, 50, 1e-4, 2.0, 40, 19),
    (102400, 10, 1.0, 1.0, 0, 0),
    (3000, 3000, 0.7, 1.5, 10, 5),        # kbar >= pbar: no coupling
    (500, 4, 0.2, math.inf, 5, 4),        # no box (kbar = 0 after J1 = 4)
    (500, 12, 0.05, math.inf, 5, 4),
    (2000, 30, 5.0, 0.3, 0, 0),           # box-active regime c > rho*M
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_prox_matches_oracle(lib, case, dtype):
    p, k, rho, M, n0, n1 = case
    rng = np.random.default_rng(p + k)
    v = synth.prox_input(p, seed=p * 7 + k, scale=3.0)
    if dtype == torch.float32:
        v = v.astype(np.float32).astype(np.float64)
    fix = rand_fix(rng, p, n0, n1) if (n0 or n1) else None
    lam2 = 0.5
    step = rho / (2 * lam2)
    want, (ntop, nnz) = R.prox_g(v, rho, fix, k, M, return_info=True)
    vin = dev(v, dtype)
    out = torch.empty_like(vin)
    counts = torch.zeros(2, dtype=torch.int32, device="cuda")
    fx = dev(fix, torch.int8) if fix is not None else None
    lib.prox_persp(vin, out, step, k, lam2, M, fx, counts)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    if dtype == torch.float64:
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14 * max(1.0, np.abs(v).max()))
    else:
        np.testing.assert_allclose(got, want, rtol=2.0 ** -22, atol=1e-30)
    c = counts.cpu().numpy()
    assert int(c[1]) == nnz
    assert int(c[0]) == ntop


def test_prox_aliasing_and_zero_input(lib):
    v = torch.zeros(333, dtype=torch.float64, device="cuda")
    lib.prox_persp(v, v, 0.1, 5, 1.0, 2.0)
    torch.cuda.synchronize()
    assert torch.count_nonzero(v).item() == 0
    x = torch.tensor(synth.prox_input(999, 3), dtype=torch.float64, device="cuda")
    want = R.prox_g(x.cpu().numpy(), 0.2, None, 7, 2.0)
    lib.prox_persp(x, x, 0.1, 7, 1.0, 2.0)     # in place
    torch.cuda.synchronize()
    np.testing.assert_allclose(x.cpu().numpy(), want, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_g_and_gstar_match_oracle(lib, case, dtype):
    p, k, rho, M, n0, n1 = case
    rng = np.random.default_rng(3 * p + k)
    fix = rand_fix(rng, p, n0, n1) if (n0 or n1) else None
    if k - (0 if fix is None else int(np.sum(fix > 0))) < 0:
        pytest.skip("k < |J1|")
    v = synth.prox_input(p, seed=p + 11, scale=2.0)
    b = R.prox_g(v, rho, fix, k, M)                 # a point of dom g (the Sec. 5.1 recipe)
    if dtype == torch.float32:
        b = b.astype(np.float32).astype(np.float64)
        if not R.in_domain(b, fix, k, M, rtol=1e-6):
            pytest.skip("rounding left the domain")
    fx = dev(fix, torch.int8) if fix is not None else None
    # FP32 rounding can put a boundary point a few ulp outside dom g; the device
    # accepts 1e-6 relative, so the oracle's Algorithm 1 is asked for the same
    want = R.g_alg1(b, fix, k, M, domain_rtol=1e-12 if dtype == torch.float64 else 1e-6)
    got = lib.gval_persp(dev(b, dtype), k, M, fx)
    assert got == pytest.approx(want, rel=1e-12 if dtype == torch.float64 else 1e-9, abs=1e-300)
    a = synth.prox_input(p, seed=p + 5, scale=1.7)
    if dtype == torch.float32:
        a = a.astype(np.float32).astype(np.float64)
    gs = lib.gstar_persp(dev(a, dtype), k, M, fx)
    assert gs == pytest.approx(R.gstar(a, fix, k, M), rel=1e-12)


def test_g_outside_domain_is_inf(lib):
    b = torch.tensor([0.0, 2.5, 0.0], dtype=torch.float64, device="cuda")
    assert math.isinf(lib.gval_persp(b, 2, 2.0))
    fix = torch.tensor([-1, 0, 0], dtype=torch.int8, device="cuda")
    b2 = torch.tensor([0.3, 0.1, 0.0], dtype=torch.float64, device="cuda")
    assert math.isinf(lib.gval_persp(b2, 2, 2.0, fix))


def test_worked_examples_on_device(lib):
    # Sec. 4.2 figure: g(1.4, 0.6; k=1) = 2.0, g(0.6, 1.2, 1.2; k=2) = 2.25
    assert lib.gval_persp(torch.tensor([1.4, 0.6], dtype=torch.float64, device="cuda"), 1, 2.0) == \
        pytest.approx(2.0, rel=1e-15)
    assert lib.gval_persp(torch.tensor([0.6, 1.2, 1.2], dtype=torch.float64, device="cuda"), 2, 1.5) == \
        pytest.approx(2.25, rel=1e-15)


def test_invalid_arguments(lib):
    v = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.RelaxError):
        lib.prox_persp(v, v, -1.0, 2, 1.0, 2.0)
    with pytest.raises(lib.RelaxError):
        lib.gval_persp(v, 2, -1.0)
