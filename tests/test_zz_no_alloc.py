"""prox_persp_noalloc (scratch in the library's fixed device array) against
the FP64 oracle's prox (Algorithm 2 + Eq. prox:gN) and against prox_persp
(stream-ordered scratch), through the C ABI, on two calls in a row.

Same tolerances as the prox parity tests: FP64 outputs to 1e-12 relative, FP32
to 2^-22 relative, threshold counts (n_top, n_nz) equal.  Collected last so
that it also runs after every other test in one process; it passes alone too.
"""
import numpy as np
import pytest

import synth
from oracle import regularizer as R

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [
    # (p, k, rho, M, n0, n1)
    (1000, 10, 0.5, 2.0, 37, 4),
    (50000, 50, 1e-4, 2.0, 40, 19),
    (102400, 10, 1.0, 1.0, 0, 0),
    (189440, 30, 0.05, 2.0, 11, 3),   # the largest p the fixed scratch admits
]


def _fix(p, n0, n1, seed):
    if not (n0 or n1):
        return None
    rng = np.random.default_rng(seed)
    f = np.zeros(p, dtype=np.int8)
    perm = rng.permutation(p)
    f[perm[:n0]] = -1
    f[perm[n0:n0 + n1]] = 1
    return torch.tensor(f, device="cuda")


def _close(got, want, dtype):
    if dtype == torch.float64:
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14 * max(1.0, np.abs(want).max()))
    else:
        np.testing.assert_allclose(got, want, rtol=2.0 ** -22, atol=1e-30)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("case", CASES)
def test_noalloc_matches_prox_persp_twice(lib, case, dtype):
    p, k, rho, M, n0, n1 = case
    lam2 = 0.5
    step = rho / (2 * lam2)
    fix = _fix(p, n0, n1, p + k)
    # two calls in a row with different inputs: the shared array must not carry
    # anything from the first call into the second
    for call, scale in enumerate((3.0, 0.7)):
        v = torch.tensor(synth.prox_input(p, seed=11 * p + call, scale=scale), dtype=dtype, device="cuda")
        ref = torch.empty_like(v)
        out = torch.full_like(v, float("nan"))
        c_ref = torch.zeros(2, dtype=torch.int32, device="cuda")
        c_out = torch.full((2,), -1, dtype=torch.int32, device="cuda")
        lib.prox_persp(v, ref, step, k, lam2, M, fix, c_ref)
        lib.prox_persp_noalloc(v, out, step, k, lam2, M, fix, c_out)
        torch.cuda.synchronize()
        _close(out.double().cpu().numpy(), ref.double().cpu().numpy(), dtype)
        assert c_out.cpu().tolist() == c_ref.cpu().tolist()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("case", CASES)
def test_noalloc_matches_oracle_twice(lib, case, dtype):
    p, k, rho, M, n0, n1 = case
    lam2 = 0.5
    step = rho / (2 * lam2)
    fix = _fix(p, n0, n1, p + k)
    fix_h = None if fix is None else fix.cpu().numpy()
    for call, scale in enumerate((2.0, 0.4)):
        v = synth.prox_input(p, seed=5 * p + call, scale=scale)
        if dtype == torch.float32:
            v = v.astype(np.float32).astype(np.float64)   # the oracle sees the values the device sees
        want, (ntop, nnz) = R.prox_g(v, rho, fix_h, k, M, return_info=True)
        vd = torch.tensor(v, dtype=dtype, device="cuda")
        out = torch.full_like(vd, float("nan"))
        c_out = torch.full((2,), -1, dtype=torch.int32, device="cuda")
        lib.prox_persp_noalloc(vd, out, step, k, lam2, M, fix, c_out)
        torch.cuda.synchronize()
        _close(out.double().cpu().numpy(), want, dtype)
        assert c_out.cpu().tolist() == [ntop, nnz]


def test_noalloc_rejects_p_beyond_its_scratch(lib):
    p = 189441            # one past the largest p the fixed array serves
    v = torch.zeros(p, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(v)
    with pytest.raises(lib.RelaxError) as ei:
        lib.prox_persp_noalloc(v, out, 0.1, 5, 1.0, 2.0)
    assert ei.value.code == 8          # RELAX_ENOTSUP
    assert "scratch" in lib.relax_error_detail()
