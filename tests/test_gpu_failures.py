"""Failure paths that are injected on the host: non-finite values in the data,
in a warm start or in a prox input (RELAX_ENUMERIC and the prox's NaN / {-1, -1}
sentinel), invalid fixings and cardinalities (RELAX_EINVAL) on a live handle.
No GPU fault is involved: every case is a value the kernels detect."""
import math

import numpy as np
import pytest

import synth
from oracle import solver

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ENUMERIC, EINVAL = 6, 1


def _problem(loss="ls", dtype=np.float64):
    w = synth.Workload("fail", 80, 200, 0.5, 5, 0.5, loss)
    X, y = synth.make_problem_cpu(w, dtype=dtype)
    return w, X, y


@pytest.mark.parametrize("loss", ["ls", "logistic"])
def test_nan_in_y_gives_enumeric(lib, loss):
    w, X, y = _problem(loss)
    L = solver.lipschitz(X, loss)
    y = y.copy()
    y[17] = math.nan
    h = lib.Handle(torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda"), loss=loss, k=w.k,
                   lambda2=w.lambda2, lipschitz=L)
    _, res, code = h.solve(gap_tol=1e-6)
    h.close()
    assert code == ENUMERIC
    assert res.status == ENUMERIC


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_nan_in_warm_start_gives_enumeric(lib, dtype):
    w, X, y = _problem(dtype=dtype)
    L = solver.lipschitz(X.astype(np.float64), "ls")
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    h = lib.Handle(torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda"), k=w.k, lambda2=w.lambda2,
                   lipschitz=L)
    warm = torch.zeros(w.p, dtype=tdt, device="cuda")
    warm[3] = float("inf")
    _, res, code = h.solve(warm_start=warm, gap_tol=1e-6)
    assert code == ENUMERIC
    # the handle still serves a clean solve afterwards
    _, res2, code2 = h.solve(gap_tol=1e-6)
    h.close()
    assert code2 == 0


def test_nan_in_x_is_rejected(lib):
    w, X, y = _problem()
    X = X.copy()
    X[5, 9] = math.nan
    Xd, yd = torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda")
    # the Lanczos estimate of L meets the NaN at create
    with pytest.raises(lib.RelaxError) as ei:
        lib.Handle(Xd, yd, k=w.k, lambda2=w.lambda2)
    assert ei.value.code == ENUMERIC
    # with L given, the solve meets it in its first fused pass
    h = lib.Handle(Xd, yd, k=w.k, lambda2=w.lambda2, lipschitz=100.0)
    _, res, code = h.solve(gap_tol=1e-6)
    h.close()
    assert code == ENUMERIC


def test_invalid_fixings_and_cardinality(lib):
    w, X, y = _problem()
    h = lib.Handle(torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda"), k=3, lambda2=w.lambda2,
                   lipschitz=solver.lipschitz(X, "ls"))
    bad = torch.zeros(w.p, dtype=torch.int8, device="cuda")
    bad[4] = 2                                   # not one of -1, 0, +1
    with pytest.raises(lib.RelaxError) as ei:
        h.solve(fixings=bad)
    assert ei.value.code == EINVAL
    many = torch.zeros(w.p, dtype=torch.int8, device="cuda")
    many[:4] = 1                                 # |J1| = 4 > k = 3
    with pytest.raises(lib.RelaxError) as ei:
        h.solve(fixings=many)
    assert ei.value.code == EINVAL
    fx2 = torch.zeros((2, w.p), dtype=torch.int8, device="cuda")
    fx2[1, :4] = 1
    with pytest.raises(lib.RelaxError) as ei:
        h.solve_batch(2, fixings=fx2)
    assert ei.value.code == EINVAL
    h.close()


@pytest.mark.parametrize("fn", ["prox_persp", "prox_persp_noalloc"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_prox_non_finite_input_gives_sentinels(lib, fn, dtype):
    """The prox does not synchronize, so a non-finite input shows in its
    outputs: beta_out all NaN and counts {-1, -1}; the next clean call on the
    same buffers is exact again."""
    p = 5000
    v = torch.tensor(synth.prox_input(p, seed=3, scale=2.0), dtype=dtype, device="cuda")
    v[123] = float("nan")
    out = torch.zeros_like(v)
    counts = torch.zeros(2, dtype=torch.int32, device="cuda")
    getattr(lib, fn)(v, out, 0.1, 10, 1.0, 2.0, None, counts)
    torch.cuda.synchronize()
    assert torch.isnan(out).all().item()
    assert counts.cpu().tolist() == [-1, -1]
    v[123] = 0.5
    getattr(lib, fn)(v, out, 0.1, 10, 1.0, 2.0, None, counts)
    torch.cuda.synchronize()
    from oracle import regularizer as R
    want, (nt, nn) = R.prox_g(v.double().cpu().numpy(), 0.2, None, 10, 2.0, return_info=True)
    tol = 1e-12 if dtype == torch.float64 else 2.0 ** -22
    np.testing.assert_allclose(out.double().cpu().numpy(), want, rtol=tol, atol=1e-30)
    assert counts.cpu().tolist() == [nt, nn]
