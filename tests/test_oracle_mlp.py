"""Pins of the warm-start network oracle (oracle/mlp.py) against facts other
than itself: central finite differences of the loss, the affine regime's
closed form, Adam's first step, BF16 values fixed by the format, and library
routines for the features."""
import numpy as np
import pytest

from oracle import losses, mlp


def _data(N=40, seed=0, out_scale=0.3):
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((N, mlp.NIN)) * np.array([0.5, 3.0, 1.0, 2.0, 0.2]) + np.array([0, 1, 0, 5, 0.3])
    theta = mlp.init(seed=seed + 1, shift=F.mean(axis=0), scale=F.std(axis=0))
    # give the output layer weight so that every parameter has a gradient
    o = mlp.NH * mlp.NIN + mlp.NH + mlp.NH * mlp.NH + mlp.NH
    theta[o:o + mlp.NH] = rng.standard_normal(mlp.NH) * out_scale
    theta[o + mlp.NH] = 0.1
    base = rng.standard_normal(N)
    target = base + 0.2 * rng.standard_normal(N)
    return theta, F, base, target


def test_gradient_matches_central_differences():
    theta, F, base, target = _data()
    _, (xs, a1, h1, a2, h2) = mlp.forward(theta, F)
    h = 1e-6
    # a step of h in one parameter moves a pre-activation by at most h times an
    # input of order 10: none sits that close to its ReLU kink
    assert min(np.abs(a1).min(), np.abs(a2).min()) > 100 * h
    L, g = mlp.loss_and_grad(theta, F, base, target)
    rng = np.random.default_rng(7)
    idx = np.concatenate([rng.choice(mlp.N_TRAIN, 200, replace=False), [0, mlp.N_TRAIN - 1]])
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, F, base, target)[0] - mlp.loss_and_grad(tm, F, base, target)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9), i
    assert np.all(g[mlp.N_TRAIN:] == 0.0)


def test_zero_output_layer_is_the_parent_start():
    theta = mlp.init(seed=3)
    F = np.random.default_rng(1).standard_normal((17, 5))
    out, _ = mlp.forward(theta, F)
    assert np.all(out == 0.0)
    base = np.arange(17.0)
    target = base + 2.0
    L, g = mlp.loss_and_grad(theta, F, base, target)
    assert L == pytest.approx(4.0)
    assert g[mlp.N_TRAIN - 1] == pytest.approx(-4.0)          # dL/db3 = 2 mean(r) = -4


def test_affine_regime_closed_form():
    # every pre-activation positive: f(x) = w3'(W2 (W1 xs + b1) + b2) + b3
    theta, F, base, target = _data(N=25, seed=4)
    W1, b1, W2, b2, w3, b3, shift, scale = mlp.unpack(theta)
    theta = theta.copy()
    o1 = mlp.NH * mlp.NIN
    theta[o1:o1 + mlp.NH] = 50.0
    o2 = o1 + mlp.NH + mlp.NH * mlp.NH
    theta[o1 + mlp.NH:o2] = np.abs(theta[o1 + mlp.NH:o2])
    theta[o2:o2 + mlp.NH] = 10.0
    W1, b1, W2, b2, w3, b3, shift, scale = mlp.unpack(theta)
    xs = (F - shift) / scale
    assert np.all(xs @ W1.T + b1 > 0)
    A = w3 @ W2 @ W1                        # the affine map's slope in xs
    c = w3 @ (W2 @ b1 + b2) + b3
    out, _ = mlp.forward(theta, F)
    np.testing.assert_allclose(out, xs @ A + c, rtol=1e-12, atol=1e-9)


def test_adam_first_step_moves_by_lr_times_sign():
    theta, F, base, target = _data(seed=5)
    _, g = mlp.loss_and_grad(theta, F, base, target)
    t1, m, v = mlp.adam_step(theta, g, np.zeros(mlp.N_TRAIN), np.zeros(mlp.N_TRAIN), 1, lr=1e-3, eps=1e-300)
    d = (t1 - theta)[:mlp.N_TRAIN]
    nz = g[:mlp.N_TRAIN] != 0
    np.testing.assert_allclose(d[nz], -1e-3 * np.sign(g[:mlp.N_TRAIN][nz]), rtol=1e-12)
    assert np.all(t1[mlp.N_TRAIN:] == theta[mlp.N_TRAIN:])
    np.testing.assert_allclose(m, 0.1 * g[:mlp.N_TRAIN])
    np.testing.assert_allclose(v, 0.001 * g[:mlp.N_TRAIN] ** 2)


def test_bf16_rounding_values():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even mantissa;
    # 1 + 3 * 2^-9 is nearer to 1 + 2^-7
    np.testing.assert_array_equal(mlp.bf16_round([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5]),
                                  [1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7, -2.5])


def test_features_against_library_routines():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((30, 7))
    X[:, 3] = 1.5                          # constant column: no correlation defined -> 0
    y = rng.standard_normal(30)
    norms, corr = mlp.column_stats(X, y)
    np.testing.assert_allclose(norms, np.linalg.norm(X, axis=0), rtol=1e-14)
    for j in (0, 1, 2, 4, 5, 6):
        assert corr[j] == pytest.approx(abs(np.corrcoef(X[:, j], y)[0, 1]), rel=1e-12)
    assert corr[3] == 0.0
    # the gradient feature is the gradient of beta -> F(X beta): central differences
    beta = rng.standard_normal(7)
    for loss in ("ls", "logistic"):
        yy = y if loss == "ls" else np.sign(y)
        g = mlp.parent_gradient(X, yy, loss, beta)
        for j in range(7):
            e = np.zeros(7)
            e[j] = 1e-6
            fd = (losses.F(X @ (beta + e), yy, loss) - losses.F(X @ (beta - e), yy, loss)) / 2e-6
            assert g[j] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    fx = np.array([0, -1, 1, 0, 0, 0, 1], dtype=np.int8)
    Fm = mlp.features(beta, g, fx, norms, corr)
    assert Fm.shape == (7, 5)
    np.testing.assert_array_equal(Fm[:, 2], fx.astype(float))
