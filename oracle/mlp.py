"""Learned per-coordinate warm start (FP64 oracle; test infrastructure).

In branch and bound every child node is warm-started from its parent's
solution (Sec. 5.3).  The learned variant keeps that start and adds a
correction predicted coordinate by coordinate:

    beta0_j = b_j + f(x_j),

where x_j holds five features of coordinate j:

    x_j = [ b_j,                            the parent's solution on the child's set
            (X' grad F(X b))_j,             the loss gradient there
            fix_j in {-1, 0, +1},           the child's fixing (J0, free, J1)
            ||X_j||_2,                      the column norm
            |corr(X_j, y)| ]                Pearson correlation with y

with b = beta^P projected onto the child's fixings (zero on the child's J0):
the gradient at b carries the effect of the branching on every other
coordinate, which the gradient at beta^P itself (the same for both children)
does not.

f is a multilayer perceptron 5 -> 64 -> 64 -> 1 with ReLU after both hidden
layers, whose inputs are standardised as (x - shift) / scale.  A network with
zero output layer is exactly the parent warm start.  Training minimises the
mean squared error between b_j + f(x_j) and the child's converged beta_j.

Parameter vector (FP32 on the device, FP64 here), in this order:
    W1 (64 x 5, row h = hidden unit), b1 (64), W2 (64 x 64, row o = output
    unit of layer 2), b2 (64), w3 (64), b3 (1)      -> 4609 trainable values,
    shift (5), scale (5)                              -> 10 fixed values.

Everything below is plain numpy in float64: the forward pass, the loss, its
gradient by the chain rule written out layer by layer, Adam (Kingma and Ba,
2015, Algorithm 1), and round-to-nearest-even to BF16 from that format's
definition.  Pinned by tests/test_oracle_mlp.py (finite differences, closed
forms of the affine regime and of Adam's first step, library routines for the
features).
"""
from __future__ import annotations

import numpy as np

from . import losses

NIN, NH = 5, 64
N_TRAIN = NH * NIN + NH + NH * NH + NH + NH + 1      # 4609
N_PARAM = N_TRAIN + 2 * NIN                          # 4619


def unpack(theta):
    """Views of the parameter vector: W1, b1, W2, b2, w3, b3, shift, scale."""
    t = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = t[o:o + NH * NIN].reshape(NH, NIN); o += NH * NIN
    b1 = t[o:o + NH]; o += NH
    W2 = t[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = t[o:o + NH]; o += NH
    w3 = t[o:o + NH]; o += NH
    b3 = t[o]; o += 1
    shift = t[o:o + NIN]; o += NIN
    scale = t[o:o + NIN]; o += NIN
    return W1, b1, W2, b2, w3, b3, shift, scale


def init(seed=0, shift=None, scale=None):
    """He-initialised hidden layers, zero output layer (so f = 0: the parent
    warm start), identity standardisation unless given."""
    rng = np.random.default_rng(seed)
    theta = np.zeros(N_PARAM)
    W1, b1, W2, b2, w3, b3, sh, sc = unpack(theta)
    theta[:NH * NIN] = rng.standard_normal(NH * NIN) * np.sqrt(2.0 / NIN)
    o = NH * NIN + NH
    theta[o:o + NH * NH] = rng.standard_normal(NH * NH) * np.sqrt(2.0 / NH)
    theta[N_TRAIN:N_TRAIN + NIN] = 0.0 if shift is None else shift
    theta[N_TRAIN + NIN:] = 1.0 if scale is None else scale
    return theta


def projected_parent(beta_parent, fix_child):
    """b: the parent's solution with the child's J0 coordinates set to zero."""
    b = np.array(beta_parent, dtype=np.float64)
    if fix_child is not None:
        b[np.asarray(fix_child) < 0] = 0.0
    return b


def parent_gradient(X, y, loss, beta):
    """X' grad F(X beta): the gradient of the loss term at the parent."""
    X = np.asarray(X, dtype=np.float64)
    return X.T @ losses.grad_F(X @ np.asarray(beta, dtype=np.float64), np.asarray(y, dtype=np.float64), loss)


def column_stats(X, y):
    """||X_j||_2 and |corr(X_j, y)| (Pearson; 0 where a column or y is constant)."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    norms = np.sqrt(np.sum(X * X, axis=0))
    Xc = X - X.mean(axis=0)
    yc = y - y.mean()
    num = Xc.T @ yc
    den = np.sqrt(np.sum(Xc * Xc, axis=0)) * np.sqrt(yc @ yc)
    corr = np.where(den > 0, np.abs(num) / np.where(den > 0, den, 1.0), 0.0)
    return norms, corr


def features(beta_parent, grad_parent, fix_child, norms, corr):
    """The (p, 5) feature matrix of one child node."""
    p = len(beta_parent)
    fx = np.zeros(p) if fix_child is None else np.asarray(fix_child, dtype=np.float64)
    return np.stack([np.asarray(beta_parent, dtype=np.float64), np.asarray(grad_parent, dtype=np.float64),
                     fx, np.asarray(norms, dtype=np.float64), np.asarray(corr, dtype=np.float64)], axis=1)


def forward(theta, F):
    """f(x) for every row of F (N x 5); returns (out, cache)."""
    W1, b1, W2, b2, w3, b3, shift, scale = unpack(theta)
    xs = (np.asarray(F, dtype=np.float64) - shift) / scale
    a1 = xs @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    out = h2 @ w3 + b3
    return out, (xs, a1, h1, a2, h2)


def start(theta, F):
    """The child's starting point: 0 on its J0 (feature 2 = -1), b + f(x)
    elsewhere, with b = feature 0."""
    F = np.asarray(F, dtype=np.float64)
    out, _ = forward(theta, F)
    return np.where(F[:, 2] < 0, 0.0, F[:, 0] + out)


def loss_and_grad(theta, F, base, target):
    """L = mean((base + f(x) - target)^2) and dL/dtheta (zero on shift, scale)."""
    W1, b1, W2, b2, w3, b3, shift, scale = unpack(theta)
    out, (xs, a1, h1, a2, h2) = forward(theta, F)
    r = np.asarray(base, dtype=np.float64) + out - np.asarray(target, dtype=np.float64)
    N = len(r)
    L = float(np.mean(r * r))
    d_out = 2.0 * r / N                       # dL/d out
    g_w3 = h2.T @ d_out
    g_b3 = np.sum(d_out)
    d_a2 = np.outer(d_out, w3) * (a2 > 0)     # through h2 = relu(a2)
    g_W2 = d_a2.T @ h1
    g_b2 = d_a2.sum(axis=0)
    d_h1 = d_a2 @ W2
    d_a1 = d_h1 * (a1 > 0)
    g_W1 = d_a1.T @ xs
    g_b1 = d_a1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3], np.zeros(2 * NIN)])
    return L, g


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1) of the trainable entries; returns
    (theta, m, v) as new arrays."""
    theta = np.array(theta, dtype=np.float64)
    g = np.asarray(grad, dtype=np.float64)[:N_TRAIN]
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    theta[:N_TRAIN] -= lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v


def bf16_round(x):
    """Round FP64 values to BF16 (via FP32, round-to-nearest-even on the 16
    dropped mantissa bits), returned as FP64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_weights(theta):
    """The network the BF16-weight kernels evaluate: trainable entries rounded
    to BF16, standardisation kept exact."""
    t = np.array(theta, dtype=np.float64)
    t[:N_TRAIN] = bf16_round(t[:N_TRAIN])
    return t
