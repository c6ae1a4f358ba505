"""Learned warm start of child nodes (include/warmstart.h): the parent's
solution on the child's set plus a per-coordinate correction from a
5 -> 64 -> 64 -> 1 network.  Training, inference and the features run in the
library's kernels; this module holds the parameter tensors and drives the
calls (argument marshalling and the minibatch schedule).
"""
from __future__ import annotations

import numpy as np

from .binding import MLP_NPARAM, MLP_NTRAIN, relax_mlp_adam, relax_mlp_forward, relax_mlp_grad

NIN, NH = 5, 64


def init_params(seed=0, shift=None, scale=None):
    """He-initialised hidden layers and a zero output layer (the network then
    returns the parent start unchanged); identity standardisation unless given.
    Host float64 vector in the layout of include/warmstart.h."""
    rng = np.random.default_rng(seed)
    th = np.zeros(MLP_NPARAM)
    th[:NH * NIN] = rng.standard_normal(NH * NIN) * np.sqrt(2.0 / NIN)
    o = NH * NIN + NH
    th[o:o + NH * NH] = rng.standard_normal(NH * NH) * np.sqrt(2.0 / NH)
    th[MLP_NTRAIN:MLP_NTRAIN + NIN] = 0.0 if shift is None else shift
    th[MLP_NTRAIN + NIN:] = 1.0 if scale is None else scale
    return th


class WarmStartNet:
    """Parameters (FP32 master on the device), Adam moments, and the calls."""

    def __init__(self, device="cuda", seed=0, bf16=True, theta=None):
        import torch
        self.device = device
        self.bf16 = bf16
        th = init_params(seed) if theta is None else np.asarray(theta, dtype=np.float64)
        self.theta = torch.tensor(th, dtype=torch.float32, device=device)
        self.m = torch.zeros(MLP_NTRAIN, dtype=torch.float32, device=device)
        self.v = torch.zeros(MLP_NTRAIN, dtype=torch.float32, device=device)
        self.grad = torch.zeros(MLP_NPARAM, dtype=torch.float32, device=device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.t = 0

    def set_standardisation(self, feat):
        """shift = mean, scale = standard deviation (1 where constant) of the
        training features (statistics of the data, computed once on the host)."""
        f = feat.double().cpu().numpy()
        sh = f.mean(axis=0)
        sc = f.std(axis=0)
        sc = np.where(sc > 0, sc, 1.0)
        th = self.theta.double().cpu().numpy()
        th[MLP_NTRAIN:MLP_NTRAIN + NIN] = sh
        th[MLP_NTRAIN + NIN:] = sc
        self.theta.copy_(self.theta.new_tensor(th))

    def predict(self, feat, out=None):
        """b + f(x) for every row of feat (float32 (rows, 5); b = column 0)."""
        import torch
        if out is None:
            out = torch.empty(feat.shape[0], dtype=torch.float32, device=feat.device)
        base = feat[:, 0].contiguous()
        return relax_mlp_forward(self.theta, feat, out, base=base, bf16=self.bf16)

    def loss_of(self, feat, target):
        """Mean squared error of b + f(x) against target (device float)."""
        base = feat[:, 0].contiguous()
        relax_mlp_grad(self.theta, feat, base, target, self.grad, self.loss, bf16=self.bf16)
        return float(self.loss.item())

    def fit(self, feat, target, epochs=4, batch=16384, lr=1e-3, seed=0, log=None):
        """Minibatch Adam over the rows of (feat, target); the rows are visited
        in one seeded permutation, cut into contiguous minibatches."""
        import torch
        g = torch.Generator(device="cpu").manual_seed(seed)
        perm = torch.randperm(feat.shape[0], generator=g).to(feat.device)
        F = feat.index_select(0, perm).contiguous()
        T = target.index_select(0, perm).contiguous()
        B = F[:, 0].contiguous()
        rows = F.shape[0]
        for ep in range(epochs):
            for s in range(0, rows, batch):
                e = min(rows, s + batch)
                relax_mlp_grad(self.theta, F[s:e], B[s:e], T[s:e], self.grad, self.loss, bf16=self.bf16)
                self.t += 1
                relax_mlp_adam(self.theta, self.grad, self.m, self.v, self.t, lr)
            if log is not None:
                log(ep, float(self.loss.item()))
        return self
