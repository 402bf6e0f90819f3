"""Learned closure of a low-order FR right-hand side, driven through the
library (include/fr.h): samples from a higher-order solve, training of one
network per element type with the library's BF16 kernels, and attaching the
trained networks to the low-order context.  Argument marshalling only:
PyTorch holds the device buffers; every sample, forward, backward and Adam
step runs in the library's kernels.

The target of element e is P RHS_hi(u_hi) - RHS_lo(u_lo) (P the order
transfer, u_lo = P u_hi or a p_lo solution at the same time); the network
sees the element's own p_lo state and corrected gradient (20 nu features)
and predicts the target divided by per-variable scales (the target's RMS
over the training samples, per conserved variable and element type).
"""
from __future__ import annotations

import numpy as np
import torch

from synth import mlp_init

from . import fr

NH = 128


class Network:
    """FP32 master parameters, gradient and Adam moments of one network."""

    def __init__(self, nin, nout, nh=NH, seed=0, device="cuda"):
        self.nin, self.nh, self.nout = int(nin), int(nh), int(nout)
        self.n = fr.mlp_nparams(nin, nh, nout)
        self.P = torch.tensor(mlp_init(nin, nh, nout, seed), dtype=torch.float32, device=device)
        assert self.P.numel() == self.n
        self.G = torch.zeros_like(self.P)
        self.m = torch.zeros_like(self.P)
        self.v = torch.zeros_like(self.P)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.steps = 0
        self._ws = None

    def _workspace(self, rows):
        need = fr.mlp_workspace(self.nin, self.nh, self.nout, rows)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.float32, device=self.P.device)
        return self._ws

    def grad(self, X, T, stream=None):
        """G = dL/dP, loss = L on (X, T); returns nothing (device values)."""
        rows = X.shape[0]
        ws = self._workspace(rows)
        fr.mlp_grad(self.nin, self.nh, self.nout, rows, X.data_ptr(), T.data_ptr(), self.P.data_ptr(),
                    self.G.data_ptr(), self.loss.data_ptr(), ws.data_ptr(), stream)

    def adam(self, lr, stream=None):
        self.steps += 1
        fr.mlp_adam(self.n, self.P.data_ptr(), self.G.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                    self.steps, lr, stream)

    def train(self, X, T, iters, lr=1e-3, batch=None, log_every=0):
        """Adam on the mean squared error; batch=None: full batch, else
        consecutive row slices of that size in turn.  Returns the logged
        losses (every log_every steps, 0: none)."""
        rows = X.shape[0]
        losses = []
        b = rows if batch is None else min(int(batch), rows)
        nb = max(1, rows // b)
        for it in range(int(iters)):
            k = it % nb
            self.grad(X[k * b:(k + 1) * b], T[k * b:(k + 1) * b])
            self.adam(lr)
            if log_every and (it % log_every == 0 or it == iters - 1):
                losses.append(float(self.loss.item()))
        return losses

    def forward(self, X, stream=None):
        rows = X.shape[0]
        Y = torch.empty(rows, self.nout, dtype=torch.float32, device=X.device)
        ws = self._workspace(rows)
        fr.mlp_forward(self.nin, self.nh, self.nout, rows, X.data_ptr(), self.P.data_ptr(), Y.data_ptr(),
                       ws.data_ptr(), stream)
        return Y

    def mse(self, X, T):
        """Mean squared error on (X, T), from the library's loss."""
        self.grad(X, T)
        return float(self.loss.item())


def _pairs(states):
    """[(u_hi, u_lo or None)] from a list of u_hi or of pairs."""
    return [st if isinstance(st, tuple) else (st, None) for st in states]


def sample_scale(ctx_hi, ctx_lo, states, etype):
    """Per-variable RMS (5) of the unscaled target of one element type."""
    pairs = _pairs(states)
    ss = torch.zeros(5, dtype=torch.float64, device=pairs[0][0].device)
    for u, ul in pairs:
        ctx_lo.closure_sample(ctx_hi, u.data_ptr(), etype, None, None, None, ss.data_ptr(),
                              u_lo_ptr=ul.data_ptr() if ul is not None else None)
    count = len(pairs) * ctx_lo.ne(etype) * ctx_lo.nu(etype)
    return np.sqrt(ss.cpu().numpy() / count)


def samples(ctx_hi, ctx_lo, states, etype, scale):
    """Features X (rows = elements of every state) and targets T / scale
    (scale: 5 per-variable values)."""
    pairs = _pairs(states)
    ne, nu = ctx_lo.ne(etype), ctx_lo.nu(etype)
    dev = pairs[0][0].device
    X = torch.empty(len(pairs) * ne, 20 * nu, dtype=torch.float32, device=dev)
    T = torch.empty(len(pairs) * ne, 5 * nu, dtype=torch.float32, device=dev)
    inv = 1.0 / np.maximum(np.asarray(scale, dtype=np.float64), 1e-300)
    for k, (u, ul) in enumerate(pairs):
        ctx_lo.closure_sample(ctx_hi, u.data_ptr(), etype, inv, X[k * ne:].data_ptr(), T[k * ne:].data_ptr(),
                              None, u_lo_ptr=ul.data_ptr() if ul is not None else None)
    return X, T


class Closure:
    """One network per element type of a low-order context.  Training
    states are p_hi states (targets against the RHS of their projection) or
    pairs (u_hi, u_lo) of a p_hi and a p_lo solution at the same time
    (targets against the RHS of u_lo, features of u_lo)."""

    def __init__(self, ctx_lo, nh=NH, seed=0):
        self.ctx = ctx_lo
        self.nets, self.scale = {}, {}
        for et in range(3):  # tets, prisms, hexes
            if ctx_lo.ne(et):
                nu = ctx_lo.nu(et)
                self.nets[et] = Network(20 * nu, 5 * nu, nh=nh, seed=seed + et)

    def fit(self, ctx_hi, states, iters=2000, lr=1e-3, batch=None, log_every=0):
        """Train on the samples of `states`; returns {etype: logged losses}."""
        log = {}
        for et, net in self.nets.items():
            self.scale[et] = sample_scale(ctx_hi, self.ctx, states, et)
            X, T = samples(ctx_hi, self.ctx, states, et, self.scale[et])
            log[et] = net.train(X, T, iters, lr=lr, batch=batch, log_every=log_every)
        return log

    def error(self, ctx_hi, states):
        """{etype: (relative RMS error of the closed RHS, of the plain RHS)}
        against the target in the scaled units the network is trained in,
        i.e. sqrt(mse / mean(T^2)) with and without it."""
        out = {}
        for et, net in self.nets.items():
            X, T = samples(ctx_hi, self.ctx, states, et, self.scale[et])
            t2 = float(torch.mean(T.double() ** 2).item())
            out[et] = (float(np.sqrt(net.mse(X, T) / t2)), 1.0)
        return out

    def attach(self):
        for et, net in self.nets.items():
            self.ctx.closure_set(et, net.P.data_ptr(), net.nh, self.scale[et])

    def detach(self):
        for et in self.nets:
            self.ctx.closure_set(et, None)
