"""Pricing surrogate for Heston calibration: labels, normalisation, training.

Labels come from the Monte Carlo method itself: for each parameter vector
theta (drawn uniformly in the Heston box, conditioned on Feller) and each of
the instruments (the maturities of the calibration set, strikes drawn
U(70, 130)), mc_price_jacobian returns the MC price E y and its pathwise
derivatives dE y/dtheta.  The network is trained on the differential loss
(value + alpha * input-gradient mismatch on the theta inputs) with Adam; all
of it runs in the library's kernels (mlp_* and mc_price_jacobian), this module
only arranges buffers.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib, inputs

PRICE_SCALE = 100.0  # network output = price / PRICE_SCALE


@dataclass
class Normaliser:
    """Affine maps of (theta, K, T) onto about [-1, 1]."""
    lo: np.ndarray
    hi: np.ndarray
    k_mid: float = 100.0
    k_half: float = 30.0
    t_mid: float = 1.125
    t_half: float = 0.875

    @property
    def th_mid(self):
        return 0.5 * (self.lo + self.hi)

    @property
    def th_half(self):
        return 0.5 * (self.hi - self.lo)

    def features(self, theta, K, T):
        """X [n, 7] (torch float32 on theta's device) for rows (theta_r, K_r, T_r)."""
        mid = torch.as_tensor(self.th_mid, dtype=theta.dtype, device=theta.device)
        half = torch.as_tensor(self.th_half, dtype=theta.dtype, device=theta.device)
        xt = (theta - mid) / half
        xk = ((K - self.k_mid) / self.k_half)[:, None]
        xT = ((T - self.t_mid) / self.t_half)[:, None]
        return torch.cat([xt, xk.to(theta.dtype), xT.to(theta.dtype)], dim=1).to(torch.float32).contiguous()

    def dprice_dtheta(self, dnet_dx):
        """d price/d theta from the network's input gradient on the theta columns."""
        half = torch.as_tensor(self.th_half, dtype=dnet_dx.dtype, device=dnet_dx.device)
        return dnet_dx[:, :5] * PRICE_SCALE / half


def default_normaliser():
    return Normaliser(lo=inputs.HESTON_RANGES["lo"].copy(), hi=inputs.HESTON_RANGES["hi"].copy())


def make_dataset(problem, n_theta, paths_per_theta, seed=0x5EED, device="cuda", chunk=4096, norm=None):
    """(X [n, 7], y [n], dy [n, 5]) float32 on the device, n = n_theta * m."""
    norm = norm or default_normaliser()
    dev = torch.device(device)
    rng = np.random.default_rng(seed)
    thetas = np.stack([inputs.draw_heston_theta(rng) for _ in range(n_theta)])
    strikes = rng.uniform(70.0, 130.0, (n_theta, problem.m))
    mc = _lib.Context(problem, max_paths=max(paths_per_theta, 32), device=dev)
    T_inst = torch.tensor(problem.mat_step * problem.dt, dtype=torch.float64, device=dev)
    Xs, ys, dys = [], [], []
    half = torch.as_tensor(norm.th_half, dtype=torch.float64, device=dev)
    for c0 in range(0, n_theta, chunk):
        c1 = min(n_theta, c0 + chunk)
        th = torch.tensor(thetas[c0:c1], dtype=torch.float64, device=dev)
        Kt = torch.tensor(strikes[c0:c1], dtype=torch.float64, device=dev)
        Ey, J = mc.price_jacobian(th, seed + c0, paths_per_theta, strikes=Kt)
        nt = c1 - c0
        th_rows = th[:, None, :].expand(nt, problem.m, 5).reshape(-1, 5)
        X = norm.features(th_rows, Kt.reshape(-1), T_inst.repeat(nt))
        Xs.append(X)
        ys.append((Ey.reshape(-1) / PRICE_SCALE).to(torch.float32))
        dys.append((J.reshape(-1, 5) * half / PRICE_SCALE).to(torch.float32))
    return torch.cat(Xs), torch.cat(ys), torch.cat(dys)


LAYER_SHAPES = [(256, 7), (256,), (256, 256), (256,), (256, 256), (256,), (256, 256), (256,), (256,), (1,)]


def init_params(seed=0):
    """Glorot-uniform weights and zero biases, flat in the library's layout."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in LAYER_SHAPES:
        if len(s) == 2:
            lim = math.sqrt(6.0 / (s[0] + s[1]))
            parts.append(rng.uniform(-lim, lim, s).ravel())
        elif s == (256,) and len(parts) == 8:  # w5
            lim = math.sqrt(6.0 / 257)
            parts.append(rng.uniform(-lim, lim, s))
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts)


class Surrogate:
    """FP32 master parameters and Adam state, with training and inference contexts."""

    def __init__(self, batch=4096, seed=0, device="cuda", norm=None, infer_rows=128):
        self.device = torch.device(device)
        self.norm = norm or default_normaliser()
        self.batch = batch
        self.train_net = _lib.Mlp(batch, self.device)
        self.infer_net = _lib.Mlp(max(128, (infer_rows + 127) // 128 * 128), self.device)
        n = self.train_net.n_params
        self.params = torch.tensor(init_params(seed), dtype=torch.float32, device=self.device)
        assert self.params.numel() == n
        self.grads = torch.zeros(n, dtype=torch.float32, device=self.device)
        self.m = torch.zeros(n, dtype=torch.float32, device=self.device)
        self.v = torch.zeros(n, dtype=torch.float32, device=self.device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.t = 0
        self.train_net.set_weights(self.params)
        self.infer_net.set_weights(self.params)
        self.history = []

    def train(self, X, y, dy, epochs=10, lr=1e-3, lr_final=1e-5, alpha=1.0, seed=0, log_every=0):
        """Adam on the differential loss over shuffled batches; returns seconds spent."""
        n = X.shape[0]
        nb = n // self.batch
        total = max(1, epochs * nb)
        g = torch.Generator(device=self.device).manual_seed(seed)
        Xb = torch.empty((self.batch, 7), dtype=torch.float32, device=self.device)
        yb = torch.empty(self.batch, dtype=torch.float32, device=self.device)
        dyb = torch.empty((self.batch, 5), dtype=torch.float32, device=self.device)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step = 0
        for ep in range(epochs):
            perm = torch.randperm(n, device=self.device, generator=g)
            for b in range(nb):
                idx = perm[b * self.batch:(b + 1) * self.batch]
                torch.index_select(X, 0, idx, out=Xb)
                torch.index_select(y, 0, idx, out=yb)
                torch.index_select(dy, 0, idx, out=dyb)
                # cosine decay of the learning rate from lr to lr_final
                a = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * step / total))
                self.t += 1
                self.train_net.train_step(self.params, Xb, yb, dyb, alpha, self.grads, self.loss, self.m, self.v,
                                          self.t, lr=a)
                step += 1
                if log_every and step % log_every == 0:
                    self.history.append((step, float(self.loss.item())))
        torch.cuda.synchronize()
        self.infer_net.set_weights(self.params)
        return time.perf_counter() - t0

    def evaluate_loss(self, X, y, dy, alpha=1.0):
        """Mean differential loss over whole batches of a data set."""
        nb = X.shape[0] // self.batch
        tot = 0.0
        for b in range(nb):
            sl = slice(b * self.batch, (b + 1) * self.batch)
            self.train_net.loss_grad(self.params, X[sl].contiguous(), y[sl].contiguous(), dy[sl].contiguous(),
                                     alpha, self.grads, self.loss)
            tot += float(self.loss.item())
        return tot / max(nb, 1)

    def prices(self, theta, K, T, with_grad=False):
        """Surrogate prices of the instruments (K, T) at theta (FP64 torch [5]), and
        d price/d theta [m, 5] when with_grad."""
        m = K.shape[0]
        th = theta.to(self.device, torch.float64)[None, :].expand(m, 5)
        X = self.norm.features(th, K.to(self.device, torch.float64), T.to(self.device, torch.float64))
        if with_grad:
            out, dx = self.infer_net.forward(self.params, X, with_grad=True)
            return out.double() * PRICE_SCALE, self.norm.dprice_dtheta(dx.double())
        return self.infer_net.forward(self.params, X).double() * PRICE_SCALE
