"""torch.autograd.Function over the MC-AAD library.

``mc_expect(ctx, theta, seed, n_paths)`` returns E y(theta) (step 1 of the
paper's two-step algorithm) and records checkpoints; its backward is the
reverse sweep seeded with the incoming gradient y-bar (eq. 0711A per path,
then the mean over paths).  For G = 1/2 |E y - C|^2, torch hands the backward
exactly the paper's lambda = E y - C, so ``G.backward()`` is steps 2-3.
Both directions run in the library's CUDA kernels.
"""
from __future__ import annotations

import torch

from . import _lib


class McExpect(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, mc: "_lib.Context", seed: int, n_paths: int, path0: int):
        th = theta.detach().to(torch.float64).contiguous()
        Ey = mc.forward(th, seed, n_paths, path0=path0, keep=True)
        mc._generation = getattr(mc, "_generation", 0) + 1
        ctx.mc, ctx.seed, ctx.n_paths, ctx.path0 = mc, seed, n_paths, path0
        ctx.generation = mc._generation
        ctx.save_for_backward(th)
        return Ey

    @staticmethod
    def backward(ctx, ybar):
        (th,) = ctx.saved_tensors
        mc = ctx.mc
        if mc._generation != ctx.generation:
            # a later forward replaced the checkpoints: re-run this one
            mc.forward(th, ctx.seed, ctx.n_paths, path0=ctx.path0, keep=True)
            mc._generation += 1
            ctx.generation = mc._generation
        g = mc.vjp(ybar.detach().to(torch.float64).contiguous())
        return g, None, None, None, None


def mc_expect(mc: "_lib.Context", theta: torch.Tensor, seed: int, n_paths: int, path0: int = 0):
    """E y(theta) as a differentiable torch op (FP64 [m] on the context's device)."""
    return McExpect.apply(theta, mc, seed, n_paths, path0)


def calibration_objective(mc, theta, C, seed, n_paths, path0=0):
    """G = 1/2 sum_i (E y_i - C_i)^2 (eq. 241118A) as a differentiable torch op."""
    Ey = mc_expect(mc, theta, seed, n_paths, path0)
    return 0.5 * torch.sum((Ey - C) ** 2)
