"""The two-step algorithm over several ranks (one GPU each), paths partitioned.

Rank r evaluates its own global path range.  The algorithm then has exactly
two exchange steps (two-step algorithm, steps 1 -> 2 and 2 -> 3):
  1. all-gather of (n_r, E_r y): every rank forms the global
     E y = sum_r n_r E_r y / sum_r n_r in rank order, then lambda and G;
  2. after each rank's reverse sweep seeded with the global lambda
     (mc_vjp), all-gather of (n_r, theta_bar_r): grad G = sum_r n_r
     theta_bar_r / sum_r n_r in rank order.
Sums run in rank order on every rank, so all ranks hold identical G and
grad G.  Only m + 1 and M + 1 FP64 numbers cross ranks per evaluation.
The compute is passed in (forward_fn, vjp_fn), so the same code runs with the
CUDA library under NCCL and with any other per-rank evaluator under gloo.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def _gather_weighted_mean(local, n_local, group=None):
    """sum_r n_r x_r / sum_r n_r over ranks, in rank order (FP64)."""
    x = torch.as_tensor(local, dtype=torch.float64).reshape(-1)
    buf = torch.cat([torch.tensor([float(n_local)], dtype=torch.float64, device=x.device), x])
    world = dist.get_world_size(group)
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    num = torch.zeros_like(x)
    den = torch.zeros(1, dtype=torch.float64, device=x.device)
    for p in parts:  # rank order
        num = num + p[0] * p[1:]
        den = den + p[0]
    return num / den


def sharded_value_and_grad(forward_fn, vjp_fn, C, n_local, group=None):
    """(E y, G, grad G) of the global estimator; forward_fn() -> local E y [m],
    vjp_fn(ybar) -> local sum_i ybar_i d(E_r y_i)/d theta [M] (after forward_fn)."""
    Ey = _gather_weighted_mean(forward_fn(), n_local, group)
    C = torch.as_tensor(C, dtype=torch.float64, device=Ey.device)
    lam = Ey - C
    G = 0.5 * torch.sum(lam * lam)
    grad = _gather_weighted_mean(vjp_fn(lam), n_local, group)
    return Ey, G, grad
