"""Heston calibration by gradient-based descent (the paper's application:
calibrating a stochastic model means minimising G = 1/2 sum_i (E y_i - C_i)^2).

Both arms use the same optimiser, fed only G and grad G: limited-memory BFGS
with box bounds (scipy's L-BFGS-B) on the parameters scaled to [0, 1]^5,
stopping as soon as G < tol (``descend`` is the plain projected gradient
descent with backtracking, kept for comparison; it is far slower on this
ill-conditioned problem).  The plain arm evaluates G and grad G by the
two-step MC-AAD algorithm at every iterate (mc_value_and_grad, common random
numbers: one seed for the whole descent); the surrogate arm first descends on
the surrogate's G (microseconds per evaluation) and then finishes with MC-AAD
steps from the surrogate's minimiser.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import inputs


@dataclass
class DescentResult:
    theta: np.ndarray
    G: float
    iters: int
    evals: int
    seconds: float
    converged: bool
    trace: list = field(default_factory=list)


def descend(value_and_grad, theta0, lo, hi, tol, max_evals=2000, step0=0.05, armijo=1e-4, min_step=1e-12,
            time_budget=None):
    """Projected preconditioned gradient descent with backtracking.
    value_and_grad(theta np[5]) -> (G float, grad np[5])."""
    D = (hi - lo) ** 2
    th = np.clip(np.asarray(theta0, dtype=np.float64), lo, hi)
    t0 = time.perf_counter()
    G, g = value_and_grad(th)
    evals, iters, step = 1, 0, step0
    trace = [(0, G)]
    while G >= tol and evals < max_evals and step > min_step:
        if time_budget and time.perf_counter() - t0 > time_budget:
            break
        cand = np.clip(th - step * D * g, lo, hi)
        d = th - cand
        Gc, gc = value_and_grad(cand)
        evals += 1
        if Gc <= G - armijo * float(g @ d) and np.isfinite(Gc):
            th, G, g = cand, Gc, gc
            iters += 1
            step *= 1.5
            trace.append((evals, G))
        else:
            step *= 0.5
    return DescentResult(th, G, iters, evals, time.perf_counter() - t0, G < tol, trace)


class _Converged(Exception):
    pass


def descend_lbfgs(value_and_grad, theta0, lo, hi, tol, max_evals=500, gtol=1e-12, restarts=20):
    """L-BFGS-B on u = (theta - lo)/(hi - lo) in [0, 1]^5; stops when G < tol.
    When the line search gives up before that, it restarts from the best point
    (fresh curvature memory) while evaluations remain."""
    from scipy.optimize import minimize
    lo = np.asarray(lo, dtype=np.float64)
    width = np.asarray(hi, dtype=np.float64) - lo
    best = {"G": np.inf, "theta": np.asarray(theta0, dtype=np.float64), "evals": 0}
    trace = []

    def f(u):
        th = lo + np.clip(u, 0.0, 1.0) * width
        G, g = value_and_grad(th)
        best["evals"] += 1
        trace.append((best["evals"], G))
        if G < best["G"]:
            best["G"], best["theta"] = G, th
        if G < tol:
            raise _Converged()
        return G, g * width

    t0 = time.perf_counter()
    iters = 0
    messages = []
    try:
        for _ in range(restarts + 1):
            left = max_evals - best["evals"]
            if left <= 0:
                break
            u0 = np.clip((best["theta"] - lo) / width, 0.0, 1.0)
            g_before = best["G"]
            res = minimize(f, u0, jac=True, method="L-BFGS-B", bounds=[(0.0, 1.0)] * len(u0),
                           options={"maxfun": left, "maxiter": left, "ftol": 0.0, "gtol": gtol})
            iters += int(res.nit)
            messages.append(str(res.message))
            if not best["G"] < g_before and res.nit == 0:
                break
    except _Converged:
        pass
    out = DescentResult(best["theta"], best["G"], iters, best["evals"], time.perf_counter() - t0,
                        best["G"] < tol, trace)
    out.messages = messages
    return out


def descend_metric(value_and_grad, metric, theta0, lo, hi, tol, max_evals=100, mu0=1e-6, mu_max=1e8):
    """Descent on G with the gradient from value_and_grad (the MC-AAD two-step
    algorithm) and the metric from metric(theta) -> J [m, 5]: in box-scaled
    coordinates the step solves (J^T J + mu diag(J^T J)) d = -grad, projected
    onto the box (Levenberg-Marquardt damping: mu grows tenfold after a step
    that does not lower G, shrinks threefold after one that does).  With J the
    surrogate's Jacobian this is a Gauss-Newton step whose curvature costs no
    Monte Carlo; with a poor J it falls back towards scaled gradient steps."""
    lo = np.asarray(lo, dtype=np.float64)
    width = np.asarray(hi, dtype=np.float64) - lo
    t0 = time.perf_counter()
    u = np.clip((np.asarray(theta0, dtype=np.float64) - lo) / width, 0.0, 1.0)
    G, g = value_and_grad(lo + u * width)
    evals, iters, mu = 1, 0, mu0
    trace = [(1, G)]
    J = metric(lo + u * width) * width[None, :]
    while G >= tol and evals < max_evals and mu <= mu_max:
        Hm = J.T @ J
        dg = np.maximum(np.diag(Hm), 1e-12 * max(np.trace(Hm), 1e-300))
        d = -np.linalg.solve(Hm + mu * np.diag(dg), g * width)
        cand = np.clip(u + d, 0.0, 1.0)
        Gc, gc = value_and_grad(lo + cand * width)
        evals += 1
        trace.append((evals, Gc))
        if np.isfinite(Gc) and Gc < G:
            u, G, g = cand, Gc, gc
            mu = max(mu / 3.0, 1e-12)
            iters += 1
            J = metric(lo + u * width) * width[None, :]
        else:
            mu *= 10.0
    return DescentResult(lo + u * width, G, iters, evals, time.perf_counter() - t0, G < tol, trace)


def surrogate_jacobian(sur, K, T):
    Kt = torch.as_tensor(K, dtype=torch.float64, device=sur.device)
    Tt = torch.as_tensor(T, dtype=torch.float64, device=sur.device)

    def f(theta):
        _, dp = sur.prices(torch.as_tensor(theta, dtype=torch.float64), Kt, Tt, with_grad=True)
        return dp.cpu().numpy()

    return f


def mc_objective(ctx, C, seed, n_paths):
    """(G, grad) of the MC-AAD path at theta, FP64 on the host (one stream sync per evaluation)."""
    Ct = torch.as_tensor(C, dtype=torch.float64, device=ctx.device)
    out = (torch.empty(1, dtype=torch.float64, device=ctx.device), torch.empty(ctx.M, dtype=torch.float64,
                                                                               device=ctx.device), None)
    th_dev = torch.empty(ctx.M, dtype=torch.float64, device=ctx.device)

    def f(theta):
        th_dev.copy_(torch.as_tensor(theta, dtype=torch.float64))
        G, g, _ = ctx.value_and_grad(th_dev, Ct, seed, n_paths, out=out)
        return float(G.item()), g.cpu().numpy()

    return f


def surrogate_objective(sur, K, T, C):
    Kt = torch.as_tensor(K, dtype=torch.float64, device=sur.device)
    Tt = torch.as_tensor(T, dtype=torch.float64, device=sur.device)
    Ct = torch.as_tensor(C, dtype=torch.float64, device=sur.device)

    def f(theta):
        p, dp = sur.prices(torch.as_tensor(theta, dtype=torch.float64), Kt, Tt, with_grad=True)
        lam = (p - Ct).cpu().numpy()
        return float(0.5 * lam @ lam), dp.cpu().numpy().T @ lam

    return f


def verify_by_mc(ctx, theta, theta_star, seed, n_paths, chunks=4):
    """Independent check of a calibrated theta: RMS difference of the prices at
    theta and at theta* over chunks * n_paths fresh paths (a seed the descent
    never used), and the standard error of that difference."""
    diffs = []
    for c in range(chunks):
        a = ctx.forward(theta, seed, n_paths, path0=c * n_paths).cpu().numpy()
        b = ctx.forward(theta_star, seed, n_paths, path0=c * n_paths).cpu().numpy()
        diffs.append(a - b)
    d = np.mean(diffs, axis=0)
    se = np.std(diffs, axis=0, ddof=1) / np.sqrt(chunks) if chunks > 1 else np.zeros_like(d)
    return {"paths": chunks * n_paths, "rms_price_diff": float(np.sqrt(np.mean(d * d))),
            "max_abs_price_diff": float(np.max(np.abs(d))), "max_stderr": float(np.max(se))}


def run_experiment(ctx, sur, theta0, C, seed, n_paths, tol=1e-8, max_evals=500, sur_evals=300):
    """Plain MC-AAD descent vs surrogate-then-MC-AAD descent from theta0 (same optimiser)."""
    lo, hi = inputs.HESTON_RANGES["lo"], inputs.HESTON_RANGES["hi"]
    pb = ctx.problem
    mc = mc_objective(ctx, C, seed, n_paths)
    mc(np.asarray(theta0))  # warm the path kernels once, outside both timings
    plain = descend_lbfgs(mc, theta0, lo, hi, tol, max_evals=max_evals)
    T = pb.mat_step * pb.dt
    sf = surrogate_objective(sur, pb.K, T, C)
    sf(np.asarray(theta0))
    s1 = descend_lbfgs(sf, theta0, lo, hi, 0.0, max_evals=sur_evals)
    s2 = descend_metric(mc, surrogate_jacobian(sur, pb.K, T), s1.theta, lo, hi, tol, max_evals=max_evals)
    return {"plain": plain, "surrogate_phase": s1, "mc_phase": s2,
            "surrogate_total_seconds": s1.seconds + s2.seconds}
