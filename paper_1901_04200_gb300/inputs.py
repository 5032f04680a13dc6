"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no arithmetic of the method: it only describes problems
(model, time grid, instruments) and draws their seeded inputs (parameters,
normals tables, targets).  The paper (arXiv 1901.04200, Heston SLV test
paragraph) names no market data; these workloads stand in for it:

* ``gbm_config``    GBM log-Euler, piecewise-constant vol in 8 buckets over 2y,
                    16 steps, 8 calls (strikes 80..120 at the bucket ends),
                    normals as a seeded FP64 input table [P x 16], FP64 path.
* ``heston_config`` Heston full-truncation Euler, 256 steps/yr over 2y, 64 calls
                    (8 maturities 0.25..2y x 8 strikes 70..130), Philox
                    normals, FP32 path arithmetic.
* ``lv_config``     bilinear local-vol surface on 20 times x 10 log-spot nodes
                    (values U(0.1, 0.4)), 5y at 500 steps, 200 calls
                    (20 maturities x 10 strikes 60..150), FP32, checkpoints
                    every 25 steps.

Targets C_i are Black-Scholes prices at hidden volatilities drawn U(0.15, 0.35).
Seeds: normals 1901, targets 4200, parameter draws 42, Philox key 0x190104200.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

SEED_NORMALS = 1901
SEED_TARGETS = 4200
SEED_PARAMS = 42
PHILOX_SEED = 0x190104200

HESTON_RANGES = {  # (kappa, theta_h, xi, rho, v0)
    "lo": np.array([0.5, 0.01, 0.2, -0.9, 0.01]),
    "hi": np.array([3.0, 0.1, 1.0, -0.3, 0.1]),
}


@dataclass
class Problem:
    """One calibration problem: model, time grid and instruments.

    kind: "gbm" | "heston" | "lv".  State x = ln(S/S0) starts at 0.
    Instrument i: call with strike K[i] paying at step mat_step[i].
    normals: optional FP64 table [P, n_steps * normals_per_step] for global
    paths normals_path0.. (GBM workload); otherwise Philox with key ``seed``.
    precision / ckpt_every / paths_per_thread are knobs of the CUDA path.
    """
    kind: str
    S0: float
    r: float
    dt: float
    n_steps: int
    K: np.ndarray
    mat_step: np.ndarray
    seed: int = PHILOX_SEED
    bucket_end: Optional[np.ndarray] = None
    nt: int = 0
    nx: int = 0
    t_max: float = 0.0
    x_lo: float = 0.0
    x_hi: float = 0.0
    normals: Optional[np.ndarray] = None
    normals_path0: int = 0
    precision: str = "fp32"
    ckpt_every: int = 0
    paths_per_thread: int = 0
    # what the reverse sweep reads: "checkpoint" (states every K steps, re-run with
    # regenerated normals), "normals" (the checkpoints and every normal drawn),
    # "full" (every step's tape), "states" (local vol: the state before every step),
    # "auto" (states for local vol, normals otherwise, if they fit a quarter of the
    # device's memory, else checkpoint)
    storage: str = "auto"

    @property
    def m(self) -> int:
        return len(self.K)

    @property
    def n_params(self) -> int:
        if self.kind == "gbm":
            return len(self.bucket_end)
        if self.kind == "heston":
            return 5
        if self.kind == "slv":
            return 5 + self.nt * self.nx
        return self.nt * self.nx

    @property
    def normals_per_step(self) -> int:
        return 2 if self.kind in ("heston", "slv") else 1

    @property
    def last_step(self) -> int:
        return int(np.max(self.mat_step))


@dataclass
class Workload:
    name: str
    problem: Problem
    theta: np.ndarray
    C: np.ndarray
    n_paths: int
    extra: dict = field(default_factory=dict)


def _bs_call(S, K, T, r, vol):
    """Black-Scholes call price (target generator only)."""
    if T <= 0 or vol <= 0:
        return max(S - K * math.exp(-r * T), 0.0)
    sd = vol * math.sqrt(T)
    d1 = (math.log(S / K) + (r + 0.5 * vol * vol) * T) / sd
    d2 = d1 - sd
    N = lambda u: 0.5 * (1.0 + math.erf(u / math.sqrt(2.0)))
    return S * N(d1) - K * math.exp(-r * T) * N(d2)


def _bs_targets(S0, r, K, T, vols_per_mat, mat_index):
    return np.array([_bs_call(S0, K[i], T[i], r, vols_per_mat[mat_index[i]]) for i in range(len(K))])


def gbm_config(n_paths: int = 4096, n_steps: int = 16, n_buckets: int = 8, T: float = 2.0,
               seed_normals: int = SEED_NORMALS, path0: int = 0) -> Workload:
    """GBM log-Euler, piecewise-constant vol; normals as a seeded FP64 table."""
    assert n_steps % n_buckets == 0
    dt = T / n_steps
    spb = n_steps // n_buckets
    bucket_end = np.arange(1, n_buckets + 1, dtype=np.int32) * spb
    K = np.linspace(80.0, 120.0, n_buckets)
    mat_step = bucket_end.copy()
    rng = np.random.default_rng(seed_normals)
    normals = rng.standard_normal((path0 + n_paths, n_steps))[path0:]
    trng = np.random.default_rng(SEED_TARGETS)
    hidden = trng.uniform(0.15, 0.35, n_buckets)
    # C_i = BS at sigma_eff with sigma_eff^2 T_i = sum_{b <= i} hidden_b^2 * (bucket length)
    Ti = mat_step * dt
    cumvar = np.cumsum(hidden ** 2 * spb * dt)
    C = np.array([_bs_call(100.0, K[i], Ti[i], 0.02, math.sqrt(cumvar[i] / Ti[i]))
                  for i in range(n_buckets)])
    pb = Problem(kind="gbm", S0=100.0, r=0.02, dt=dt, n_steps=n_steps, K=K, mat_step=mat_step,
                 bucket_end=bucket_end, normals=normals, normals_path0=path0,
                 precision="fp64", ckpt_every=spb)
    theta = np.full(n_buckets, 0.25)
    return Workload("gbm_pwc_m8_s16_fp64", pb, theta, C, n_paths, {"hidden_vol": hidden})


def heston_instruments(steps_per_year: int, n_mat: int = 8, n_strike: int = 8,
                       t_lo: float = 0.25, t_hi: float = 2.0, k_lo: float = 70.0, k_hi: float = 130.0):
    Tm = np.linspace(t_lo, t_hi, n_mat)
    steps = np.rint(Tm * steps_per_year).astype(np.int32)
    strikes = np.linspace(k_lo, k_hi, n_strike)
    K = np.tile(strikes, n_mat)
    mat_step = np.repeat(steps, n_strike).astype(np.int32)
    mat_index = np.repeat(np.arange(n_mat), n_strike)
    return K, mat_step, mat_index


def draw_heston_theta(rng, feller: bool = True) -> np.ndarray:
    """Uniform draw from the parameter box; with ``feller`` the draw is
    repeated until 2 kappa theta_h > xi^2 (the pathwise gradient of the
    full-truncation scheme is heavy-tailed in v^-1/2 otherwise)."""
    while True:
        th = rng.uniform(HESTON_RANGES["lo"], HESTON_RANGES["hi"])
        if not feller or 2.0 * th[0] * th[1] > th[2] ** 2:
            return th


def heston_config(n_paths: int = 1 << 20, steps_per_year: int = 256, T: float = 2.0,
                  n_mat: int = 8, n_strike: int = 8, seed: int = PHILOX_SEED,
                  ckpt_every: int = 8, feller: bool = True) -> Workload:
    """Heston full-truncation Euler with Philox normals; FP32 path arithmetic."""
    dt = 1.0 / steps_per_year
    n_steps = int(round(T * steps_per_year))
    K, mat_step, mat_index = heston_instruments(steps_per_year, n_mat, n_strike, T / n_mat, T)
    theta = draw_heston_theta(np.random.default_rng(SEED_PARAMS), feller)
    trng = np.random.default_rng(SEED_TARGETS)
    hidden = trng.uniform(0.15, 0.35, n_mat)
    C = _bs_targets(100.0, 0.02, K, mat_step * dt, hidden, mat_index)
    pb = Problem(kind="heston", S0=100.0, r=0.02, dt=dt, n_steps=n_steps, K=K, mat_step=mat_step,
                 seed=seed, precision="fp32", ckpt_every=ckpt_every)
    return Workload("heston_ft_m64_s512_fp32", pb, theta, C, n_paths, {"hidden_vol": hidden})


def lv_config(n_paths: int = 1 << 22, n_steps: int = 500, T: float = 5.0, nt: int = 20,
              nx: int = 10, n_mat: int = 20, n_strike: int = 10, seed: int = PHILOX_SEED,
              ckpt_every: int = 5, paths_per_thread: int = 4) -> Workload:
    """Bilinear local-vol surface over (t, ln S/S0); FP32 path arithmetic.  Segments of 5
    steps with four paths per thread: the fastest launch shape measured on 2^22 x 500 with the
    stored states the library picks for local vol (7.1 ms per value and gradient; with two paths
    per thread it measured 8.1 ms and with stored normals 8.5 ms, in earlier builds)."""
    dt = T / n_steps
    steps = (np.arange(1, n_mat + 1) * (n_steps // n_mat)).astype(np.int32)
    strikes = np.linspace(60.0, 150.0, n_strike)
    K = np.tile(strikes, n_mat)
    mat_step = np.repeat(steps, n_strike).astype(np.int32)
    mat_index = np.repeat(np.arange(n_mat), n_strike)
    theta = np.random.default_rng(SEED_PARAMS).uniform(0.1, 0.4, nt * nx)
    trng = np.random.default_rng(SEED_TARGETS)
    hidden = trng.uniform(0.15, 0.35, n_mat)
    C = _bs_targets(100.0, 0.02, K, mat_step * dt, hidden, mat_index)
    pb = Problem(kind="lv", S0=100.0, r=0.02, dt=dt, n_steps=n_steps, K=K, mat_step=mat_step,
                 seed=seed, nt=nt, nx=nx, t_max=T, x_lo=-1.0, x_hi=1.0,
                 precision="fp32", ckpt_every=ckpt_every, paths_per_thread=paths_per_thread)
    return Workload("lv_bilinear_m200_s500_fp32", pb, theta, C, n_paths, {"hidden_vol": hidden})


def slv_config(n_paths: int = 1 << 20, steps_per_year: int = 256, T: float = 2.0, n_mat: int = 8,
               n_strike: int = 8, nt: int = 9, nx: int = 10, seed: int = PHILOX_SEED,
               ckpt_every: int = 8) -> Workload:
    """Heston stochastic local volatility (the paper's test model): Heston parameters drawn as in
    heston_config and a leverage surface L(t, x) on nt x nx nodes (t_j = j T/(nt-1), x in [-1, 1]),
    values U(0.8, 1.2); parameters (kappa, theta_h, xi, rho, v0, L...)."""
    w = heston_config(n_paths=n_paths, steps_per_year=steps_per_year, T=T, n_mat=n_mat, n_strike=n_strike,
                      seed=seed, ckpt_every=ckpt_every)
    lev = np.random.default_rng(SEED_PARAMS + 1).uniform(0.8, 1.2, nt * nx)
    pb = replace(w.problem, kind="slv", nt=nt, nx=nx, t_max=T, x_lo=-1.0, x_hi=1.0)
    theta = np.concatenate([w.theta, lev])
    return Workload("heston_slv_m%d_s%d_fp32" % (pb.m, pb.n_steps), pb, theta, w.C, n_paths, w.extra)


def with_paths(w: Workload, n_paths: int) -> Workload:
    return replace(w, n_paths=n_paths)
