"""Pins of the FP64 oracle against what the paper and the mathematics fix.

* the gradient identity of the paper (dG/dx_j = E(sum_i (E y_i - C_i) dy_i/dx_j)):
  the two-step gradient equals the derivative of the whole program with the
  expectation differentiated through (Fries' expected backward AD, Appendix);
* Black-Scholes closed forms: GBM log-Euler with piecewise-constant vol,
  Heston with xi = 0 and a local-vol surface constant in x all give a
  lognormal S_T with a known total variance;
* the martingale property E[exp(-rT) S_T] = S0 of all three discretisations;
* central finite differences of the oracle's own G with common random numbers;
* the paper's cost table agrees with eq. 0711C.
"""
import json
import math
import os
from dataclasses import replace

import numpy as np
import pytest
from scipy.stats import norm

from paper_1901_04200_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def bs_call(S, K, T, r, vol):
    sd = vol * math.sqrt(T)
    d1 = (math.log(S / K) + (r + 0.5 * vol * vol) * T) / sd
    return S * norm.cdf(d1) - K * math.exp(-r * T) * norm.cdf(d1 - sd)


def bs_vega(S, K, T, r, vol):
    sd = vol * math.sqrt(T)
    d1 = (math.log(S / K) + (r + 0.5 * vol * vol) * T) / sd
    return S * norm.pdf(d1) * math.sqrt(T)


def batched(fn, n_paths, n_batches=16):
    """Mean and standard error of a path mean from independent path batches."""
    b = n_paths // n_batches
    vals = np.array([fn(k * b, b) for k in range(n_batches)])
    return vals.mean(0), vals.std(0, ddof=1) / math.sqrt(n_batches)


def gbm_philox(n_steps=16, n_buckets=8):
    w = inputs.gbm_config(n_paths=16, n_steps=n_steps, n_buckets=n_buckets)
    pb = replace(w.problem, normals=None)
    return w, pb


# ----------------------------------------------------------- gradient identity

@pytest.mark.parametrize("kind", ["gbm", "heston", "lv", "heston_nofeller"])
def test_two_step_equals_full_tape_fries(orc, kind):
    from oracle import tape
    P = 16
    if kind == "gbm":
        w = inputs.gbm_config(n_paths=P, n_steps=4, n_buckets=2)
    elif kind.startswith("heston"):
        w = inputs.heston_config(n_paths=P, steps_per_year=4, T=1.0, n_mat=2, n_strike=3,
                                 feller=(kind == "heston"))
    else:
        w = inputs.lv_config(n_paths=P, n_steps=4, T=4.0, nt=3, nx=4, n_mat=2, n_strike=3)
    pb = w.problem
    Z = pb.normals if pb.normals is not None else orc.normals_fill(pb.seed, 0, P, pb.n_steps * pb.normals_per_step)
    Ey, G, g = orc.value_and_grad(pb, w.theta, w.C, P)
    Gt, gt = tape.full_tape_value_and_grad(pb, w.theta, w.C, Z)
    assert math.isclose(G, Gt, rel_tol=1e-13)
    assert np.max(np.abs(g - gt)) <= 1e-13 * np.max(np.abs(gt))


def test_lv_full_tape_with_clamping(orc):
    """Paths leaving the surface's x range (flat extrapolation) still agree."""
    from oracle import tape
    P = 16
    w = inputs.lv_config(n_paths=P, n_steps=4, T=4.0, nt=3, nx=4, n_mat=2, n_strike=3)
    pb = replace(w.problem, x_lo=-0.05, x_hi=0.05)
    Z = orc.normals_fill(pb.seed, 0, P, pb.n_steps)
    _, G, g = orc.value_and_grad(pb, w.theta, w.C, P)
    st = np.array([orc.path_forward(pb, w.theta, p)[0][:, 0] for p in range(P)])
    assert (st > 0.05).any() and (st < -0.05).any()
    Gt, gt = tape.full_tape_value_and_grad(pb, w.theta, w.C, Z)
    assert math.isclose(G, Gt, rel_tol=1e-13)
    assert np.max(np.abs(g - gt)) <= 1e-13 * np.max(np.abs(gt))


def test_vjp_is_linear_and_matches_value_and_grad(orc):
    w = inputs.heston_config(n_paths=256, steps_per_year=16, T=1.0, n_mat=4, n_strike=3)
    pb, P = w.problem, 256
    Ey, G, g = orc.value_and_grad(pb, w.theta, w.C, P)
    assert math.isclose(G, 0.5 * np.sum((Ey - w.C) ** 2), rel_tol=1e-14)
    gv = orc.vjp(pb, w.theta, Ey - w.C, P)
    assert np.allclose(gv, g, rtol=1e-13, atol=0)
    a = np.random.default_rng(0).standard_normal(pb.m)
    b = np.random.default_rng(1).standard_normal(pb.m)
    lhs = orc.vjp(pb, w.theta, 2.0 * a - 3.0 * b, P)
    rhs = 2.0 * orc.vjp(pb, w.theta, a, P) - 3.0 * orc.vjp(pb, w.theta, b, P)
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(lhs))


# --------------------------------------------------------------- closed forms

@pytest.mark.slow
def test_gbm_matches_black_scholes(orc):
    """Log-Euler is exact for GBM: E y_i -> BS at sigma_eff^2 T_i = sum_b theta_b^2 dt_b."""
    w, pb = gbm_philox()
    theta = np.array([0.15, 0.3, 0.22, 0.18, 0.35, 0.25, 0.2, 0.28])
    P = 1 << 20
    Ey, se = batched(lambda p0, n: orc.forward(pb, theta, n, path0=p0), P)
    dt = pb.dt
    spb = pb.n_steps // len(theta)
    for i in range(pb.m):
        Ti = pb.mat_step[i] * dt
        var = np.sum(theta[: i + 1] ** 2) * spb * dt
        ref = bs_call(pb.S0, pb.K[i], Ti, pb.r, math.sqrt(var / Ti))
        assert abs(Ey[i] - ref) < 5 * se[i] + 1e-12, (i, Ey[i], ref, se[i])
    # gradient: dE y_i/dtheta_b = vega_i * theta_b dt_b / (sigma_eff_i T_i), b <= bucket(i)
    for i in [1, 4, 7]:
        e = np.zeros(pb.m)
        e[i] = 1.0
        gi, gse = batched(lambda p0, n: orc.vjp(pb, theta, e, n, path0=p0), P)
        Ti = pb.mat_step[i] * dt
        var = np.sum(theta[: i + 1] ** 2) * spb * dt
        s_eff = math.sqrt(var / Ti)
        vega = bs_vega(pb.S0, pb.K[i], Ti, pb.r, s_eff)
        ref = np.array([vega * theta[b] * spb * dt / (s_eff * Ti) if b <= i else 0.0 for b in range(8)])
        assert np.all(np.abs(gi - ref) <= 5 * gse + 1e-12), (i, gi, ref, gse)
        assert np.all(gi[i + 1:] == 0.0)


@pytest.mark.slow
def test_heston_xi0_reduces_to_black_scholes(orc):
    """xi = 0: v is deterministic, S_T lognormal with variance sum_n v_n dt."""
    w = inputs.heston_config(n_paths=16, steps_per_year=64, T=1.0, n_mat=4, n_strike=4)
    pb = w.problem
    theta = np.array([1.5, 0.05, 0.0, -0.6, 0.02])
    kappa, thh, _, _, v0 = theta
    dt = pb.dt
    nl = pb.last_step
    v = np.zeros(nl + 1)
    dv = np.zeros((nl + 1, 3))  # d v_n / d(kappa, theta_h, v0)
    v[0], dv[0] = v0, (0.0, 0.0, 1.0)
    for n in range(nl):
        v[n + 1] = v[n] + kappa * (thh - v[n]) * dt
        dv[n + 1, 0] = dv[n, 0] * (1 - kappa * dt) + (thh - v[n]) * dt
        dv[n + 1, 1] = dv[n, 1] * (1 - kappa * dt) + kappa * dt
        dv[n + 1, 2] = dv[n, 2] * (1 - kappa * dt)
    P = 1 << 18
    Ey, se = batched(lambda p0, n: orc.forward(pb, theta, n, path0=p0), P)
    for i in range(pb.m):
        ni = pb.mat_step[i]
        Ti = ni * dt
        var = np.sum(v[:ni]) * dt
        ref = bs_call(pb.S0, pb.K[i], Ti, pb.r, math.sqrt(var / Ti))
        assert abs(Ey[i] - ref) < 5 * se[i] + 1e-12
    for i in [0, 5, 15]:
        e = np.zeros(pb.m)
        e[i] = 1.0
        gi, gse = batched(lambda p0, n: orc.vjp(pb, theta, e, n, path0=p0), P)
        ni = pb.mat_step[i]
        Ti = ni * dt
        var = np.sum(v[:ni]) * dt
        s_eff = math.sqrt(var / Ti)
        vega = bs_vega(pb.S0, pb.K[i], Ti, pb.r, s_eff)
        dvar = np.sum(dv[:ni], axis=0) * dt
        ref = vega * dvar / (2 * s_eff * Ti)
        got = gi[[0, 1, 4]]
        assert np.all(np.abs(got - ref) <= 5 * gse[[0, 1, 4]] + 1e-12), (i, got, ref)
        assert gi[3] == 0.0  # rho only acts through xi


@pytest.mark.slow
def test_lv_constant_in_x_reduces_to_black_scholes(orc):
    """A surface constant in x: sigma(t_n) deterministic, S_T lognormal."""
    w = inputs.lv_config(n_paths=16, n_steps=100, T=2.0, nt=5, nx=6, n_mat=4, n_strike=3)
    pb = w.problem
    s = np.array([0.15, 0.3, 0.2, 0.25, 0.35])
    theta = np.repeat(s, pb.nx)
    dt = pb.dt
    ht = pb.t_max / (pb.nt - 1)
    nl = pb.last_step
    sig = np.zeros(nl)
    wt = np.zeros((nl, pb.nt))  # hat weights of the time nodes
    for n in range(nl):
        u = n * dt / ht
        for j in range(pb.nt):
            wt[n, j] = max(0.0, 1.0 - abs(u - j))
        sig[n] = wt[n] @ s
    P = 1 << 18
    Ey, se = batched(lambda p0, n: orc.forward(pb, theta, n, path0=p0), P)
    for i in range(pb.m):
        ni = pb.mat_step[i]
        Ti = ni * dt
        ref = bs_call(pb.S0, pb.K[i], Ti, pb.r, math.sqrt(np.sum(sig[:ni] ** 2) * dt / Ti))
        assert abs(Ey[i] - ref) < 5 * se[i] + 1e-12
    for i in [1, 7, 11]:
        e = np.zeros(pb.m)
        e[i] = 1.0
        gi, gse = batched(lambda p0, n: orc.vjp(pb, theta, e, n, path0=p0).reshape(pb.nt, pb.nx).sum(1), P)
        ni = pb.mat_step[i]
        Ti = ni * dt
        var = np.sum(sig[:ni] ** 2) * dt
        s_eff = math.sqrt(var / Ti)
        vega = bs_vega(pb.S0, pb.K[i], Ti, pb.r, s_eff)
        dvar = 2.0 * (sig[:ni, None] * wt[:ni]).sum(0) * dt
        ref = vega * dvar / (2 * s_eff * Ti)
        assert np.all(np.abs(gi - ref) <= 5 * gse + 1e-12), (i, gi, ref, gse)


@pytest.mark.parametrize("kind", ["gbm", "heston", "lv"])
def test_martingale(orc, kind):
    """E[exp(-r T) S_T] = S0 for every discretisation; its gradient has mean 0."""
    if kind == "gbm":
        w, pb = gbm_philox()
    elif kind == "heston":
        w = inputs.heston_config(n_paths=16, steps_per_year=32, T=1.0, n_mat=2, n_strike=2)
        pb = w.problem
    else:
        w = inputs.lv_config(n_paths=16, n_steps=50, T=1.0, nt=4, nx=5, n_mat=2, n_strike=2)
        pb = w.problem
    pb = replace(pb, K=np.zeros(pb.m))
    P = 1 << 16
    Ey, se = batched(lambda p0, n: orc.forward(pb, w.theta, n, path0=p0), P)
    assert np.all(np.abs(Ey - pb.S0) < 5 * se)
    e = np.ones(pb.m)
    g, gse = batched(lambda p0, n: orc.vjp(pb, w.theta, e, n, path0=p0), P)
    assert np.all(np.abs(g) <= 5 * gse + 1e-9)


# --------------------------------------------------------- finite differences

@pytest.mark.parametrize("kind", ["gbm", "heston", "lv"])
def test_fd_common_random_numbers(orc, kind):
    if kind == "gbm":
        w = inputs.gbm_config(n_paths=4096)
        P = 4096
        idx = range(8)
    elif kind == "heston":
        w = inputs.heston_config(n_paths=1 << 11, steps_per_year=64)
        P = 1 << 11
        idx = range(5)
    else:
        w = inputs.lv_config(n_paths=1 << 10, n_steps=100, T=2.0, nt=5, nx=6, n_mat=4, n_strike=5)
        P = 1 << 10
        idx = [0, 7, 8, 13, 14, 20, 26, 29]
    pb = w.problem
    _, G, g = orc.value_and_grad(pb, w.theta, w.C, P)
    for j in idx:
        h = 1e-6 * max(1.0, abs(w.theta[j]))
        tp, tm = w.theta.copy(), w.theta.copy()
        tp[j] += h
        tm[j] -= h
        fd = (orc.value_and_grad(pb, tp, w.C, P)[1] - orc.value_and_grad(pb, tm, w.C, P)[1]) / (2 * h)
        assert abs(fd - g[j]) <= 1e-5 * np.max(np.abs(g)) + 1e-9, (kind, j, fd, g[j])


# ------------------------------------------------------ oracle bookkeeping

def test_partition_invariance(orc):
    w = inputs.heston_config(n_paths=3000, steps_per_year=16, T=1.0, n_mat=2, n_strike=3)
    pb = w.problem
    full = orc.forward(pb, w.theta, 3000)
    parts = (1000 * orc.forward(pb, w.theta, 1000) + 2000 * orc.forward(pb, w.theta, 2000, path0=1000)) / 3000
    assert np.allclose(full, parts, rtol=1e-13, atol=0)
    a = orc.forward(pb, w.theta, 3000, n_threads=1)
    b = orc.forward(pb, w.theta, 3000, n_threads=5)
    assert np.array_equal(a, b)  # fixed chunk order: thread count does not matter


def test_normals_table_equals_philox(orc):
    """A normals table filled from the generator reproduces Philox mode exactly."""
    w = inputs.lv_config(n_paths=64, n_steps=20, T=1.0, nt=3, nx=4, n_mat=2, n_strike=2)
    pb = w.problem
    Z = orc.normals_fill(pb.seed, 10, 64, pb.n_steps)
    a = orc.value_and_grad(pb, w.theta, w.C, 64, path0=10)
    b = orc.value_and_grad(replace(pb, normals=Z, normals_path0=10), w.theta, w.C, 64, path0=10)
    assert np.array_equal(a[0], b[0]) and a[1] == b[1] and np.array_equal(a[2], b[2])


def test_invalid_problems_rejected(orc):
    w = inputs.heston_config(n_paths=16, steps_per_year=16, T=1.0, n_mat=2, n_strike=2)
    pb = w.problem
    with pytest.raises(ValueError):
        orc.forward(pb, w.theta, 0)
    bad = w.theta.copy()
    bad[3] = 1.0
    with pytest.raises(ValueError):
        orc.forward(pb, bad, 16)
    with pytest.raises(ValueError):
        orc.forward(replace(pb, mat_step=pb.mat_step + pb.n_steps), w.theta, 16)


def test_paper_cost_table_satisfies_eq_0711C():
    """The table's last column is (2 K_F + K_R)/c, eq. 0711C, to print rounding."""
    with open(os.path.join(HERE, "golden", "paper_cost_table.json")) as f:
        tab = json.load(f)
    for row in tab["rows"]:
        total = 2 * row["KF_over_c"] + row["KR_over_c"]
        assert abs(total - row["cost_G_over_paths_costF"]) <= 0.005 + 1e-12, row


# ------------------------------------------------------- Heston SLV (paper's model)

def slv_small(P=16, nt=3, nx=4):
    return inputs.slv_config(n_paths=P, steps_per_year=4, T=1.0, n_mat=2, n_strike=3, nt=nt, nx=nx)


def test_slv_two_step_equals_full_tape(orc):
    from oracle import tape
    w = slv_small()
    pb, P = w.problem, 16
    Z = orc.normals_fill(pb.seed, 0, P, pb.n_steps * 2)
    _, G, g = orc.value_and_grad(pb, w.theta, w.C, P)
    Gt, gt = tape.full_tape_value_and_grad(pb, w.theta, w.C, Z)
    assert math.isclose(G, Gt, rel_tol=1e-13)
    assert np.max(np.abs(g - gt)) <= 1e-13 * np.max(np.abs(gt))


def test_slv_with_unit_leverage_is_heston(orc):
    """L = 1 everywhere gives exactly the Heston prices and Heston-parameter gradient."""
    w = inputs.slv_config(n_paths=512, steps_per_year=32, T=1.0, n_mat=4, n_strike=4)
    pb = w.problem
    th = w.theta.copy()
    th[5:] = 1.0
    wh = inputs.heston_config(n_paths=512, steps_per_year=32, T=1.0, n_mat=4, n_strike=4)
    Ey_s, G_s, g_s = orc.value_and_grad(pb, th, w.C, 512)
    Ey_h, G_h, g_h = orc.value_and_grad(wh.problem, th[:5], w.C, 512)
    assert np.array_equal(Ey_s, Ey_h) and G_s == G_h
    assert np.allclose(g_s[:5], g_h, rtol=1e-12, atol=1e-12 * np.max(np.abs(g_h)))


def test_slv_leverage_gradient_against_global_scale(orc):
    """d E y_i / d c of E y_i(L = c L0) at c = 1 equals sum_nodes L0 * dE y_i/dL (bilinear
    weights sum to one), by central differences with common random numbers."""
    w = inputs.slv_config(n_paths=2048, steps_per_year=32, T=1.0, n_mat=4, n_strike=4)
    pb, n = w.problem, 2048
    e = np.zeros(pb.m)
    e[9] = 1.0
    g = orc.vjp(pb, w.theta, e, n)
    h = 1e-6
    tp, tm = w.theta.copy(), w.theta.copy()
    tp[5:] *= 1 + h
    tm[5:] *= 1 - h
    fd = (orc.forward(pb, tp, n)[9] - orc.forward(pb, tm, n)[9]) / (2 * h)
    assert abs(fd - np.dot(w.theta[5:], g[5:])) <= 1e-6 * max(1.0, abs(fd))


def test_slv_fd_and_martingale(orc):
    w = inputs.slv_config(n_paths=1024, steps_per_year=32, T=1.0, n_mat=4, n_strike=4, nt=5, nx=6)
    pb, n = w.problem, 1024
    _, G, g = orc.value_and_grad(pb, w.theta, w.C, n)
    for j in [0, 1, 2, 3, 4, 5, 12, 20, 33]:
        hh = 1e-6 * max(1.0, abs(w.theta[j]))
        tp, tm = w.theta.copy(), w.theta.copy()
        tp[j] += hh
        tm[j] -= hh
        fd = (orc.value_and_grad(pb, tp, w.C, n)[1] - orc.value_and_grad(pb, tm, w.C, n)[1]) / (2 * hh)
        assert abs(fd - g[j]) <= 1e-5 * np.max(np.abs(g)) + 1e-9, (j, fd, g[j])
    pb0 = replace(pb, K=np.zeros(pb.m))
    Ey, se = batched(lambda p0, k: orc.forward(pb0, w.theta, k, path0=p0), 1 << 15)
    assert np.all(np.abs(Ey - pb.S0) < 5 * se)


# ------------------------------------------- Heston / SLV variance dynamics

def one_step_problem(kind, dt=0.25):
    """One Euler step of the Heston or SLV variance model (Heston SLV model paragraph:
    dV = kappa (theta_h - V) dt + xi sqrt(V) dW^V, d<W^S, W^V> = rho dt)."""
    pb = inputs.Problem(kind=kind, S0=100.0, r=0.02, dt=dt, n_steps=1,
                        K=np.array([100.0]), mat_step=np.array([1], dtype=np.int32))
    if kind == "slv":
        pb = replace(pb, nt=2, nx=2, t_max=1.0, x_lo=-1.0, x_hi=1.0)
    return pb


def moment_se(a, b):
    """Sample covariance of a and b and its standard error (delta method on the products)."""
    da, db = a - a.mean(), b - b.mean()
    prod = da * db
    return prod.mean(), prod.std(ddof=1) / math.sqrt(len(a))


@pytest.mark.parametrize("kind,lev", [("heston", 1.0), ("slv", 1.3), ("slv", 0.7)])
def test_one_step_conditional_moments(orc, kind, lev):
    """From a fixed v0 > 0 one full-truncation Euler step has exactly
    E dx = (r - L^2 v0/2) dt, Var dx = L^2 v0 dt, E dv = kappa (theta_h - v0) dt,
    Var dv = xi^2 v0 dt and Cov(dx, dv) = rho xi L v0 dt (L the leverage, 1 for Heston):
    the drift, diffusion and correlation of both equations, independent of the adjoint."""
    kappa, thh, xi, rho, v0 = 1.5, 0.06, 0.7, -0.3, 0.04
    theta = np.array([kappa, thh, xi, rho, v0])
    pb = one_step_problem(kind)
    if kind == "slv":
        theta = np.concatenate([theta, np.full(4, lev)])
    N = 1 << 20
    st = orc.states_at(pb, theta, 1, N)
    dx, dv = st[:, 0], st[:, 1] - v0
    dt, r = pb.dt, pb.r
    sd_x, sd_v = math.sqrt(dx.var()), math.sqrt(dv.var())
    assert abs(dx.mean() - (r - 0.5 * lev * lev * v0) * dt) < 5 * sd_x / math.sqrt(N)
    assert abs(dv.mean() - kappa * (thh - v0) * dt) < 5 * sd_v / math.sqrt(N)
    for a, b, ref in [(dx, dx, lev * lev * v0 * dt), (dv, dv, xi * xi * v0 * dt),
                      (dx, dv, rho * xi * lev * v0 * dt)]:
        got, se = moment_se(a, b)
        assert abs(got - ref) < 5 * se, (got, ref, se)


def test_one_step_full_truncation(orc):
    """From v0 < 0 the step uses v+ = 0: no diffusion in x or v, and v moves by
    kappa theta_h dt exactly."""
    kappa, thh, xi, rho, v0 = 1.5, 0.06, 0.7, -0.3, -0.01
    pb = one_step_problem("heston")
    st = orc.states_at(pb, np.array([kappa, thh, xi, rho, v0]), 1, 1024)
    assert np.all(st[:, 0] == pb.r * pb.dt)
    assert np.allclose(st[:, 1], v0 + kappa * thh * pb.dt, rtol=0, atol=1e-17)


def heston_cf_call(S0, K, T, r, kappa, thh, xi, rho, v0):
    """Heston (1993) call price from the characteristic function of ln S_T, in the form of
    Albrecher, Mayer, Schoutens and Tistaert (2007, "the little Heston trap"), which stays
    on the principal branch of the complex logarithm: C = S0 P1 - K e^{-rT} P2 with
    P_j = 1/2 + (1/pi) int_0^inf Re[e^{-iu ln K} f_j(u) / (iu)] du,
    f_2(u) = phi(u), f_1(u) = phi(u - i) / phi(-i)."""
    from scipy.integrate import quad

    def phi(u):
        iu = 1j * u
        b = kappa - rho * xi * iu
        d = np.sqrt(b * b + xi * xi * (iu + u * u))
        g = (b - d) / (b + d)
        e = np.exp(-d * T)
        C = r * iu * T + kappa * thh / (xi * xi) * ((b - d) * T - 2.0 * np.log((1.0 - g * e) / (1.0 - g)))
        D = (b - d) / (xi * xi) * (1.0 - e) / (1.0 - g * e)
        return np.exp(C + D * v0 + iu * math.log(S0))

    lk = math.log(K)
    fwd = phi(-1j)

    def p1(u):
        return (np.exp(-1j * u * lk) * phi(u - 1j) / (1j * u * fwd)).real

    def p2(u):
        return (np.exp(-1j * u * lk) * phi(u) / (1j * u)).real

    P1 = 0.5 + quad(p1, 1e-10, 200.0, limit=500, epsabs=1e-12)[0] / math.pi
    P2 = 0.5 + quad(p2, 1e-10, 200.0, limit=500, epsabs=1e-12)[0] / math.pi
    return S0 * P1 - K * math.exp(-r * T) * P2


def test_heston_cf_pricer_reduces_to_black_scholes():
    """The pricer itself: at a tiny vol of vol the variance is deterministic, so the price is
    Black-Scholes at the integrated variance theta_h T + (v0 - theta_h)(1 - e^{-kappa T})/kappa."""
    kappa, thh, v0, T, r = 2.0, 0.05, 0.03, 1.0, 0.02
    var = thh * T + (v0 - thh) * (1.0 - math.exp(-kappa * T)) / kappa
    for K in (80.0, 100.0, 120.0):
        got = heston_cf_call(100.0, K, T, r, kappa, thh, 1e-3, -0.5, v0)
        ref = bs_call(100.0, K, T, r, math.sqrt(var / T))
        assert abs(got - ref) < 2e-3, (K, got, ref)


@pytest.mark.slow
def test_heston_matches_characteristic_function_price(orc):
    """The full-truncation Euler prices converge to Heston's closed-form price: at dt/2 the oracle's
    price lies within 5 standard errors plus the Euler bias, estimated by halving the step
    (weak order one: bias(dt/2) ~ price(dt) - price(dt/2)).  The two step sizes share their
    Brownian increments (a coarse normal is the scaled sum of two fine ones), so the bias estimate
    carries little noise."""
    kappa, thh, xi, rho, v0 = 3.0, 0.05, 0.5, -0.7, 0.03
    theta = np.array([kappa, thh, xi, rho, v0])
    strikes = np.array([80.0, 100.0, 120.0])
    T, n = 1.0, 64
    P, nb = 1 << 19, 16
    b = P // nb

    def problem(steps, Z, p0):
        return inputs.Problem(kind="heston", S0=100.0, r=0.02, dt=T / steps, n_steps=steps, K=strikes,
                              mat_step=np.full(3, steps, dtype=np.int32), normals=Z, normals_path0=p0)

    fine, diff = [], []
    for k in range(nb):
        Zf = np.random.default_rng(7000 + k).standard_normal((b, 2 * n, 2))  # [path, fine step, (z1, z2)]
        Zc = (Zf[:, 0::2, :] + Zf[:, 1::2, :]) / math.sqrt(2.0)
        yf = orc.forward(problem(2 * n, Zf.reshape(b, -1), k * b), theta, b, path0=k * b)
        yc = orc.forward(problem(n, np.ascontiguousarray(Zc.reshape(b, -1)), k * b), theta, b, path0=k * b)
        fine.append(yf)
        diff.append(yc - yf)
    fine, diff = np.array(fine), np.array(diff)
    pf, sf = fine.mean(0), fine.std(0, ddof=1) / math.sqrt(nb)
    bias, sb = diff.mean(0), diff.std(0, ddof=1) / math.sqrt(nb)
    ref = np.array([heston_cf_call(100.0, K, T, 0.02, kappa, thh, xi, rho, v0) for K in strikes])
    tol = 5 * sf + np.abs(bias) + 5 * sb
    assert np.all(np.abs(pf - ref) < tol), (pf, ref, sf, bias, sb)
    # the tolerance is a small part of each price: the pin sees the dynamics' shape
    assert np.all(tol < 0.02 * ref + 0.02), tol
