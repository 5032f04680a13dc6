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
