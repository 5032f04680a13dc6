"""Calibration host logic on the oracle: the optimisers driven by the FP64
oracle's G and grad G recover the hidden parameters when the targets are
priced with the same seed and paths (common random numbers: G = 0 at theta*)."""
import numpy as np
import pytest

from paper_1901_04200_gb300 import calibrate, inputs

LO, HI = inputs.HESTON_RANGES["lo"], inputs.HESTON_RANGES["hi"]


def small_problem():
    w = inputs.heston_config(n_paths=2048, steps_per_year=32, T=1.0, n_mat=4, n_strike=4)
    return w.problem


def oracle_objective(orc, pb, C, n):
    def f(theta):
        _, G, g = orc.value_and_grad(pb, theta, C, n, n_threads=4)
        return G, g
    return f


@pytest.mark.parametrize("start", [0.1, 0.9])
def test_lbfgs_wrapper_on_a_quadratic(start):
    """L-BFGS-B in box-scaled coordinates reaches the minimiser of a convex
    quadratic G = 1/2 |A (theta - theta*)|^2 (interior and on a bound) and stops
    as soon as G < tol."""
    rng = np.random.default_rng(0)
    A = rng.normal(size=(8, 5)) * (HI - LO)[None, :] ** -1
    for theta_star in [LO + 0.37 * (HI - LO), np.where(np.arange(5) == 2, HI, LO + 0.5 * (HI - LO))]:
        def f(th):
            r = A @ (th - theta_star)
            return 0.5 * float(r @ r), A.T @ r
        r = calibrate.descend_lbfgs(f, LO + start * (HI - LO), LO, HI, 1e-20, max_evals=500)
        assert r.converged
        assert np.max(np.abs(r.theta - theta_star) / (HI - LO)) < 1e-8


def test_metric_descent_with_exact_jacobian_on_oracle(orc):
    """descend_metric with the exact Jacobian (the oracle's unit-seed vjps) is Gauss-Newton."""
    pb, n = small_problem(), 2048
    rng = np.random.default_rng(8)
    theta_star, theta0 = inputs.draw_heston_theta(rng), inputs.draw_heston_theta(rng)
    C = orc.forward(pb, theta_star, n, n_threads=4)
    eye = np.eye(pb.m)
    jac = lambda th: np.stack([orc.vjp(pb, th, eye[i], n, n_threads=4) for i in range(pb.m)])
    r = calibrate.descend_metric(oracle_objective(orc, pb, C, n), jac, theta0, LO, HI, 1e-12, max_evals=60)
    assert r.converged and r.evals < 40


def test_projected_gradient_descent_decreases_monotonically(orc):
    pb, n = small_problem(), 1024
    rng = np.random.default_rng(2)
    theta_star, theta0 = inputs.draw_heston_theta(rng), inputs.draw_heston_theta(rng)
    C = orc.forward(pb, theta_star, n, n_threads=4)
    r = calibrate.descend(oracle_objective(orc, pb, C, n), theta0, LO, HI, 1e-14, max_evals=60)
    Gs = [G for _, G in r.trace]
    assert all(b < a for a, b in zip(Gs, Gs[1:]))
    assert np.all(r.theta >= LO) and np.all(r.theta <= HI)
