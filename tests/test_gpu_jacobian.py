"""Forward-mode Jacobian (surrogate labels) against the oracle.

Row i of d E y/d theta is the oracle's vector-Jacobian product with the unit
seed e_i; J^T lambda must equal grad G of the two-step algorithm on the same
paths (the gradient identity)."""
from dataclasses import replace

import numpy as np
import pytest

from paper_1901_04200_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_04200_gb300 import build as b
    b.build()
    from paper_1901_04200_gb300 import _lib
    return _lib


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_jacobian_matches_oracle(L, orc, precision, tol):
    w = inputs.heston_config(n_paths=1500, steps_per_year=32, T=1.0, n_mat=4, n_strike=4)
    pb = replace(w.problem, precision=precision)
    n, seed = 1500, 5
    rng = np.random.default_rng(7)
    thetas = np.stack([w.theta] + [inputs.draw_heston_theta(rng) for _ in range(2)])
    strikes = rng.uniform(70.0, 130.0, (3, pb.m))
    ctx = L.Context(pb, max_paths=n)
    Ey, J = ctx.price_jacobian(thetas, seed, n, strikes=strikes)
    Ey, J = Ey.cpu().numpy(), J.cpu().numpy()
    for t in range(3):
        pbt = replace(pb, K=strikes[t], seed=seed)
        Eo = orc.forward(pbt, thetas[t], n, path0=t * n)
        Jo = np.stack([orc.vjp(pbt, thetas[t], np.eye(pb.m)[i], n, path0=t * n) for i in range(pb.m)])
        assert rel(Ey[t], Eo) <= (1e-12 if precision == "fp64" else 2e-6)
        assert rel(J[t], Jo) <= tol, (t, rel(J[t], Jo))


def test_jacobian_transpose_lambda_is_grad_G(L):
    w = inputs.heston_config(n_paths=1 << 14, steps_per_year=64, T=1.0, n_mat=4, n_strike=4)
    pb = replace(w.problem, precision="fp64")
    n, seed = 1 << 14, 21
    ctx = L.Context(pb, max_paths=n)
    G, g, Ey = ctx.value_and_grad(w.theta, w.C, seed, n)
    Ey2, J = ctx.price_jacobian(w.theta[None, :], seed, n)
    lam = Ey2[0] - torch.tensor(w.C, dtype=torch.float64, device="cuda")
    g2 = J[0].T @ lam
    assert rel(Ey2[0].cpu().numpy(), Ey.cpu().numpy()) <= 1e-12
    assert rel(g2.cpu().numpy(), g.cpu().numpy()) <= 1e-10


def test_jacobian_many_thetas_fp32(L, orc):
    """The label-generation shape: many parameter vectors, one block each."""
    w = inputs.heston_config(n_paths=1024, steps_per_year=64, T=2.0)
    pb = w.problem
    rng = np.random.default_rng(11)
    nt, n = 2048, 1024
    thetas = np.stack([inputs.draw_heston_theta(rng) for _ in range(nt)])
    ctx = L.Context(pb, max_paths=n)
    Ey, J = ctx.price_jacobian(thetas, 3, n)
    Ey, J = Ey.cpu().numpy(), J.cpu().numpy()
    assert np.all(np.isfinite(Ey)) and np.all(np.isfinite(J))
    for t in [0, 777, nt - 1]:
        pbt = replace(pb, seed=3)
        Eo = orc.forward(pbt, thetas[t], n, path0=t * n)
        assert rel(Ey[t], Eo) <= 2e-6
        gi = orc.vjp(pbt, thetas[t], np.eye(pb.m)[10], n, path0=t * n)
        assert rel(J[t, 10], gi) <= 1e-4


# ------------------------------------- G and grad G by forward-mode tangents

@pytest.mark.parametrize("path0", [0, 12345])
def test_tangent_value_and_grad_fp64_matches_oracle(L, orc, path0):
    """mc_value_and_grad_tangent = the oracle's two-step G and grad G on the same paths."""
    w = inputs.heston_config(n_paths=2001, steps_per_year=32, T=1.0, n_mat=4, n_strike=5)
    pb = replace(w.problem, precision="fp64")
    ctx = L.Context(pb, max_paths=w.n_paths)
    G, g, Ey = ctx.value_and_grad_tangent(w.theta, w.C, pb.seed, w.n_paths, path0=path0)
    Eo, Go, go = orc.value_and_grad(pb, w.theta, w.C, w.n_paths, path0=path0)
    assert rel(Ey.cpu().numpy(), Eo) <= 1e-12
    assert abs(G.item() - Go) <= 1e-10 * abs(Go)
    assert rel(g.cpu().numpy(), go) <= 1e-10


def test_tangent_equals_adjoint_fp32(L):
    """Forward mode and the adjoint give the same estimator: E y to FP32 summation order,
    the gradient to FP32 rounding of the path arithmetic."""
    w = inputs.heston_config(n_paths=1 << 16, steps_per_year=64, T=2.0)
    ctx = L.Context(w.problem, max_paths=w.n_paths)
    Ga, ga, Ea = [t.cpu().numpy() for t in ctx.value_and_grad(w.theta, w.C, w.problem.seed, w.n_paths)]
    Gt, gt, Et = [t.cpu().numpy() for t in ctx.value_and_grad_tangent(w.theta, w.C, w.problem.seed, w.n_paths)]
    assert rel(Et, Ea) <= 1e-6
    assert rel(gt, ga) <= 1e-4
    assert abs(Gt[0] - Ga[0]) <= 1e-4 * abs(Ga[0])


def test_tangent_rejects_other_models(L):
    w = inputs.lv_config(n_paths=64, n_steps=100, T=2.0, nt=5, nx=6, n_mat=4, n_strike=5)
    ctx = L.Context(w.problem, max_paths=64)
    with pytest.raises(L.McError) as e:
        ctx.value_and_grad_tangent(w.theta, w.C, w.problem.seed, 64)
    assert e.value.status == L.MC_ERR_UNSUPPORTED


@pytest.mark.slow
def test_tangent_full_size_equals_adjoint(L):
    """The bench's forward-mode arm (2^20 x 512) against the adjoint on the same paths."""
    w = inputs.heston_config()
    ctx = L.Context(w.problem, max_paths=w.n_paths)
    Ga, ga, Ea = [t.cpu().numpy() for t in ctx.value_and_grad(w.theta, w.C, w.problem.seed, w.n_paths)]
    Gt, gt, Et = [t.cpu().numpy() for t in ctx.value_and_grad_tangent(w.theta, w.C, w.problem.seed, w.n_paths)]
    assert rel(Et, Ea) <= 1e-6
    assert rel(gt, ga) <= 1e-4
