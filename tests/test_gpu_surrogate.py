"""What the trained surrogate gains: calibration to G < 1e-8 with fewer MC-AAD
evaluations than plain MC-AAD descent from the same starts (the MC-AAD phase
stays the judge: every accepted point is an MC-AAD evaluation)."""
import numpy as np
import pytest

from paper_1901_04200_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def trained():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_04200_gb300 import build as b
    b.build()
    from paper_1901_04200_gb300 import surrogate
    pb = inputs.heston_config().problem
    X, y, dy = surrogate.make_dataset(pb, 16384, 1 << 15, seed=31)
    Xv, yv, dyv = surrogate.make_dataset(pb, 256, 1 << 15, seed=32)
    sur = surrogate.Surrogate(batch=4096, seed=1)
    loss0 = sur.evaluate_loss(Xv, yv, dyv)
    sur.train(X, y, dy, epochs=30, lr=2e-3)
    return pb, sur, loss0, sur.evaluate_loss(Xv, yv, dyv)


def test_training_reduces_held_out_loss(trained):
    _, _, loss0, loss1 = trained
    assert loss1 < 1e-2 * loss0


def test_surrogate_assisted_calibration_beats_plain(trained):
    from paper_1901_04200_gb300 import _lib, calibrate
    pb, sur, _, _ = trained
    P, seed = 1 << 21, 777
    ctx = _lib.Context(pb, max_paths=P)
    plain_evals, sur_evals, sur_conv = [], [], []
    for sd in range(4):
        rng = np.random.default_rng(1000 + sd)
        theta_star, theta0 = inputs.draw_heston_theta(rng), inputs.draw_heston_theta(rng)
        C = ctx.forward(theta_star, seed, P).cpu().numpy()
        r = calibrate.run_experiment(ctx, sur, theta0, C, seed, P, tol=1e-8, max_evals=200)
        plain_evals.append(r["plain"].evals if r["plain"].converged else 200)
        sur_evals.append(r["mc_phase"].evals)
        sur_conv.append(r["mc_phase"].converged)
        if r["mc_phase"].converged:
            assert r["mc_phase"].G < 1e-8
    assert sum(sur_conv) >= 3
    assert np.median(sur_evals) < np.median(plain_evals)


def test_gpu_calibration_matches_oracle_calibration(orc):
    """Gauss-Newton-metric descent on the FP64 CUDA path (Jacobian from the
    forward-mode kernel) and on the oracle (Jacobian from unit-seed vjps), from
    a start near theta*, both recover theta* under common random numbers (the
    landscape has boundary local minima far from theta*)."""
    from dataclasses import replace
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_04200_gb300 import _lib, calibrate
    from paper_1901_04200_gb300 import build as b
    b.build()
    w = inputs.heston_config(n_paths=2048, steps_per_year=32, T=1.0, n_mat=4, n_strike=4)
    n, seed = 2048, 99
    pb = replace(w.problem, precision="fp64", seed=seed)
    rng = np.random.default_rng(5)
    theta_star = inputs.draw_heston_theta(rng)
    lo, hi = inputs.HESTON_RANGES["lo"], inputs.HESTON_RANGES["hi"]
    theta0 = np.clip(theta_star + 0.05 * (hi - lo) * rng.choice([-1.0, 1.0], 5), lo, hi)
    C = orc.forward(pb, theta_star, n, n_threads=4)
    ctx = _lib.Context(pb, max_paths=n)
    jac_gpu = lambda th: ctx.price_jacobian(np.asarray(th)[None, :], seed, n)[1][0].cpu().numpy()
    r_gpu = calibrate.descend_metric(calibrate.mc_objective(ctx, C, seed, n), jac_gpu, theta0, lo, hi, 1e-12,
                                     max_evals=80)
    eye = np.eye(pb.m)

    def of(th):
        _, G, g = orc.value_and_grad(pb, th, C, n, n_threads=4)
        return G, g
    jac_cpu = lambda th: np.stack([orc.vjp(pb, th, eye[i], n, n_threads=4) for i in range(pb.m)])
    r_cpu = calibrate.descend_metric(of, jac_cpu, theta0, lo, hi, 1e-12, max_evals=80)
    assert r_gpu.converged and r_cpu.converged
    assert np.max(np.abs(r_gpu.theta - theta_star) / (hi - lo)) < 1e-4
    assert np.max(np.abs(r_cpu.theta - theta_star) / (hi - lo)) < 1e-4
