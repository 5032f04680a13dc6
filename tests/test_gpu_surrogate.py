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
