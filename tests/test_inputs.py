"""The synthetic workloads follow their stated recipe: time grids, instrument sets,
parameter boxes, surfaces and sizes (no GPU)."""
import numpy as np

from paper_1901_04200_gb300 import inputs


def _by_maturity(pb):
    steps = sorted(set(np.asarray(pb.mat_step).tolist()))
    return steps, [np.asarray(pb.K)[np.asarray(pb.mat_step) == s] for s in steps]


def test_gbm_workload():
    w = inputs.gbm_config()
    pb = w.problem
    assert pb.kind == "gbm" and pb.n_steps == 16 and pb.dt == 0.125 and pb.precision == "fp64"
    assert np.array_equal(pb.bucket_end, np.arange(2, 17, 2))
    assert np.array_equal(pb.mat_step, pb.bucket_end)
    assert np.allclose(pb.K, np.linspace(80.0, 120.0, 8))
    assert pb.normals.shape == (4096, 16) and np.all(w.theta == 0.25)
    ref = np.random.default_rng(inputs.SEED_NORMALS).standard_normal((4096, 16))
    assert np.array_equal(pb.normals, ref)


def test_heston_bench_workload():
    w = inputs.heston_config()
    pb = w.problem
    assert w.n_paths == 1 << 20 and pb.kind == "heston" and pb.precision == "fp32"
    assert pb.n_steps == 512 and pb.dt == 1.0 / 256 and pb.ckpt_every == 8 and pb.storage == "auto"
    assert pb.m == 64 and pb.S0 == 100.0 and pb.r == 0.02 and pb.seed == inputs.PHILOX_SEED
    steps, strikes = _by_maturity(pb)
    assert steps == [64 * k for k in range(1, 9)]  # 0.25 .. 2 years
    for k in strikes:
        assert np.allclose(np.sort(k), np.linspace(70.0, 130.0, 8))
    th = w.theta
    lo, hi = inputs.HESTON_RANGES["lo"], inputs.HESTON_RANGES["hi"]
    assert th.shape == (5,) and np.all(th >= lo) and np.all(th <= hi)
    assert 2.0 * th[0] * th[1] > th[2] ** 2  # Feller
    assert len(w.C) == 64 and np.all(np.asarray(w.C) > 0)


def test_local_vol_workload():
    w = inputs.lv_config()
    pb = w.problem
    assert w.n_paths == 1 << 22 and pb.kind == "lv" and pb.n_steps == 500 and abs(pb.dt - 0.01) < 1e-15
    assert (pb.nt, pb.nx, pb.x_lo, pb.x_hi, pb.t_max) == (20, 10, -1.0, 1.0, 5.0)
    assert pb.ckpt_every == 5 and pb.paths_per_thread == 4 and pb.m == 200
    steps, strikes = _by_maturity(pb)
    assert steps == [25 * k for k in range(1, 21)]
    for k in strikes:
        assert np.allclose(np.sort(k), np.linspace(60.0, 150.0, 10))
    assert w.theta.shape == (200,) and np.all((w.theta >= 0.1) & (w.theta <= 0.4))


def test_slv_workload():
    w = inputs.slv_config()
    pb, h = w.problem, inputs.heston_config()
    assert pb.kind == "slv" and (pb.nt, pb.nx) == (9, 10) and pb.n_params == 95
    assert np.array_equal(w.theta[:5], h.theta) and np.array_equal(pb.mat_step, h.problem.mat_step)
    lev = w.theta[5:]
    assert lev.shape == (90,) and np.all((lev >= 0.8) & (lev <= 1.2))


def test_heston_draws_stay_in_the_box():
    rng = np.random.default_rng(5)
    lo, hi = inputs.HESTON_RANGES["lo"], inputs.HESTON_RANGES["hi"]
    for _ in range(200):
        th = inputs.draw_heston_theta(rng)
        assert np.all(th >= lo) and np.all(th <= hi) and 2.0 * th[0] * th[1] > th[2] ** 2
