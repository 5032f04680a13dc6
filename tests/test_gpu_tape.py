"""Expected-backward AD on the GPU (include/mctape.h) against the oracle.

The oracle's whole-program tape (oracle/tape.py, the Appendix's rule in FP64
numpy) differentiates the same program on the same normals; for the Heston
calibration objective the two-step algorithm (the oracle's C path, and the
GPU's mc_value_and_grad) gives the same G and gradient (the gradient identity)."""
from dataclasses import replace

import numpy as np
import pytest

from paper_1901_04200_gb300 import inputs

import tape_programs as TP

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_04200_gb300 import build as b
    b.build()
    from paper_1901_04200_gb300 import tape
    return tape


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("seed,P", [(1, 1000), (2, 33), (3, 4096), (4, 1)])
def test_random_programs_match_oracle_tape(T, orc, seed, P):
    ops, obj = TP.random_program(seed)
    theta = np.random.default_rng(100 + seed).uniform(0.2, 0.8, 4)
    phil = 0x190104200 + seed
    Z = orc.normals_fill(phil, 0, P, 6)
    G_o, g_o, vals = TP.run_oracle(ops, obj, theta, Z)
    prog, nodes = TP.build_product(ops, T)
    ctx = T.TapeContext(prog, nodes[obj], 4, max_paths=P)
    G, g = ctx.value_and_grad(theta, phil, P)
    assert abs(G.item() - G_o) <= 1e-12 * max(abs(G_o), 1.0)
    assert rel(g.cpu().numpy(), g_o) <= 1e-10
    # per-path values of nodes always kept on the tape: expectation arguments and arguments of
    # products (other per-path nodes may live only in the shared-memory window)
    kept = {a for op, a, b, _ in ops if op == "expect"} | {x for op, a, b, _ in ops if op == "mul" for x in (a, b)}
    checked = 0
    for k in sorted(kept):
        if not _is_det(ops, k):
            assert rel(ctx.path_values(nodes[k]).cpu().numpy(), vals[k].v) <= 1e-12, k
            checked += 1
    assert checked >= 6


def _is_det(ops, k):
    op, a, b, _ = ops[k]
    if op in ("param", "const", "expect"):
        return True
    if op == "normal":
        return False
    return all(_is_det(ops, x) for x in (a, b) if x >= 0)


def test_path_offset_and_partition(T, orc):
    """Paths [path0, path0 + n): the normals follow the global path index."""
    ops, obj = TP.random_program(7)
    theta = np.full(4, 0.5)
    Z = orc.normals_fill(99, 5000, 700, 6)
    G_o, g_o, _ = TP.run_oracle(ops, obj, theta, Z)
    prog, nodes = TP.build_product(ops, T)
    ctx = T.TapeContext(prog, nodes[obj], 4, max_paths=1000)
    G, g = ctx.value_and_grad(theta, 99, 700, path0=5000)
    assert abs(G.item() - G_o) <= 1e-12 * max(abs(G_o), 1.0)
    assert rel(g.cpu().numpy(), g_o) <= 1e-10


def test_expectation_inside_paths_control_variate(T, orc):
    """G = E[(y - E y)^2] with y = theta0 exp(theta1 z): the expectation feeds every path."""
    P = 2048
    ops = [("param", -1, -1, 0), ("param", -1, -1, 1), ("normal", -1, -1, 0)]
    ops += [("mul", 1, 2, 0.0), ("exp", 3, -1, 0.0), ("mul", 0, 4, 0.0), ("expect", 5, -1, 0.0),
            ("sub", 5, 6, 0.0), ("mul", 7, 7, 0.0), ("expect", 8, -1, 0.0)]
    theta = np.array([1.3, 0.4])
    Z = orc.normals_fill(11, 0, P, 1)
    G_o, g_o, _ = TP.run_oracle(ops, 9, theta, Z)
    prog, nodes = TP.build_product(ops, T)
    ctx = T.TapeContext(prog, nodes[9], 2, max_paths=P)
    G, g = ctx.value_and_grad(theta, 11, P)
    assert abs(G.item() - G_o) <= 1e-12 * abs(G_o)
    assert rel(g.cpu().numpy(), g_o) <= 1e-10
    # closed form of the sample variance's gradient on these paths
    z = Z[:, 0]
    y = theta[0] * np.exp(theta[1] * z)
    dy0, dy1 = np.exp(theta[1] * z), y * z
    c = y - y.mean()
    assert rel(g.cpu().numpy(), [2 * np.mean(c * (dy0 - dy0.mean())), 2 * np.mean(c * (dy1 - dy1.mean()))]) <= 1e-10


@pytest.mark.parametrize("n_paths", [1000, 4096])
def test_heston_objective_equals_two_step(T, orc, n_paths):
    """The whole-program tape of G and the two-step algorithm agree (gradient identity)."""
    w = inputs.heston_config(n_paths=n_paths, steps_per_year=16, T=1.0, n_mat=4, n_strike=3)
    pb = replace(w.problem, precision="fp64", ckpt_every=4)  # maturities at steps 4, 8, 12, 16
    prog, G = T.heston_objective(pb, w.C)
    ctx = T.TapeContext(prog, G, 5, max_paths=n_paths)
    Gt, gt = ctx.value_and_grad(w.theta, pb.seed, n_paths)
    _, Go, go = orc.value_and_grad(pb, w.theta, w.C, n_paths)
    assert abs(Gt.item() - Go) <= 1e-10 * abs(Go)
    assert rel(gt.cpu().numpy(), go) <= 1e-9
    from paper_1901_04200_gb300 import _lib
    c2 = _lib.Context(pb, max_paths=n_paths)
    G2, g2, _ = c2.value_and_grad(w.theta, w.C, pb.seed, n_paths)
    assert abs(Gt.item() - G2.item()) <= 1e-10 * abs(G2.item())
    assert rel(gt.cpu().numpy(), g2.cpu().numpy()) <= 1e-9


def test_deterministic_repeat(T):
    ops, obj = TP.random_program(5)
    prog, nodes = TP.build_product(ops, T)
    ctx = T.TapeContext(prog, nodes[obj], 4, max_paths=5000)
    a = [x.cpu().numpy().copy() for x in ctx.value_and_grad(np.full(4, 0.4), 3, 5000)]
    b = [x.cpu().numpy().copy() for x in ctx.value_and_grad(np.full(4, 0.4), 3, 5000)]
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("mode", ["interpret", "compiled", "compiled_recompute"])
def test_reused_context_fewer_paths(T, orc, mode):
    """A context evaluated again with fewer paths, another seed and other parameters gives a
    fresh context's result and the oracle's: before each backward sweep every adjoint row that
    accumulates in HBM is cleared for the evaluated paths."""
    ops, obj = TP.random_program(3)
    prog, nodes = TP.build_product(ops, T)

    def make():
        c = T.TapeContext(prog, nodes[obj], 4, max_paths=3000)
        if mode != "interpret":
            c.compile(seg_nodes=7, recompute=(mode == "compiled_recompute"))
        return c

    used = make()
    used.value_and_grad(np.full(4, 0.7), 0x1234, 3000)
    theta = np.random.default_rng(7).uniform(0.2, 0.8, 4)
    G1, g1 = used.value_and_grad(theta, 0x5678, 1234)
    G2, g2 = make().value_and_grad(theta, 0x5678, 1234)
    assert G1.item() == G2.item() and np.array_equal(g1.cpu().numpy(), g2.cpu().numpy())
    Z = orc.normals_fill(0x5678, 0, 1234, 6)
    G_o, g_o, _ = TP.run_oracle(ops, obj, theta, Z)
    assert abs(G1.item() - G_o) <= 1e-12 * max(abs(G_o), 1.0)
    assert rel(g1.cpu().numpy(), g_o) <= 1e-10


def test_call_errors(T):
    from paper_1901_04200_gb300 import _lib
    ops, obj = TP.random_program(6)
    prog, nodes = TP.build_product(ops, T)
    ctx = T.TapeContext(prog, nodes[obj], 4, max_paths=64)
    with pytest.raises(_lib.McError):
        ctx.value_and_grad(np.full(4, 0.4), 3, 65)
    ctx.value_and_grad(np.full(4, 0.4), 3, 64)
    with pytest.raises(_lib.McError):
        ctx.path_values(nodes[obj])
    # a per-path node read only by the next node, through an addition, is not kept
    p2 = T.Program()
    z = p2.normal(0)
    u = z + 1.0
    G = T.expect(u * u)
    c2 = T.TapeContext(p2, G, 0, max_paths=64)
    c2.value_and_grad(np.zeros(1), 3, 64)
    with pytest.raises(_lib.McError) as e:
        c2.path_values(z)
    assert e.value.status == _lib.MC_ERR_UNSUPPORTED
    from oracle import normals_fill
    assert np.allclose(c2.path_values(u).cpu().numpy(), normals_fill(3, 0, 64, 1)[:, 0] + 1.0, rtol=0, atol=1e-14)


# ---------------------------------------------------------------- FP32 tape

@pytest.mark.parametrize("seed", [1, 3])
def test_random_programs_fp32(T, orc, seed):
    """FP32 per-path values and adjoints, FP64 sums: within FP32 rounding of the FP64 oracle."""
    P = 3000
    ops, obj = TP.random_program(seed)
    theta = np.random.default_rng(100 + seed).uniform(0.2, 0.8, 4)
    phil = 0x190104200 + seed
    Z = orc.normals_fill(phil, 0, P, 6)
    G_o, g_o, _ = TP.run_oracle(ops, obj, theta, Z)
    prog, nodes = TP.build_product(ops, T)
    ctx = T.TapeContext(prog, nodes[obj], 4, max_paths=P, precision="fp32")
    G, g = ctx.value_and_grad(theta, phil, P)
    assert abs(G.item() - G_o) <= 1e-5 * max(abs(G_o), 1.0)
    assert rel(g.cpu().numpy(), g_o) <= 1e-4


def test_heston_objective_fp32_equals_two_step_fp32(T):
    """The FP32 tape of the Heston objective and the FP32 two-step kernels (same FP32 normals)."""
    w = inputs.heston_config(n_paths=1 << 14, steps_per_year=64, T=2.0)
    pb = w.problem
    prog, G = T.heston_objective(pb, w.C)
    ctx = T.TapeContext(prog, G, 5, max_paths=w.n_paths, precision="fp32")
    Gt, gt = ctx.value_and_grad(w.theta, pb.seed, w.n_paths)
    from paper_1901_04200_gb300 import _lib
    c2 = _lib.Context(pb, max_paths=w.n_paths)
    G2, g2, _ = c2.value_and_grad(w.theta, w.C, pb.seed, w.n_paths)
    assert abs(Gt.item() - G2.item()) <= 1e-5 * abs(G2.item())
    assert rel(gt.cpu().numpy(), g2.cpu().numpy()) <= 1e-4


@pytest.mark.slow
def test_heston_tape_bench_size_equals_two_step(T):
    """The bench's tape run (2^18 paths x 512 steps, FP32) against the FP32 two-step kernels."""
    w = inputs.heston_config(n_paths=1 << 18)
    prog, G = T.heston_objective(w.problem, w.C)
    ctx = T.TapeContext(prog, G, 5, max_paths=w.n_paths, precision="fp32")
    Gt, gt = ctx.value_and_grad(w.theta, w.problem.seed, w.n_paths)
    from paper_1901_04200_gb300 import _lib
    c2 = _lib.Context(w.problem, max_paths=w.n_paths)
    G2, g2, _ = c2.value_and_grad(w.theta, w.C, w.problem.seed, w.n_paths)
    assert abs(Gt.item() - G2.item()) <= 1e-5 * abs(G2.item())
    assert rel(gt.cpu().numpy(), g2.cpu().numpy()) <= 1e-4


# ------------------------------------------------------ compiled programs

@pytest.mark.parametrize("recompute,piece", [(False, 0), (True, 0), (True, 3), (True, 16)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("seed,seg", [(1, 40), (3, 7), (4, 1000)])
def test_compiled_equals_interpreter_and_oracle(T, orc, seed, seg, precision, tol, recompute, piece):
    """mc_tape_compile: straight-line segment kernels give the interpreter's results (to the
    rounding of reordered sums) and the oracle's."""
    P = 3000
    ops, obj = TP.random_program(seed)
    theta = np.random.default_rng(100 + seed).uniform(0.2, 0.8, 4)
    phil = 0x190104200 + seed
    prog, nodes = TP.build_product(ops, T)
    a = T.TapeContext(prog, nodes[obj], 4, max_paths=P, precision=precision)
    Ga, ga = a.value_and_grad(theta, phil, P)
    b = T.TapeContext(prog, nodes[obj], 4, max_paths=P, precision=precision)
    sec, hb = b.compile(seg_nodes=seg, recompute=recompute, piece=piece)
    assert sec > 0 and hb > 0
    Gb, gb = b.value_and_grad(theta, phil, P)
    assert abs(Gb.item() - Ga.item()) <= tol * max(abs(Ga.item()), 1.0)
    assert rel(gb.cpu().numpy(), ga.cpu().numpy()) <= 10 * tol
    if precision == "fp64":
        Z = orc.normals_fill(phil, 0, P, 6)
        G_o, g_o, vals = TP.run_oracle(ops, obj, theta, Z)
        assert abs(Gb.item() - G_o) <= 1e-12 * max(abs(G_o), 1.0)
        assert rel(gb.cpu().numpy(), g_o) <= 1e-10
        for k in sorted({x for op, x, _, _ in ops if op == "expect"}):
            if not _is_det(ops, k):
                assert rel(b.path_values(nodes[k]).cpu().numpy(), vals[k].v) <= 1e-12


@pytest.mark.parametrize("piece", [0, 16])
def test_compiled_heston_objective_equals_two_step(T, orc, piece):
    w = inputs.heston_config(n_paths=2000, steps_per_year=16, T=1.0, n_mat=4, n_strike=3)
    pb = replace(w.problem, precision="fp64", ckpt_every=4)
    prog, G = T.heston_objective(pb, w.C)
    ctx = T.TapeContext(prog, G, 5, max_paths=2000)
    ctx.compile(seg_nodes=64, recompute=True, piece=piece)
    Gt, gt = ctx.value_and_grad(w.theta, pb.seed, 2000, path0=77)
    _, Go, go = orc.value_and_grad(pb, w.theta, w.C, 2000, path0=77)
    assert abs(Gt.item() - Go) <= 1e-10 * abs(Go)
    assert rel(gt.cpu().numpy(), go) <= 1e-9
