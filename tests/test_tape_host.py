"""Expected-backward tape: host planning through the C ABI (no GPU) and the
oracle tape's log pin."""
import math

import numpy as np
import pytest

from paper_1901_04200_gb300 import _lib, inputs
from paper_1901_04200_gb300 import tape


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1901_04200_gb300 import build
    build.build()


def test_heston_program_has_two_stages():
    w = inputs.heston_config(n_paths=64, steps_per_year=8, T=1.0, n_mat=2, n_strike=2)
    prog, G = tape.heston_objective(w.problem, w.C)
    st, ns, nrows, ws, hb = tape.plan(prog, G, 5, 1000)
    assert st == _lib.MC_OK and ns == 2
    assert 0 < nrows < len(prog.nodes) and ws >= 2 * nrows * 1024 * 8
    # the shared-memory window keeps most values and adjoints out of HBM
    assert 0 < hb < 3 * 8 * nrows


def test_stages_follow_expectation_use():
    p = tape.Program()
    th, z = p.param(0), p.normal(0)
    y = th * z
    e1 = tape.expect(y)                 # stage 0
    y2 = (y - e1) * (y - e1)            # needs e1: stage 1
    e2 = tape.expect(y2)                # end of stage 1
    y3 = tape.exp(z * 0.1) + e2         # stage 2
    G = tape.expect(y3) * 2.0           # deterministic, after E(y3): stage 3
    assert tape.plan(p, G, 1)[1] == 4
    q = tape.Program()                  # every node is evaluated, so a separate program:
    th, z = q.param(0), q.normal(0)
    e1 = tape.expect(th * z)
    H = e1 * e1 + th                    # deterministic, after E(th z): stage 1
    assert tape.plan(q, H, 1)[1] == 2


@pytest.mark.parametrize("bad", ["forward_ref", "self_ref", "path_objective", "param_range", "unknown_op",
                                 "extra_arg"])
def test_invalid_programs_rejected(bad):
    p = tape.Program()
    th, z = p.param(0), p.normal(0)
    y = th * z
    G = tape.expect(y)
    obj, n_params = G, 1
    if bad == "forward_ref":
        p.nodes.append((tape.OPS["add"], 0, len(p.nodes) + 3, 0.0))
    elif bad == "self_ref":
        p.nodes.append((tape.OPS["neg"], len(p.nodes), -1, 0.0))
    elif bad == "path_objective":
        obj = y
    elif bad == "param_range":
        n_params = 0
    elif bad == "unknown_op":
        p.nodes.append((99, -1, -1, 0.0))
    elif bad == "extra_arg":
        p.nodes.append((tape.OPS["const"], 0, -1, 1.0))
    assert tape.plan(p, obj, n_params)[0] == _lib.MC_ERR_INVALID_ARG


def test_builder_encodes_scalars_exactly():
    p = tape.Program()
    a = p.param(0)
    b = 2.0 - a
    c = a / 4.0
    d = 3.0 * a
    assert p.nodes[b.i][0] == tape.OPS["addc"] and p.nodes[b.i][3] == 2.0
    assert p.nodes[p.nodes[b.i][1]][0] == tape.OPS["neg"]
    assert p.nodes[c.i][0] == tape.OPS["div"] and p.nodes[p.nodes[c.i][2]][3] == 4.0
    assert p.nodes[d.i][0] == tape.OPS["mulc"] and p.nodes[d.i][3] == 3.0


def test_oracle_tape_log_by_finite_differences():
    """d/dtheta E[log(theta + z^2)] of the oracle's tape against central differences."""
    from oracle import tape as T
    z = np.random.default_rng(3).standard_normal(257)

    def value(theta):
        tp = T.Tape(len(z))
        th = tp.input(theta)
        out = T.expectation(T.log(th + tp.const(z * z)))
        return out, tp, th

    out, tp, th = value(0.8)
    D = tp.backward(out)
    g = np.mean(D[th.idx])
    h = 1e-6
    fd = (value(0.8 + h)[0].v[0] - value(0.8 - h)[0].v[0]) / (2 * h)
    assert math.isclose(g, fd, rel_tol=1e-8)
    assert math.isclose(g, np.mean(1.0 / (0.8 + z * z)), rel_tol=1e-14)


def test_oracle_tape_product_of_expectations():
    """G = E[Y E[X]] with X = theta a, Y = theta b: G = theta^2 mean(a) mean(b), so dG/dtheta =
    2 theta mean(a) mean(b).  The adjoint reaching E[X] differs from path to path (Y), so the
    expectation's rule must take its mean over the paths."""
    from oracle import tape as T
    rng = np.random.default_rng(11)
    a, b = rng.standard_normal(301), rng.uniform(0.5, 1.5, 301)
    tp = T.Tape(len(a))
    th = tp.input(0.7)
    ex = T.expectation(th * tp.const(a))
    out = T.expectation((th * tp.const(b)) * ex)
    D = tp.backward(out)
    g = np.mean(D[th.idx])
    assert math.isclose(out.v[0], 0.7 * 0.7 * np.mean(a) * np.mean(b), rel_tol=1e-12)
    assert math.isclose(g, 2 * 0.7 * np.mean(a) * np.mean(b), rel_tol=1e-12)


def test_stage_limits():
    """More than 2048 expectations in one stage is refused as unsupported, 2048 is accepted."""
    for n, want in [(2048, _lib.MC_OK), (2049, _lib.MC_ERR_UNSUPPORTED)]:
        p = tape.Program()
        z = p.normal(0)
        G = None
        for k in range(n):
            e = tape.expect(z * float(k + 1))
            G = e if G is None else G + e
        assert tape.plan(p, G, 0)[0] == want
