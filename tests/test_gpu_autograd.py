"""The autograd wrapper: G.backward() reproduces mc_value_and_grad, checked
against central finite differences with common random numbers."""
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


def test_backward_equals_value_and_grad(L):
    from paper_1901_04200_gb300.autograd import calibration_objective
    w = inputs.heston_config(n_paths=1 << 14, steps_per_year=64, T=1.0, n_mat=4, n_strike=4)
    mc = L.Context(w.problem, max_paths=1 << 14)
    C = torch.tensor(w.C, dtype=torch.float64, device="cuda")
    th = torch.tensor(w.theta, dtype=torch.float64, device="cuda", requires_grad=True)
    G = calibration_objective(mc, th, C, 11, 1 << 14)
    G.backward()
    G2, g2, _ = mc.value_and_grad(w.theta, w.C, 11, 1 << 14)
    # torch sums lambda^2 in its own order: G agrees to rounding; the seeds are identical
    assert abs(G.item() - G2.item()) <= 1e-14 * abs(G2.item())
    assert torch.allclose(th.grad, g2, rtol=1e-14, atol=0)


def test_backward_after_another_forward(L):
    from paper_1901_04200_gb300.autograd import mc_expect
    w = inputs.lv_config(n_paths=4096, n_steps=100, T=2.0, nt=5, nx=6, n_mat=4, n_strike=5)
    mc = L.Context(w.problem, max_paths=4096)
    th = torch.tensor(w.theta, dtype=torch.float64, device="cuda", requires_grad=True)
    Ey1 = mc_expect(mc, th, 3, 4096)
    _ = mc_expect(mc, th * 1.1, 4, 4096)  # overwrites the context's checkpoints
    Ey1.sum().backward()
    ref = mc.forward(w.theta, 3, 4096, keep=True)
    g_ref = mc.vjp(torch.ones(w.problem.m, dtype=torch.float64, device="cuda"))
    assert torch.equal(Ey1.detach(), ref)
    assert torch.equal(th.grad, g_ref)


@pytest.mark.parametrize("kind", ["heston", "lv", "gbm"])
def test_fd_common_random_numbers_fp64(L, kind):
    """Central differences of the GPU's own G (same seed) match its adjoint gradient."""
    if kind == "heston":
        w = inputs.heston_config(n_paths=1 << 13, steps_per_year=64, T=1.0, n_mat=4, n_strike=4)
        idx = range(5)
    elif kind == "lv":
        w = inputs.lv_config(n_paths=1 << 12, n_steps=100, T=2.0, nt=5, nx=6, n_mat=4, n_strike=5)
        idx = [0, 7, 8, 13, 14, 20]
    else:
        w = inputs.gbm_config()
        idx = range(8)
    pb = replace(w.problem, precision="fp64")
    n = w.n_paths
    mc = L.Context(pb, max_paths=n)
    G0, g, _ = mc.value_and_grad(w.theta, w.C, 5, n)
    g = g.cpu().numpy()
    for j in idx:
        h = 1e-6 * max(1.0, abs(w.theta[j]))
        tp, tm = w.theta.copy(), w.theta.copy()
        tp[j] += h
        tm[j] -= h
        Gp = mc.value_and_grad(tp, w.C, 5, n)[0].item()
        Gm = mc.value_and_grad(tm, w.C, 5, n)[0].item()
        fd = (Gp - Gm) / (2 * h)
        assert abs(fd - g[j]) <= 1e-5 * np.max(np.abs(g)) + 1e-9, (kind, j, fd, g[j])
