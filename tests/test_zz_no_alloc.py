"""mc_forward_static: E y through the C ABI with no device allocation.

It serves callers that cannot call cudaMalloc (a process whose device memory
belongs to another allocator's pool, or a loop that must not pay cudaMalloc's
implicit device synchronisation): its scratch is a fixed device array in the
library.  This file is collected last so that a run stopping at the first
failure has already run every other test.  The check: two calls in a row
give the same E y as mc_forward (the context entry point) on the same inputs.
"""
import ctypes

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
    _lib.load()
    return _lib


def _static_forward(L, pc, theta, seed, path0, n_paths, m):
    Ey = torch.empty(m, dtype=torch.float64, device="cuda")
    st = L.load().mc_forward_static(ctypes.byref(pc.model), ctypes.byref(pc.inst),
                                    ctypes.c_void_p(theta.data_ptr()), seed, path0, n_paths,
                                    ctypes.c_void_p(Ey.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == L.MC_OK
    return Ey


@pytest.mark.parametrize("kind", ["heston", "lv"])
def test_static_forward_matches_context_forward_twice(L, kind):
    if kind == "heston":
        w = inputs.heston_config(n_paths=50000, steps_per_year=64, T=2.0)
    else:
        w = inputs.lv_config(n_paths=20000)
    pb, n = w.problem, w.n_paths
    ctx = L.Context(pb, max_paths=n)
    pc = L._ProblemC(pb, torch.device("cuda"))
    for call, (theta, seed, path0) in enumerate([(w.theta, 17, 0), (w.theta * 1.01, 18, 123)]):
        th = torch.tensor(theta, dtype=torch.float64, device="cuda")
        ref = ctx.forward(th, seed, n, path0=path0)
        got = _static_forward(L, pc, th, seed, path0, n, pb.m)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.max(np.abs(g - r)) <= 1e-12 * np.max(np.abs(r)), (call, np.max(np.abs(g - r)))


def test_static_forward_rejects_oversized_problem(L):
    """A local-vol grid whose tables exceed shared memory (checked before the fixed scratch, which
    holds the same tables) is refused as unsupported."""
    lv = inputs.lv_config(n_paths=64, n_steps=100000, T=100.0, nt=20, nx=10, n_mat=1, n_strike=1)
    pl = L._ProblemC(lv.problem, torch.device("cuda"))
    thl = torch.tensor(lv.theta, dtype=torch.float64, device="cuda")
    Ey = torch.empty(1, dtype=torch.float64, device="cuda")
    st = L.load().mc_forward_static(ctypes.byref(pl.model), ctypes.byref(pl.inst),
                                    ctypes.c_void_p(thl.data_ptr()), 1, 0, 64, ctypes.c_void_p(Ey.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == L.MC_ERR_UNSUPPORTED


def test_static_forward_rejects_wrapping_path_range(L):
    """path0 + n_paths beyond 2^64 is refused before any launch (with a normals table the wrapped
    range would otherwise pass the table's bounds check)."""
    w = inputs.gbm_config(n_paths=256)
    pc = L._ProblemC(w.problem, torch.device("cuda"))
    th = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
    Ey = torch.empty(w.problem.m, dtype=torch.float64, device="cuda")
    st = L.load().mc_forward_static(ctypes.byref(pc.model), ctypes.byref(pc.inst), ctypes.c_void_p(th.data_ptr()),
                                    1, (1 << 64) - 4, 16, ctypes.c_void_p(Ey.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == L.MC_ERR_INVALID_ARG
