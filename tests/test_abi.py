"""The C ABI without a GPU: the library loads, exports every declared entry
point, and rejects invalid problems on the host before touching the device."""
import ctypes
import os
import re
from dataclasses import replace

import numpy as np
import pytest

from paper_1901_04200_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1901_04200_gb300 import build as b
    b.build()
    from paper_1901_04200_gb300 import _lib
    return _lib.load()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*((?:mc|mlp)_[a-z0-9_]+)\s*\(",
                                src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_symbol():
    from paper_1901_04200_gb300 import _lib
    assert sorted(s[0] for s in _lib.SIGNATURES) == declared_functions()


def _ws(lib, pb, max_paths=1024):
    from paper_1901_04200_gb300 import _lib
    c = _lib._ProblemC(pb, device=None) if pb.normals is None else None
    n = ctypes.c_size_t(0)
    return lib.mc_workspace_size(ctypes.byref(c.model), ctypes.byref(c.inst), max_paths, 0, ctypes.byref(n))


@pytest.mark.parametrize("mutate", [
    lambda p: replace(p, mat_step=p.mat_step + 100000),           # maturity beyond the grid
    lambda p: replace(p, mat_step=np.zeros_like(p.mat_step)),     # maturity at step 0
    lambda p: replace(p, dt=0.0),
    lambda p: replace(p, S0=-1.0),
    lambda p: replace(p, ckpt_every=3),                            # does not divide the maturities
    lambda p: replace(p, K=np.full(p.m, np.nan)),
])
def test_invalid_problems_rejected_on_host(lib, mutate):
    from paper_1901_04200_gb300 import _lib
    pb = mutate(inputs.heston_config(n_paths=64, steps_per_year=16, T=1.0, n_mat=2, n_strike=2).problem)
    assert _ws(lib, pb) == _lib.MC_ERR_INVALID_ARG


def test_lv_and_gbm_rejections(lib):
    from paper_1901_04200_gb300 import _lib
    lv = inputs.lv_config(n_paths=64, n_steps=50, T=1.0, nt=3, nx=4, n_mat=2, n_strike=2).problem
    assert _ws(lib, replace(lv, nx=1)) == _lib.MC_ERR_INVALID_ARG
    assert _ws(lib, replace(lv, x_hi=lv.x_lo)) == _lib.MC_ERR_INVALID_ARG
    g = replace(inputs.gbm_config(n_paths=16).problem, normals=None)
    assert _ws(lib, replace(g, bucket_end=g.bucket_end[::-1].copy())) == _lib.MC_ERR_INVALID_ARG
    assert _ws(lib, replace(g, bucket_end=g.bucket_end[:2].copy())) == _lib.MC_ERR_INVALID_ARG


def test_unsupported_segment_length(lib):
    from paper_1901_04200_gb300 import _lib
    pb = inputs.heston_config(n_paths=64, steps_per_year=64, T=1.0, n_mat=2, n_strike=2).problem
    assert _ws(lib, replace(pb, ckpt_every=32)) == _lib.MC_ERR_UNSUPPORTED


def test_fill_hooks_reject_bad_arguments(lib):
    from paper_1901_04200_gb300 import _lib
    assert lib.mc_philox_fill(1, 0, 0, 4, None, None) == _lib.MC_ERR_INVALID_ARG
    assert lib.mc_normals_fill(1, 0, 4, 4, 7, ctypes.c_void_p(256), None) == _lib.MC_ERR_INVALID_ARG


def test_unbuilt_paths_per_thread_is_unsupported(lib):
    """paths_per_thread up to 4 is accepted by the ABI; a combination without kernels is refused."""
    from paper_1901_04200_gb300 import _lib
    pb = inputs.heston_config(n_paths=64, steps_per_year=16, T=1.0, n_mat=2, n_strike=2).problem
    assert _ws(lib, replace(pb, paths_per_thread=4, ckpt_every=4)) == _lib.MC_ERR_UNSUPPORTED
    assert _ws(lib, replace(pb, paths_per_thread=5)) == _lib.MC_ERR_INVALID_ARG
