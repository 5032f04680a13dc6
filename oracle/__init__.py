"""FP64 CPU oracle for G = 1/2 sum_i (E y_i - C_i)^2 and grad G.

TEST INFRASTRUCTURE ONLY (arXiv 1901.04200, eq. 241118A and the two-step
algorithm).  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the CUDA
library: the C source here is compiled with gcc into ``liboracle.so`` and
called through ctypes.  A problem is any object with the attributes of
``paper_1901_04200_gb300.inputs.Problem`` (read by duck typing, so this package
imports nothing from the product).

Readings of the paper that this oracle fixes:
state x = ln(S/S0); call payoffs discounted with exp(-r T); payoff kink
derivative 1{S > K}; Heston full truncation with derivative 1{v > 0} of
max(v, 0); local volatility bilinear with flat extrapolation; normals from
Philox-4x32-10 + Box-Muller with the counter layout in ``mcaad_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcaad_oracle.c")
_HDR = os.path.join(_HERE, "mcaad_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

KIND = {"gbm": 0, "heston": 1, "lv": 2, "slv": 3}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE FP64: no fast-math, no FMA contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
               "-fno-fast-math", "-pthread", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("S0", ctypes.c_double), ("r", ctypes.c_double), ("dt", ctypes.c_double),
        ("n_steps", ctypes.c_int),
        ("n_buckets", ctypes.c_int),
        ("bucket_end", ctypes.POINTER(ctypes.c_int)),
        ("nt", ctypes.c_int), ("nx", ctypes.c_int),
        ("t_max", ctypes.c_double), ("x_lo", ctypes.c_double), ("x_hi", ctypes.c_double),
        ("m", ctypes.c_int),
        ("K", ctypes.POINTER(ctypes.c_double)),
        ("mat_step", ctypes.POINTER(ctypes.c_int)),
        ("normals", ctypes.POINTER(ctypes.c_double)),
        ("normals_path0", ctypes.c_uint64),
        ("seed", ctypes.c_uint64),
    ]


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d, i, u64, u32 = ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32
            P = ctypes.POINTER
            lib.orc_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
            lib.orc_philox_fill.argtypes = [u64, u64, u32, u32, P(ctypes.c_uint32)]
            lib.orc_uniform.argtypes = [u32]
            lib.orc_uniform.restype = d
            lib.orc_normal.argtypes = [u64, u64, u64]
            lib.orc_normal.restype = d
            lib.orc_normals_fill.argtypes = [u64, u64, u32, u32, P(d)]
            for fn in ("orc_state_dim", "orc_normals_per_step", "orc_n_params", "orc_last_step"):
                getattr(lib, fn).argtypes = [P(_Problem)]
                getattr(lib, fn).restype = i
            lib.orc_check.argtypes = [P(_Problem), P(d)]
            lib.orc_path_forward.argtypes = [P(_Problem), P(d), u64, P(d), P(d), P(d)]
            lib.orc_path_adjoint.argtypes = [P(_Problem), P(d), P(d), P(d), P(d), P(d)]
            lib.orc_forward.argtypes = [P(_Problem), P(d), u64, u64, i, P(d)]
            lib.orc_vjp.argtypes = [P(_Problem), P(d), P(d), u64, u64, i, P(d)]
            lib.orc_value_and_grad.argtypes = [P(_Problem), P(d), P(d), u64, u64, i, P(d), P(d), P(d)]
            lib.orc_states_at.argtypes = [P(_Problem), P(d), u64, u64, i, i, P(d)]
            _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


class _Bound:
    """A ctypes view of a problem; keeps the numpy buffers alive."""

    def __init__(self, pb):
        self.keep = []

        def arr(x, dt):
            a = np.ascontiguousarray(np.asarray(x, dtype=dt))
            self.keep.append(a)
            return a

        s = _Problem()
        s.kind = KIND[pb.kind]
        s.S0, s.r, s.dt = float(pb.S0), float(pb.r), float(pb.dt)
        s.n_steps = int(pb.n_steps)
        if pb.kind == "gbm":
            be = arr(pb.bucket_end, np.int32)
            s.n_buckets = len(be)
            s.bucket_end = _iptr(be)
        if pb.kind in ("lv", "slv"):
            s.nt, s.nx = int(pb.nt), int(pb.nx)
            s.t_max, s.x_lo, s.x_hi = float(pb.t_max), float(pb.x_lo), float(pb.x_hi)
        K = arr(pb.K, np.float64)
        ms = arr(pb.mat_step, np.int32)
        s.m = len(K)
        s.K = _dptr(K)
        s.mat_step = _iptr(ms)
        if getattr(pb, "normals", None) is not None:
            z = arr(pb.normals, np.float64)
            s.normals = _dptr(z)
            s.normals_path0 = int(getattr(pb, "normals_path0", 0))
        s.seed = int(pb.seed) & 0xFFFFFFFFFFFFFFFF
        self.s = s
        self.ref = ctypes.byref(s)


def _threads(n_threads):
    return int(n_threads) if n_threads else (os.cpu_count() or 1)


# ------------------------------------------------------------------ RNG

def philox4x32_10(ctr, key):
    """One Philox-4x32-10 block: ctr = 4 uint32 words, key = 2 uint32 words."""
    lib = _lib_handle()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def philox_fill(seed, path0, n_paths, n_calls):
    """uint32 [n_paths, n_calls, 4]: block (call c, path p) with counter (c, 0, p_lo, p_hi)."""
    lib = _lib_handle()
    out = np.zeros((n_paths, n_calls, 4), dtype=np.uint32)
    lib.orc_philox_fill(seed, path0, n_paths, n_calls,
                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return out


def uniform(w):
    return _lib_handle().orc_uniform(int(w) & 0xFFFFFFFF)


def normals_fill(seed, path0, n_paths, n_per_path):
    """FP64 normals [n_paths, n_per_path]; normal j of path p as in mcaad_oracle.c."""
    lib = _lib_handle()
    out = np.zeros((n_paths, n_per_path), dtype=np.float64)
    lib.orc_normals_fill(seed, path0, n_paths, n_per_path, _dptr(out))
    return out


# ---------------------------------------------------------------- paths

def n_params(pb):
    return _lib_handle().orc_n_params(_Bound(pb).ref)


def last_step(pb):
    return _lib_handle().orc_last_step(_Bound(pb).ref)


def check(pb, theta):
    b = _Bound(pb)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    return _lib_handle().orc_check(b.ref, _dptr(th)) == 0


def path_forward(pb, theta, p):
    """One path of F: returns (states [n_last+1, state_dim], z [n_last, dz], y [m])."""
    lib = _lib_handle()
    b = _Bound(pb)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    nl = lib.orc_last_step(b.ref)
    sd = lib.orc_state_dim(b.ref)
    dz = lib.orc_normals_per_step(b.ref)
    states = np.zeros((nl + 1, sd))
    z = np.zeros((max(nl, 1), dz))
    y = np.zeros(b.s.m)
    if lib.orc_path_forward(b.ref, _dptr(th), int(p), _dptr(states), _dptr(z), _dptr(y)):
        raise ValueError("oracle: invalid problem")
    return states, z[:nl], y


def path_adjoint(pb, theta, p, lam):
    """One path of R seeded with lam: g_j = sum_i lam_i dy_i/dtheta_j."""
    lib = _lib_handle()
    b = _Bound(pb)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    states, z, _ = path_forward(pb, theta, p)
    zz = np.ascontiguousarray(z if len(z) else np.zeros((1, 1)))
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    g = np.zeros(lib.orc_n_params(b.ref))
    lib.orc_path_adjoint(b.ref, _dptr(th), _dptr(states), _dptr(zz), _dptr(lam), _dptr(g))
    return g


def forward(pb, theta, n_paths, path0=0, n_threads=None):
    """E y over global paths [path0, path0+n_paths)."""
    lib = _lib_handle()
    b = _Bound(pb)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    Ey = np.zeros(b.s.m)
    if lib.orc_forward(b.ref, _dptr(th), path0, n_paths, _threads(n_threads), _dptr(Ey)):
        raise ValueError("oracle: invalid problem")
    return Ey


def vjp(pb, theta, ybar, n_paths, path0=0, n_threads=None):
    """sum_i ybar_i d(E y_i)/dtheta over global paths [path0, path0+n_paths)."""
    lib = _lib_handle()
    b = _Bound(pb)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    yb = np.ascontiguousarray(ybar, dtype=np.float64)
    out = np.zeros(lib.orc_n_params(b.ref))
    if lib.orc_vjp(b.ref, _dptr(th), _dptr(yb), path0, n_paths, _threads(n_threads), _dptr(out)):
        raise ValueError("oracle: invalid problem")
    return out


def value_and_grad(pb, theta, C, n_paths, path0=0, n_threads=None):
    """The two-step algorithm: returns (E y [m], G, grad G [M])."""
    lib = _lib_handle()
    b = _Bound(pb)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    Cc = np.ascontiguousarray(C, dtype=np.float64)
    Ey = np.zeros(b.s.m)
    G = ctypes.c_double(0.0)
    grad = np.zeros(lib.orc_n_params(b.ref))
    if lib.orc_value_and_grad(b.ref, _dptr(th), _dptr(Cc), path0, n_paths, _threads(n_threads),
                              _dptr(Ey), ctypes.byref(G), _dptr(grad)):
        raise ValueError("oracle: invalid problem")
    return Ey, G.value, grad


def states_at(pb, theta, step, n_paths, path0=0, n_threads=None):
    """State after `step` steps of each path: [n_paths, state_dim] (x, and v for Heston/SLV)."""
    lib = _lib_handle()
    b = _Bound(pb)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    out = np.zeros((n_paths, lib.orc_state_dim(b.ref)))
    if lib.orc_states_at(b.ref, _dptr(th), path0, n_paths, int(step), _threads(n_threads), _dptr(out)):
        raise ValueError("oracle: invalid problem")
    return out
