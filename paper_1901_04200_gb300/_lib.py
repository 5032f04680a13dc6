"""ctypes binding of libmcaad.so (include/mcaad.h), argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module
converts a ``Problem`` into the C structs, hands device pointers of torch
tensors and the current torch stream to the C entry points, and raises on a
non-zero ``mc_status``.  There is no CPU fallback: if the library is missing,
``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmcaad.so")

MC_OK, MC_ERR_INVALID_ARG, MC_ERR_CUDA, MC_ERR_OOM, MC_ERR_UNSUPPORTED, MC_ERR_STATE = range(6)
MC_FP64, MC_FP32 = 0, 1
KIND = {"gbm": 0, "heston": 1, "lv": 2, "slv": 3}
STORAGE = {"checkpoint": 0, "full": 1, "normals": 2, "auto": 3, "states": 4}  # mc_storage
_STATUS = {1: "MC_ERR_INVALID_ARG", 2: "MC_ERR_CUDA", 3: "MC_ERR_OOM", 4: "MC_ERR_UNSUPPORTED",
           5: "MC_ERR_STATE"}


class McError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class mc_model(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("S0", ctypes.c_double), ("r", ctypes.c_double), ("dt", ctypes.c_double),
        ("n_steps", ctypes.c_int32), ("ckpt_every", ctypes.c_int32),
        ("n_buckets", ctypes.c_int32), ("bucket_end_host", ctypes.POINTER(ctypes.c_int32)),
        ("nt", ctypes.c_int32), ("nx", ctypes.c_int32),
        ("t_max", ctypes.c_double), ("x_lo", ctypes.c_double), ("x_hi", ctypes.c_double),
        ("normals", ctypes.c_void_p), ("normals_path0", ctypes.c_uint64),
        ("normals_rows", ctypes.c_uint64), ("paths_per_thread", ctypes.c_int32),
        ("storage", ctypes.c_int32),
    ]


class mc_instruments(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("K_host", ctypes.POINTER(ctypes.c_double)),
                ("mat_step_host", ctypes.POINTER(ctypes.c_int32))]


_lib = None
_lock = threading.Lock()

# (name, restype, argtypes) of every entry point in include/mcaad.h
_P, _V, _U64, _U32, _I32, _SZ = ctypes.POINTER, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, \
    ctypes.c_int32, ctypes.c_size_t
SIGNATURES = [
    ("mc_workspace_size", ctypes.c_int, [_P(mc_model), _P(mc_instruments), _U64, ctypes.c_int, _P(_SZ)]),
    ("mc_context_create", ctypes.c_int, [ctypes.c_int, _P(mc_model), _P(mc_instruments), _U64, _V, _SZ,
                                         _P(_V)]),
    ("mc_context_destroy", None, [_V]),
    ("mc_last_error", ctypes.c_char_p, [_V]),
    ("mc_n_params", _I32, [_V]),
    ("mc_n_instruments", _I32, [_V]),
    ("mc_storage_mode", _I32, [_V]),
    ("mc_sync", ctypes.c_int, [_V, _V]),
    ("mc_forward", ctypes.c_int, [_V, _V, _U64, _U64, _U64, _V, ctypes.c_int, _V]),
    ("mc_vjp", ctypes.c_int, [_V, _V, _V, _V]),
    ("mc_value_and_grad", ctypes.c_int, [_V, _V, _V, _U64, _U64, _U64, _V, _V, _V, _V]),
    ("mc_philox_fill", ctypes.c_int, [_U64, _U64, _U32, _U32, _V, _V]),
    ("mc_normals_fill", ctypes.c_int, [_U64, _U64, _U32, _U32, _I32, _V, _V]),
    ("mc_profile_begin", ctypes.c_int, [_V, _I32]),
    ("mc_profile_end", ctypes.c_int, [_V, _P(ctypes.c_double), _P(_I32)]),
    ("mc_forward_static", ctypes.c_int, [_P(mc_model), _P(mc_instruments), _V, _U64, _U64, _U64, _V, _V]),
    ("mc_price_jacobian_scratch_size", ctypes.c_int, [_V, _I32, _U64, _P(_SZ)]),
    ("mc_price_jacobian", ctypes.c_int, [_V, _V, _V, _I32, _U64, _U64, _V, _V, _V, _SZ, _V]),
    ("mc_value_and_grad_tangent_scratch_size", ctypes.c_int, [_V, _U64, _P(_SZ)]),
    # expected-backward tape (include/mctape.h); nodes passed as a ctypes array of mc_tape_node
    ("mc_tape_plan", ctypes.c_int, [_V, _I32, _I32, _I32, _I32, _U64, _P(_I32), _P(_I32), _P(_SZ), _P(_SZ)]),
    ("mc_tape_create", ctypes.c_int, [ctypes.c_int, _V, _I32, _I32, _I32, _I32, _U64, _V, _SZ, _P(_V)]),
    ("mc_tape_destroy", None, [_V]),
    ("mc_tape_last_error", ctypes.c_char_p, [_V]),
    ("mc_tape_value_and_grad", ctypes.c_int, [_V, _V, _U64, _U64, _U64, _V, _V, _V]),
    ("mc_tape_path_values", ctypes.c_int, [_V, _I32, _V, _V]),
    ("mc_tape_compile", ctypes.c_int, [_V, _I32, _I32, _I32, _P(ctypes.c_double), _P(_SZ)]),
    ("mc_value_and_grad_tangent", ctypes.c_int, [_V, _V, _V, _U64, _U64, _U64, _V, _V, _V, _V, _SZ, _V]),
    ("mc_tc_gemm_bf16", ctypes.c_int, [_V, ctypes.c_int64, _V, ctypes.c_int64, _I32, _I32, _I32, _I32, _V,
                                       ctypes.c_int64, _V, _V]),
    ("mlp_n_params", ctypes.c_int64, []),
    ("mlp_workspace_size", ctypes.c_int, [_I32, _P(_SZ)]),
    ("mlp_create", ctypes.c_int, [ctypes.c_int, _I32, _V, _SZ, _P(_V)]),
    ("mlp_destroy", None, [_V]),
    ("mlp_set_weights", ctypes.c_int, [_V, _V, _V]),
    ("mlp_forward", ctypes.c_int, [_V, _V, _V, _I32, _V, _V, _V]),
    ("mlp_loss_grad", ctypes.c_int, [_V, _V, _V, _V, _V, ctypes.c_float, _V, _V, _V]),
    ("mlp_adam_step", ctypes.c_int, [_V, _V, _V, _V, _V, _I32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float, _V]),
    ("mlp_train_step", ctypes.c_int, [_V, _V, _V, _V, _V, ctypes.c_float, _V, _V, _V, _V, _I32, ctypes.c_float,
                                      ctypes.c_float, ctypes.c_float, ctypes.c_float, _V]),
    ("mlp_error_flag", ctypes.c_int, [_V, _P(_I32)]),
]
KERNEL_NAMES = ["forward_sweep", "finalize_y", "seed", "reverse_sweep", "finalize_grad", "tangent_sweep",
                "finalize_tangent"]  # mc_profile kernel ids 0 .. MC_N_KERNELS-1


def load():
    """Load libmcaad.so (built by ``paper_1901_04200_gb300.build``); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libmcaad.so is not built: run paper_1901_04200_gb300.build.build() "
                                   "(or __graft_entry__.build()) first")
            lib = ctypes.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _check(st, ctx=None, what=""):
    if st != MC_OK:
        msg = load().mc_last_error(ctx).decode() if ctx else what
        raise McError(st, msg or what)


class _ProblemC:
    """C views of a Problem; keeps host arrays (and the device normals table) alive."""

    def __init__(self, pb, device):
        self.keep = []
        md = mc_model()
        md.kind = KIND[pb.kind]
        md.precision = MC_FP64 if pb.precision == "fp64" else MC_FP32
        md.S0, md.r, md.dt = float(pb.S0), float(pb.r), float(pb.dt)
        md.n_steps = int(pb.n_steps)
        md.ckpt_every = int(pb.ckpt_every or 0)
        md.paths_per_thread = int(getattr(pb, "paths_per_thread", 0) or 0)
        md.storage = STORAGE[getattr(pb, "storage", "auto")]
        if pb.kind == "gbm":
            be = np.ascontiguousarray(pb.bucket_end, dtype=np.int32)
            self.keep.append(be)
            md.n_buckets = len(be)
            md.bucket_end_host = be.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        if pb.kind in ("lv", "slv"):
            md.nt, md.nx = int(pb.nt), int(pb.nx)
            md.t_max, md.x_lo, md.x_hi = float(pb.t_max), float(pb.x_lo), float(pb.x_hi)
        if pb.normals is not None:
            z = torch.as_tensor(np.ascontiguousarray(pb.normals, dtype=np.float64)).to(device)
            self.normals = z
            md.normals = z.data_ptr()
            md.normals_path0 = int(pb.normals_path0)
            md.normals_rows = int(z.shape[0])
        K = np.ascontiguousarray(pb.K, dtype=np.float64)
        ms = np.ascontiguousarray(pb.mat_step, dtype=np.int32)
        self.keep += [K, ms]
        ins = mc_instruments()
        ins.m = len(K)
        ins.K_host = K.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        ins.mat_step_host = ms.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        self.model, self.inst = md, ins


class Context:
    """An mc_ctx: one model + instrument set, workspace allocated by torch."""

    def __init__(self, problem, max_paths: int, device=None):
        lib = load()
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.problem = problem
        self._c = _ProblemC(problem, self.device)
        nbytes = ctypes.c_size_t(0)
        _check(lib.mc_workspace_size(ctypes.byref(self._c.model), ctypes.byref(self._c.inst),
                                     int(max_paths), self.device.index, ctypes.byref(nbytes)),
               what="mc_workspace_size rejected the problem")
        self.workspace = torch.empty(max(int(nbytes.value), 256) + 256, dtype=torch.uint8,
                                     device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        h = ctypes.c_void_p()
        _check(lib.mc_context_create(self.device.index, ctypes.byref(self._c.model),
                                     ctypes.byref(self._c.inst), int(max_paths),
                                     ctypes.c_void_p(aligned), int(nbytes.value), ctypes.byref(h)),
               what="mc_context_create rejected the problem")
        self.handle = h
        self.M = lib.mc_n_params(h)
        self.m = lib.mc_n_instruments(h)
        # the storage mode the context runs ("auto" resolved by the library)
        self.storage = {v: k for k, v in STORAGE.items()}[lib.mc_storage_mode(h)]
        self.max_paths = int(max_paths)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.mc_context_destroy(h)
            self.handle = None

    def _f64(self, x, n):
        t = torch.as_tensor(x, dtype=torch.float64, device=self.device).contiguous()
        if t.numel() != n:
            raise ValueError("expected %d values, got %d" % (n, t.numel()))
        return t

    def forward(self, theta, seed: int, n_paths: int, path0: int = 0, keep: bool = False, stream=None):
        """E y [m] over global paths [path0, path0 + n_paths) (mc_forward)."""
        th = self._f64(theta, self.M)
        Ey = torch.empty(self.m, dtype=torch.float64, device=self.device)
        _check(load().mc_forward(self.handle, _ptr(th), int(seed), int(path0), int(n_paths), _ptr(Ey),
                                 1 if keep else 0, _stream(stream)), self.handle)
        self._theta_keep = th if keep else None
        return Ey

    def vjp(self, ybar, stream=None):
        """sum_i ybar_i dE y_i/dtheta for the last kept forward (mc_vjp)."""
        yb = self._f64(ybar, self.m)
        out = torch.empty(self.M, dtype=torch.float64, device=self.device)
        _check(load().mc_vjp(self.handle, _ptr(yb), _ptr(out), _stream(stream)), self.handle)
        return out

    def value_and_grad(self, theta, C, seed: int, n_paths: int, path0: int = 0, with_ey: bool = True,
                       stream=None, out=None):
        """(G [1], grad G [M], E y [m] or None) by the two-step algorithm (mc_value_and_grad)."""
        th = self._f64(theta, self.M)
        Ct = self._f64(C, self.m)
        if out is None:
            G = torch.empty(1, dtype=torch.float64, device=self.device)
            grad = torch.empty(self.M, dtype=torch.float64, device=self.device)
            Ey = torch.empty(self.m, dtype=torch.float64, device=self.device) if with_ey else None
        else:
            G, grad, Ey = out
        _check(load().mc_value_and_grad(self.handle, _ptr(th), _ptr(Ct), int(seed), int(path0), int(n_paths),
                                        _ptr(G), _ptr(grad), _ptr(Ey) if Ey is not None else None,
                                        _stream(stream)), self.handle)
        self._theta_keep = th
        return G, grad, Ey

    def value_and_grad_tangent(self, theta, C, seed: int, n_paths: int, path0: int = 0, with_ey: bool = True,
                               stream=None, out=None):
        """(G [1], grad G [M], E y [m] or None) by forward-mode tangents (mc_value_and_grad_tangent)."""
        th = self._f64(theta, self.M)
        Ct = self._f64(C, self.m)
        if out is None:
            G = torch.empty(1, dtype=torch.float64, device=self.device)
            grad = torch.empty(self.M, dtype=torch.float64, device=self.device)
            Ey = torch.empty(self.m, dtype=torch.float64, device=self.device) if with_ey else None
        else:
            G, grad, Ey = out
        nbytes = ctypes.c_size_t(0)
        _check(load().mc_value_and_grad_tangent_scratch_size(self.handle, int(n_paths), ctypes.byref(nbytes)),
               self.handle)
        key = int(nbytes.value)
        if getattr(self, "_tan_scratch", None) is None or self._tan_scratch[0] < key:
            buf = torch.empty(key + 256, dtype=torch.uint8, device=self.device)
            self._tan_scratch = (key, buf)
        buf = self._tan_scratch[1]
        base = (buf.data_ptr() + 255) // 256 * 256
        _check(load().mc_value_and_grad_tangent(self.handle, _ptr(th), _ptr(Ct), int(seed), int(path0),
                                                int(n_paths), _ptr(G), _ptr(grad),
                                                _ptr(Ey) if Ey is not None else None, ctypes.c_void_p(base),
                                                key, _stream(stream)), self.handle)
        self._theta_keep = (th, Ct)
        return G, grad, Ey

    def price_jacobian(self, thetas, seed: int, n_paths: int, strikes=None, stream=None):
        """(E y [n_theta, m], J [n_theta, m, 5]) by forward-mode tangents (mc_price_jacobian)."""
        th = torch.as_tensor(thetas, dtype=torch.float64, device=self.device).reshape(-1, self.M).contiguous()
        nt = th.shape[0]
        kt = None
        if strikes is not None:
            kt = torch.as_tensor(strikes, dtype=torch.float64, device=self.device).reshape(nt, self.m).contiguous()
        nbytes = ctypes.c_size_t(0)
        _check(load().mc_price_jacobian_scratch_size(self.handle, nt, int(n_paths), ctypes.byref(nbytes)),
               self.handle)
        scratch = torch.empty(max(int(nbytes.value), 8) // 8 + 1, dtype=torch.float64, device=self.device)
        Ey = torch.empty((nt, self.m), dtype=torch.float64, device=self.device)
        J = torch.empty((nt, self.m, self.M), dtype=torch.float64, device=self.device)
        _check(load().mc_price_jacobian(self.handle, _ptr(th), _ptr(kt) if kt is not None else None, nt, int(seed),
                                        int(n_paths), _ptr(Ey), _ptr(J), _ptr(scratch), scratch.numel() * 8,
                                        _stream(stream)), self.handle)
        self._jac_keep = (th, kt, scratch)
        return Ey, J

    def profile_begin(self, max_launches: int):
        _check(load().mc_profile_begin(self.handle, int(max_launches)), self.handle)

    def profile_end(self):
        """{kernel name: (total ms, launches)} for the launches since profile_begin."""
        nk = len(KERNEL_NAMES)
        ms = (ctypes.c_double * nk)()
        n = (ctypes.c_int32 * nk)()
        _check(load().mc_profile_end(self.handle, ms, n), self.handle)
        return {KERNEL_NAMES[k]: (ms[k], n[k]) for k in range(nk)}

    def sync(self, stream=None):
        _check(load().mc_sync(self.handle, _stream(stream)), self.handle)


def tc_gemm_bf16(A: torch.Tensor, B: torch.Tensor, k_slice: int = 0, err: torch.Tensor = None):
    """FP32 [K/k_slice, M, N] = A [M,K] @ B [N,K]^T per K slice on the tensor cores (mc_tc_gemm_bf16)."""
    M, K = A.shape
    N = B.shape[0]
    ks = k_slice or K
    D = torch.empty((K // ks, M, N), dtype=torch.float32, device=A.device)
    _check(load().mc_tc_gemm_bf16(_ptr(A), A.stride(0), _ptr(B), B.stride(0), M, N, K, ks, _ptr(D), N,
                                  _ptr(err) if err is not None else None, _stream()), what="mc_tc_gemm_bf16")
    return D


def philox_fill(seed: int, path0: int, n_paths: int, n_calls: int, device="cuda"):
    """uint32 Philox blocks [n_paths, n_calls, 4] (as int64 numpy after copy-back)."""
    out = torch.empty((n_paths, n_calls, 4), dtype=torch.int32, device=device)
    _check(load().mc_philox_fill(int(seed), int(path0), int(n_paths), int(n_calls), _ptr(out), _stream()),
           what="mc_philox_fill")
    return out


def normals_fill(seed: int, path0: int, n_paths: int, n_per_path: int, precision="fp32", device="cuda"):
    dt = torch.float64 if precision == "fp64" else torch.float32
    out = torch.empty((n_paths, n_per_path), dtype=dt, device=device)
    _check(load().mc_normals_fill(int(seed), int(path0), int(n_paths), int(n_per_path),
                                  MC_FP64 if precision == "fp64" else MC_FP32, _ptr(out), _stream()),
           what="mc_normals_fill")
    return out


class Mlp:
    """An mlp_ctx: the surrogate's activation workspace for `batch` rows (torch-allocated)."""

    def __init__(self, batch: int, device=None):
        lib = load()
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        nbytes = ctypes.c_size_t(0)
        _check(lib.mlp_workspace_size(int(batch), ctypes.byref(nbytes)), what="mlp_workspace_size")
        self.workspace = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device=self.device)
        aligned = (self.workspace.data_ptr() + 255) // 256 * 256
        h = ctypes.c_void_p()
        _check(lib.mlp_create(self.device.index, int(batch), ctypes.c_void_p(aligned), int(nbytes.value),
                              ctypes.byref(h)), what="mlp_create")
        self.handle = h
        self.batch = int(batch)
        self.n_params = int(lib.mlp_n_params())

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.mlp_destroy(h)
            self.handle = None

    def set_weights(self, params, stream=None):
        _check(load().mlp_set_weights(self.handle, _ptr(params), _stream(stream)), what="mlp_set_weights")

    def forward(self, params, X, with_grad=False, stream=None):
        n = X.shape[0]
        out = torch.empty(n, dtype=torch.float32, device=self.device)
        dx = torch.empty((n, 7), dtype=torch.float32, device=self.device) if with_grad else None
        _check(load().mlp_forward(self.handle, _ptr(params), _ptr(X), n, _ptr(out), _ptr(dx) if dx is not None else None,
                                  _stream(stream)), what="mlp_forward")
        return (out, dx) if with_grad else out

    def loss_grad(self, params, X, y, dy, alpha, grads, loss=None, stream=None):
        _check(load().mlp_loss_grad(self.handle, _ptr(params), _ptr(X), _ptr(y), _ptr(dy), float(alpha),
                                    _ptr(loss) if loss is not None else None, _ptr(grads), _stream(stream)),
               what="mlp_loss_grad")

    def adam_step(self, params, grads, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        _check(load().mlp_adam_step(self.handle, _ptr(params), _ptr(grads), _ptr(m), _ptr(v), int(t), float(lr),
                                    float(beta1), float(beta2), float(eps), _stream(stream)), what="mlp_adam_step")

    def train_step(self, params, X, y, dy, alpha, grads, loss, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                   stream=None):
        """mlp_loss_grad then mlp_adam_step, replayed as a captured graph after the first call."""
        _check(load().mlp_train_step(self.handle, _ptr(params), _ptr(X), _ptr(y), _ptr(dy), float(alpha), _ptr(grads),
                                     _ptr(loss) if loss is not None else None, _ptr(m), _ptr(v), int(t), float(lr),
                                     float(beta1), float(beta2), float(eps), _stream(stream)),
               what="mlp_train_step")

    def error_flag(self):
        f = ctypes.c_int32(0)
        _check(load().mlp_error_flag(self.handle, ctypes.byref(f)), what="mlp_error_flag")
        return f.value
