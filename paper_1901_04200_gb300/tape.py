"""Programs for expected-backward AD on the GPU (include/mctape.h).

A ``Program`` records operations on ``Node`` objects (operator overloading
with Python floats mixed in) into the node list that ``mc_tape_create``
takes; ``TapeContext`` evaluates the objective and its gradient through the
C ABI.  ``heston_objective`` writes the calibration objective
G = 1/2 sum_i (E y_i - C_i)^2 of the Heston full-truncation model as such a
program -- the whole program, expectations included, differentiated by the
Appendix's rule instead of the two-step algorithm.
"""
from __future__ import annotations

import ctypes

import numpy as np

OPS = {"param": 0, "const": 1, "normal": 2, "add": 3, "sub": 4, "mul": 5, "div": 6, "addc": 7, "mulc": 8,
       "neg": 9, "exp": 10, "log": 11, "sqrt": 12, "relu": 13, "abs": 14, "expect": 15}


class mc_tape_node(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("a", ctypes.c_int32), ("b", ctypes.c_int32), ("c", ctypes.c_double)]


class Node:
    __slots__ = ("prog", "i")
    __array_priority__ = 100

    def __init__(self, prog: "Program", i: int):
        self.prog, self.i = prog, i

    def _bin(self, op, o, swap=False):
        o = o if isinstance(o, Node) else self.prog.const(float(o))
        a, b = (o, self) if swap else (self, o)
        return self.prog.node(op, a.i, b.i)

    def __add__(self, o):
        return self.prog.node("addc", self.i, c=float(o)) if not isinstance(o, Node) else self._bin("add", o)

    __radd__ = __add__

    def __sub__(self, o):
        return self.prog.node("addc", self.i, c=-float(o)) if not isinstance(o, Node) else self._bin("sub", o)

    def __rsub__(self, o):
        return self.prog.node("addc", (-self).i, c=float(o))

    def __mul__(self, o):
        return self.prog.node("mulc", self.i, c=float(o)) if not isinstance(o, Node) else self._bin("mul", o)

    __rmul__ = __mul__

    def __truediv__(self, o):
        return self._bin("div", o)

    def __rtruediv__(self, o):
        return self._bin("div", o, swap=True)

    def __neg__(self):
        return self.prog.node("neg", self.i)


class Program:
    def __init__(self):
        self.nodes = []

    def node(self, op: str, a: int = -1, b: int = -1, c: float = 0.0) -> Node:
        self.nodes.append((OPS[op], int(a), int(b), float(c)))
        return Node(self, len(self.nodes) - 1)

    def param(self, k: int) -> Node:
        return self.node("param", c=k)

    def const(self, v: float) -> Node:
        return self.node("const", c=v)

    def normal(self, j: int) -> Node:
        return self.node("normal", c=j)

    def c_nodes(self):
        arr = (mc_tape_node * len(self.nodes))()
        for k, (op, a, b, c) in enumerate(self.nodes):
            arr[k].op, arr[k].a, arr[k].b, arr[k].c = op, a, b, c
        return arr


def exp(a: Node) -> Node:
    return a.prog.node("exp", a.i)


def log(a: Node) -> Node:
    return a.prog.node("log", a.i)


def sqrt(a: Node) -> Node:
    return a.prog.node("sqrt", a.i)


def relu(a: Node) -> Node:
    return a.prog.node("relu", a.i)


def absv(a: Node) -> Node:
    return a.prog.node("abs", a.i)


def expect(a: Node) -> Node:
    return a.prog.node("expect", a.i)


PRECISION = {"fp64": 0, "fp32": 1}  # mc_precision


def plan(prog: Program, objective: Node, n_params: int, max_paths: int = 1, precision: str = "fp64"):
    """(status, stages, per-path nodes, workspace bytes, HBM bytes per path of one value and
    gradient) from mc_tape_plan (host only)."""
    from . import _lib
    ns, nr, ws, hb = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_size_t(0), ctypes.c_size_t(0)
    st = _lib.load().mc_tape_plan(prog.c_nodes(), len(prog.nodes), objective.i, n_params, PRECISION[precision], max_paths,
                                  ctypes.byref(ns), ctypes.byref(nr), ctypes.byref(ws), ctypes.byref(hb))
    return st, ns.value, nr.value, ws.value, hb.value


class TapeContext:
    """A program on one GPU with tapes for up to max_paths paths (mc_tape_create); precision
    "fp64" or "fp32" (per-path values, adjoints and normals; sums over paths stay FP64)."""

    def __init__(self, prog: Program, objective: Node, n_params: int, max_paths: int, device=None,
                 precision: str = "fp64"):
        import torch
        from . import _lib
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.n_params = int(n_params)
        self.objective = objective.i
        lib = _lib.load()
        h = ctypes.c_void_p()
        _lib._check(lib.mc_tape_create(self.device.index, prog.c_nodes(), len(prog.nodes), objective.i,
                                       self.n_params, PRECISION[precision], int(max_paths), None, 0,
                                       ctypes.byref(h)),
                    what="mc_tape_create rejected the program")
        self.handle = h
        self._destroy = lib.mc_tape_destroy  # kept: no imports while the interpreter shuts down
        self.max_paths = int(max_paths)
        self._n = 0

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            self._destroy(h)
            self.handle = None

    def _check(self, st):
        from . import _lib
        if st != _lib.MC_OK:
            raise _lib.McError(st, _lib.load().mc_tape_last_error(self.handle).decode())

    def value_and_grad(self, theta, seed: int, n_paths: int, path0: int = 0, stream=None, out=None):
        """(objective [1], gradient [n_params]) over global paths [path0, path0 + n_paths)."""
        import torch
        from . import _lib
        th = torch.as_tensor(np.asarray(theta, dtype=np.float64) if not isinstance(theta, torch.Tensor) else theta,
                             dtype=torch.float64, device=self.device).contiguous()
        if out is None:
            val = torch.empty(1, dtype=torch.float64, device=self.device)
            grad = torch.empty(max(self.n_params, 1), dtype=torch.float64, device=self.device)
        else:
            val, grad = out
        self._check(_lib.load().mc_tape_value_and_grad(self.handle, _lib._ptr(th), int(seed), int(path0),
                                                       int(n_paths), _lib._ptr(val), _lib._ptr(grad),
                                                       _lib._stream(stream)))
        self._keep = th
        self._n = int(n_paths)
        return val, grad[:self.n_params]

    def compile(self, seg_nodes: int = 0, recompute: bool = False, threads: int = 0, piece: int = 0):
        """Compile the program into straight-line kernels (mc_tape_compile); with recompute the
        backward kernels re-run their segment's forward instead of reloading values, in pieces of
        `piece` nodes when piece >= 2 (each piece's inputs kept on the tape by the forward kernel).
        Returns (compile seconds, HBM bytes per path of one compiled value and gradient)."""
        from . import _lib
        sec, hb = ctypes.c_double(0.0), ctypes.c_size_t(0)
        mode = (int(piece) if piece >= 2 else 1) if recompute else 0
        self._check(_lib.load().mc_tape_compile(self.handle, int(seg_nodes), mode, int(threads),
                                                ctypes.byref(sec), ctypes.byref(hb)))
        return sec.value, hb.value

    def path_values(self, node: Node, stream=None):
        """Per-path values of a per-path node on the last evaluated paths."""
        import torch
        from . import _lib
        out = torch.empty(self._n, dtype=torch.float64, device=self.device)
        self._check(_lib.load().mc_tape_path_values(self.handle, node.i, _lib._ptr(out), _lib._stream(stream)))
        return out


def heston_objective(pb, C):
    """G = 1/2 sum_i (E y_i - C_i)^2 of the Heston full-truncation model (parameters 0..4 =
    kappa, theta_h, xi, rho, v0) as one program: per step v+ = max(v, 0), vdt = v+ dt,
    sq = sqrt(vdt), w = rho z1 + sqrt(1 - rho^2) z2, x += r dt - vdt/2 + sq z1,
    v += kappa (theta_h - v+) dt + xi sq w; normals 2n and 2n+1 of step n; payoff
    e^{-r T_i} max(S0 e^{x_{n_i}} - K_i, 0).  Returns (program, objective node)."""
    prog = Program()
    kappa, thh, xi, rho, v0 = (prog.param(k) for k in range(5))
    dt, r = float(pb.dt), float(pb.r)
    rhob = sqrt(1.0 - rho * rho)
    kdt = kappa * dt
    kthdt = kdt * thh
    x = prog.const(0.0)
    v = v0
    mat = np.asarray(pb.mat_step)
    last = int(mat.max())
    xs = {}
    for n in range(last):
        z1, z2 = prog.normal(2 * n), prog.normal(2 * n + 1)
        vdt = relu(v) * dt
        sq = sqrt(vdt)
        w = rho * z1 + rhob * z2
        x = x + ((r * dt) - 0.5 * vdt + sq * z1)
        v = v + (kthdt - kappa * vdt + xi * sq * w)
        if n + 1 in set(mat.tolist()):
            xs[n + 1] = x
    G = None
    for i in range(len(mat)):
        ni = int(mat[i])
        S = exp(xs[ni]) * float(pb.S0)
        y = relu(S - float(pb.K[i])) * float(np.exp(-r * ni * dt))
        lam = expect(y) - float(C[i])
        term = 0.5 * (lam * lam)
        G = term if G is None else G + term
    return prog, G
