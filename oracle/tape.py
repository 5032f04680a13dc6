"""Expected backward automatic differentiation over a whole-program tape.

TEST INFRASTRUCTURE ONLY.  This follows the paper's Appendix (after Fries):
a program is a list of operations x_m = f_m(x_tau...), one of which may be an
expectation operator; the backward sweep starts from D_N = 1, walks the list
from last to first, adds D_m * df_m/dx_j to each argument's adjoint for an
ordinary operation and E(D_m) for the expectation, and the derivative of the
output with respect to input i is E(D_i).

Values are random variables, stored as numpy vectors over all Monte Carlo
paths (a deterministic value is a constant vector).  Unlike the two-step
algorithm of the paper, this differentiates THROUGH the expectations: the
whole computation of G -- all paths, the means E y_i, lambda and G -- is on
one tape.  On tiny inputs it is the independent check that the two-step
gradient equals the gradient of G (the gradient identity of the paper).

Kink conventions match the two-step oracle: d max(u,0)/du = 1{u > 0};
d sqrt(u)/du is taken as 0 at u = 0; clamp has derivative 1 strictly inside.
"""
from __future__ import annotations

import numpy as np


class Tape:
    def __init__(self, n_paths: int):
        self.P = n_paths
        self.ops = []  # list of (kind, [(arg_index, partial_vector)])

    def _push(self, value, parents, kind="op"):
        idx = len(self.ops)
        self.ops.append((kind, parents))
        return Var(self, idx, np.broadcast_to(np.asarray(value, dtype=np.float64), (self.P,)).copy())

    def input(self, value):
        return self._push(value, [], "input")

    def const(self, value):
        return self._push(value, [], "const")

    def backward(self, out: "Var"):
        """Fries' rule; returns the list of adjoint vectors D_i."""
        D = [np.zeros(self.P) for _ in self.ops]
        D[out.idx] = np.ones(self.P)
        for m in range(len(self.ops) - 1, -1, -1):
            kind, parents = self.ops[m]
            for j, partial in parents:
                if kind == "expectation":
                    D[j] = D[j] + np.mean(D[m])
                else:
                    D[j] = D[j] + D[m] * partial
        return D


class Var:
    __array_priority__ = 100

    def __init__(self, tape: Tape, idx: int, value: np.ndarray):
        self.t, self.idx, self.v = tape, idx, value

    def _lift(self, o):
        return o if isinstance(o, Var) else self.t.const(o)

    def __add__(self, o):
        o = self._lift(o)
        return self.t._push(self.v + o.v, [(self.idx, 1.0), (o.idx, 1.0)])

    __radd__ = __add__

    def __sub__(self, o):
        o = self._lift(o)
        return self.t._push(self.v - o.v, [(self.idx, 1.0), (o.idx, -1.0)])

    def __rsub__(self, o):
        return self._lift(o) - self

    def __mul__(self, o):
        o = self._lift(o)
        return self.t._push(self.v * o.v, [(self.idx, o.v), (o.idx, self.v)])

    __rmul__ = __mul__

    def __truediv__(self, o):
        o = self._lift(o)
        return self.t._push(self.v / o.v, [(self.idx, 1.0 / o.v), (o.idx, -self.v / (o.v * o.v))])

    def __neg__(self):
        return self.t._push(-self.v, [(self.idx, -1.0)])


def exp(a: Var) -> Var:
    e = np.exp(a.v)
    return a.t._push(e, [(a.idx, e)])


def log(a: Var) -> Var:
    return a.t._push(np.log(a.v), [(a.idx, 1.0 / a.v)])


def sqrt(a: Var) -> Var:
    s = np.sqrt(a.v)
    with np.errstate(divide="ignore"):
        d = np.where(a.v > 0.0, 0.5 / np.where(s > 0, s, 1.0), 0.0)
    return a.t._push(s, [(a.idx, d)])


def relu(a: Var) -> Var:
    """max(a, 0) with derivative 1{a > 0}."""
    return a.t._push(np.maximum(a.v, 0.0), [(a.idx, (a.v > 0.0).astype(np.float64))])


def clamp(a: Var, lo: float, hi: float) -> Var:
    inside = ((a.v > lo) & (a.v < hi)).astype(np.float64)
    return a.t._push(np.clip(a.v, lo, hi), [(a.idx, inside)])


def absv(a: Var) -> Var:
    return a.t._push(np.abs(a.v), [(a.idx, np.sign(a.v))])


def expectation(a: Var) -> Var:
    """The expectation operator: a deterministic value, Fries' adjoint rule."""
    return a.t._push(np.full(a.t.P, np.mean(a.v)), [(a.idx, None)], "expectation")


def full_tape_value_and_grad(pb, theta, C, normals):
    """G and grad G by differentiating the whole program, expectations included.

    pb: a problem (attributes of ``Problem``); normals: [P, n_steps*dz] FP64.
    Written independently of the two-step oracle: the local-vol surface is a
    sum of tensor-product hat functions over all nodes rather than a cell
    lookup, and the payoff, state recursions and G are plain tape expressions.
    """
    P = normals.shape[0]
    T = Tape(P)
    th = [T.input(float(v)) for v in theta]
    dt, r = float(pb.dt), float(pb.r)
    sdt = float(np.sqrt(dt))
    last = int(np.max(pb.mat_step))
    x = T.const(0.0)
    states = [x]
    if pb.kind in ("heston", "slv"):
        kappa, thh, xi, rho, v0 = th[:5]
        v = v0 * 1.0
        rhob = sqrt(1.0 - rho * rho)

    def surface(nodes, xv, n):
        """Bilinear node surface at (t_n, x) as a sum of tensor-product hat functions."""
        nt, nx = int(pb.nt), int(pb.nx)
        ht = pb.t_max / (nt - 1)
        hx = (pb.x_hi - pb.x_lo) / (nx - 1)
        ut = min(max(n * dt / ht, 0.0), nt - 1.0)
        ux = clamp((xv - pb.x_lo) * (1.0 / hx), 0.0, nx - 1.0)
        acc = None
        for j in range(nt):
            wt = max(0.0, 1.0 - abs(ut - j))
            if wt == 0.0:
                continue
            for c in range(nx):
                term = nodes[j * nx + c] * relu(1.0 - absv(ux - float(c))) * wt
                acc = term if acc is None else acc + term
        return acc
    for n in range(last):
        if pb.kind == "gbm":
            b = int(np.searchsorted(np.asarray(pb.bucket_end), n, side="right"))
            vol = th[b]
            z = T.const(normals[:, n])
            x = x + (r - 0.5 * vol * vol) * dt + vol * sdt * z
        elif pb.kind == "heston":
            z1 = T.const(normals[:, 2 * n])
            z2 = T.const(normals[:, 2 * n + 1])
            vp = relu(v)
            sq = sqrt(vp * dt)
            w = rho * z1 + rhob * z2
            x_new = x + (r - 0.5 * vp) * dt + sq * z1
            v = v + kappa * (thh - vp) * dt + xi * sq * w
            x = x_new
        elif pb.kind == "slv":
            z1 = T.const(normals[:, 2 * n])
            z2 = T.const(normals[:, 2 * n + 1])
            lev = surface(th[5:], x, n)
            vp = relu(v)
            sq = sqrt(vp * dt)
            w = rho * z1 + rhob * z2
            x_new = x + (r - 0.5 * lev * lev * vp) * dt + lev * sq * z1
            v = v + kappa * (thh - vp) * dt + xi * sq * w
            x = x_new
        else:
            sigma = surface(th, x, n)
            z = T.const(normals[:, n])
            x = x + (r - 0.5 * sigma * sigma) * dt + sigma * sdt * z
        states.append(x)
    G = None
    for i in range(len(pb.K)):
        ni = int(pb.mat_step[i])
        S = exp(states[ni]) * float(pb.S0)
        y = relu(S - float(pb.K[i])) * float(np.exp(-r * ni * dt))
        lam = expectation(y) - float(C[i])
        term = lam * lam * 0.5
        G = term if G is None else G + term
    D = T.backward(G)
    grad = np.array([np.mean(D[t.idx]) for t in th])
    return float(G.v[0]), grad
