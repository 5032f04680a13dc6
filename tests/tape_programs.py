"""Seeded random programs for the expected-backward tape tests, as neutral op
lists (name, a, b, c) that each side builds with its own API.  Holds none of
the method's arithmetic: it only chooses operations and constants."""
from __future__ import annotations

import numpy as np


def random_program(seed: int, n_params: int = 4, n_normals: int = 6, n_ops: int = 120, n_expect: int = 4):
    """Ops over bounded values: every value-growing op is followed by x / (|x| + 1); exp takes
    bounded inputs, log takes x^2 + 1, sqrt takes relu or abs.  Expectations appear mid-program
    and feed later per-path operations.  Returns (ops, objective index)."""
    rng = np.random.default_rng(seed)
    ops = []

    def add(op, a=-1, b=-1, c=0.0):
        ops.append((op, int(a), int(b), float(c)))
        return len(ops) - 1

    pool = [add("param", c=k) for k in range(n_params)]
    pool += [add("normal", c=j) for j in range(n_normals)]
    pool.append(add("const", c=0.7))
    expects = []

    def squash(i):
        ab = add("abs", i)
        den = add("addc", ab, c=1.0)
        return add("div", i, den)

    while len(ops) < n_ops:
        a, b = (int(x) for x in rng.choice(pool, 2))
        kind = rng.integers(0, 12)
        if kind == 0:
            r = squash(add("add", a, b))
        elif kind == 1:
            r = squash(add("sub", a, b))
        elif kind == 2:
            r = squash(add("mul", a, b))
        elif kind == 3:
            r = add("addc", a, c=float(rng.uniform(-1, 1)))
        elif kind == 4:
            r = add("mulc", a, c=float(rng.uniform(-1.5, 1.5)))
        elif kind == 5:
            r = add("neg", a)
        elif kind == 6:
            r = squash(add("exp", a))
        elif kind == 7:
            sq = add("mul", a, a)
            r = add("log", add("addc", sq, c=1.0))
        elif kind == 8:
            r = add("sqrt", add("relu" if rng.integers(0, 2) else "abs", a))
        elif kind == 9:
            r = add("relu", a)
        elif kind == 10 and len(expects) < n_expect:
            r = add("expect", a)
            expects.append(r)
        else:
            den = add("addc", add("abs", b), c=1.5)
            r = add("div", a, den)
        pool.append(r)
    # objective: 1/2 sum of squared expectations of the last few values, plus the first expectation
    G = None
    for i in pool[-5:] + expects:
        e = add("expect", i)
        t = add("mulc", add("mul", e, e), c=0.5)
        G = t if G is None else add("add", G, t)
    return ops, G


def build_product(ops, tape_mod):
    """The program in the product's builder (paper_1901_04200_gb300.tape)."""
    prog = tape_mod.Program()
    nodes = [prog.node(op, a, b, c) for op, a, b, c in ops]
    return prog, nodes


def run_oracle(ops, objective, theta, Z):
    """Value and gradient of the program by the oracle's whole-program tape."""
    from oracle import tape as T
    tp = T.Tape(Z.shape[0])
    vals, inputs = [], {}
    for op, a, b, c in ops:
        A = vals[a] if a >= 0 else None
        B = vals[b] if b >= 0 else None
        if op == "param":
            v = tp.input(float(theta[int(c)]))
            inputs[int(c)] = v
        elif op == "const":
            v = tp.const(c)
        elif op == "normal":
            v = tp.const(Z[:, int(c)])
        elif op == "add":
            v = A + B
        elif op == "sub":
            v = A - B
        elif op == "mul":
            v = A * B
        elif op == "div":
            v = A / B
        elif op == "addc":
            v = A + c
        elif op == "mulc":
            v = A * c
        elif op == "neg":
            v = -A
        elif op == "exp":
            v = T.exp(A)
        elif op == "log":
            v = T.log(A)
        elif op == "sqrt":
            v = T.sqrt(A)
        elif op == "relu":
            v = T.relu(A)
        elif op == "abs":
            v = T.absv(A)
        elif op == "expect":
            v = T.expectation(A)
        else:
            raise ValueError(op)
        vals.append(v)
    D = tp.backward(vals[objective])
    grad = np.array([np.mean(D[inputs[k].idx]) for k in sorted(inputs)])
    return float(vals[objective].v[0]), grad, vals
