"""FP64 oracle of the pricing surrogate: MLP 7 -> 256 -> 256 -> 256 -> 256 -> 1 with SiLU.

TEST INFRASTRUCTURE ONLY (only tests, the smoke check and the benchmark's
CPU-baseline leg may use it).  Plain numpy, one matrix product per layer.

The network maps (Heston theta [5], strike, maturity) to a price; it is trained
with the differential loss
    L = mean_b (out_b - y_b)^2 + alpha * mean_b sum_{j<5} (d out_b / d x_bj - dy_bj)^2,
whose labels y and dy = d price / d theta come from the Monte Carlo method
itself (forward sweep and pathwise derivatives).  The gradient of L with
respect to the weights needs the derivative of the input gradient, written
here by hand (no autodiff library):

  forward      z_l = h_{l-1} W_l^T + b_l,  h_l = silu(z_l),  out = h_4 . w5 + b5
  input grad   g_4 = w5,  p_l = g_l * silu'(z_l),  g_{l-1} = p_l W_l,  d out/dx = g_0
  adjoints     out_bar = 2 (out - y)/B,  g0_bar = 2 alpha (g_0 - dy)/B on the theta columns
               up the tangent chain (l = 1..4):
                 p_bar_l = g_bar_{l-1} W_l^T,   dW_l += p_l^T g_bar_{l-1}
                 g_bar_l = p_bar_l * silu'(z_l), z_bar_l(tangent) = p_bar_l * g_l * silu''(z_l)
                 (l = 4: dw5 += column sums of g_bar_4)
               down the forward chain (l = 4..1):
                 h_bar_4 = out_bar w5^T,  dw5 += h_4^T out_bar,  db5 = sum out_bar
                 z_bar_l = h_bar_l * silu'(z_l) + z_bar_l(tangent)
                 dW_l += z_bar_l^T h_{l-1},  db_l = column sums of z_bar_l,  h_bar_{l-1} = z_bar_l W_l

With ``bf16=True`` every operand of a matrix product is rounded to bfloat16
(round to nearest even) first, at the same points as the tensor-core kernels;
everything else stays FP64.
"""
from __future__ import annotations

import numpy as np

D_IN, H, N_LAYERS, N_THETA = 7, 256, 4, 5
SHAPES = [("W1", (H, D_IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
          ("W4", (H, H)), ("b4", (H,)), ("w5", (H,)), ("b5", (1,))]


def n_params():
    return int(sum(np.prod(s) for _, s in SHAPES))


def unflatten(vec):
    p, o = {}, 0
    for name, s in SHAPES:
        n = int(np.prod(s))
        p[name] = np.asarray(vec[o:o + n], dtype=np.float64).reshape(s)
        o += n
    return p


def flatten(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init_params(seed=0):
    """Glorot-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, s in SHAPES:
        if name.startswith("W"):
            lim = np.sqrt(6.0 / (s[0] + s[1]))
            p[name] = rng.uniform(-lim, lim, s)
        elif name == "w5":
            lim = np.sqrt(6.0 / (H + 1))
            p[name] = rng.uniform(-lim, lim, s)
        else:
            p[name] = np.zeros(s)
    return p


def round_bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def silu(z):
    return z * sigmoid(z)


def dsilu(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def d2silu(z):
    s = sigmoid(z)
    return s * (1.0 - s) * (2.0 + z * (1.0 - 2.0 * s))


def _mm(a, b, bf16):
    if bf16:
        return round_bf16(a) @ round_bf16(b)
    return a @ b


def forward(p, X, bf16=False):
    """out [B] and the cache (z_l, h_l for l = 0..4)."""
    h = [np.asarray(X, dtype=np.float64)]
    z = [None]
    for l in range(1, N_LAYERS + 1):
        zl = _mm(h[l - 1], p["W%d" % l].T, bf16) + p["b%d" % l]
        z.append(zl)
        h.append(silu(zl))
    out = h[4] @ p["w5"] + p["b5"][0]
    return out, {"z": z, "h": h}


def input_grad(p, cache, bf16=False):
    """d out / d x [B, 7] and the tangent chain (g_l, p_l)."""
    z = cache["z"]
    B = z[1].shape[0]
    g = [None] * (N_LAYERS + 1)
    pl = [None] * (N_LAYERS + 1)
    g[4] = np.broadcast_to(p["w5"], (B, H))
    for l in range(N_LAYERS, 0, -1):
        pl[l] = g[l] * dsilu(z[l])
        g[l - 1] = _mm(pl[l], p["W%d" % l], bf16)
    return g[0], {"g": g, "p": pl}


def loss(p, X, y, dy, alpha, bf16=False):
    out, cache = forward(p, X, bf16)
    g0, _ = input_grad(p, cache, bf16)
    B = len(y)
    return float(np.sum((out - y) ** 2) / B + alpha * np.sum((g0[:, :N_THETA] - dy) ** 2) / B)


def loss_grad(p, X, y, dy, alpha, bf16=False):
    """(L, dL/dparams as a dict, out, d out/dx) by the explicit double-backward chain above."""
    X = np.asarray(X, dtype=np.float64)
    B = X.shape[0]
    out, cache = forward(p, X, bf16)
    g0, tan = input_grad(p, cache, bf16)
    z, h = cache["z"], cache["h"]
    g, pl = tan["g"], tan["p"]
    L = float(np.sum((out - y) ** 2) / B + alpha * np.sum((g0[:, :N_THETA] - dy) ** 2) / B)
    grads = {name: np.zeros(s) for name, s in SHAPES}
    out_bar = 2.0 * (out - y) / B
    gbar = np.zeros_like(g0)
    gbar[:, :N_THETA] = 2.0 * alpha * (g0[:, :N_THETA] - dy) / B
    zbar_t = [None] * (N_LAYERS + 1)
    for l in range(1, N_LAYERS + 1):
        W = p["W%d" % l]
        pbar = _mm(gbar, W.T, bf16)
        grads["W%d" % l] += _mm(pl[l].T, gbar, bf16)
        gbar_l = pbar * dsilu(z[l])
        zbar_t[l] = pbar * g[l] * d2silu(z[l])
        gbar = gbar_l
    grads["w5"] += gbar.sum(axis=0)
    hbar = np.outer(out_bar, p["w5"])
    grads["w5"] += (round_bf16(h[4]) if bf16 else h[4]).T @ out_bar
    grads["b5"][0] = out_bar.sum()
    for l in range(N_LAYERS, 0, -1):
        zbar = hbar * dsilu(z[l]) + zbar_t[l]
        grads["W%d" % l] += _mm(zbar.T, h[l - 1], bf16)
        grads["b%d" % l] = zbar.sum(axis=0)
        if l > 1:
            hbar = _mm(zbar, p["W%d" % l], bf16)
    return L, grads, out, g0


def adam(vec, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba) on flat FP64 vectors; t counts from 1."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return vec - lr * mh / (np.sqrt(vh) + eps), m, v
