"""Pins of the FP64 surrogate oracle: finite differences of its own loss and
output, closed-form SiLU derivatives, bfloat16 rounding, and Adam's
sign property under a constant gradient."""
import numpy as np
import pytest

from oracle import mlp


def data(B=64, seed=1):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, (B, mlp.D_IN))
    y = rng.normal(size=B)
    dy = rng.normal(size=(B, mlp.N_THETA))
    return X, y, dy


def test_silu_derivatives_fd():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    assert np.allclose((mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), mlp.dsilu(z), atol=1e-9)
    assert np.allclose((mlp.dsilu(z + h) - mlp.dsilu(z - h)) / (2 * h), mlp.d2silu(z), atol=1e-9)


def test_input_grad_fd():
    p = mlp.init_params(3)
    X, _, _ = data(8)
    out, cache = mlp.forward(p, X)
    g0, _ = mlp.input_grad(p, cache)
    h = 1e-6
    for j in range(mlp.D_IN):
        e = np.zeros(mlp.D_IN)
        e[j] = h
        fd = (mlp.forward(p, X + e)[0] - mlp.forward(p, X - e)[0]) / (2 * h)
        assert np.allclose(fd, g0[:, j], rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("alpha", [0.0, 0.7])
def test_loss_grad_fd(alpha):
    p = mlp.init_params(5)
    for k in p:
        if k.startswith("b"):
            p[k] = np.random.default_rng(9).normal(scale=0.1, size=p[k].shape)
    X, y, dy = data(32)
    L, grads, _, _ = mlp.loss_grad(p, X, y, dy, alpha)
    assert np.isclose(L, mlp.loss(p, X, y, dy, alpha), rtol=1e-14)
    rng = np.random.default_rng(2)
    for name, s in mlp.SHAPES:
        for _ in range(4):
            idx = tuple(rng.integers(0, n) for n in s)
            h = 1e-6
            pp = {k: v.copy() for k, v in p.items()}
            pm = {k: v.copy() for k, v in p.items()}
            pp[name][idx] += h
            pm[name][idx] -= h
            fd = (mlp.loss(pp, X, y, dy, alpha) - mlp.loss(pm, X, y, dy, alpha)) / (2 * h)
            assert abs(fd - grads[name][idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, grads[name][idx])


def test_flatten_roundtrip_and_count():
    p = mlp.init_params(0)
    v = mlp.flatten(p)
    assert v.size == mlp.n_params() == 199681
    q = mlp.unflatten(v)
    assert all(np.array_equal(p[k], q[k]) for k in p)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7 + 2 ** -8, 3.0e38, -2.5, 0.1])
    r = mlp.round_bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                    # tie -> even mantissa
    assert r[2] == 1.0 + 2 ** -6          # tie -> even (rounds up)
    assert r[4] == -2.5
    assert abs(r[5] - 0.1) <= 0.1 * 2 ** -8
    assert np.all(np.frexp(r[[0, 1, 2, 4, 5]])[0] * 256 % 1 == 0)  # 8 significant bits


def test_adam_constant_gradient_moves_by_lr_times_sign():
    """With a constant gradient the bias-corrected ratio m^/sqrt(v^) is sign(g) exactly."""
    vec = np.zeros(4)
    g = np.array([3.0, -0.5, 2e-3, -7.0])
    m = np.zeros(4)
    v = np.zeros(4)
    for t in range(1, 6):
        vec, m, v = mlp.adam(vec, g, m, v, t, lr=0.01, eps=0.0)
        assert np.allclose(vec, -0.01 * t * np.sign(g), rtol=1e-12, atol=1e-15)


def test_bf16_mode_is_close_to_fp64():
    p = mlp.init_params(7)
    X, y, dy = data(128)
    L0, g0, _, _ = mlp.loss_grad(p, X, y, dy, 0.5)
    L1, g1, _, _ = mlp.loss_grad(p, X, y, dy, 0.5, bf16=True)
    assert abs(L1 - L0) <= 0.05 * abs(L0)
    a, b = mlp.flatten(g0), mlp.flatten(g1)
    assert np.max(np.abs(a - b)) <= 0.05 * np.max(np.abs(a))
