"""The tensor-core surrogate kernels against the FP64 oracle run with the same
bfloat16 rounding of every matrix-product operand."""
import numpy as np
import pytest

from oracle import mlp as omlp

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


def setup(B, seed=3):
    rng = np.random.default_rng(seed)
    p = omlp.init_params(seed)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.normal(scale=0.05, size=p[k].shape)
    X = rng.uniform(-1, 1, (B, 7)).astype(np.float32).astype(np.float64)
    y = rng.normal(size=B).astype(np.float32).astype(np.float64)
    dy = rng.normal(size=(B, 5)).astype(np.float32).astype(np.float64)
    return p, X, y, dy


def cuda32(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("B,n", [(128, 128), (256, 200), (4096, 4096)])
def test_forward_and_input_grad(L, B, n):
    p, X, _, _ = setup(n)
    net = L.Mlp(B)
    prm = cuda32(omlp.flatten(p))
    net.set_weights(prm)
    out, dx = net.forward(prm, cuda32(X), with_grad=True)
    torch.cuda.synchronize()
    assert net.error_flag() == 0
    o_ref, cache = omlp.forward(p, X, bf16=True)
    g_ref, _ = omlp.input_grad(p, cache, bf16=True)
    assert rel(out.cpu().numpy(), o_ref) <= 2e-3
    assert rel(dx.cpu().numpy(), g_ref) <= 5e-3


@pytest.mark.parametrize("alpha,B", [(0.0, 512), (0.5, 512), (1.0, 4096), (1.0, 128), (0.5, 640)])
def test_loss_grad_matches_oracle(L, alpha, B):
    """B = 4096, alpha = 1 is the training step the bench times; B = 128 and 640 take the
    weight-gradient GEMMs' smaller K splits (4 slices of 64 and 320 rows)."""
    p, X, y, dy = setup(B, seed=11)
    net = L.Mlp(B)
    prm = cuda32(omlp.flatten(p))
    net.set_weights(prm)
    grads = torch.zeros(net.n_params, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    net.loss_grad(prm, cuda32(X), cuda32(y), cuda32(dy), alpha, grads, loss)
    torch.cuda.synchronize()
    assert net.error_flag() == 0
    L_ref, g_ref, _, _ = omlp.loss_grad(p, X, y, dy, alpha, bf16=True)
    assert abs(loss.item() - L_ref) <= 2e-3 * abs(L_ref)
    gv = grads.cpu().numpy().astype(np.float64)
    gr = omlp.flatten(g_ref)
    for name, s in omlp.SHAPES:
        a = omlp.unflatten(gv)[name]
        b = omlp.unflatten(gr)[name]
        # each parameter block against its own scale: the oracle rounds to BF16 at the kernels'
        # storage points, so what is left is FP32 accumulation order (and the odd BF16 rounding
        # tie it moves)
        assert np.max(np.abs(a - b)) <= 5e-3 * np.max(np.abs(b)), (name, np.max(np.abs(a - b)), np.max(np.abs(b)))
    assert rel(gv, gr) <= 2e-3


@pytest.mark.parametrize("mode", ["1", "2"])
@pytest.mark.parametrize("B", [128, 4096])
def test_row_chain_kernel_matches_oracle(L, B, mode, monkeypatch):
    """The opt-in single-launch row chains (MCAAD_MLP_CHAIN=1: F, T, R, D of each 128-row block in
    one CTA; 2: in a cluster of eight CTAs, 32 columns each) match the oracle as the per-GEMM path
    does."""
    monkeypatch.setenv("MCAAD_MLP_CHAIN", mode)
    p, X, y, dy = setup(B, seed=5)
    net = L.Mlp(B)
    prm = cuda32(omlp.flatten(p))
    net.set_weights(prm)
    grads = torch.zeros(net.n_params, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    net.loss_grad(prm, cuda32(X), cuda32(y), cuda32(dy), 1.0, grads, loss)
    torch.cuda.synchronize()
    assert net.error_flag() == 0
    L_ref, g_ref, _, _ = omlp.loss_grad(p, X, y, dy, 1.0, bf16=True)
    assert abs(loss.item() - L_ref) <= 2e-3 * abs(L_ref)
    gv = grads.cpu().numpy().astype(np.float64)
    gr = omlp.flatten(g_ref)
    for name, s in omlp.SHAPES:
        a = omlp.unflatten(gv)[name]
        b = omlp.unflatten(gr)[name]
        assert np.max(np.abs(a - b)) <= 5e-3 * np.max(np.abs(b)), (name, np.max(np.abs(a - b)), np.max(np.abs(b)))


def test_adam_step_matches_oracle(L):
    B = 128
    p, X, y, dy = setup(B, seed=2)
    net = L.Mlp(B)
    vec = omlp.flatten(p)
    prm = cuda32(vec)
    g = np.random.default_rng(0).normal(size=vec.size)
    m = torch.zeros_like(prm)
    v = torch.zeros_like(prm)
    pv, mv, vv = vec.copy(), np.zeros_like(vec), np.zeros_like(vec)
    for t in range(1, 4):
        net.adam_step(prm, cuda32(g * t), m, v, t, lr=1e-3)
        pv, mv, vv = omlp.adam(pv, g * t, mv, vv, t, lr=1e-3)
    torch.cuda.synchronize()
    assert np.max(np.abs(prm.cpu().numpy() - pv)) <= 1e-6


def test_train_step_graph_equals_eager_steps(L):
    """mlp_train_step (first call eager, then a replayed CUDA graph with the step's learning rate
    and bias corrections patched in) gives bit-identical parameters, moments and loss to
    mlp_loss_grad + mlp_adam_step, over batches that live at different addresses each step."""
    B, steps = 512, 6
    p, _, _, _ = setup(B, seed=5)
    rng = np.random.default_rng(9)
    batches = [(cuda32(rng.uniform(-1, 1, (B, 7))), cuda32(rng.normal(size=B)), cuda32(rng.normal(size=(B, 5))))
               for _ in range(steps)]
    runs = []
    for graph in (False, True):
        net = L.Mlp(B)
        prm = cuda32(omlp.flatten(p))
        net.set_weights(prm)
        g = torch.zeros_like(prm)
        m, v = torch.zeros_like(prm), torch.zeros_like(prm)
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        losses = []
        for t in range(1, steps + 1):
            X, y, dy = batches[t - 1]
            lr = 1e-3 / t
            if graph:
                net.train_step(prm, X, y, dy, 0.7, g, loss, m, v, t, lr=lr)
            else:
                net.loss_grad(prm, X, y, dy, 0.7, g, loss)
                net.adam_step(prm, g, m, v, t, lr=lr)
            losses.append(loss.clone())
        torch.cuda.synchronize()
        assert net.error_flag() == 0
        runs.append((prm.cpu(), m.cpu(), v.cpu(), torch.cat(losses).cpu()))
    for a, b in zip(*runs):
        assert torch.equal(a, b)
