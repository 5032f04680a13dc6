"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: Philox blocks bit-exact; FP64 paths: E y, G and grad G within
1e-10 relative (normwise for vectors); FP32 paths: grad G within 1e-4
normwise, E y within 2e-6 of max |E y|, G within 1e-4 relative.
"""
from dataclasses import replace

import numpy as np
import pytest

from paper_1901_04200_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_04200_gb300 import build as b
    b.build()
    from paper_1901_04200_gb300 import _lib
    _lib.load()
    return _lib


def gpu_vg(L, w, n_paths=None, path0=0, seed=None):
    n = n_paths or w.n_paths
    ctx = L.Context(w.problem, max_paths=n)
    G, g, Ey = ctx.value_and_grad(w.theta, w.C, w.problem.seed if seed is None else seed, n, path0=path0)
    torch.cuda.synchronize()
    return Ey.cpu().numpy(), G.item(), g.cpu().numpy()


def check(L, orc, w, tol_g, tol_ey, n_paths=None, path0=0):
    n = n_paths or w.n_paths
    Ey, G, g = gpu_vg(L, w, n, path0)
    Eo, Go, go = orc.value_and_grad(w.problem, w.theta, w.C, n, path0=path0)
    assert rel(Ey, Eo) <= tol_ey, ("Ey", rel(Ey, Eo))
    assert abs(G - Go) <= tol_g * abs(Go), ("G", G, Go)
    assert rel(g, go) <= tol_g, ("grad", rel(g, go), g, go)
    return Ey, G, g


# ------------------------------------------------------------- generator

@pytest.mark.parametrize("seed,path0", [(0x190104200, 0), (0, (1 << 32) - 7), (0xFFFFFFFFFFFFFFFF, 12345)])
def test_philox_bit_exact(L, orc, seed, path0):
    n_paths, n_calls = 37, 9
    got = L.philox_fill(seed, path0, n_paths, n_calls).cpu().numpy().view(np.uint32)
    ref = orc.philox_fill(seed, path0, n_paths, n_calls)
    assert np.array_equal(got, ref)


def test_normals_match_oracle(L, orc):
    seed, path0, n_paths, n = 0x190104200, 1000, 257, 61
    ref = orc.normals_fill(seed, path0, n_paths, n)
    z64 = L.normals_fill(seed, path0, n_paths, n, "fp64").cpu().numpy()
    assert np.max(np.abs(z64 - ref)) <= 1e-13
    z32 = L.normals_fill(seed, path0, n_paths, n, "fp32").cpu().numpy().astype(np.float64)
    err = np.abs(z32 - ref)
    assert np.max(err) <= 5e-5 and np.mean(err) <= 2e-6, (np.max(err), np.mean(err))


def test_philox_against_curand_device_api(L, tmp_path):
    """Counter layout = cuRAND device API philox4_32_10 with subsequence = path, offset = 4 * call."""
    import os
    import subprocess
    src = os.path.join(os.path.dirname(__file__), "cuda", "curand_philox_dump.cu")
    exe = str(tmp_path / "curand_dump")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", src, "-o", exe], check=True)
    for seed, path0 in [(0x190104200, 0), (7, (1 << 32) - 3), (0xDEADBEEFCAFEF00D, (5 << 32) + 11)]:
        out = subprocess.run([exe, str(seed), str(path0), "40", "6"], check=True, capture_output=True).stdout
        ref = np.frombuffer(out, dtype=np.uint32).reshape(40, 6, 4)
        got = L.philox_fill(seed, path0, 40, 6).cpu().numpy().view(np.uint32)
        assert np.array_equal(got, ref), (seed, path0)


# ----------------------------------------------------------- FP64 exact

def test_gbm_fp64_config(L, orc):
    """The GBM workload (normals table input, FP64 path) within 1e-10."""
    w = inputs.gbm_config()
    check(L, orc, w, 1e-10, 1e-12)


def test_gbm_fp64_philox_ragged(L, orc):
    w = inputs.gbm_config(n_paths=16)
    w = replace(w, problem=replace(w.problem, normals=None))
    check(L, orc, w, 1e-10, 1e-12, n_paths=1001, path0=(1 << 32) - 500)


@pytest.mark.parametrize("n_steps", [7, 14])
def test_gbm_fp64_philox_partial_period(L, orc, n_steps):
    """Seven segments of one step (groups of four per Philox block) or two steps (groups of two)."""
    w = inputs.gbm_config(n_paths=16, n_steps=n_steps, n_buckets=7)
    w = replace(w, problem=replace(w.problem, normals=None))
    check(L, orc, w, 1e-10, 1e-12, n_paths=777)


@pytest.mark.parametrize("storage", ["checkpoint", "normals"])
@pytest.mark.parametrize("K,ppt", [(1, 1), (2, 1), (4, 1), (8, 1), (2, 2), (4, 2), (8, 2)])
def test_heston_fp64_all_segment_lengths(L, orc, K, ppt, storage):
    w = inputs.heston_config(n_paths=3000, steps_per_year=32, T=1.0, n_mat=4, n_strike=5)
    w = replace(w, problem=replace(w.problem, precision="fp64", ckpt_every=K, paths_per_thread=ppt,
                                   storage=storage))
    check(L, orc, w, 1e-10, 1e-12, n_paths=3000, path0=77)


def test_heston_fp64_no_feller(L, orc):
    """Exact arithmetic agrees even where v often truncates (FP64 on both sides)."""
    w = inputs.heston_config(n_paths=2048, steps_per_year=32, T=1.0, n_mat=4, n_strike=5, feller=False)
    w = replace(w, problem=replace(w.problem, precision="fp64"))
    check(L, orc, w, 1e-9, 1e-12)


@pytest.mark.parametrize("storage", ["checkpoint", "normals", "states"])
@pytest.mark.parametrize("K,ppt", [(1, 1), (5, 1), (25, 1), (5, 2), (5, 4)])
def test_lv_fp64(L, orc, K, ppt, storage):
    w = inputs.lv_config(n_paths=1500, n_steps=100, T=2.0, nt=5, nx=6, n_mat=4, n_strike=5)
    w = replace(w, problem=replace(w.problem, precision="fp64", ckpt_every=K, paths_per_thread=ppt,
                                   storage=storage))
    check(L, orc, w, 1e-10, 1e-12)


@pytest.mark.parametrize("storage", ["checkpoint", "normals", "states"])
@pytest.mark.parametrize("K,ppt", [(1, 1), (5, 1), (5, 2), (5, 4)])
def test_lv_fp64_partial_philox_period(L, orc, K, ppt, storage):
    """95 steps: 19 segments at K = 5 and 95 at K = 1, so the forward sweep's last group of
    segments (four per Philox period of 20 or 4 normals) is partial."""
    w = inputs.lv_config(n_paths=1100, n_steps=95, T=1.9, nt=5, nx=6, n_mat=19, n_strike=2)
    w = replace(w, problem=replace(w.problem, precision="fp64", ckpt_every=K, paths_per_thread=ppt,
                                   storage=storage))
    check(L, orc, w, 1e-10, 1e-12)


@pytest.mark.parametrize("storage", ["normals", "states"])
def test_lv_fp64_clamped_surface(L, orc, storage):
    w = inputs.lv_config(n_paths=999, n_steps=100, T=2.0, nt=5, nx=6, n_mat=4, n_strike=5)
    w = replace(w, problem=replace(w.problem, precision="fp64", x_lo=-0.1, x_hi=0.15, storage=storage))
    check(L, orc, w, 1e-10, 1e-12)


# ------------------------------------------------------------ FP32 paths

@pytest.mark.parametrize("storage", ["checkpoint", "normals"])
@pytest.mark.parametrize("K,ppt", [(8, 1), (4, 2), (2, 2)])
def test_heston_fp32_small(L, orc, K, ppt, storage):
    w = inputs.heston_config(n_paths=1 << 14, steps_per_year=64, T=2.0)
    w = replace(w, problem=replace(w.problem, ckpt_every=K, paths_per_thread=ppt, storage=storage))
    check(L, orc, w, 1e-4, 2e-6)


def test_lv_fp32_small(L, orc):
    w = inputs.lv_config(n_paths=1 << 13)
    check(L, orc, w, 1e-4, 2e-6)


@pytest.mark.parametrize("K,ppt", [(25, 1), (25, 2), (5, 4)])
def test_lv_fp32_recompute(L, orc, K, ppt):
    """Checkpoints only, each segment re-run into shared memory (25 steps, two paths per thread:
    the bench's recompute arm), on the workload's own grid and instruments, ragged path count."""
    w = inputs.lv_config(n_paths=(1 << 13) - 17)
    w = replace(w, problem=replace(w.problem, storage="checkpoint", ckpt_every=K, paths_per_thread=ppt))
    check(L, orc, w, 1e-4, 2e-6)


def test_gbm_fp32(L, orc):
    w = inputs.gbm_config()
    w = replace(w, problem=replace(w.problem, precision="fp32"))
    check(L, orc, w, 1e-4, 2e-6)


# -------------------------------------------------------------- edge cases

@pytest.mark.parametrize("storage", ["checkpoint", "normals"])
@pytest.mark.parametrize("n", [1, 31, 33, 4097])
def test_ragged_path_counts(L, orc, n, storage):
    w = inputs.heston_config(n_paths=n, steps_per_year=16, T=1.0, n_mat=2, n_strike=3)
    w = replace(w, problem=replace(w.problem, precision="fp64", storage=storage))
    check(L, orc, w, 1e-10, 1e-12)


def test_unsorted_instruments_and_single_segment(L, orc):
    w = inputs.heston_config(n_paths=700, steps_per_year=16, T=1.0, n_mat=4, n_strike=3)
    pb = w.problem
    rng = np.random.default_rng(5)
    order = rng.permutation(pb.m)
    pb = replace(pb, K=pb.K[order], mat_step=pb.mat_step[order], precision="fp64", ckpt_every=4)
    w = replace(w, problem=pb, C=w.C[order])
    check(L, orc, w, 1e-10, 1e-12)
    # a single maturity at the first segment end
    pb1 = replace(pb, K=np.array([95.0, 100.0, 105.0]), mat_step=np.array([4, 4, 4], dtype=np.int32))
    w1 = replace(w, problem=pb1, C=np.array([5.0, 2.0, 1.0]))
    check(L, orc, w1, 1e-10, 1e-12)


def test_vjp_and_forward_match_oracle(L, orc):
    w = inputs.lv_config(n_paths=2000, n_steps=100, T=2.0, nt=5, nx=6, n_mat=4, n_strike=5)
    w = replace(w, problem=replace(w.problem, precision="fp64"))
    ctx = L.Context(w.problem, max_paths=2000)
    ybar = np.random.default_rng(3).standard_normal(w.problem.m)
    Ey = ctx.forward(w.theta, w.problem.seed, 2000, path0=5, keep=True)
    tb = ctx.vjp(ybar)
    torch.cuda.synchronize()
    assert rel(Ey.cpu().numpy(), orc.forward(w.problem, w.theta, 2000, path0=5)) <= 1e-12
    assert rel(tb.cpu().numpy(), orc.vjp(w.problem, w.theta, ybar, 2000, path0=5)) <= 1e-10


def test_vjp_requires_kept_checkpoints(L):
    w = inputs.heston_config(n_paths=64, steps_per_year=16, T=1.0, n_mat=2, n_strike=2)
    ctx = L.Context(w.problem, max_paths=64)
    ctx.forward(w.theta, 1, 64, keep=False)
    with pytest.raises(L.McError) as e:
        ctx.vjp(np.ones(w.problem.m))
    assert e.value.status == L.MC_ERR_STATE


def test_call_argument_errors(L):
    w = inputs.heston_config(n_paths=64, steps_per_year=16, T=1.0, n_mat=2, n_strike=2)
    ctx = L.Context(w.problem, max_paths=64)
    with pytest.raises(L.McError) as e:
        ctx.forward(w.theta, 1, 65)
    assert e.value.status == L.MC_ERR_INVALID_ARG
    for call in (lambda: ctx.forward(w.theta, 1, 0), lambda: ctx.value_and_grad(w.theta, w.C, 1, 0)):
        with pytest.raises(L.McError) as e:  # no paths: an empty estimator
            call()
        assert e.value.status == L.MC_ERR_INVALID_ARG


@pytest.mark.parametrize("split,tol", [(6016, 1e-13), (6000, 1e-7)])
def test_partition_invariance(L, split, tol):
    """Global path indices: two ranges combine to the full range.  A split on a
    32-path boundary keeps every FP32 warp sum identical (only the FP64 order
    changes); any other split regroups the FP32 warp sums."""
    n = 1 << 14
    w = inputs.heston_config(n_paths=n, steps_per_year=64, T=1.0, n_mat=4, n_strike=4)
    ctx = L.Context(w.problem, max_paths=n)
    full = ctx.forward(w.theta, 9, n).cpu().numpy()
    a = ctx.forward(w.theta, 9, split).cpu().numpy()
    b = ctx.forward(w.theta, 9, n - split, path0=split).cpu().numpy()
    comb = (split * a + (n - split) * b) / n
    assert rel(comb, full) <= tol


def test_deterministic_repeat(L):
    w = inputs.heston_config(n_paths=1 << 15, steps_per_year=64, T=1.0, n_mat=4, n_strike=4)
    a = gpu_vg(L, w)
    b = gpu_vg(L, w)
    assert np.array_equal(a[0], b[0]) and a[1] == b[1] and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("kind", ["heston", "lv"])
def test_reused_context_queue_and_repeat(L, orc, kind):
    """One context, calls of different path counts in a row (each sweep takes its chunks from a
    queue the previous launch reset): every call equals the oracle, and repeating a call gives
    the same bits whatever chunks the warps took."""
    w = small_case(kind, n_paths=5000)
    pb = with_pb(w, precision="fp64").problem
    ctx = L.Context(pb, max_paths=5000)
    runs = []
    for n, p0 in [(1000, 0), (4097, 9), (33, 100), (1000, 0)]:
        G, g, Ey = (x.cpu().numpy() for x in ctx.value_and_grad(w.theta, w.C, pb.seed, n, path0=p0))
        Eo, Go, go = orc.value_and_grad(pb, w.theta, w.C, n, path0=p0)
        assert rel(Ey, Eo) <= 1e-12 and abs(G[0] - Go) <= 1e-10 * abs(Go) and rel(g, go) <= 1e-10
        runs.append((G, g, Ey))
    assert all(np.array_equal(a, b) for a, b in zip(runs[0], runs[3]))


# ------------------------------------------------------------ full sizes

@pytest.mark.slow
def test_heston_full_size(L, orc):
    """The benchmark workload (2^20 paths x 512 steps, launch shape of the bench) vs the oracle,
    checkpoint/recompute arm."""
    w = inputs.heston_config()
    check(L, orc, replace(w, problem=replace(w.problem, storage="checkpoint")), 1e-4, 2e-6)


def full_size_sampled(L, orc, w, n_slice):
    """A full-size workload in the bench's context: a slice of n_slice paths at the top of the
    range against the oracle -- E y, G and grad G of the slice, and the full run's lambda pulled
    back through the slice (vjp) -- and the full run's E y and grad G equal the size-weighted
    combination of its two halves (the gradient rebuilt from the halves' vjp with the full run's
    lambda)."""
    n = w.n_paths
    ctx = L.Context(w.problem, max_paths=n)
    p0 = n - n_slice
    Gs, gs, Eys = (x.cpu().numpy() for x in ctx.value_and_grad(w.theta, w.C, w.problem.seed, n_slice, path0=p0))
    Eo, Go, go = orc.value_and_grad(w.problem, w.theta, w.C, n_slice, path0=p0)
    assert rel(Eys, Eo) <= 2e-6, ("Ey", rel(Eys, Eo))
    assert abs(Gs[0] - Go) <= 1e-4 * abs(Go), ("G", Gs[0], Go)
    assert rel(gs, go) <= 1e-4, ("grad", rel(gs, go))
    G, g, Ey = ctx.value_and_grad(w.theta, w.C, w.problem.seed, n)
    Ey, g = Ey.cpu().numpy(), g.cpu().numpy()
    lam = Ey - w.C
    ctx.forward(w.theta, w.problem.seed, n_slice, path0=p0, keep=True)
    vs = ctx.vjp(lam).cpu().numpy()
    assert rel(vs, orc.vjp(w.problem, w.theta, lam, n_slice, path0=p0)) <= 1e-4
    h = n // 2
    a = ctx.forward(w.theta, w.problem.seed, h, keep=True).cpu().numpy()
    va = ctx.vjp(lam).cpu().numpy()
    b = ctx.forward(w.theta, w.problem.seed, n - h, path0=h, keep=True).cpu().numpy()
    vb = ctx.vjp(lam).cpu().numpy()
    assert rel((a + b) / 2, Ey) <= 1e-12
    assert rel((va + vb) / 2, g) <= 1e-5
    return ctx


@pytest.mark.slow
def test_lv_full_size_sampled(L, orc):
    """2^22 x 500 local vol (the bench's headline workload and launch shape)."""
    ctx = full_size_sampled(L, orc, inputs.lv_config(), 1 << 13)
    assert ctx.storage == "states"


@pytest.mark.slow
def test_lv_full_size_sampled_recompute(L, orc):
    """The same workload by checkpoints every 25 steps and recompute, two paths per thread (the
    bench's recompute arm and launch shape)."""
    w = inputs.lv_config()
    w = replace(w, problem=replace(w.problem, storage="checkpoint", ckpt_every=25, paths_per_thread=2))
    ctx = full_size_sampled(L, orc, w, 1 << 12)
    assert ctx.storage == "checkpoint"


# ------------------------------------------------- Heston SLV (the paper's model)

@pytest.mark.parametrize("storage", ["checkpoint", "normals"])
@pytest.mark.parametrize("K", [1, 2, 4, 8])
def test_slv_fp64(L, orc, K, storage):
    w = inputs.slv_config(n_paths=1500, steps_per_year=32, T=1.0, n_mat=4, n_strike=4, nt=5, nx=6)
    w = replace(w, problem=replace(w.problem, precision="fp64", ckpt_every=K, storage=storage))
    check(L, orc, w, 1e-10, 1e-12, path0=33)


def test_slv_fp32(L, orc):
    w = inputs.slv_config(n_paths=1 << 14, steps_per_year=64, T=2.0)
    check(L, orc, w, 1e-4, 2e-6)


def test_slv_unit_leverage_matches_heston_gpu(L):
    """At L = 1 the SLV kernels reproduce the Heston kernels' prices exactly (FP64)."""
    ws = inputs.slv_config(n_paths=4096, steps_per_year=32, T=1.0, n_mat=4, n_strike=4)
    wh = inputs.heston_config(n_paths=4096, steps_per_year=32, T=1.0, n_mat=4, n_strike=4)
    th = ws.theta.copy()
    th[5:] = 1.0
    ps = replace(ws.problem, precision="fp64")
    ph = replace(wh.problem, precision="fp64", paths_per_thread=1)
    a = L.Context(ps, max_paths=4096).forward(th, 7, 4096).cpu().numpy()
    b = L.Context(ph, max_paths=4096).forward(th[:5], 7, 4096).cpu().numpy()
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))


# ------------------------------------- stored variants: full tape, stored normals
# "full": the forward sweep stores every step's tape and the reverse sweep runs
# only the adjoint; "normals": the forward sweep stores its normals next to the
# checkpoints and the reverse sweep re-runs each segment on them.

STORED = ["full", "normals"]


def small_case(kind, n_paths=None):
    if kind == "gbm":
        return inputs.gbm_config()
    if kind == "heston":
        return inputs.heston_config(n_paths=n_paths or 2000, steps_per_year=32, T=1.0, n_mat=4, n_strike=5)
    if kind == "lv":
        return inputs.lv_config(n_paths=n_paths or 1500, n_steps=100, T=2.0, nt=5, nx=6, n_mat=4, n_strike=5)
    return inputs.slv_config(n_paths=n_paths or 1500, steps_per_year=32, T=1.0, n_mat=4, n_strike=4, nt=5, nx=6)


def with_pb(w, **kw):
    return replace(w, problem=replace(w.problem, **kw))


@pytest.mark.parametrize("storage", STORED)
@pytest.mark.parametrize("kind", ["gbm", "heston", "lv", "slv"])
def test_stored_variants_fp64(L, orc, kind, storage):
    check(L, orc, with_pb(small_case(kind), precision="fp64", storage=storage), 1e-10, 1e-12)


@pytest.mark.parametrize("kind,K,ppt", [("gbm", 1, 1), ("gbm", 16, 1), ("heston", 1, 1), ("heston", 2, 2),
                                        ("heston", 4, 1), ("heston", 8, 2), ("lv", 1, 1), ("lv", 5, 2),
                                        ("lv", 25, 1), ("slv", 2, 1), ("slv", 8, 1)])
def test_stored_normals_staging_shapes_fp64(L, orc, kind, K, ppt):
    """Every staging geometry: rows per warp K*DZ*PPT from 1 to 32, copies that do not fill
    the warp's lanes, 256-byte FP64 rows, ragged path counts."""
    if kind == "gbm":  # one bucket, so that K = 16 divides the only maturity step
        w = with_pb(inputs.gbm_config(n_paths=1001, n_buckets=8 if K < 16 else 1), normals=None)
    else:
        w = small_case(kind, n_paths=1001)
    check(L, orc, with_pb(w, precision="fp64", storage="normals", ckpt_every=K, paths_per_thread=ppt),
          1e-10, 1e-12)


@pytest.mark.parametrize("kind,storage", [(k, st) for k in ("heston", "lv", "slv") for st in STORED]
                         + [("lv", "states")])
def test_stored_equals_recompute_fp32(L, kind, storage):
    """The stored variants run the same step arithmetic as checkpoint/recompute: the same
    E y, and the gradient to FP32 rounding of the re-run segments."""
    if kind == "heston":
        w = inputs.heston_config(n_paths=1 << 15, steps_per_year=64, T=2.0)
    elif kind == "lv":
        w = inputs.lv_config(n_paths=1 << 14)
    else:
        w = inputs.slv_config(n_paths=1 << 14, steps_per_year=64, T=2.0)
    a = gpu_vg(L, with_pb(w, storage="checkpoint"))
    b = gpu_vg(L, with_pb(w, storage=storage))
    assert rel(a[0], b[0]) <= 1e-13
    assert rel(a[2], b[2]) <= 1e-5


@pytest.mark.parametrize("n", [1, 33, 4097])
def test_stored_normals_ragged_fp32(L, orc, n):
    w = inputs.heston_config(n_paths=n, steps_per_year=16, T=1.0, n_mat=2, n_strike=3)
    check(L, orc, with_pb(w, storage="normals"), 1e-4, 2e-6)


def test_stored_normals_vjp_after_forward(L, orc):
    """mc_forward with kept results, then mc_vjp, on the stored normals."""
    w = with_pb(small_case("lv"), precision="fp64", storage="normals")
    ctx = L.Context(w.problem, max_paths=w.n_paths)
    Ey = ctx.forward(w.theta, w.problem.seed, w.n_paths, keep=True).cpu().numpy()
    ybar = np.linspace(-1.0, 1.0, len(Ey))
    g = ctx.vjp(ybar).cpu().numpy()
    assert rel(Ey, orc.forward(w.problem, w.theta, w.n_paths)) <= 1e-12
    assert rel(g, orc.vjp(w.problem, w.theta, ybar, w.n_paths)) <= 1e-10


@pytest.mark.slow
def test_heston_full_size_stored_normals(L, orc):
    """The benchmark workload with stored normals (4.3 GB of them) vs the oracle."""
    check(L, orc, with_pb(inputs.heston_config(), storage="normals"), 1e-4, 2e-6)


def test_auto_storage_resolves(L):
    """"auto" picks the stored normals (local vol: the stored states) when they fit a quarter of
    the device's memory."""
    w = inputs.heston_config(n_paths=4096, steps_per_year=16, T=1.0, n_mat=2, n_strike=3)
    assert L.Context(w.problem, max_paths=4096).storage == "normals"
    for st in ("checkpoint", "normals", "full"):
        assert L.Context(with_pb(w, storage=st).problem, max_paths=4096).storage == st
    wl = small_case("lv", n_paths=4096)
    assert L.Context(wl.problem, max_paths=4096).storage == "states"


# ----------------------------------------------- stored states (local vol)
# The forward sweep stores the state before every step; the reverse sweep runs only the
# adjoint, with each step's sqrt(dt) z taken from the states at its two ends.

@pytest.mark.parametrize("n", [1, 31, 33, 4097])
@pytest.mark.parametrize("precision,tol_g,tol_ey", [("fp64", 1e-10, 1e-12), ("fp32", 1e-4, 2e-6)])
def test_states_ragged(L, orc, n, precision, tol_g, tol_ey):
    w = with_pb(small_case("lv", n_paths=n), precision=precision, storage="states")
    check(L, orc, w, tol_g, tol_ey, path0=5)


def test_states_vjp_after_forward(L, orc):
    """mc_forward with kept results, then mc_vjp with an arbitrary seed, on the stored states."""
    w = with_pb(small_case("lv"), precision="fp64", storage="states")
    ctx = L.Context(w.problem, max_paths=w.n_paths)
    Ey = ctx.forward(w.theta, w.problem.seed, w.n_paths, path0=3, keep=True).cpu().numpy()
    ybar = np.linspace(-1.0, 1.0, len(Ey))
    g = ctx.vjp(ybar).cpu().numpy()
    assert rel(Ey, orc.forward(w.problem, w.theta, w.n_paths, path0=3)) <= 1e-12
    assert rel(g, orc.vjp(w.problem, w.theta, ybar, w.n_paths, path0=3)) <= 1e-10


def test_states_single_segment_and_reuse(L, orc):
    """One segment (K = 25 over 25 steps: the extra tile follows directly), and a context reused
    with fewer paths, another seed and other node values."""
    w = with_pb(inputs.lv_config(n_paths=700, n_steps=25, T=0.5, nt=3, nx=4, n_mat=1, n_strike=4),
                precision="fp64", storage="states", ckpt_every=25, paths_per_thread=1)
    check(L, orc, w, 1e-10, 1e-12)
    ctx = L.Context(w.problem, max_paths=700)
    th = w.theta * 1.1
    G, g, Ey = (x.cpu().numpy() for x in ctx.value_and_grad(th, w.C, 99, 400, path0=11))
    pb = replace(w.problem, seed=99)
    Eo, Go, go = orc.value_and_grad(pb, th, w.C, 400, path0=11)
    assert rel(Ey, Eo) <= 1e-12 and abs(G[0] - Go) <= 1e-10 * abs(Go) and rel(g, go) <= 1e-10


@pytest.mark.parametrize("kind", ["gbm", "heston", "slv"])
def test_states_only_for_local_vol(L, kind):
    w = with_pb(small_case(kind, n_paths=64), storage="states")
    with pytest.raises(L.McError) as e:
        L.Context(w.problem, max_paths=64)
    assert e.value.status == L.MC_ERR_UNSUPPORTED


@pytest.mark.slow
def test_slv_full_size_sampled(L, orc):
    """Heston SLV at the bench's size (2^20 x 512, M = 95, stored normals)."""
    ctx = full_size_sampled(L, orc, inputs.slv_config(), 1 << 12)
    assert ctx.storage == "normals"


# ------------------------------------------------------------- size limits

@pytest.mark.parametrize("storage", ["checkpoint", "normals"])
def test_heston_1024_instruments_fp64(L, orc, storage):
    """The instrument limit (m = 1024: 8 maturities x 128 strikes) against the oracle."""
    w = inputs.heston_config(n_paths=700, steps_per_year=16, T=1.0, n_mat=8, n_strike=128)
    assert w.problem.m == 1024
    check(L, orc, replace(w, problem=replace(w.problem, precision="fp64", ckpt_every=2, storage=storage)),
          1e-10, 1e-12)


@pytest.mark.parametrize("storage", ["checkpoint", "normals"])
def test_lv_256_parameters_fp64(L, orc, storage):
    """The parameter limit (M = 256: an 8 x 32 node surface, the 32-node axis limit) against the oracle."""
    w = inputs.lv_config(n_paths=900, n_steps=100, T=2.0, nt=8, nx=32, n_mat=4, n_strike=5)
    assert w.problem.n_params == 256
    check(L, orc, replace(w, problem=replace(w.problem, precision="fp64", storage=storage)), 1e-10, 1e-12)


def test_beyond_limits_rejected(L):
    w = inputs.heston_config(n_paths=64, steps_per_year=16, T=1.0, n_mat=8, n_strike=129)
    with pytest.raises(L.McError) as e:
        L.Context(w.problem, max_paths=64)
    assert e.value.status == L.MC_ERR_INVALID_ARG
    w = inputs.lv_config(n_paths=64, n_steps=100, T=2.0, nt=9, nx=32, n_mat=4, n_strike=5)
    with pytest.raises(L.McError):
        L.Context(w.problem, max_paths=64)
