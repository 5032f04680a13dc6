"""The sharded two-step algorithm on CPU: two gloo ranks, each evaluating its
own path range with the oracle, reproduce the single-process oracle's G and
grad G, identically on both ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, splits, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    import oracle
    from paper_1901_04200_gb300 import inputs
    from paper_1901_04200_gb300.sharding import sharded_value_and_grad
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = inputs.heston_config(n_paths=16, steps_per_year=32, T=1.0, n_mat=4, n_strike=3)
    p0, n = splits[rank]
    fwd = lambda: oracle.forward(w.problem, w.theta, n, path0=p0, n_threads=2)
    vjp = lambda ybar: oracle.vjp(w.problem, w.theta, ybar.numpy(), n, path0=p0, n_threads=2)
    Ey, G, g = sharded_value_and_grad(fwd, vjp, w.C, n)
    np.save(os.path.join(out_dir, "r%d.npy" % rank), np.concatenate([Ey.numpy(), [G.item()], g.numpy()]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("splits", [[(0, 3000), (3000, 2000)], [(0, 2500), (2500, 2500)]])
def test_two_rank_gloo_matches_single_process(orc, tmp_path, splits):
    port = _free_port()
    mp.spawn(_worker, args=(2, port, splits, str(tmp_path)), nprocs=2, join=True)
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert np.array_equal(r0, r1)  # rank-order sums: identical on every rank
    from paper_1901_04200_gb300 import inputs
    w = inputs.heston_config(n_paths=16, steps_per_year=32, T=1.0, n_mat=4, n_strike=3)
    total = sum(n for _, n in splits)
    Ey, G, g = orc.value_and_grad(w.problem, w.theta, w.C, total, n_threads=2)
    m = w.problem.m
    assert np.allclose(r0[:m], Ey, rtol=1e-13, atol=0)
    assert abs(r0[m] - G) <= 1e-12 * abs(G)
    assert np.allclose(r0[m + 1:], g, rtol=1e-12, atol=1e-12 * np.max(np.abs(g)))
