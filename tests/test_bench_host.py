"""Host-side arithmetic of bench.py's roofline entries (no GPU)."""
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

N_SM, MHZ = 152, 2070.0
ISSUE = 128 * N_SM * MHZ * 1e6
HBM = 6800.3e9


def test_algorithmic_bytes_per_path_step():
    """Stored normals: two normals and a checkpoint of two words every K steps, 4 B each."""
    assert bench.kernel_bytes("heston", "normals", 8, 512, 8)["forward_sweep"] == 4.0 * 2 / 8 + 8.0
    assert bench.kernel_bytes("heston", "checkpoint", 8, 512, 8)["reverse_sweep"] == 1.0
    assert bench.kernel_bytes("lv", "normals", 5, 500, 20)["forward_sweep"] == 4.0 / 5 + 4.0
    # full tape: four Heston fields per step and x at each of 8 maturity steps out of 512
    assert bench.kernel_bytes("heston", "full", 8, 512, 8)["forward_sweep"] == 16.0 + 4.0 * 8 / 512


@pytest.mark.parametrize("storage", ["normals", "checkpoint"])
def test_pipe_fractions(storage):
    P, S = 1 << 20, 512
    prof = {"forward_sweep": (11.3, 10), "reverse_sweep": (7.7, 10)}
    r = bench.kernel_rooflines("heston", storage, 8, 2, P, S, 8, prof, ISSUE, HBM, "measured", N_SM, MHZ)
    for name, k in r["kernels"].items():
        t = k["ms"] * 1e-3
        by = k["ops_by_pipe"]
        assert sum(by.values()) == k["ops_per_path_step"] == bench.kernel_ops("heston", storage, name)
        assert math.isclose(k["pipe_fracs"]["issue"], k["alu_frac"], rel_tol=1e-12)
        for kind, v in by.items():
            want = P * S * v / t / (bench.PIPE_RATES[kind] * N_SM * MHZ * 1e6)
            assert math.isclose(k["pipe_fracs"][kind], want, rel_tol=1e-12)
        assert k["alu_pipe_bound"] == max(k["pipe_fracs"], key=k["pipe_fracs"].get)
    dom = r["kernels"]["forward_sweep"]  # the longer kernel
    assert r["bound"] == "alu" and r["frac"] == dom["alu_frac"] and r["fp32_pipe_frac"] == dom["pipe_fracs"]["fp32"]
    assert r["hbm"]["frac"] == dom["hbm_frac"]


def test_tangent_sweep_counts_f_and_the_tangents():
    prof = {"tangent_sweep": (19.1, 10)}
    r = bench.kernel_rooflines("heston", "tangent", 8, 1, 1 << 20, 512, 8, prof, ISSUE, HBM, "measured",
                               N_SM, MHZ)
    k = r["kernels"]["tangent_sweep"]
    assert k["ops_per_path_step"] == sum(bench.OPS["heston"]["F"].values()) + bench.OPS_TANGENT["heston"]["fp32"]
    assert r["bound"] == "alu" and k["bytes_per_path_step"] == 0.0


def test_measured_traffic_only_for_the_profiled_sources(monkeypatch):
    """The stored DRAM bytes are reported while the kernel sources hash to the captured version,
    and null once they differ."""
    key = ("heston", "normals", 8, 2, "forward_sweep")
    rec = bench.MEASURED_TRAFFIC[key]
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda model="heston": rec["sources"])
    assert bench.measured_traffic(*key) == rec["bytes"]
    assert bench.measured_traffic("heston", "normals", 4, 2, "forward_sweep") is None
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda model="heston": "another version")
    assert bench.measured_traffic(*key) is None


def test_local_vol_kernel_parts_by_storage():
    """Local vol: the stored-states reverse sweep runs the adjoint alone (Rs), its checkpoint
    reverse sweep re-runs each segment with the surface from the node table (Fn) and then runs the
    same adjoint; the other models' checkpoint reverse sweeps re-run F and its tape adjoint R."""
    ops = lambda part: sum(bench.OPS["lv"][part].values())  # noqa: E731
    assert bench.kernel_ops("lv", "states", "reverse_sweep") == ops("Rs")
    assert bench.kernel_ops("lv", "checkpoint", "reverse_sweep") == ops("Fn") + ops("Rs")
    assert bench.kernel_ops("lv", "checkpoint", "forward_sweep") == ops("F")
    assert ops("Fn") == ops("F") + 2
    assert bench.kernel_ops("heston", "checkpoint", "reverse_sweep") == (
        sum(bench.OPS["heston"]["F"].values()) + sum(bench.OPS["heston"]["R"].values()))
    # stored states: 4 B per path-step and the final state once per 500 steps
    assert bench.kernel_bytes("lv", "states", 5, 500, 20)["reverse_sweep"] == 4.0 + 4.0 / 500


def test_kernel_sources_hash_covers_the_model_table():
    """The hash that keys measured traffic reads every file the kernels are built from."""
    files = bench.KERNEL_SOURCES + bench.MODEL_SOURCE["lv"]
    assert "mc_paths_lv.cuh" in files and "mc_paths.cuh" in files
    for f in files:
        assert os.path.exists(os.path.join(ROOT, "paper_1901_04200_gb300", "csrc", f)), f
