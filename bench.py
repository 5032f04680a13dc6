"""Benchmark: G + grad G path-steps/s of the two-step MC-AAD algorithm on GB300.

One step = one mc_value_and_grad call (forward sweep, E y / lambda / G, reverse
sweep, grad G).  The headline workload is the largest one: local volatility on a
bilinear 20 x 10 node surface, 2^22 paths x 500 steps (Delta = 0.01, 5y), 200
calls, 200 parameters, FP32 paths, FP64 sums.  The Heston workload (2^20 paths x
512 steps, 64 calls) is measured after it and reported under "workloads", and
the surrogate-assisted against plain calibration under "calibration".  The
metric is path-steps per second, P * S / (time per step); the roofline is the
per-pipe ALU issue bound of the dominant kernel, with its HBM fraction beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: rank r evaluates global paths [r P, (r+1) P) of
one estimator over N P paths (weak scaling); the two exchange steps of the
algorithm (E y partials before lambda, gradient partials after the reverse
sweep) are NCCL all-gathers of m + 1 and M + 1 numbers.
--impl reference times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
from dataclasses import replace
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "G+grad G path-steps/s (Heston FT, 2^20 paths x 512 steps, m=64, M=5)"
UNIT = "path-steps/s"

# Algorithmic ALU operations per path-step, counted from the formulas with
# ideal fusion (one FMA per a*b+c, one wide multiply for both halves of a
# 32x32 product, one three-input logic op, one MUFU per log2/sqrt/rsqrt/sin/cos):
#   "F"    one Euler step with its normals: Philox-4x32-10 (10 rounds x (2 wide
#          multiplies + 2 xor3) per block of 4 normals), uniforms (bit op + or,
#          FADD), Box-Muller (FP32 scale of log, clamp, shift, angle scalings,
#          products; MUFU lg2, sqrt, sin, cos per pair), the model step;
#   "step" the model step alone (normals given);
#   "R"    the adjoint of one step.
# Heston: F = 22 FP32 + 5 MUFU + 24 INT, step = 13 FP32 + rsqrt, R = 17 FP32.
# Local vol (one normal per step): F = Philox 10 INT + uniform 2 INT, half a
# Box-Muller pair (3.5 FP32 + 2 MUFU, 1 FADD), bilinear step 16 FP32 (cell, clamp,
# lerp, Euler); R = cell and lerp again 12, sigma-bar and weights 6, four row-adjoint
# FMAs 4, d sigma/dx 2 (shared-memory traffic not counted).
# Heston SLV: the Heston step plus the leverage lookup (10) and L^2 vdt, L sq (2);
# R adds the lookup again (10), L-bar and weights (4), four row-adjoint FMAs (4), the
# extra L factors (3) and dL/dx (2) to the Heston adjoint.
# Local vol from stored states ("Rs", the adjoint alone): the cell and lerp once 12, the step's
# sqrt(dt) z from its two end states (difference, drift and sigma^2 terms) 4 and one reciprocal,
# sigma-bar and weights 6, four row-adjoint FMAs 4, d sigma/dx 2.
OPS = {"heston": {"F": {"fp32": 22, "mufu": 5, "int": 24}, "step": {"fp32": 13, "mufu": 1}, "R": {"fp32": 17}},
       "lv": {"F": {"fp32": 20, "mufu": 2, "int": 12}, "step": {"fp32": 15}, "R": {"fp32": 23},
              "Rs": {"fp32": 28, "mufu": 1},
              # F with the surface from per-time-cell node pairs (two more FMAs per step)
              "Fn": {"fp32": 22, "mufu": 2, "int": 12}},
       "slv": {"F": {"fp32": 34, "mufu": 5, "int": 24}, "step": {"fp32": 25, "mufu": 1}, "R": {"fp32": 40}}}
# Forward-mode tangents of the Heston step (mc_value_and_grad_tangent), per path-step on top of
# F: shared factors 10 FP32 (the 1{v>0} dt select; the x and v coefficients of d vdt, 2 + 2; the
# explicit derivatives in kappa, xi, rho, 1 + 1 + 3) and per parameter j the chain d vdt_j, dx_j,
# dv_j (3), plus the explicit term for j < 4 (1): 10 + 5 x 3 + 4 = 29.
OPS_TANGENT = {"heston": {"fp32": 29}}
# What each path kernel runs per path-step, by storage mode.
KERNEL_PARTS = {"checkpoint": {"forward_sweep": ["F"], "reverse_sweep": ["F", "R"]},
                "normals": {"forward_sweep": ["F"], "reverse_sweep": ["step", "R"]},
                "full": {"forward_sweep": ["F"], "reverse_sweep": ["R"]},
                "states": {"forward_sweep": ["F"], "reverse_sweep": ["Rs"]}}
# Local vol's checkpoint reverse sweep re-runs each segment into shared memory and runs the
# stored-states adjoint over it.
KERNEL_PARTS_MODEL = {("lv", "checkpoint"): {"forward_sweep": ["F"], "reverse_sweep": ["Fn", "Rs"]}}
# State words, normals per step and tape words per step of each model.
DIMS = {"heston": (2, 2, 4), "lv": (1, 1, 2), "slv": (2, 2, 5)}


def kernel_ops(model, storage, kernel, kind=None):
    table = KERNEL_PARTS_MODEL.get((model, storage), KERNEL_PARTS[storage])
    parts = [OPS[model][q] for q in table[kernel]]
    return sum(v for d in parts for k, v in d.items() if kind is None or k == kind)


def kernel_bytes(model, storage, K, S, n_groups):
    """Algorithmic HBM bytes per path-step of the forward and reverse sweeps (FP32): each
    kernel writes (forward) or reads (reverse) the same stored data once."""
    sd, dz, nf = DIMS[model]
    if storage == "checkpoint":
        b = 4.0 * sd / K
    elif storage == "normals":
        b = 4.0 * sd / K + 4.0 * dz
    elif storage == "states":
        b = 4.0 * sd + 4.0 * sd / S  # the state before every step, and the final state
    else:
        b = 4.0 * nf + 4.0 * n_groups / S
    return {"forward_sweep": b, "reverse_sweep": b}


# DRAM bytes (read + write) per launch of a path kernel, from one ncu capture of a small case of
# the bench workload (profiles/), scaled to the full launch by its paths (the traffic is
# proportional to the paths; dirty lines still in L2 when the kernel ends are not counted, so a
# write-heavy kernel reads a little under its algorithmic bytes); reported only while the kernel
# sources' code (comments and layout aside) hashes to the captured version.  Key: (model,
# storage, K, paths per thread, kernel).
MEASURED_TRAFFIC = {
    # stored states, 2^20 of 2^22 paths (x 4): read 2.118220 GB + write 14.198 MB; read 0.536 MB + write 2.054537 GB
    ("lv", "states", 5, 4, "reverse_sweep"): {"bytes": 8529672000, "sources": "6263506f6fa9e9c9"},
    ("lv", "states", 5, 4, "forward_sweep"): {"bytes": 8218292000, "sources": "6263506f6fa9e9c9"},
    # checkpoints every 25 steps, two paths per thread (the recompute arm), 2^21 of 2^22 paths (x 2):
    # read 335.837 MB + write 39.257 MB; read 0.134 MB + write 326.978 MB (each 4-row checkpoint
    # group holds the two path slots and two padding rows, twice the algorithmic bytes)
    ("lv", "checkpoint", 25, 2, "reverse_sweep"): {"bytes": 750189000, "sources": "6263506f6fa9e9c9"},
    ("lv", "checkpoint", 25, 2, "forward_sweep"): {"bytes": 654223000, "sources": "6263506f6fa9e9c9"},
    # stored normals, 2^18 of 2^20 paths (x 4): read 1.208061 GB + write 0.248 MB; read 0.066 MB + write 1.148159 GB
    ("heston", "normals", 8, 2, "reverse_sweep"): {"bytes": 4833235000, "sources": "882aaba6c5a33637"},
    ("heston", "normals", 8, 2, "forward_sweep"): {"bytes": 4592903000, "sources": "882aaba6c5a33637"},
}
KERNEL_SOURCES = ["mc_common.cuh", "mc_paths.cuh"]
MODEL_SOURCE = {"gbm": ["mc_paths_gbm.cu"], "heston": ["mc_paths_heston.cu"],
                "lv": ["mc_paths_lv.cuh", "mc_paths_lv.cu"], "slv": ["mc_paths_slv.cu"]}


def code_tokens(src):
    """C++ source without its comments, whitespace runs collapsed: what the compiler sees, so a
    comment or layout edit keeps the hash (string and character literals are kept as written)."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_sources_hash(model="heston"):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES + MODEL_SOURCE[model]:
        with open(os.path.join(ROOT, "paper_1901_04200_gb300", "csrc", f)) as fh:
            h.update(code_tokens(fh.read()).encode())
    return h.hexdigest()[:16]


def measured_traffic(model, storage, k, ppt, kernel):
    rec = MEASURED_TRAFFIC.get((model, storage, k, ppt, kernel))
    if rec and rec["sources"] == kernel_sources_hash(model):
        return rec["bytes"]
    return None


# Per-SM thread-operation rates per clock of the pipes the path kernels use (the CUDA
# throughput table for compute capability 10.x): FP32 add/multiply/FMA 128, 32-bit integer and
# logical operations 64, special functions (lg2, sqrt, rsqrt, sin, cos) 16; instruction issue
# (four warp instructions) 128.
PIPE_RATES = {"issue": 128, "fp32": 128, "int": 64, "mufu": 16}


def kernel_rooflines(model, storage, K, ppt, P, S, n_groups, prof, issue_peak, hbm_peak, peak_src, n_sm,
                     sm_mhz_peak):
    """Per path kernel: achieved algorithmic ops and bytes per second (CUDA-event durations from
    the context's profile) against the issue-rate and HBM peaks, and each ALU pipe's fraction of
    its own rate (the per-pipe roofline: the pipe with the largest fraction binds); the roofline
    entry of the JSON line for the kernel with the longest time, with the bound of the larger of
    its issue and HBM fractions."""
    if storage == "tangent":
        f = OPS[model]["F"]
        table = {"tangent_sweep": ({"fp32": f["fp32"] + OPS_TANGENT[model]["fp32"], "int": f["int"],
                                    "mufu": f["mufu"]}, 0.0)}
    else:
        by = kernel_bytes(model, storage, K, S, n_groups)
        table = {k: ({kind: kernel_ops(model, storage, k, kind) for kind in ("fp32", "int", "mufu")}, by[k])
                 for k in ("forward_sweep", "reverse_sweep")}
    clock = n_sm * sm_mhz_peak * 1e6
    kern = {}
    for kname, (by_kind, byts) in table.items():
        ops = sum(by_kind.values())
        ms, n = prof[kname]
        t = ms / max(n, 1) * 1e-3
        a_ops, a_bytes = P * S * ops / t, P * S * byts / t
        pipes = {"issue": a_ops / (PIPE_RATES["issue"] * clock)}
        pipes.update({kind: P * S * v / t / (PIPE_RATES[kind] * clock) for kind, v in by_kind.items()})
        kern[kname] = {"ms": t * 1e3, "ops_per_path_step": ops, "bytes_per_path_step": byts,
                       "alu_frac": a_ops / issue_peak, "hbm_frac": a_bytes / hbm_peak,
                       "alu_tops": a_ops / 1e12, "hbm_gbs": a_bytes / 1e9,
                       "fp32_frac": P * S * by_kind["fp32"] / t / issue_peak,
                       "ops_by_pipe": by_kind, "pipe_fracs": pipes,
                       "alu_pipe_bound": max(pipes, key=pipes.get)}
    dom = max(kern, key=lambda k: kern[k]["ms"])
    d = kern[dom]
    # The path is ALU work (the per-pipe issue bound); the HBM fraction of the bytes the storage
    # mode moves is reported beside it.
    return {"bound": "alu",
            "achieved": d["alu_tops"], "peak": issue_peak / 1e12, "unit": "Tops/s", "frac": d["alu_frac"],
            "fp32_pipe_frac": d["pipe_fracs"]["fp32"], "pipe_fracs": d["pipe_fracs"],
            "alu_pipe_bound": d["alu_pipe_bound"],
            "hbm": {"achieved": d["hbm_gbs"], "peak": hbm_peak / 1e9, "unit": "GB/s", "frac": d["hbm_frac"],
                    "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs, %s)" % peak_src},
            "traffic": measured_traffic(model, storage, K, ppt, dom),
            "algorithmic_bytes": P * S * d["bytes_per_path_step"],
            "kernel": "%s (%s, %s, K=%d, %d paths/thread)" % (dom, model, storage if storage == "tangent"
                                                               else storage + " storage", K, ppt),
            "peak_basis": "SM issue rate 128 thread-ops/clk x %d SMs x %.0f MHz (%s max clock); each pipe "
                          "against its own rate in pipe_fracs" % (n_sm, sm_mhz_peak, peak_src),
            "kernels": kern}


def time_arm(ctx, step, steps, stream):
    """ms per step (CUDA events on the launching stream, 3 warm-up steps) and the context's
    per-kernel profile."""
    import torch
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    ctx.profile_begin(8 * steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, ctx.profile_end()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:  # no nvidia-smi: the line reports no clock samples
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.proc:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        out.update(sm_mhz=statistics.median(loaded) if loaded else None,
                   sm_max_mhz=max(mx) if mx else None, reasons=reasons, samples=len(rows))
        return out


def cpu_baseline(workload, n_paths, threads=None, keep=None):
    """The FP64 oracle's value_and_grad on a bounded sample of the same workload (paths
    [0, n_paths)); its (E y, G, grad G) go to keep[0] when a list is given."""
    import oracle
    oracle.build()
    threads = threads or os.cpu_count() or 1
    pb = workload.problem
    t0 = time.perf_counter()
    res = oracle.value_and_grad(pb, workload.theta, workload.C, n_paths, n_threads=threads)
    dt = time.perf_counter() - t0
    if keep is not None:
        keep.append(res)
    steps = pb.last_step
    return {"value": n_paths * steps / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d of the workload's paths x %d steps, FP64, value+grad, %.1f s wall" % (n_paths, steps, dt)}


def oracle_single_path_cost(workload, n_paths=512):
    """Cost(F) of the paper's table: seconds of the oracle's forward sweep per path on one core."""
    import oracle
    t0 = time.perf_counter()
    oracle.forward(workload.problem, workload.theta, n_paths, n_threads=1)
    return (time.perf_counter() - t0) / n_paths


def cpu_baseline_tape(pb, theta, C, n_paths):
    """The oracle's whole-program tape (FP64 numpy) on a bounded sample of the same program."""
    import oracle
    from oracle import tape as otape
    Z = oracle.normals_fill(pb.seed, 0, n_paths, 2 * pb.n_steps)
    t0 = time.perf_counter()
    otape.full_tape_value_and_grad(pb, theta, C, Z)
    dt = time.perf_counter() - t0
    return {"value": n_paths * pb.last_step / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d paths x %d steps through the oracle's whole-program tape (FP64 numpy), %.1f s wall"
                      % (n_paths, pb.last_step, dt)}


def cpu_baseline_surrogate(B=4096, steps=3):
    """The oracle MLP's differential-loss gradient and Adam step (FP64 numpy) at the same batch."""
    import numpy as np
    from oracle import mlp as omlp
    rng = np.random.default_rng(0)
    pv = omlp.flatten(omlp.init_params(0))
    X = rng.uniform(-1, 1, (B, 7))
    y = rng.uniform(0, 0.3, B)
    dy = rng.standard_normal((B, 5)) * 0.05
    m, v = np.zeros_like(pv), np.zeros_like(pv)
    t0 = time.perf_counter()
    for t in range(1, steps + 1):
        _, g, _, _ = omlp.loss_grad(omlp.unflatten(pv), X, y, dy, 1.0)
        pv, m, v = omlp.adam(pv, omlp.flatten(g), m, v, t, 1e-4)
    dt = (time.perf_counter() - t0) / steps
    return {"value": B / dt, "unit": "samples/s", "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": "%d training steps at batch %d, FP64 numpy (BLAS threads), %.2f s per step" % (steps, B, dt)}


def surrogate_flops_per_step(B=4096):
    """Dense FLOPs of the tensor-core GEMMs of one training step (2 M N K each,
    padded shapes as launched)."""
    H, KX, NX = 256, 64, 16
    f = 0
    f += 2 * B * H * KX + 3 * 2 * B * H * H          # F1..F4
    f += 3 * 2 * B * H * H + 2 * B * NX * H          # T4..T1
    f += 2 * B * H * KX + 3 * 2 * B * H * H          # R1..R4
    f += 3 * 2 * B * H * H                           # D4..D2
    f += 3 * 2 * H * H * (2 * B) + 2 * H * NX * (2 * B)  # G1..G4
    return f


def surrogate_step_bench(args, rank, world):
    """Training-step throughput of the pricing surrogate (differential loss + Adam), batch 4096."""
    import torch

    from paper_1901_04200_gb300 import surrogate
    B = 4096
    dev = torch.device("cuda", torch.cuda.current_device())
    g = torch.Generator(device=dev).manual_seed(rank)
    X = torch.rand((B, 7), device=dev, generator=g) * 2 - 1
    y = torch.rand(B, device=dev, generator=g) * 0.3
    dy = torch.randn((B, 5), device=dev, generator=g) * 0.05
    sur = surrogate.Surrogate(batch=B, device=dev)

    def step(t):
        sur.train_net.train_step(sur.params, X, y, dy, 1.0, sur.grads, sur.loss, sur.m, sur.v, t, lr=1e-4)

    for t in range(1, max(args.warmup, 3) + 1):
        step(t)
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for t in range(args.steps):
        step(100 + t)
    e1.record()
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    peaks, src = load_peaks()
    flops = surrogate_flops_per_step(B)
    if rank == 0:
        base = cpu_baseline_surrogate(B) if (world == 1 and not args.no_cpu_baseline) else None
        print(json.dumps({
            "cpu_baseline": base,
            "metric": "surrogate training samples/s (MLP 7->256x4->1, differential loss, batch 4096)",
            "value": world * B / (ms * 1e-3), "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "surrogate_mlp_train_step", "batch": B, "params": sur.params.numel()},
            "roofline": {"bound": "tensor", "achieved": flops / (ms * 1e-3) / 1e12,
                         "peak": float(peaks.get("bf16_tflops", 1900.0)), "unit": "TFLOP/s",
                         "frac": flops / (ms * 1e-3) / 1e12 / float(peaks.get("bf16_tflops", 1900.0)),
                         "traffic": None, "kernel": "all tcgen05 GEMMs of the step (whole-step time)",
                         "flops_per_step": flops, "peak_basis": "%s bf16 dense burst" % src},
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]}}))


def tape_bench(args, rank, world):
    """G and grad G of the Heston objective by the expected-backward tape (the whole program,
    expectations included, differentiated by the Appendix's rule)."""
    import numpy as np
    import torch

    from paper_1901_04200_gb300 import inputs, tape
    P = args.tape_paths
    w = inputs.heston_config(n_paths=P)
    pb, S = w.problem, w.problem.last_step
    prog, G = tape.heston_objective(pb, w.C)
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = tape.TapeContext(prog, G, 5, max_paths=P, device=dev, precision=args.tape_precision)
    compile_s, per_path = None, tape.plan(prog, G, 5, P, args.tape_precision)[4]  # interpreter HBM bytes per path
    if not args.tape_interpret:
        compile_s, per_path = ctx.compile(seg_nodes=args.tape_seg, recompute=args.tape_recompute,
                                          piece=args.tape_piece)  # untimed
    theta = torch.tensor(w.theta, dtype=torch.float64, device=dev)
    out = (torch.empty(1, dtype=torch.float64, device=dev), torch.empty(5, dtype=torch.float64, device=dev))
    path0 = rank * P

    def step():
        ctx.value_and_grad(theta, pb.seed, P, path0=path0, out=out)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    peaks, src = load_peaks()
    byts = P * per_path
    hbm = float(peaks["hbm_gbs"]) * 1e9
    if rank == 0:
        base = cpu_baseline_tape(pb, w.theta, w.C, 4096) if (world == 1 and not args.no_cpu_baseline) else None
        print(json.dumps({
            "cpu_baseline": base,
            "metric": "G+grad G path-steps/s by the expected-backward tape (Heston FT, %d paths x %d steps, "
                      "m=64, M=5)" % (P, S),
            "value": world * P * S / (ms * 1e-3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.tape_precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": "tape_" + w.name, "paths_per_gpu": P, "steps": S, "nodes": len(prog.nodes),
                       "precision": args.tape_precision + " per-path values and adjoints, fp64 sums",
                       "execution": "interpreter" if args.tape_interpret else
                                    "compiled (segments of %s nodes%s, %.1f s run-time compilation)"
                                    % (args.tape_seg or 384,
                                       (", backward recomputes in pieces of %d nodes" % args.tape_piece
                                        if args.tape_piece >= 2 else ", backward recomputes")
                                       if args.tape_recompute else "", compile_s),
                       "l2": "inputs larger than L2: %.1f GB of tape and adjoints" % (byts / 1e9)},
            "roofline": {"bound": "hbm", "achieved": byts / (ms * 1e-3) / 1e9, "peak": hbm / 1e9, "unit": "GB/s",
                         "frac": byts / (ms * 1e-3) / hbm, "traffic": None,
                         "algorithmic_bytes": byts, "bytes_per_path": per_path,
                         "kernel": "all tape kernels of the step (whole-step time)",
                         "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs, %s)" % src},
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]}}))


def calibration_experiment(cases, epochs=40, label_paths=1 << 16, n_theta=16384, label_steps_per_year=32):
    """Surrogate labels and training (the learned part), then Heston calibration to
    G < 1e-8 at 2^22 paths: surrogate-assisted vs plain MC-AAD descent from the same starts."""
    import numpy as np
    import torch

    from paper_1901_04200_gb300 import _lib, calibrate, inputs, surrogate
    pb = inputs.heston_config().problem
    # the labels' time grid (the maturities lie on every grid that divides a quarter year)
    pb_labels = pb if label_steps_per_year == 256 else inputs.heston_config(steps_per_year=label_steps_per_year).problem
    n_paths = label_paths
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, y, dy = surrogate.make_dataset(pb_labels, n_theta, n_paths)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    sur = surrogate.Surrogate(batch=4096)
    t_train = sur.train(X, y, dy, epochs=epochs, lr=2e-3)
    P, seed = 1 << 22, 777
    ctx = _lib.Context(pb, max_paths=P)
    plain, sur_rows = [], []
    for sd in range(cases):
        rng = np.random.default_rng(1000 + sd)
        theta_star, theta0 = inputs.draw_heston_theta(rng), inputs.draw_heston_theta(rng)
        C = ctx.forward(theta_star, seed, P).cpu().numpy()
        r = calibrate.run_experiment(ctx, sur, theta0, C, seed, P, tol=1e-8, max_evals=300)
        pl, mc = r["plain"], r["mc_phase"]
        plain.append({"converged": bool(pl.converged), "mc_evals": int(pl.evals), "seconds": float(pl.seconds),
                      "final_G": float(pl.G), "stopped": (getattr(pl, "messages", None) or [""])[-1][:80]})
        sur_rows.append({"converged": bool(mc.converged), "mc_evals": int(mc.evals),
                         "seconds_excl_training": float(r["surrogate_phase"].seconds + mc.seconds),
                         "final_G": float(mc.G)})
        if sd == 0:
            verified = calibrate.verify_by_mc(ctx, mc.theta, theta_star, seed + 1, P)
    n_samples = n_theta * pb.m

    one_off = t_data + t_train

    def summary(rows, seconds_key):
        ok = [x for x in rows if x["converged"]]
        secs = [x[seconds_key] for x in rows]
        return {"converged": len(ok) / len(rows), "n_converged": len(ok),
                "median_mc_evals_all": float(np.median([x["mc_evals"] for x in rows])),
                "median_seconds_all": float(np.median(secs)), "mean_seconds_all": float(np.mean(secs)),
                "median_mc_evals_converged": float(np.median([x["mc_evals"] for x in ok])) if ok else None,
                "median_seconds_converged": float(np.median([x[seconds_key] for x in ok])) if ok else None,
                "cases": rows}

    ps, ss = summary(plain, "seconds"), summary(sur_rows, "seconds_excl_training")
    ss["median_seconds_all_incl_one_off"] = ss["median_seconds_all"] + one_off
    ss["mean_seconds_all_incl_one_off"] = ss["mean_seconds_all"] + one_off
    gain = ps["mean_seconds_all"] - ss["mean_seconds_all"]
    return {"tol": 1e-8, "paths": P, "cases": cases, "start": "theta*, theta0 drawn in the Heston box (Feller)",
            "all_cases_note": "medians and means over all cases; a case that stops before G < tol (evaluation "
                              "cap or a stalled line search) counts at its stopping time, a lower bound on its "
                              "time to tolerance",
            "labels": {"samples": n_samples, "paths_per_sample": n_paths, "steps": int(pb_labels.n_steps),
                       "seconds": t_data},
            "training": {"epochs": epochs, "batch": 4096, "seconds": t_train,
                         "samples_per_s": epochs * (n_samples // 4096) * 4096 / t_train},
            "plain": dict(ps, method="L-BFGS-B on MC-AAD G and grad G, restarts, 300 evaluations"),
            "surrogate": dict(ss, one_off_seconds=one_off,
                              method="L-BFGS-B on the surrogate, then MC-AAD steps with its Gauss-Newton metric"),
            "break_even_recalibrations": (one_off / gain) if gain > 0 else None,
            "break_even_note": "calibrations after which the one-off labels + training cost is repaid: one-off "
                               "seconds / (plain - surrogate mean seconds per calibration, all cases)",
            "verified_by_mc": dict(verified, case=0, note="prices at the calibrated theta vs theta*, fresh seed")}


def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args):
    """The oracle timed on the host cores, as the reference arm."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1901_04200_gb300 import inputs
    w = inputs.heston_config()
    # size the per-step sample from a short probe of the host's rate, so the whole run
    # (warm-ups at an eighth of the sample) takes about --ref-seconds
    rate = cpu_baseline(w, 2048)["value"]
    budget_steps = args.steps + args.warmup / 8.0
    n = int(rate * args.ref_seconds / max(budget_steps, 1.0) / w.problem.last_step) // 1024 * 1024
    n = max(1024, min(n, args.ref_paths))
    for _ in range(args.warmup):
        cpu_baseline(w, max(n // 8, 256))
    vals = [cpu_baseline(w, n) for _ in range(args.steps)]
    v = statistics.median(x["value"] for x in vals)
    ms = w.problem.last_step * w.n_paths / v * 1e3
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name, "paths": w.n_paths, "steps": w.problem.last_step,
                       "sample_paths_per_step": n},
            "cpu_baseline": dict(vals[0], value=v),
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


WORKLOAD_TITLES = {"lv": "local vol, 2^22 paths x 500 steps, m=200, M=200",
                   "heston": "Heston FT, 2^20 paths x 512 steps, m=64, M=5",
                   "slv": "Heston SLV, 2^20 paths x 512 steps, m=64, M=95"}


def make_workload(model, args):
    from paper_1901_04200_gb300 import inputs
    if model == "lv":
        w = inputs.lv_config(n_paths=args.paths or (1 << 22))
    elif model == "slv":
        w = inputs.slv_config(n_paths=args.paths or (1 << 20))
    else:
        w = inputs.heston_config(n_paths=args.paths or (1 << 20))
    return w


def oracle_precision(ctx, w, theta, C, keep, n_cpu):
    """The FP32 path's error against the FP64 oracle, per result, on the same paths."""
    import numpy as np
    Ey_o, G_o, g_o = keep
    Gs, gs, Eys = (x.cpu().numpy() for x in ctx.value_and_grad(theta, C, w.problem.seed, n_cpu))
    return {"sample": "paths [0, %d) of the workload: GPU FP32 paths and FP64 sums vs the FP64 oracle" % n_cpu,
            "Ey_max_rel": float(np.max(np.abs(Eys - Ey_o)) / np.max(np.abs(Ey_o))),
            "G_rel": float(abs(Gs[0] - G_o) / abs(G_o)),
            "grad_normwise_rel": float(np.max(np.abs(gs - g_o)) / np.max(np.abs(g_o)))}


def run_path_workload(model, args, rank, world, local, headline):
    """Times mc_value_and_grad on one path workload: the device-timed steps (inputs resident),
    the end-to-end steps through host buffers, and (one GPU) the comparison arms.  Returns the
    JSON fields of that workload."""
    import numpy as np
    import torch

    from paper_1901_04200_gb300 import _lib

    w = make_workload(model, args)
    if headline and (args.ppt or args.ckpt):
        w.problem.paths_per_thread = args.ppt or w.problem.paths_per_thread
        w.problem.ckpt_every = args.ckpt or w.problem.ckpt_every
    w.problem.storage = args.storage if headline else "auto"
    pb, P, S = w.problem, w.n_paths, w.problem.last_step
    path0 = rank * P
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = _lib.Context(pb, max_paths=P, device=dev)
    theta = torch.tensor(w.theta, dtype=torch.float64, device=dev)
    C = torch.tensor(w.C, dtype=torch.float64, device=dev)
    out = (torch.empty(1, dtype=torch.float64, device=dev), torch.empty(ctx.M, dtype=torch.float64, device=dev),
           torch.empty(ctx.m, dtype=torch.float64, device=dev))
    seed = pb.seed
    stream = torch.cuda.current_stream()
    steps = args.steps if headline else max(3, args.steps // 2)

    if world > 1:
        from paper_1901_04200_gb300.sharding import sharded_value_and_grad

        def step():
            sharded_value_and_grad(lambda: ctx.forward(theta, seed, P, path0=path0, keep=True), ctx.vjp, C, P)
    else:
        def step():
            ctx.value_and_grad(theta, C, seed, P, path0=path0, out=out)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # ---------------- device-timed region (inputs resident in HBM)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    ctx.profile_begin(8 * steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    prof = ctx.profile_end()
    ms_total = e0.elapsed_time(e1)
    # ---------------- end to end: host buffers in, host results out, every step
    th_h = torch.tensor(w.theta, dtype=torch.float64).pin_memory()
    C_h = torch.tensor(w.C, dtype=torch.float64).pin_memory()
    res_h = torch.empty(1 + ctx.M + ctx.m, dtype=torch.float64).pin_memory()
    th_d = torch.empty_like(theta)
    C_d = torch.empty_like(C)
    res_d = torch.empty(1 + ctx.M + ctx.m, dtype=torch.float64, device=dev)
    outs = (res_d[0:1], res_d[1:1 + ctx.M], res_d[1 + ctx.M:])

    def e2e_step():
        th_d.copy_(th_h, non_blocking=True)
        C_d.copy_(C_h, non_blocking=True)
        if world > 1:
            Ey_g, G_g, g_g = sharded_value_and_grad(lambda: ctx.forward(th_d, seed, P, path0=path0, keep=True),
                                                    ctx.vjp, C_d, P)
            res_d[0:1].copy_(G_g.reshape(1))
            res_d[1:1 + ctx.M].copy_(g_g)
            res_d[1 + ctx.M:].copy_(Ey_g)
        else:
            ctx.value_and_grad(th_d, C_d, seed, P, path0=path0, out=outs)
        res_h.copy_(res_d, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(steps):
        e2e_step()
        torch.cuda.current_stream().synchronize()
    e2e_s = time.perf_counter() - t0
    clk = clocks.stop()

    ms_step = max_over_ranks(ms_total / steps, world)
    e2e_ms = max_over_ranks(e2e_s * 1e3 / steps, world)
    value = world * P * S / (ms_step * 1e-3)
    peaks, peak_src = load_peaks()
    sm_mhz_peak = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    issue_peak = 128 * n_sm * sm_mhz_peak * 1e6  # thread-ops/s: 4 warp instructions per SM per clock
    hbm_peak = float(peaks["hbm_gbs"]) * 1e9
    storage = ctx.storage
    K = pb.ckpt_every
    ppt = pb.paths_per_thread or 2
    n_groups = len(set(np.asarray(pb.mat_step).tolist()))
    bytes_ps = kernel_bytes(model, storage, K, S, n_groups)
    roof_args = (P, S, n_groups)
    peak_args = (issue_peak, hbm_peak, peak_src, n_sm, sm_mhz_peak)
    roofline = kernel_rooflines(model, storage, K, ppt, *roof_args, prof, *peak_args)
    res = {
        "metric": "G+grad G path-steps/s (%s)" % WORKLOAD_TITLES[model],
        "value": value, "unit": UNIT, "ms_per_step": ms_step, "steps": steps,
        "config": {"workload": w.name, "paths_per_gpu": P, "steps": S, "instruments": pb.m, "params": pb.n_params,
                   "storage": storage, "ckpt_every": pb.ckpt_every, "paths_per_thread": ppt,
                   "precision": "fp32 paths, fp64 sums",
                   "l2": "inputs larger than L2: %.0f MB stored and re-read per step" %
                         (P * S * bytes_ps["forward_sweep"] / 1e6)},
        "roofline": roofline,
        "kernels_ms_per_step": {k: v[0] / steps for k, v in prof.items() if v[1]},
        "gpu_launches": sum(n for _, n in prof.values()),
        "e2e": {"value": world * P * S / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": 8 * (ctx.M + ctx.m), "d2h_bytes_per_step": 8 * (1 + ctx.M + ctx.m)},
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
    }
    if world == 1 and not args.no_arms:
        # the same workload by the design that regenerates the normals and recomputes every
        # segment (checkpoints only; local vol at the 25-step interval the workload names), and
        # for Heston by forward-mode tangents (no reverse sweep)
        if storage != "checkpoint":
            K_r, ppt_r = (25, 2) if model == "lv" else (K, pb.paths_per_thread)
            pb_r = replace(pb, storage="checkpoint", ckpt_every=K_r, paths_per_thread=ppt_r)
            ctx_r = _lib.Context(pb_r, max_paths=P, device=dev)
            ms_r, prof_r = time_arm(ctx_r, lambda: ctx_r.value_and_grad(theta, C, seed, P, path0=path0, out=out),
                                    steps, stream)
            res["recompute_arm"] = {"ms_per_step": ms_r, "value": P * S / (ms_r * 1e-3), "unit": UNIT,
                                    "storage": "checkpoint", "ckpt_every": K_r, "paths_per_thread": ppt_r or 2,
                                    "roofline": kernel_rooflines(model, "checkpoint", K_r, ppt_r or 2, *roof_args,
                                                                 prof_r, *peak_args)}
            del ctx_r
        if model == "heston":
            ms_t, prof_t = time_arm(ctx, lambda: ctx.value_and_grad_tangent(theta, C, seed, P, path0=path0,
                                                                            out=out), steps, stream)
            res["tangent_arm"] = {"ms_per_step": ms_t, "value": P * S / (ms_t * 1e-3), "unit": UNIT,
                                  "method": "forward-mode tangents, grad G = J^T lambda",
                                  "roofline": kernel_rooflines(model, "tangent", K, 1, *roof_args, prof_t,
                                                               *peak_args)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_cpu = args.cpu_paths or (1 << 18 if model == "lv" else 1 << 17)
        keep = []
        res["cpu_baseline"] = cpu_baseline(w, n_cpu, keep=keep)
        res["precision"] = oracle_precision(ctx, w, theta, C, keep[0], n_cpu)
        # the GPU analogues of the paper's cost table (eq. 1311A with c = one GPU)
        cost_f = oracle_single_path_cost(w)
        kf = roofline["kernels"]["forward_sweep"]["ms"] * 1e-3
        kr = roofline["kernels"]["reverse_sweep"]["ms"] * 1e-3
        res["paper_table"] = {"cost_F_one_core_s": cost_f, "K_F_over_c": kf / (P * cost_f),
                              "K_R_over_c": kr / (P * cost_f), "cost_G_over_P_cost_F": ms_step * 1e-3 / (P * cost_f),
                              "note": "Cost(F): the oracle's FP64 forward sweep of one path on one host core"}
    del ctx
    torch.cuda.empty_cache()
    return res


def run_reference(args):
    """The oracle timed on the host cores, as the reference arm: each step one bounded sample of
    the headline workload's paths (the whole workload would take hours on the host)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = make_workload(args.workload, args)
    S = w.problem.last_step
    # size the per-step sample from a short probe of the host's rate, so the whole run
    # (warm-ups at an eighth of the sample) takes about --ref-seconds
    rate = cpu_baseline(w, 2048)["value"]
    budget_steps = args.steps + args.warmup / 8.0
    n = int(rate * args.ref_seconds / max(budget_steps, 1.0) / S) // 1024 * 1024
    n = max(1024, min(n, args.ref_paths))
    for _ in range(args.warmup):
        cpu_baseline(w, max(n // 8, 256))
    vals = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        vals.append(cpu_baseline(w, n))
        vals[-1]["wall_s"] = time.perf_counter() - t0
    v = statistics.median(x["value"] for x in vals)
    line = {"metric": "G+grad G path-steps/s (%s)" % WORKLOAD_TITLES[args.workload], "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.median(x["wall_s"] for x in vals) * 1e3,
            "ms_per_step_is": "the timed sample step (%d of the workload's %d paths)" % (n, w.n_paths),
            "full_workload_ms_per_step_extrapolated": S * w.n_paths / v * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name, "paths_per_gpu": w.n_paths, "steps": S, "instruments": w.problem.m,
                       "params": w.problem.n_params},
            "sample_paths_per_step": n,
            "cpu_baseline": dict(vals[0], value=v),
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--paths", type=int, default=0, help="paths per GPU (0 = the workload's own count)")
    ap.add_argument("--cpu-paths", type=int, default=0,
                    help="oracle sample for cpu_baseline and precision (0 = 2^18 local vol, 2^17 Heston)")
    ap.add_argument("--ref-paths", type=int, default=1 << 15, help="--impl reference: largest sample per step")
    ap.add_argument("--ref-seconds", type=float, default=90.0,
                    help="--impl reference: host time the whole run is sized for")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ppt", type=int, default=0, help="paths per GPU thread (0 = library default)")
    ap.add_argument("--tape-paths", type=int, default=1 << 18, help="paths of the --workload tape run")
    ap.add_argument("--tape-precision", default="fp32", choices=["fp32", "fp64"],
                    help="per-path values and adjoints of the --workload tape run")
    ap.add_argument("--tape-interpret", action="store_true",
                    help="--workload tape: run the interpreter instead of the compiled program")
    ap.add_argument("--tape-piece", type=int, default=256,
                    help="--workload tape: backward recompute in pieces of this many nodes (0: whole segments); "
                         "256 measured fastest with 768-node segments")
    ap.add_argument("--tape-seg", type=int, default=768,
                    help="--workload tape: nodes per compiled segment (0 = library default, 384)")
    ap.add_argument("--tape-store", dest="tape_recompute", action="store_false",
                    help="--workload tape: compiled backward kernels read every value they need from the "
                         "tape; by default they re-run their segment's forward, which measured faster")
    ap.add_argument("--workload", default="lv", choices=["lv", "heston", "slv", "surrogate", "tape"],
                    help="lv (the largest workload, 2^22 x 500 local vol: the headline), heston (2^20 x 512), "
                         "slv (Heston SLV), surrogate (one differential-loss training step of the pricing "
                         "network) or tape (the expected-backward tape)")
    ap.add_argument("--also", default="heston",
                    help="comma-separated path workloads measured after the headline, reported under "
                         "'workloads' ('' for none)")
    ap.add_argument("--no-calibration", action="store_true", help="skip the surrogate vs plain calibration")
    ap.add_argument("--no-arms", action="store_true",
                    help="skip the recompute and forward-mode comparison arms")
    ap.add_argument("--calib-cases", type=int, default=16)
    ap.add_argument("--calib-epochs", type=int, default=40, help="surrogate training epochs")
    ap.add_argument("--calib-label-paths", type=int, default=1 << 16, help="MC paths per surrogate label")
    ap.add_argument("--calib-label-steps-per-year", type=int, default=32,
                    help="time grid of the surrogate labels (the calibration itself runs at 256; 32 measured "
                         "as effective as 256 for the surrogate phase at a third of the label time)")
    ap.add_argument("--calib-thetas", type=int, default=16384,
                    help="parameter draws for the surrogate labels (64 instruments each)")
    ap.add_argument("--ckpt", type=int, default=0, help="checkpoint interval (0 = workload default)")
    ap.add_argument("--storage", default="auto", choices=["auto", "checkpoint", "normals", "full", "states"],
                    help="what the reverse sweep reads: checkpoints (re-run with regenerated normals), "
                         "checkpoints and stored normals, the whole stored tape, or the library's choice")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.workload not in WORKLOAD_TITLES:
            args.workload = "lv"
        return run_reference(args)

    from paper_1901_04200_gb300 import build as _build

    rank, world, local = dist_setup(args.gpus)
    if rank == 0:
        _build.build()
    barrier(world)
    if args.workload == "surrogate":
        return surrogate_step_bench(args, rank, world)
    if args.workload == "tape":
        return tape_bench(args, rank, world)
    head = run_path_workload(args.workload, args, rank, world, local, headline=True)
    line = {}
    if rank == 0:
        line = {"metric": head.pop("metric"), "value": head.pop("value"), "unit": UNIT, "n_gpus": world,
                "steps": head.pop("steps"), "warmup": max(args.warmup, 3), "ms_per_step": head.pop("ms_per_step"),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic"}
        line.update(head)
    others = [m for m in args.also.split(",") if m and m != args.workload] if not args.paths else []
    if others:
        line["workloads"] = {}
    for m in others:
        r = run_path_workload(m, args, rank, world, local, headline=False)
        if rank == 0:
            line["workloads"][r["config"]["workload"]] = r
    if rank == 0 and not args.no_calibration and world == 1:
        line["calibration"] = calibration_experiment(args.calib_cases, args.calib_epochs, args.calib_label_paths,
                                                     args.calib_thetas, args.calib_label_steps_per_year)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
