#!/usr/bin/env python
"""Throughput of the conservative spectral collision step on GB300.

One bench "step" is one Strang-split time step of the 1-D wall boundary-layer
problem (transport dt/2, Heun collision dt = two evaluations of the collision
operator with the conservation projection, transport dt/2): every step of the
hot path.  The metric is nominal pair-updates per second,
    (collision evaluations) x (cells) x N^6 / time,
the count the paper's N^6 cost model uses.

Default workload (N=1): N = 16, L = 6, lambda = 1, 128 cells of width
min(dx0 1.05^j, 0.5), dx0 = 1/8, wall at T_w = 1.5 against a unit Maxwellian
gas, dt = 0.01; transforms and convolution in float, weights, projection,
transport and state in double.  Secondary objects in the same line: the same
step in double precision ("fp64") and the N = 32, 256-cell workload ("n32").

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs its own replica (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Q(f) pair-updates/s FP32+FP64-cons vs FP64 at N=16/32, err; serve p50/p99"
UNIT = "pair-updates/s"
L_BOX = 6.0
LAM = 1.0
DT = 0.01
WALL_T = 1.5
WORKLOADS = {
    "wall16": dict(N=16, ncells=128),
    "wall32": dict(N=32, ncells=256),
}
MAX_SM_MHZ = 2070.0
# DRAM bytes (read + write) per convolution launch from ncu captures of the
# current kernel (profiles/), keyed by (N, cells); None where not captured
TRAFFIC = {(16, 128): 18415616, (32, 256): 3028994304 + 67706112}
SMS = 152
FP32_LANES = 128


def describe(wl: str) -> str:
    p = WORKLOADS[wl]
    return (f"1-D wall boundary layer, N={p['N']}, L=6, lambda=1, {p['ncells']} cells "
            f"(dx_j=min(0.125*1.05^j,0.5)), T_w=1.5 vs unit Maxwellian, dt=0.01, one Strang step "
            f"(2 collision evaluations + 4 transport stages)")


def tiles_total(N: int) -> int:
    h = N // 2
    tot = 0
    for k1 in range(N):
        for k2 in range(N):
            v1 = min(k1 + h, N - 1) - max(0, k1 + h - N + 1) + 1
            v2 = min(k2 + h, N - 1) - max(0, k2 + h - N + 1) + 1
            tot += (v1 * v2 + 1) // 2
    return tot


def unique_pairs_per_cell(N: int) -> int:
    """Pairs the symmetrised half-tile convolution visits per cell per evaluation."""
    return tiles_total(N) * (3 * N * N // 4)


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # the raw samples go to $CS_CLOCKS_DIR when set (kept), else to a temporary folder
        folder = os.environ.get("CS_CLOCKS_DIR") or tempfile.mkdtemp(prefix="cs_clocks_")
        self.path = os.path.join(folder, f"clocks_rank{index}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names[1:], parts[5:9]):
                if val.lower() in ("active", "0x1") or val == "1":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def conv_ms_in_mode(api, torch, h, f, n, mode, reps=5):
    """Average convolution launch (ms) of cs_collide on n cells with the
    weights read from the stored tiles (mode 1) or rebuilt from the radius
    tables (mode 2), the launch shape left as tuned."""
    keep = api.cs_tune_get(h.ptr, api.CS_TUNE_WEIGHTS)
    api.cs_tune(h.ptr, api.CS_TUNE_WEIGHTS, mode)
    q = torch.empty_like(f)
    api.cs_collide(h.ptr, f, n, 1.0, q, 1)
    api.cs_profile(h.ptr, True)
    api.cs_profile_read(h.ptr, reset=True)
    for _ in range(reps):
        api.cs_collide(h.ptr, f, n, 1.0, q, 1)
    torch.cuda.synchronize()
    p = api.cs_profile_read(h.ptr, reset=True)
    api.cs_profile(h.ptr, False)
    api.cs_tune(h.ptr, api.CS_TUNE_WEIGHTS, keep)
    return p["convolve"][0] / max(p["convolve"][1], 1)


WEIGHT_MODES = {0: "automatic", 1: "stored tiles", 2: "radius tables"}


def max_over_ranks(x: float, device) -> float:
    """The largest of every rank's x (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- our arm
def make_state(api, inputs, torch, N, ncells, device):
    dx = inputs.wall_grid(ncells)
    f0 = inputs.wall_initial(N, L_BOX, ncells)
    far = inputs.maxwellian(N, L_BOX, 1.0, (0.0, 0.0, 0.0), 1.0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    return f0, t(f0), t(dx), t(far)


def time_steps(torch, h, fd, dxd, fard, K, W, flush, profile=False):
    """W untimed warm-up steps, then K steps each timed with CUDA events on the
    current stream, the L2 flushed before each; returns the summed device ms."""
    from paper_1301_4195_gb300 import api
    for _ in range(W):
        h.step(fd, dxd, fard, WALL_T, (0.0, 0.0, 0.0), DT, nsteps=1)
    torch.cuda.synchronize()
    if profile:
        api.cs_profile(h.ptr, True)
        api.cs_profile_read(h.ptr, reset=True)
    evs = []
    for _ in range(K):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        h.step(fd, dxd, fard, WALL_T, (0.0, 0.0, 0.0), DT, nsteps=1)
        b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    total = sum(a.elapsed_time(b) for a, b in evs)
    prof = None
    if profile:
        prof = api.cs_profile_read(h.ptr, reset=True)
        api.cs_profile(h.ptr, False)
    return total, prof


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1301_4195_gb300 import api, build, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.gpus > 1 and world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} needs torchrun with {args.gpus} ranks (WORLD_SIZE={world})")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=device)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    build.build()

    wl = WORKLOADS[args.workload]
    N, ncells = wl["N"], (args.cells or wl["ncells"])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)  # > L2 (129 MB)

    h32 = api.Handle(N, L_BOX, LAM, "fp32")
    h32.reserve(ncells)
    if args.tune:  # fixed launch choices (profiling runs: timings under a profiler would mislead the autotuner)
        for param, v in zip((api.CS_TUNE_GROUPS_PER_CTA, api.CS_TUNE_CTAS_PER_SM, api.CS_TUNE_SPLIT,
                             api.CS_TUNE_WEIGHTS), (int(x) for x in args.tune.split(","))):
            api.cs_tune(h32.ptr, param, v)
        tuned_ms = None
    else:
        tuned_ms = api.cs_autotune(h32.ptr, ncells)  # launch shape of the convolution (outside the timed region)
    f0, fd, dxd, fard = make_state(api, inputs, torch, N, ncells, device)

    # warm-up + timed region (barrier and synchronize on both sides, max over ranks)
    for _ in range(args.warmup):
        h32.step(fd, dxd, fard, WALL_T, (0.0, 0.0, 0.0), DT, nsteps=1)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # timed region: K steps (CUDA graph replays), barrier + synchronize on both
    # sides, max over ranks; clocks sampled throughout
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    api.cs_launch_count(reset=True)
    plain_ms, _ = time_steps(torch, h32, fd, dxd, fard, args.steps, 0, flush, profile=False)
    launches = api.cs_launch_count(reset=True)  # kernels of ours in the timed steps (graph nodes x replays)
    barrier()
    plain_ms = max_over_ranks(plain_ms, device)
    # the same K steps again with per-stage events (direct launches) for the
    # stage times and the convolution's average launch duration
    _, prof = time_steps(torch, h32, fd, dxd, fard, args.steps, 0, flush, profile=True)
    barrier()
    clk = clocks.stop()
    ms_step = plain_ms / args.steps
    evals_per_step = 2
    pairs_step = evals_per_step * ncells * N ** 6
    value = world * pairs_step / (ms_step * 1e-3)

    # roofline of the dominant kernel (the convolution), timed live above:
    # FP32 FMA-pipe lane operations, 6 per (pair, cell) (one FMUL2 + two FFMA2), against
    # 152 SMs x 128 lanes x 2070 MHz; flops (10 per pair) reported beside it
    conv_ms, conv_n = prof["convolve"]
    conv_avg = conv_ms / max(conv_n, 1)
    pair_cells = unique_pairs_per_cell(N) * ncells
    flops_launch = 10.0 * pair_cells
    peak_tflops = SMS * FP32_LANES * 2 * MAX_SM_MHZ * 1e6 / 1e12
    peak_tops = SMS * FP32_LANES * MAX_SM_MHZ * 1e6 / 1e12
    achieved_ops = 6.0 * pair_cells / (conv_avg * 1e-3) / 1e12
    achieved = flops_launch / (conv_avg * 1e-3) / 1e12
    step_stage_ms = {k: v[0] / args.steps for k, v in prof.items()}

    # e2e: host state in pinned memory, copied in and out around the public call every step
    fh = torch.from_numpy(f0.copy()).pin_memory()
    fdev = torch.empty_like(fd)
    for _ in range(2):
        fdev.copy_(fh, non_blocking=True)
        h32.step(fdev, dxd, fard, WALL_T, (0.0, 0.0, 0.0), DT, nsteps=1)
        fh.copy_(fdev, non_blocking=True)
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fdev.copy_(fh, non_blocking=True)
        h32.step(fdev, dxd, fard, WALL_T, (0.0, 0.0, 0.0), DT, nsteps=1)
        fh.copy_(fdev, non_blocking=True)
        b.record()
        b.synchronize()
        e2e_ms += a.elapsed_time(b)
    e2e_ms = max_over_ranks(e2e_ms, device)
    state_bytes = ncells * N ** 3 * 8
    e2e = {"value": world * pairs_step * args.steps / (e2e_ms * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes}

    # measured pipe peaks beside the derived one (lane operations per second)
    probe = {"ffma_tlane_ops": api.cs_fma_probe(0) / 1e12, "ffma2_tlane_ops": api.cs_fma_probe(1) / 1e12,
             "dfma_tlane_ops": api.cs_fma_probe(2) / 1e12}
    probe["frac_of_best_fp32_probe"] = achieved_ops / max(probe["ffma_tlane_ops"], probe["ffma2_tlane_ops"])

    # the operator alone (t_Q = forward transform + convolution + inverse +
    # projection, one cs_collide on the workload's state), graph-free direct launches
    qd = torch.empty_like(fd)
    for _ in range(3):
        api.cs_collide(h32.ptr, fd, ncells, 1.0, qd, 1)
    torch.cuda.synchronize()
    ta, tb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nq = 20
    ta.record()
    for _ in range(nq):
        api.cs_collide(h32.ptr, fd, ncells, 1.0, qd, 1)
    tb.record()
    tb.synchronize()
    tq = ta.elapsed_time(tb) / nq
    q_eval = {"ms_per_evaluation": tq, "value": world * ncells * N ** 6 / (tq * 1e-3), "unit": UNIT,
              "note": "one collision evaluation Q(f) of the workload's cells (t_Q: transforms, convolution, "
                      "projection), L2 not flushed between evaluations"}

    # store versus recompute: the convolution with stored weight tiles and with
    # tiles rebuilt from the radius tables (the autotuner keeps the faster)
    weights = {"chosen": WEIGHT_MODES[api.cs_tune_get(h32.ptr, api.CS_TUNE_WEIGHTS)],
               "stored_conv_ms": conv_ms_in_mode(api, torch, h32, fd, ncells, 1),
               "radius_conv_ms": conv_ms_in_mode(api, torch, h32, fd, ncells, 2)}

    # the same step in double precision (the plain FP64 GPU form)
    h64, fp64 = None, None
    if not args.skip_fp64:
        h64 = api.Handle(N, L_BOX, LAM, "fp64")
        h64.reserve(ncells)
        _, fd64, _, _ = make_state(api, inputs, torch, N, ncells, device)
        k64 = max(2, min(args.steps, 5))
        ms64, _ = time_steps(torch, h64, fd64, dxd, fard, k64, 1, flush)
        fp64 = {"value": pairs_step / (ms64 / k64 * 1e-3), "ms_per_step": ms64 / k64}

    # the N = 32, 256-cell workload (secondary)
    n32 = None
    if args.workload == "wall16" and not args.skip_n32:
        N2, nc2 = WORKLOADS["wall32"]["N"], WORKLOADS["wall32"]["ncells"]
        hb = api.Handle(N2, L_BOX, LAM, "fp32")
        hb.reserve(nc2)
        api.cs_autotune(hb.ptr, nc2)
        _, fb, dxb, farb = make_state(api, inputs, torch, N2, nc2, device)
        kb = max(2, min(args.steps, 4))
        msb, profb = time_steps(torch, hb, fb, dxb, farb, kb, 1, flush, profile=True)
        cms, cn = profb["convolve"]
        cavg = cms / max(cn, 1)
        fl2 = 10.0 * unique_pairs_per_cell(N2) * nc2
        pc2 = unique_pairs_per_cell(N2) * nc2
        n32 = {"workload": describe("wall32"), "value": 2 * nc2 * N2 ** 6 / (msb / kb * 1e-3),
               "ms_per_step": msb / kb, "conv_ms": cavg,
               "weights": {"chosen": WEIGHT_MODES[api.cs_tune_get(hb.ptr, api.CS_TUNE_WEIGHTS)],
                           "stored_conv_ms": cavg, "radius_conv_ms": conv_ms_in_mode(api, torch, hb, fb, nc2, 2, 2)},
               "roofline": {"bound": "alu", "achieved": 6.0 * pc2 / (cavg * 1e-3) / 1e12, "peak": peak_tops,
                            "unit": "T FP32 FMA-pipe lane-ops/s",
                            "frac": 6.0 * pc2 / (cavg * 1e-3) / 1e12 / peak_tops,
                            "tflops": fl2 / (cavg * 1e-3) / 1e12,
                            "flop_frac": fl2 / (cavg * 1e-3) / 1e12 / peak_tflops,
                            "traffic": TRAFFIC.get((N2, nc2))}}
        hb.close()

    # N = 64 (the largest grid; a 40 GB float weight table): one collision
    # evaluation of 32 random-mixture cells, and its convolution's roofline
    n64 = None
    if args.workload == "wall16" and not args.skip_n64:
        N6, nc6 = 64, 32
        t0 = time.perf_counter()
        h6 = api.Handle(N6, L_BOX, LAM, "fp32")
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        h6.reserve(nc6)
        f6 = torch.from_numpy(inputs.random_mixture_cells(N6, L_BOX, nc6, first_id=7000)).to(device)
        q6 = torch.empty_like(f6)
        api.cs_collide(h6.ptr, f6, nc6, 1.0, q6, 1)
        torch.cuda.synchronize()
        api.cs_profile(h6.ptr, True)
        api.cs_profile_read(h6.ptr, reset=True)
        reps6 = 2
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps6):
            api.cs_collide(h6.ptr, f6, nc6, 1.0, q6, 1)
        b.record()
        b.synchronize()
        p6 = api.cs_profile_read(h6.ptr, reset=True)
        api.cs_profile(h6.ptr, False)
        ms6 = a.elapsed_time(b) / reps6
        c6 = p6["convolve"][0] / max(p6["convolve"][1], 1)
        pc6 = unique_pairs_per_cell(N6) * nc6
        n64 = {"workload": f"one collision evaluation, N={N6}, {nc6} random-mixture cells (L=6, lambda=1)",
               "ms_per_evaluation": ms6, "value": nc6 * N6 ** 6 / (ms6 * 1e-3), "unit": UNIT,
               "weights_build_s": build_s, "weight_bytes": h6.weight_bytes(), "conv_ms": c6,
               "roofline": {"bound": "alu", "achieved": 6.0 * pc6 / (c6 * 1e-3) / 1e12, "peak": peak_tops,
                            "unit": "T FP32 FMA-pipe lane-ops/s",
                            "frac": 6.0 * pc6 / (c6 * 1e-3) / 1e12 / peak_tops, "traffic": None}}
        h6.close()
        # the same evaluation from a handle holding the radius tables only
        t0 = time.perf_counter()
        h6 = api.Handle(N6, L_BOX, LAM, "fp32-radius")
        torch.cuda.synchronize()
        n64["radius_only"] = {"weights_build_s": time.perf_counter() - t0, "weight_bytes": h6.weight_bytes(),
                              "conv_ms": conv_ms_in_mode(api, torch, h6, f6, nc6, 2, 2)}
        h6.close()

    # the wall problem in two space dimensions (secondary): 32 x-cells by 8
    # periodic y-cells, the same step with the 2-D transport
    wall2d = None
    if args.workload == "wall16" and not args.skip_2d:
        N2, nx, ny, Y = 16, 32, 8, 2.0
        hw = api.Handle(N2, L_BOX, LAM, "fp32")
        hw.reserve(nx * ny)
        api.cs_autotune(hw.ptr, nx * ny)
        dx2 = torch.from_numpy(inputs.wall_grid(nx)).to(device)
        far2 = torch.from_numpy(inputs.maxwellian(N2, L_BOX, 1.0, (0.0, 0.0, 0.0), 1.0)).to(device)
        f2 = torch.from_numpy(inputs.wall2d_initial(N2, L_BOX, nx, ny, Y)).to(device)
        for _ in range(3):
            hw.step2d(f2, dx2, far2, WALL_T, (0.0, 0.0, 0.0), ny, Y / ny, DT)
        torch.cuda.synchronize()
        k2, ms2 = max(2, min(args.steps, 10)), 0.0
        for _ in range(k2):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            hw.step2d(f2, dx2, far2, WALL_T, (0.0, 0.0, 0.0), ny, Y / ny, DT)
            b.record()
            b.synchronize()
            ms2 += a.elapsed_time(b)
        wall2d = {"workload": f"wall problem in 2-D: N={N2}, {nx} x-cells (dx_j=min(0.125*1.05^j,0.5)) x {ny} "
                              f"periodic y-cells (Y={Y}), density 1+0.2 sin(2 pi y/Y), one Strang step",
                  "ms_per_step": ms2 / k2, "value": 2 * nx * ny * N2 ** 6 / (ms2 / k2 * 1e-3), "unit": UNIT}
        hw.close()

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": describe(args.workload), "N": N, "cells_per_gpu": ncells, "L": L_BOX,
                   "lambda": LAM, "dt": DT, "precision": "f32 transforms+convolution, f64 weights/projection/"
                   "transport/state", "l2": "256 MiB buffer written before every timed step",
                   "parallelism": f"replicas x{world} (cells are independent)"},
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": launches,
        # the same rate in valid pairs (27 N^6 / 64 per cell and evaluation) instead of the nominal N^6
        "effective": {"value": value * 27.0 / 64.0, "unit": "valid pair-updates/s (27 N^6/64 per cell)"},
        "gpu_launches_per_step": launches / args.steps,
        "roofline": {"bound": "alu", "achieved": achieved_ops, "peak": peak_tops,
                     "unit": "T FP32 FMA-pipe lane-ops/s", "frac": achieved_ops / peak_tops,
                     "traffic": TRAFFIC.get((N, ncells)),
                     "kernel": "conv_strip_kernel (step a2)", "avg_launch_ms": conv_avg,
                     "peak_basis": "152 SMs x 128 FP32 lanes x 2070 MHz (max SM clock)",
                     "ops_per_launch": 6.0 * pair_cells, "tflops": achieved,
                     "flop_frac": achieved / peak_tflops, "autotuned_ms": tuned_ms,
                     "launch": {"groups_per_cta": api.cs_tune_get(h32.ptr, api.CS_TUNE_GROUPS_PER_CTA),
                                "ctas_per_sm": api.cs_tune_get(h32.ptr, api.CS_TUNE_CTAS_PER_SM),
                                "tile_split": api.cs_tune_get(h32.ptr, api.CS_TUNE_SPLIT)},
                     "probe": probe},
        "stage_ms_per_step": step_stage_ms,
        "q_eval": q_eval,
        "weights": weights,
        "fp64": fp64,
        "speedup_vs_fp64": fp64["ms_per_step"] / ms_step if fp64 else None,
    }
    if n32:
        out["n32"] = n32
    if wall2d:
        out["wall2d"] = wall2d
    if n64:
        out["n64"] = n64
    if not args.skip_batched and world == 1:
        out["batched"] = batched_run(api, inputs, torch, device, args)
    if not args.skip_serve and world == 1:
        from paper_1301_4195_gb300 import serve
        torch.cuda.synchronize()
        out["serve"] = serve.serve_bench(48, args.serve_rate, horizon=(0.1, 0.5))
        out["serve"]["load"] = (f"48 Poisson requests at {args.serve_rate}/s, N in {{12,16,24,32}}, "
                                f"lambda in {{0,1}}, 2-4 Maxwellian mixtures, horizon U[0.1,0.5] at dt=0.01, "
                                f"weight tables resident")
        # the same load with one cs_relax_batched call per iteration instead of one cs_relax per class
        pc = serve.serve_bench(48, args.serve_rate, horizon=(0.1, 0.5), batched=True)
        out["serve"]["batched_relax"] = {k: pc[k] for k in ("p50_s", "p99_s", "requests_per_s",
                                                           "throughput_pair_updates_per_s")}
        # the arrival rate swept around the measured capacity (requests completed per second)
        cap = out["serve"]["requests_per_s"]
        out["serve"]["sweep"] = []
        for factor in (0.5, 2.0):
            r = serve.serve_bench(48, factor * cap, horizon=(0.1, 0.5))
            out["serve"]["sweep"].append({"rate_per_s": r["rate_per_s"], "rate_vs_capacity": factor,
                                          "p50_s": r["p50_s"], "p99_s": r["p99_s"],
                                          "requests_per_s": r["requests_per_s"],
                                          "throughput_pair_updates_per_s": r["throughput_pair_updates_per_s"]})
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"], out["error_vs_oracle"] = cpu_baseline(args, api, inputs, torch, device, h32, h64)
    h32.close()
    if h64:
        h64.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def batched_run(api, inputs, torch, device, args):
    """Uneven cells in one replayed graph: 4096 cells at N = 16 and 1024 at
    N = 24, half lambda = 0 and half lambda = 1, random 2-3 Maxwellian
    mixtures; one cs_collide_batched call = one collision evaluation of all."""
    specs = [(16, 0.0, 2048), (16, 1.0, 2048), (24, 0.0, 512), (24, 1.0, 512)]
    hs, fs, qs, first = [], [], [], 20000
    for N, lam, n in specs:
        h = api.Handle(N, L_BOX, lam, "fp32")
        h.reserve(n)
        api.cs_autotune(h.ptr, n)
        hs.append(h)
        fs.append(torch.from_numpy(inputs.random_mixture_cells(N, L_BOX, n, first_id=first)).to(device))
        qs.append(torch.empty_like(fs[-1]))
        first += n
    entries = [(h.ptr, f, q, n) for h, f, q, (_, _, n) in zip(hs, fs, qs, specs)]
    for _ in range(2):
        api.cs_collide_batched(entries)
    torch.cuda.synchronize()
    reps, total = 3, 0.0
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        api.cs_collide_batched(entries)
        b.record()
        b.synchronize()
        total += a.elapsed_time(b)
    ms = total / reps
    pairs = sum(n * N ** 6 for N, _, n in specs)
    for h in hs:
        h.close()
    return {"workload": "4096 cells N=16 + 1024 cells N=24, lambda 0/1 half each, random mixtures, "
                        "one graph replay per collision evaluation (cs_collide_batched), autotuned",
            "ms_per_call": ms, "value": pairs / (ms * 1e-3), "unit": UNIT}


def cpu_baseline(args, api, inputs, torch, device, h32, h64):
    """The oracle, as it stands, on this host's cores: one collision evaluation
    (transform, convolution, inverse, projection) of a sample of the workload's
    cells; also the GPU results' error against it on that sample."""
    import oracle
    oracle.build()
    wl = WORKLOADS[args.workload]
    N = wl["N"]
    nsample = 16
    # sample cells: the wall state after a few steps has non-trivial collisions
    f0 = inputs.random_mixture_cells(N, L_BOX, nsample, first_id=5000)
    cores = os.cpu_count() or 1
    reps, t_total = 0, 0.0
    ref = None
    while t_total < 10.0 and reps < 200:
        t0 = time.perf_counter()
        ref = oracle.collide(f0, N, L_BOX, LAM, nthreads=cores)
        t_total += time.perf_counter() - t0
        reps += 1
    cpu = {"value": reps * nsample * N ** 6 / t_total, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{reps} x one collision evaluation of {nsample} random-mixture cells at N={N} "
                     f"(L=6, lambda=1), OpenMP over zeta outputs"}
    # the same on one core, and one N = 32 cell on all cores (the paper's Tables 1-4
    # time one evaluation on 1..16 cores)
    t0 = time.perf_counter()
    oracle.collide(f0[:4], N, L_BOX, LAM, nthreads=1)
    cpu["single_thread"] = {"value": 4 * N ** 6 / (time.perf_counter() - t0), "cores": 1,
                            "sample": f"one evaluation of 4 of the cells at N={N}"}
    f32 = inputs.random_mixture_cells(32, L_BOX, 1, first_id=5000)
    t0 = time.perf_counter()
    oracle.collide(f32, 32, L_BOX, LAM, nthreads=cores)
    cpu["n32_one_cell"] = {"value": 32 ** 6 / (time.perf_counter() - t0), "cores": cores,
                           "sample": "one evaluation of one random-mixture cell at N=32"}
    # the space-homogeneous two-stream case whole: N = 8, one cell, 100 Heun steps
    # of dt = 0.01 (200 evaluations), one core, and the GPU's Heun steps beside it
    f8 = inputs.two_stream(8, L_BOX)[None]
    t0 = time.perf_counter()
    r8 = oracle.rk2_homogeneous(f8, 8, L_BOX, 1.0, 0.01, 100, nthreads=1)
    t8 = time.perf_counter() - t0
    h8 = api.Handle(8, L_BOX, 1.0, "fp64")
    g8 = torch.from_numpy(f8.copy()).to(device)
    h8.relax(g8, 0.01, 100)
    torch.cuda.synchronize()
    cpu["two_stream_n8"] = {"value": 200 * 8 ** 6 / t8, "cores": 1, "seconds": t8,
                            "sample": "N=8, one two-stream cell, 100 Heun steps of dt=0.01 (200 evaluations)",
                            "gpu_fp64_error": float(np.abs(g8.cpu().numpy() - r8).max() / np.abs(r8).max())}
    h8.close()
    err = {}
    fd = torch.from_numpy(f0).to(device)
    for name, h in (("fp32", h32), ("fp64", h64)):
        if h is None:
            continue
        q = h.collide(fd).cpu().numpy()
        err[name] = float(np.abs(q - ref).max() / np.abs(ref).max())
    return cpu, err


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    """The CPU oracle as the reference arm: each step is one Strang step of a
    bounded sample (16 of the workload's cells) on this host's cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1301_4195_gb300 import inputs
    oracle.build()
    wl = WORKLOADS[args.workload]
    N, ncells = wl["N"], 16
    dx = inputs.wall_grid(wl["ncells"])[:ncells]
    f = inputs.wall_initial(N, L_BOX, ncells)
    far = inputs.maxwellian(N, L_BOX, 1.0, (0, 0, 0), 1.0)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        f = oracle.strang_step(f, N, L_BOX, LAM, dx, WALL_T, (0, 0, 0), far, DT, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = oracle.strang_step(f, N, L_BOX, LAM, dx, WALL_T, (0, 0, 0), far, DT, nthreads=cores)
    el = time.perf_counter() - t0
    value = args.steps * 2 * ncells * N ** 6 / el
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": describe(args.workload), "N": N, "cells_per_step_sample": ncells,
                      "note": "reference = the FP64 CPU oracle (the paper has no code)"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"Strang steps of {ncells} of the {wl['ncells']} cells"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="wall16")
    ap.add_argument("--cells", type=int, default=0, help="override the workload's cell count (profiling runs)")
    ap.add_argument("--tune", default="", help="fixed launch choices instead of the autotuner: "
                    "groups_per_cta,ctas_per_sm,tile_split,weights (profiling runs)")
    ap.add_argument("--skip-n32", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true", help="omit the double-precision comparison")
    ap.add_argument("--skip-serve", action="store_true", help="omit the serving run")
    ap.add_argument("--skip-batched", action="store_true", help="omit the uneven-N batched run")
    ap.add_argument("--skip-2d", action="store_true", help="omit the two-dimensional wall problem")
    ap.add_argument("--skip-n64", action="store_true", help="omit the N = 64 collision evaluation")
    ap.add_argument("--serve-rate", type=float, default=100.0, help="Poisson arrival rate of the serving run (1/s)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
