#!/usr/bin/env python
"""Throughput of the conservative spectral collision step on GB300.

One bench "step" is one Strang-split time step of the 1-D wall boundary-layer
problem (transport dt/2, Heun collision dt = two evaluations of the collision
operator with the conservation projection, transport dt/2): every step of the
hot path.  The metric is nominal pair-updates per second,
    (collision evaluations) x (cells) x N^6 / time,
the count the paper's N^6 cost model uses.

Default workload (N=1): N = 32, L = 6, lambda = 1, 256 cells of width
min(dx0 1.05^j, 0.5), dx0 = 1/8, wall at T_w = 1.5 against a unit Maxwellian
gas, dt = 0.01; transforms and convolution in float, weights, projection,
transport and state in double.  Secondary objects in the same line: the same
step in double precision ("fp64"); the N = 16, 128-cell workload ("wall16");
the N = 32 run of 2000 steps with its error and moment drift ("config4"); the
uneven batch ("batched"); the serving sweep ("serve"); N = 64 ("n64"); the
wall problem in two space dimensions ("wall2d").

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
# current kernels (profiles/), keyed by (N, cells, groups per CTA, tile
# ranges per pencil) with the default tile, stored weights and L2
# priorities; absent (reported as null) where that launch was not captured
TRAFFIC = {
    (32, 256, 4, 1): 1491404544 + 67005696,
    (32, 256, 2, 1): 2499984640 + 66020608,
    (32, 256, 2, 2): 3038963968 + 138928896,
    (16, 128, 2, 4): 18435584,
}
# the same for the few-cell kernel, keyed by (N, cells, tile ranges per pencil)
LANE_TRAFFIC = {(32, 1, 2): 915300864 + 3899648}


def traffic_key(N: int, ncells: int, launch: dict):
    """The TRAFFIC key of the launch the handle's choices select, or None when
    the choices are not the captured defaults (tile, weights, L2 priorities)."""
    if launch is None or launch.get("tile") not in (0, 1) or launch.get("weights") != "stored tiles" or \
            launch.get("l2_hint") not in (0, 2):
        return None
    groups = -(-ncells // 32)
    g = launch["groups_per_cta"] or (2 if N <= 32 and groups % 2 == 0 else 1)
    if g == 4 and (N != 32 or groups % 4):
        g = 2 if groups % 2 == 0 else 1
    split = launch["tile_split"] or (2 if N == 16 else 1)
    return (N, ncells, g, split)
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


def valid_pairs_per_cell(N: int) -> int:
    """The valid (not dropped) pairs of the convolution per cell: (3 N^2 / 4)^3."""
    return (3 * N * N // 4) ** 3


PEAK_TOPS = SMS * FP32_LANES * MAX_SM_MHZ * 1e6 / 1e12        # FP32 FMA-pipe lane operations, T/s
PEAK_TFLOPS = 2 * PEAK_TOPS                                   # one FMA = 2 flops


def conv_roofline(N: int, ncells: int, avg_ms: float, probe=None, launch=None) -> dict:
    """Roofline of one convolution launch over ncells cells at grid N.  The
    kernel visits P(N) symmetrised pairs per cell, 6 FP32 FMA-pipe lane
    operations each (one packed FMUL2 + two FFMA2); frac_executed counts
    those, frac_effective_pairs counts the 27 N^6 / 64 valid pairs the
    unsymmetrised sum has, at the same 6 lane operations each (the work a
    kernel without the symmetrisation would have to do)."""
    ops = 6.0 * unique_pairs_per_cell(N) * ncells
    ops_eff = 6.0 * valid_pairs_per_cell(N) * ncells
    t = avg_ms * 1e-3
    ach = ops / t / 1e12
    out = {"bound": "alu", "achieved": ach, "peak": PEAK_TOPS, "unit": "T FP32 FMA-pipe lane-ops/s",
           "frac": ach / PEAK_TOPS, "frac_executed": ach / PEAK_TOPS,
           "frac_effective_pairs": ops_eff / t / 1e12 / PEAK_TOPS,
           "traffic": TRAFFIC.get(traffic_key(N, ncells, launch)), "avg_launch_ms": avg_ms,
           "ops_per_launch": ops, "effective_ops_per_launch": ops_eff,
           "tflops": 10.0 * unique_pairs_per_cell(N) * ncells / t / 1e12,
           "peak_basis": "152 SMs x 128 FP32 lanes x 2070 MHz (max SM clock), derived"}
    out["flop_frac"] = out["tflops"] / PEAK_TFLOPS
    if probe:
        out["frac_of_best_fp32_probe"] = ach / max(probe["ffma_tlane_ops"], probe["ffma2_tlane_ops"])
    return out


def moment_rows(N: int) -> np.ndarray:
    """The integration matrix C of the conservation step: rows dv^3 (1, v1, v2, v3, |v|^2)."""
    from paper_1301_4195_gb300 import inputs
    v = inputs.velocity_grid(N, L_BOX)
    w = (2 * L_BOX / N) ** 3
    return np.stack([np.ones_like(v[0]), v[0], v[1], v[2], v[0] ** 2 + v[1] ** 2 + v[2] ** 2]).reshape(5, -1) * w


def drift_of(Q: np.ndarray, N: int) -> float:
    """max over cells and rows of |C Q| / (|C| |Q|): the moment drift of a collision
    term relative to the rounding scale of its moments."""
    C = moment_rows(N)
    q = Q.reshape(Q.shape[0], -1)
    return float((np.abs(q @ C.T) / (np.abs(q) @ np.abs(C).T)).max())


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


def step_workload(api, inputs, torch, device, N, ncells, K, W, flush, tune="", profile_stages=True):
    """One Strang-step workload on a float handle: autotune (or fixed choices),
    W warm-up steps, K timed steps (replayed graphs, events per step, L2
    flushed before each), then the same K steps with per-stage events for
    the convolution's average launch.  Returns the handle, its state and the
    measurements."""
    h = api.Handle(N, L_BOX, LAM, "fp32")
    h.reserve(ncells)
    if tune:  # fixed launch choices (profiling runs: timings under a profiler would mislead the autotuner)
        for param, v in zip((api.CS_TUNE_GROUPS_PER_CTA, api.CS_TUNE_CTAS_PER_SM, api.CS_TUNE_SPLIT,
                             api.CS_TUNE_WEIGHTS, api.CS_TUNE_L2_HINT, api.CS_TUNE_TILE),
                            (int(x) for x in tune.split(","))):
            api.cs_tune(h.ptr, param, v)
        tuned_ms = None
    else:
        tuned_ms = api.cs_autotune(h.ptr, ncells)  # launch shape of the convolution (outside the timed region)
    f0, fd, dxd, fard = make_state(api, inputs, torch, N, ncells, device)
    for _ in range(W):
        h.step(fd, dxd, fard, WALL_T, (0.0, 0.0, 0.0), DT, nsteps=1)
    torch.cuda.synchronize()
    return h, f0, fd, dxd, fard, tuned_ms


def launch_choice(api, h) -> dict:
    return {"groups_per_cta": api.cs_tune_get(h.ptr, api.CS_TUNE_GROUPS_PER_CTA),
            "ctas_per_sm": api.cs_tune_get(h.ptr, api.CS_TUNE_CTAS_PER_SM),
            "tile_split": api.cs_tune_get(h.ptr, api.CS_TUNE_SPLIT),
            "weights": WEIGHT_MODES[api.cs_tune_get(h.ptr, api.CS_TUNE_WEIGHTS)],
            "l2_hint": api.cs_tune_get(h.ptr, api.CS_TUNE_L2_HINT),
            "tile": api.cs_tune_get(h.ptr, api.CS_TUNE_TILE)}


def q_eval_run(api, torch, h, fd, N, ncells, world=1):
    """The operator alone (t_Q = forward transform + convolution + inverse +
    projection, one cs_collide on the workload's state), direct launches."""
    qd = torch.empty_like(fd)
    for _ in range(3):
        api.cs_collide(h.ptr, fd, ncells, 1.0, qd, 1)
    torch.cuda.synchronize()
    ta, tb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nq = 10
    ta.record()
    for _ in range(nq):
        api.cs_collide(h.ptr, fd, ncells, 1.0, qd, 1)
    tb.record()
    tb.synchronize()
    tq = ta.elapsed_time(tb) / nq
    return {"ms_per_evaluation": tq, "value": world * ncells * N ** 6 / (tq * 1e-3), "unit": UNIT,
            "note": "one collision evaluation Q(f) of the workload's cells (t_Q: transforms, convolution, "
                    "projection), L2 not flushed between evaluations"}


def fp64_step(api, inputs, torch, device, N, ncells, dxd, fard, flush, k64):
    """The same Strang step in double precision (the plain FP64 GPU form)."""
    h64 = api.Handle(N, L_BOX, LAM, "fp64")
    h64.reserve(ncells)
    _, fd64, _, _ = make_state(api, inputs, torch, N, ncells, device)
    ms64, _ = time_steps(torch, h64, fd64, dxd, fard, k64, 1, flush)
    return h64, {"value": 2 * ncells * N ** 6 / (ms64 / k64 * 1e-3), "ms_per_step": ms64 / k64, "steps": k64}


def secondary_workload(api, inputs, torch, device, args, wl, flush, probe):
    """A Strang-step workload beside the headline one: its rate, the
    convolution's roofline, the operator alone, both weight modes and the
    double-precision form of the same step."""
    N, ncells = WORKLOADS[wl]["N"], WORKLOADS[wl]["ncells"]
    h, f0, fd, dxd, fard, tuned = step_workload(api, inputs, torch, device, N, ncells, args.steps, 3, flush)
    k = max(3, min(args.steps, 20))
    ms, _ = time_steps(torch, h, fd, dxd, fard, k, 0, flush, profile=False)
    _, prof = time_steps(torch, h, fd, dxd, fard, k, 0, flush, profile=True)
    cavg = prof["convolve"][0] / max(prof["convolve"][1], 1)
    out = {"workload": describe(wl), "value": 2 * ncells * N ** 6 / (ms / k * 1e-3), "unit": UNIT,
           "ms_per_step": ms / k, "steps": k, "conv_ms": cavg,
           "roofline": conv_roofline(N, ncells, cavg, probe, launch_choice(api, h)), "launch": launch_choice(api, h),
           "autotuned_ms": tuned, "stage_ms_per_step": {kk: v[0] / k for kk, v in prof.items()},
           "q_eval": q_eval_run(api, torch, h, fd, N, ncells),
           "weights": {"stored_conv_ms": conv_ms_in_mode(api, torch, h, fd, ncells, 1),
                       "radius_conv_ms": conv_ms_in_mode(api, torch, h, fd, ncells, 2)}}
    if not args.skip_fp64:
        h64, fp = fp64_step(api, inputs, torch, device, N, ncells, dxd, fard, flush, max(2, min(args.steps, 5)))
        h64.close()
        out["fp64"] = fp
        out["speedup_vs_fp64"] = fp["ms_per_step"] / out["ms_per_step"]
    h.close()
    return out


def config4_run(api, inputs, torch, device, h32, args):
    """The large-grid wall problem run whole: N = 32, 256 cells, 2000 Strang
    steps of dt = 0.01 in float (convolution with compensated xi-sums,
    projection in double), from the unit Maxwellian, on the headline's
    handle.  Reported: the moment drift of the collision step at ten points
    of the run (the moments of every cell before and after one Heun collision
    step of its current state, relative to the largest moment of the cell),
    |C Q| / (|C| |Q|) of the final state's collision term in every cell, the
    final state's collision term on cells 0, 1, 64 and 255 (wall, next to it,
    interior, far end) against the oracle, relative to its largest value and
    to the rounding scale S of the float sum (cells where S / |Q| > 100 are
    flagged), and the float state against the plain double form after the
    first 10 steps."""
    import oracle
    oracle.build()
    N, nc, total = 32, 256, args.config4_steps
    _, f, dx, far = make_state(api, inputs, torch, N, nc, device)
    chunk = max(1, total // 10)
    drift_steps, drifts = [], []
    ta, tb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f10 = None
    run_ms, done = 0.0, 0
    g = torch.empty_like(f)
    m0 = torch.empty((nc, 5), dtype=torch.float64, device=device)
    m1 = torch.empty_like(m0)
    while done < total:
        n = 10 if done == 0 else min(chunk, total - done)
        ta.record()
        h32.step(f, dx, far, WALL_T, (0.0, 0.0, 0.0), DT, nsteps=n)
        tb.record()
        tb.synchronize()
        run_ms += ta.elapsed_time(tb)
        done += n
        if done == 10:
            f10 = f.cpu().numpy()
        # the collision step's moment drift on the current state
        g.copy_(f)
        api.cs_moments(h32.ptr, g, nc, m0)
        api.cs_relax(h32.ptr, g, nc, DT, 1.0, 1)
        api.cs_moments(h32.ptr, g, nc, m1)
        a, b = m0.cpu().numpy(), m1.cpu().numpy()
        drift_steps.append(done)
        drifts.append(float((np.abs(b - a).max(axis=1) / np.abs(a).max(axis=1)).max()))
    api.cs_status(h32.ptr)
    fin = f.cpu().numpy()
    q = torch.empty_like(f)
    api.cs_collide(h32.ptr, f, nc, 1.0, q, 1)
    Q = q.cpu().numpy()
    sample = [0, 1, 64, 255]
    cores = os.cpu_count() or 1
    ref = oracle.collide(fin[sample], N, L_BOX, LAM, nthreads=cores)
    S = oracle.rounding_scale(fin[sample], N, L_BOX, LAM, nthreads=cores)
    cells = []
    for i, c in enumerate(sample):
        err = float(np.abs(Q[c] - ref[i]).max())
        qmax = float(np.abs(ref[i]).max())
        cells.append({"cell": c, "rel_err": err / qmax, "err_over_S": err / S[i], "S_over_Qmax": S[i] / qmax,
                      "flagged": bool(S[i] / qmax > 100.0)})
    out = {"workload": f"N=32, L=6, lambda=1, 256 cells of the wall grid, unit Maxwellian start, T_w=1.5, "
                       f"{total} Strang steps of dt=0.01 (float transforms and convolution with compensated "
                       f"xi-sums, double projection, transport and state)",
           "steps": total, "ms_per_step": run_ms / total, "run_s": run_ms / 1e3,
           "value": 2 * nc * N ** 6 / (run_ms / total * 1e-3), "unit": UNIT,
           "finite": bool(np.isfinite(fin).all()),
           "collision_step_drift": {"steps": drift_steps, "max_rel": max(drifts), "per_check": drifts},
           "final_q_drift": drift_of(Q, N),
           "oracle_err": {"cells": cells, "max_rel_err": max(c["rel_err"] for c in cells),
                          "max_err_over_S": max(c["err_over_S"] for c in cells), "tolerance": 1e-5}}
    # the plain double form over the first 10 steps
    if not args.skip_fp64:
        h64 = api.Handle(N, L_BOX, LAM, "fp64")
        h64.reserve(nc)
        _, f64, _, _ = make_state(api, inputs, torch, N, nc, device)
        h64.step(f64, dx, far, WALL_T, (0.0, 0.0, 0.0), DT, nsteps=2)
        torch.cuda.synchronize()
        ta.record()
        h64.step(f64, dx, far, WALL_T, (0.0, 0.0, 0.0), DT, nsteps=8)
        tb.record()
        tb.synchronize()
        ms64 = ta.elapsed_time(tb) / 8
        d = f64.cpu().numpy()
        out["fp64_10_steps"] = {"state_rel_diff": float(np.abs(f10 - d).max() / np.abs(d).max()),
                                "ms_per_step": ms64, "value": 2 * nc * N ** 6 / (ms64 * 1e-3)}
        h64.close()
    return out


def serve_sweep(args):
    """Config 5: Poisson arrivals of space-homogeneous relaxation requests,
    N in {12, 16, 24, 32}, lambda in {0, 1}, 2-4 Maxwellian mixtures, horizons
    U[1, 20] time units at dt = 0.01 (100 to 2000 Heun steps), every eighth
    request a Maxwell-molecule one from BKW data checked against the closed
    form.  First a saturating run measures the capacity (requests completed
    per second with every request waiting at the start), then the rate is set
    to 0.5x, 1x and 2x that capacity; each run has args.serve_requests
    requests."""
    from paper_1301_4195_gb300 import serve
    n, hz = args.serve_requests, (1.0, 20.0)
    sat = serve.serve_bench(n, 1e4, horizon=hz, bkw_every=8)
    cap = sat["requests_per_s"]
    out = {"load": f"{n} Poisson requests per rate, N in {{12,16,24,32}}, lambda in {{0,1}}, 2-4 Maxwellian "
                   f"mixtures, horizon U[1,20] time units at dt=0.01, every 8th request BKW (lambda=0, K0=0.6), "
                   f"weight tables resident, every class on its own stream advancing in chunks of up to 8 Heun steps "
                   f"as soon as its previous chunk completes",
           "capacity_requests_per_s": cap, "saturated": sat, "sweep": []}
    for factor in (0.5, 1.0, 2.0):
        r = serve.serve_bench(n, factor * cap, horizon=hz, bkw_every=8)
        r["rate_vs_capacity"] = factor
        out["sweep"].append(r)
    one = out["sweep"][1]
    out.update({"p50_s": one["p50_s"], "p99_s": one["p99_s"], "rate_per_s": one["rate_per_s"],
                "throughput_pair_updates_per_s": one["throughput_pair_updates_per_s"]})
    return out


def n64_run(api, inputs, torch, device):
    """N = 64 (a 58 GB float weight table): one collision evaluation of 32
    random-mixture cells, its convolution's roofline, and the same from a
    handle holding the radius tables only."""
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
    out = {"workload": f"one collision evaluation, N={N6}, {nc6} random-mixture cells (L=6, lambda=1)",
           "ms_per_evaluation": ms6, "value": nc6 * N6 ** 6 / (ms6 * 1e-3), "unit": UNIT,
           "weights_build_s": build_s, "weight_bytes": h6.weight_bytes(), "conv_ms": c6,
           "roofline": conv_roofline(N6, nc6, c6), "drift": drift_of(q6.cpu().numpy(), N6)}
    h6.close()
    t0 = time.perf_counter()
    h6 = api.Handle(N6, L_BOX, LAM, "fp32-radius")
    torch.cuda.synchronize()
    out["radius_only"] = {"weights_build_s": time.perf_counter() - t0, "weight_bytes": h6.weight_bytes(),
                          "conv_ms": conv_ms_in_mode(api, torch, h6, f6, nc6, 2, 2)}
    h6.close()
    return out


def few_cells_run(api, inputs, torch, device, h):
    """Convolutions over a few cells at N = 32 (the serving case): the
    few-cell kernel (one warp per cell, a pencil's outputs over its lanes)
    against the strip kernels (two strips per warp), same bits.  At one cell
    the launch must at least stream the weight table, so its roofline is HBM:
    the table's bytes per launch against the measured copy bandwidth."""
    N = 32
    f_all = torch.from_numpy(inputs.random_mixture_cells(N, L_BOX, 8, first_id=7600)).to(device)
    keep = api.cs_tune_get(h.ptr, api.CS_TUNE_FEW_CELLS)
    keep_split = api.cs_tune_get(h.ptr, api.CS_TUNE_SPLIT)
    rows = []
    for split in (0, 2):  # whole pencils; two tile ranges per pencil (the serving loop's choice)
        api.cs_tune(h.ptr, api.CS_TUNE_SPLIT, split)
        for n in (1, 2, 4, 6):
            f = f_all[:n].contiguous()
            q = torch.empty_like(f)
            r = {"cells": n, "tile_ranges": max(split, 1)}
            outs = []
            for key, mode in (("few_cell_ms", 16), ("strip_ms", -1)):
                api.cs_tune(h.ptr, api.CS_TUNE_FEW_CELLS, mode)
                r[key] = conv_ms_in_mode(api, torch, h, f, n, 1)
                api.cs_collide(h.ptr, f, n, 1.0, q, 1)
                outs.append(q.cpu().numpy())
            r["identical"] = bool(np.array_equal(outs[0], outs[1]))
            rows.append(r)
    api.cs_tune(h.ptr, api.CS_TUNE_FEW_CELLS, keep)
    api.cs_tune(h.ptr, api.CS_TUNE_SPLIT, keep_split)
    table = h.weight_bytes()
    one = min((r for r in rows if r["cells"] == 1), key=lambda r: r["few_cell_ms"])
    ms1 = one["few_cell_ms"]
    peak = None
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as fp:
            peak = json.load(fp)["hbm_gbs"]
    except (OSError, KeyError, ValueError):
        pass
    achieved = table / (ms1 * 1e-3) / 1e9
    return {"workload": f"the convolution of one collision evaluation, N={N}, 1-6 random-mixture cells "
                        "(L=6, lambda=1), few-cell kernel against strip kernels",
            "rows": rows,
            "roofline_one_cell": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                  "frac": achieved / peak if peak else None,
                                  "traffic": LANE_TRAFFIC.get((N, 1, one["tile_ranges"])), "bytes": table,
                                  "tile_ranges": one["tile_ranges"],
                                  "note": "the weight table once per launch, against the measured HBM copy bandwidth"}}


def wall2d_run(api, inputs, torch, device, args, flush):
    """The wall problem in two space dimensions: 32 x-cells by 8 periodic
    y-cells at N = 16, the same step with the 2-D transport."""
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
    hw.close()
    return {"workload": f"wall problem in 2-D: N={N2}, {nx} x-cells (dx_j=min(0.125*1.05^j,0.5)) x {ny} "
                        f"periodic y-cells (Y={Y}), density 1+0.2 sin(2 pi y/Y), one Strang step",
            "ms_per_step": ms2 / k2, "value": 2 * nx * ny * N2 ** 6 / (ms2 / k2 * 1e-3), "unit": UNIT}


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

    h32, f0, fd, dxd, fard, tuned_ms = step_workload(api, inputs, torch, device, N, ncells, args.steps,
                                                     args.warmup, flush, tune=args.tune)

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
    pairs_step = 2 * ncells * N ** 6
    value = world * pairs_step / (ms_step * 1e-3)
    conv_avg = prof["convolve"][0] / max(prof["convolve"][1], 1)
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
    roof = conv_roofline(N, ncells, conv_avg, probe, launch_choice(api, h32))
    roof.update({"kernel": "conv_strip_kernel (step a2)", "autotuned_ms": tuned_ms,
                 "launch": launch_choice(api, h32), "probe": probe})

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
        "roofline": roof,
        # the same rate in valid pairs (27 N^6 / 64 per cell and evaluation) instead of the nominal N^6
        "effective": {"value": value * 27.0 / 64.0, "unit": "valid pair-updates/s (27 N^6/64 per cell)"},
        "gpu_launches_per_step": launches / args.steps,
        "stage_ms_per_step": step_stage_ms,
        "q_eval": q_eval_run(api, torch, h32, fd, N, ncells, world),
        "weights": {"chosen": WEIGHT_MODES[api.cs_tune_get(h32.ptr, api.CS_TUNE_WEIGHTS)],
                    "stored_conv_ms": conv_ms_in_mode(api, torch, h32, fd, ncells, 1),
                    "radius_conv_ms": conv_ms_in_mode(api, torch, h32, fd, ncells, 2)},
    }
    # the plain FP64 GPU form of the same step
    h64 = None
    if not args.skip_fp64:
        h64, fp = fp64_step(api, inputs, torch, device, N, ncells, dxd, fard, flush,
                            2 if N >= 32 else max(2, min(args.steps, 5)))
        out["fp64"] = fp
        out["speedup_vs_fp64"] = fp["ms_per_step"] / ms_step
    if world == 1:
        other = "wall16" if args.workload == "wall32" else "wall32"
        if not args.skip_secondary:
            out[other] = secondary_workload(api, inputs, torch, device, args, other, flush, probe)
        if N == 32 and ncells == 256 and args.config4_steps > 0:
            out["config4"] = config4_run(api, inputs, torch, device, h32, args)
        if not args.skip_batched:
            out["batched"] = batched_run(api, inputs, torch, device, args)
        if not args.skip_2d:
            out["wall2d"] = wall2d_run(api, inputs, torch, device, args, flush)
        if not args.skip_n64:
            out["n64"] = n64_run(api, inputs, torch, device)
        if N == 32 and not args.skip_few:
            out["few_cells"] = few_cells_run(api, inputs, torch, device, h32)
        if not args.skip_serve:
            torch.cuda.synchronize()
            out["serve"] = serve_sweep(args)
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
    mixtures; one cs_collide_batched call = one collision evaluation of all.
    The roofline counts the whole call's time (transforms and projections
    included) against the convolutions' lane operations, so it is a lower
    bound on the shared convolution launch's own fraction.  Two cells of
    every entry (the first and the last) are checked against the oracle."""
    import oracle
    oracle.build()
    specs = [(16, 0.0, 2048), (16, 1.0, 2048), (24, 0.0, 512), (24, 1.0, 512)]
    hs, fs, qs, first, firsts = [], [], [], 20000, []
    for N, lam, n in specs:
        h = api.Handle(N, L_BOX, lam, "fp32")
        h.reserve(n)
        api.cs_autotune(h.ptr, n)
        hs.append(h)
        fs.append(torch.from_numpy(inputs.random_mixture_cells(N, L_BOX, n, first_id=first)).to(device))
        qs.append(torch.empty_like(fs[-1]))
        firsts.append(first)
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
    ops = sum(6.0 * unique_pairs_per_cell(N) * n for N, _, n in specs)
    ops_eff = sum(6.0 * valid_pairs_per_cell(N) * n for N, _, n in specs)
    errs, drift = [], 0.0
    cores = os.cpu_count() or 1
    for (N, lam, n), f, q, fid in zip(specs, fs, qs, firsts):
        Q = q.cpu().numpy()
        drift = max(drift, drift_of(Q, N))
        idx = [0, n - 1]
        fc = np.concatenate([inputs.random_mixture_cells(N, L_BOX, 1, first_id=fid + c) for c in idx])
        ref = oracle.collide(fc, N, L_BOX, lam, nthreads=cores)
        for j, c in enumerate(idx):
            errs.append(float(np.abs(Q[c] - ref[j]).max() / np.abs(ref[j]).max()))
    for h in hs:
        h.close()
    t = ms * 1e-3
    return {"workload": "4096 cells N=16 + 1024 cells N=24, lambda 0/1 half each, random mixtures, "
                        "one graph replay per collision evaluation (cs_collide_batched), autotuned",
            "ms_per_call": ms, "value": pairs / t, "unit": UNIT,
            "roofline": {"bound": "alu", "achieved": ops / t / 1e12, "peak": PEAK_TOPS,
                         "unit": "T FP32 FMA-pipe lane-ops/s", "frac": ops / t / 1e12 / PEAK_TOPS,
                         "frac_executed": ops / t / 1e12 / PEAK_TOPS,
                         "frac_effective_pairs": ops_eff / t / 1e12 / PEAK_TOPS, "traffic": None,
                         "timed": "the whole call (transforms, shared convolution launch, projections)"},
            "error_vs_oracle": {"max_rel": max(errs), "cells": "first and last cell of every entry"},
            "drift": drift}


def cpu_baseline(args, api, inputs, torch, device, h32, h64):
    """The oracle, as it stands, on this host's cores: one collision evaluation
    (transform, convolution, inverse, projection) of a sample of random-mixture
    cells at the workload's N; also the GPU results' error against it on that
    sample, relative to the largest value of Q and (float) to the rounding
    scale S of the float sum."""
    import oracle
    oracle.build()
    wl = WORKLOADS[args.workload]
    N = wl["N"]
    nsample = 8 if N >= 32 else 16
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
    # the same on one core (the paper's Tables 1-4 time one evaluation on 1..16 cores)
    t0 = time.perf_counter()
    oracle.collide(f0[:1], N, L_BOX, LAM, nthreads=1)
    cpu["single_thread"] = {"value": N ** 6 / (time.perf_counter() - t0), "cores": 1,
                            "sample": f"one evaluation of one of the cells at N={N}"}
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
    err = {"cells": f"{nsample} random-mixture cells at N={N}"}
    fd = torch.from_numpy(f0).to(device)
    for name, h in (("fp32", h32), ("fp64", h64)):
        if h is None:
            continue
        q = h.collide(fd).cpu().numpy()
        err[name] = float(np.abs(q - ref).max() / np.abs(ref).max())
        err[name + "_drift"] = drift_of(q, N)
        if name == "fp32":
            S = oracle.rounding_scale(f0, N, L_BOX, LAM, nthreads=cores)
            qmax = np.abs(ref.reshape(nsample, -1)).max(axis=1)
            e = np.abs(q - ref).reshape(nsample, -1).max(axis=1)
            err["fp32_err_over_S"] = float((e / S).max())
            err["S_over_Qmax_max"] = float((S / qmax).max())
            err["flagged_cells"] = int((S / qmax > 100.0).sum())
    return cpu, err


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    """The CPU oracle as the reference arm: each step is one Strang step of a
    bounded sample (the first cells of the workload's grid, a grid of their
    own with the same boundaries) on this host's cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1301_4195_gb300 import inputs
    oracle.build()
    wl = WORKLOADS[args.workload]
    N = wl["N"]
    ncells = 2 if N >= 32 else 16
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
                            "sample": f"Strang steps of the first {ncells} of the {wl['ncells']} cells"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="wall32")
    ap.add_argument("--cells", type=int, default=0, help="override the workload's cell count (profiling runs)")
    ap.add_argument("--tune", default="", help="fixed launch choices instead of the autotuner: "
                    "groups_per_cta,ctas_per_sm,tile_split,weights[,l2_hint[,tile]] (profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true", help="omit the double-precision comparison")
    ap.add_argument("--skip-secondary", action="store_true", help="omit the other wall workload")
    ap.add_argument("--skip-serve", action="store_true", help="omit the serving sweep")
    ap.add_argument("--skip-batched", action="store_true", help="omit the uneven-N batched run")
    ap.add_argument("--skip-2d", action="store_true", help="omit the two-dimensional wall problem")
    ap.add_argument("--skip-n64", action="store_true", help="omit the N = 64 collision evaluation")
    ap.add_argument("--skip-few", action="store_true", help="omit the few-cell convolutions")
    ap.add_argument("--config4-steps", type=int, default=2000,
                    help="Strang steps of the N = 32 run with error and drift (0: omit)")
    ap.add_argument("--serve-requests", type=int, default=200, help="requests per rate of the serving sweep")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
