"""Continuous-batching server for space-homogeneous relaxation requests.

A request asks for the solution of df/dt = P_N Qt(f) / eps (Sec. 3.1, 3.3) on an
N^3 grid over [-L, L]^3 with collision exponent lambda, from an initial f0 to
a horizon t_end, in Heun steps of dt (cs_relax).  The server

* keeps, per (N, lambda), one library handle (the weight table, resident on
  the device and shared by all requests of that class), a CUDA stream and a
  dense device buffer of the active requests' states;
* admits waiting requests at iteration boundaries while the device-memory
  budget allows (weight table of a new class + per-cell state and
  workspace), in arrival order; a float class whose table of every pair
  does not fit is built from the radius tables alone (CS_WEIGHTS_RADIUS:
  9 MB instead of 0.9 GB at N = 32), slower per step but admitted;
* runs every class on its own: a class advances all its active requests by
  a chunk of Heun steps (one cs_relax, a replayed graph, on the class's
  stream; at most max_chunk steps and never past the end of any of its
  requests, so each request takes exactly its own number of steps), and as
  soon as that chunk has completed (an event, polled) it retires its
  finished requests, admits waiting ones and launches the next chunk.  No
  class waits for another: the chunks of all classes overlap on the device,
  a small grid's requests are not held to the pace of the largest, and a
  request that arrives while its class runs joins at the class's next chunk.
  With batched=True the classes instead advance in lock step, one
  cs_relax_batched call over all of them per iteration (a replayed graph
  with one branch per class and the float classes' convolutions as one
  persistent launch per evaluation).  Per-class streams are the default:
  with classes of a few requests each, the shared launch pads every small
  class to whole pairs of 32-cell groups and the batched graph is captured
  again whenever a class's size changes, and at 100 requests/s it measured
  15 % lower throughput;
* retires finished requests (their final state is copied out) and compacts
  the class buffer by moving the last active state into the freed slot.

Each cell's arithmetic in the library depends only on that cell (one cell per
warp lane, fixed summation order), so a request's result does not depend on
which other requests share its batch.  The loop runs on the host; every step
of the method runs in libcs.
"""
from __future__ import annotations

import dataclasses
import heapq
import time
from typing import Dict, List, Optional, Tuple

import numpy as np
import torch

from . import api


@dataclasses.dataclass
class Request:
    rid: int
    N: int
    lam: float
    f0: np.ndarray            # [N, N, N] float64
    t_end: float              # horizon (time units)
    arrival: float = 0.0      # seconds on the server clock
    bkw_K0: Optional[float] = None  # Maxwell-molecule request started from BKW data with this K
    # filled by the server
    steps_done: int = 0
    steps_total: int = 0
    admitted: Optional[float] = None
    finished: Optional[float] = None
    result: Optional[np.ndarray] = None

    @property
    def latency(self) -> Optional[float]:
        return None if self.finished is None else self.finished - self.arrival


class _Class:
    """Requests of one (N, lambda): handle, stream, dense state buffer."""

    def __init__(self, N: int, lam: float, L: float, precision: str, device, capacity: int, radius: bool = False,
                 stream=None):
        self.N, self.lam, self.radius = N, lam, radius
        self.handle = api.Handle(N, L, lam, "fp32-radius" if radius else precision)
        if N == 32 and precision == "fp32" and not radius:
            # classes hold a handful of requests: two tile ranges per pencil
            # make those launches shorter (one request 0.43 -> 0.30 ms, 7 to 16
            # requests 1.37 -> 1.26 ms) at the cost of 1-2 % from 64 cells up;
            # a request's result still does not depend on its class's size
            api.cs_tune(self.handle.ptr, api.CS_TUNE_SPLIT, 2)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        self.capacity = capacity
        self.buf = torch.empty((capacity, N, N, N), dtype=torch.float64, device=device)
        self.reqs: List[Request] = []
        self.handle.reserve(capacity)
        # the chunk in flight: completion event, its cells and steps
        self.event = None
        self.inflight_n = 0
        self.inflight_k = 0

    @property
    def idle(self) -> bool:
        return self.event is None

    def grow(self, capacity: int):
        if capacity <= self.capacity:
            return
        nb = torch.empty((capacity,) + tuple(self.buf.shape[1:]), dtype=torch.float64, device=self.buf.device)
        n = len(self.reqs)
        with torch.cuda.stream(self.stream):
            nb[:n].copy_(self.buf[:n])
        self.buf = nb
        self.capacity = capacity
        self.handle.reserve(capacity)


class Server:
    """Continuous batching over (N, lambda) classes; see the module docstring."""

    def __init__(self, L: float = 6.0, dt: float = 0.01, eps: float = 1.0, precision: str = "fp32",
                 mem_budget: Optional[int] = None, device=None, max_cells_per_class: int = 4096,
                 radius_fallback: bool = True, batched: bool = False, max_chunk: int = 8):
        self.L, self.dt, self.eps, self.precision = L, dt, eps, precision
        self.max_chunk = max(1, int(max_chunk))
        self.radius_fallback = radius_fallback
        self.batched = batched
        self.device = torch.device(device or "cuda")
        # batched: every class works on one stream, the batched call's
        self.stream = torch.cuda.Stream(device=self.device) if batched else None
        if mem_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            mem_budget = int(0.8 * free)
        self.mem_budget = mem_budget
        self.max_cells = max_cells_per_class
        self.classes: Dict[Tuple[int, float], _Class] = {}
        self.waiting: List[Tuple[float, int, Request]] = []
        self.done: List[Request] = []
        self.t0 = time.perf_counter()
        self.iterations = 0

    # ------------------------------------------------------------ memory model
    def _cell_bytes(self, N: int) -> int:
        """Device bytes per active cell: state + workspace (4 spectral buffers,
        2 state-sized, transport tables are unused here) rounded up."""
        es = 8 if self.precision == "fp64" else 4
        return N ** 3 * (8 + 4 * 2 * es + 2 * 8) + 4096

    def _class_bytes(self, N: int, radius: bool = False) -> int:
        p = api.CS_FP64 if self.precision == "fp64" else api.CS_FP32
        return api.cs_weights_bytes(N, p | (api.CS_WEIGHTS_RADIUS if radius else 0))

    def _radius_possible(self, N: int) -> bool:
        return self.radius_fallback and self.precision == "fp32" and N in (8, 16, 24, 32, 48, 64)

    def used_bytes(self) -> int:
        total = 0
        for (N, _), c in self.classes.items():
            total += self._class_bytes(N, c.radius) + c.capacity * self._cell_bytes(N)
        return total

    # ------------------------------------------------------------ requests
    def now(self) -> float:
        return time.perf_counter() - self.t0

    def warm(self, classes, capacity: int = 32):
        """Build the weight tables (and buffers) of the given (N, lambda) classes
        ahead of traffic, so no request waits for a table build."""
        for N, lam in classes:
            key = (int(N), float(lam))
            if key not in self.classes:
                self.classes[key] = _Class(int(N), float(lam), self.L, self.precision, self.device, capacity,
                                           stream=self.stream)
        torch.cuda.synchronize(self.device)
        self.t0 = time.perf_counter()

    def submit(self, req: Request):
        req.steps_total = max(1, int(round(req.t_end / self.dt)))
        heapq.heappush(self.waiting, (req.arrival, req.rid, req))

    def _admit(self):
        """Admit arrived requests in arrival order into classes that have no
        chunk in flight (their buffers may then move and grow); a request
        whose class is busy waits for its next chunk boundary, and those
        behind it in other classes are not held up by it."""
        now = self.now()
        held = []
        while self.waiting and self.waiting[0][0] <= now:
            _, _, r = self.waiting[0]
            key = (r.N, float(r.lam))
            c = self.classes.get(key)
            if c is not None and not c.idle:
                held.append(heapq.heappop(self.waiting))
                continue
            extra, radius = 0, False
            if c is None:
                extra += self._class_bytes(r.N) + 32 * self._cell_bytes(r.N)
            elif len(c.reqs) + 1 > c.capacity:
                extra += c.capacity * self._cell_bytes(r.N)  # capacity doubles
            if c is None and self.used_bytes() + extra > self.mem_budget:
                self._evict_idle()
            if c is None and self.used_bytes() + extra > self.mem_budget and self._radius_possible(r.N):
                # the table of every pair does not fit: the radius tables alone
                rx = self._class_bytes(r.N, True) + 32 * self._cell_bytes(r.N)
                if self.used_bytes() + rx <= self.mem_budget:
                    extra, radius = rx, True
            if self.used_bytes() + extra > self.mem_budget or (c is not None and len(c.reqs) >= self.max_cells):
                break  # head of line waits until memory frees up (arrival order kept)
            heapq.heappop(self.waiting)
            if c is None:
                c = _Class(r.N, r.lam, self.L, self.precision, self.device, 32, radius, stream=self.stream)
                self.classes[key] = c
            if len(c.reqs) + 1 > c.capacity:
                c.grow(2 * c.capacity)
            slot = len(c.reqs)
            with torch.cuda.stream(c.stream):
                c.buf[slot].copy_(torch.from_numpy(np.ascontiguousarray(r.f0)).to(self.device, non_blocking=False))
            c.reqs.append(r)
            r.admitted = now
        for item in held:
            heapq.heappush(self.waiting, item)

    def _evict_idle(self):
        """Free the weight tables and buffers of classes with no active request."""
        for key in [k for k, c in self.classes.items() if not c.reqs and c.idle]:
            c = self.classes.pop(key)
            c.stream.synchronize()
            c.handle.close()
            del c

    def _retire(self, c: _Class):
        i = 0
        while i < len(c.reqs):
            r = c.reqs[i]
            if r.steps_done >= r.steps_total:
                with torch.cuda.stream(c.stream):
                    r.result = c.buf[i].cpu().numpy()
                r.finished = self.now()
                self.done.append(r)
                last = len(c.reqs) - 1
                if i != last:
                    with torch.cuda.stream(c.stream):
                        c.buf[i].copy_(c.buf[last])
                    c.reqs[i] = c.reqs[last]
                c.reqs.pop()
            else:
                i += 1

    def _chunk(self, reqs) -> int:
        """Heun steps the next chunk may take: max_chunk, but no request's end passed."""
        return max(1, min([self.max_chunk] + [r.steps_total - r.steps_done for r in reqs]))

    def iterate(self) -> bool:
        """One pass of the loop; returns False when nothing is active or waiting."""
        return self._iterate_batched() if self.batched else self._iterate_async()

    def _iterate_async(self) -> bool:
        """Complete the chunks that have finished (steps counted, requests
        retired), admit, and launch the next chunk of every idle class."""
        progressed = False
        for c in self.classes.values():
            if c.event is not None and c.event.query():
                for r in c.reqs[:c.inflight_n]:
                    r.steps_done += c.inflight_k
                c.event = None
                self._retire(c)
                progressed = True
        self._admit()
        for c in self.classes.values():
            if c.idle and c.reqs:
                n, k = len(c.reqs), self._chunk(c.reqs)
                api.cs_relax(c.handle.ptr, c.buf[:n], n, self.dt, self.eps, k, stream=c.stream)
                c.event = torch.cuda.Event()
                c.event.record(c.stream)
                c.inflight_n, c.inflight_k = n, k
                self.iterations += 1
                progressed = True
        if all(c.idle for c in self.classes.values()) and not self.waiting:
            return False
        if not progressed:
            time.sleep(5e-5)  # nothing finished or arrived yet
        return True

    def _iterate_batched(self) -> bool:
        """Lock step: admit, one chunk of Heun steps for every active request in
        one cs_relax_batched call, retire."""
        self._admit()
        active = [c for c in self.classes.values() if c.reqs]
        if not active and not self.waiting:
            return False
        if active:
            k = self._chunk([r for c in active for r in c.reqs])  # one chunk for the shared graph
            for j in range(0, len(active), 16):  # at most 16 entries per batched call
                part = active[j:j + 16]
                api.cs_relax_batched([(c.handle.ptr, c.buf[:len(c.reqs)], len(c.reqs)) for c in part], self.dt,
                                     k, self.eps, stream=self.stream)
            self.stream.synchronize()
            for c in active:
                for r in c.reqs:
                    r.steps_done += k
                self._retire(c)
            self.iterations += 1
        else:
            time.sleep(1e-4)  # idle until the next arrival
        if not any(c.reqs for c in self.classes.values()) and not self.waiting:
            return False
        return True

    def run(self, requests: List[Request], timeout: float = 600.0) -> List[Request]:
        for r in requests:
            self.submit(r)
        t_stop = self.now() + timeout
        while self.iterate():
            if self.now() > t_stop:
                raise TimeoutError("serving run exceeded its time limit")
        return self.done

    def close(self):
        for c in self.classes.values():
            c.handle.close()
        self.classes.clear()


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q / 100.0
    lo, hi = int(np.floor(k)), int(np.ceil(k))
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


def poisson_requests(n: int, rate: float, seed: int = 13014195, Ns=(12, 16, 24, 32), lams=(0.0, 1.0),
                     horizon=(0.1, 1.0), L: float = 6.0, bkw_every: int = 0, bkw_K0: float = 0.6):
    """n requests with exponential inter-arrival times (mean 1/rate seconds),
    N and lambda uniform over the given sets, f0 a random 2-4 Maxwellian
    mixture seeded per request id, horizon uniform in time units.  With
    bkw_every = k > 0 every k-th request is a Maxwell-molecule one (lambda =
    0) started from the BKW distribution with K = bkw_K0, whose exact
    solution is known at every time."""
    from . import inputs
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        N = int(rng.choice(Ns))
        lam = float(rng.choice(lams))
        t_end = float(rng.uniform(*horizon))
        if bkw_every and i % bkw_every == bkw_every - 1:
            out.append(Request(rid=i, N=N, lam=0.0, f0=inputs.bkw(N, L, bkw_K0), t_end=t_end, arrival=t,
                               bkw_K0=bkw_K0))
            continue
        f0 = inputs.mixture(N, L, inputs.random_mixture_params(seed + i, 2, 4))
        out.append(Request(rid=i, N=N, lam=lam, f0=f0, t_end=t_end, arrival=t))
    return out


def bkw_errors(done, L: float = 6.0, dt: float = 0.01) -> dict:
    """Maxwell-molecule requests started from BKW data against the closed form
    at their final time, K(t) = 1 - (1 - K0) exp(-t/6): the largest error
    relative to the state's maximum and to the change of the exact solution
    over the run."""
    from . import inputs
    out = {"requests": 0, "max_rel_to_state": 0.0, "max_rel_to_change": 0.0}
    for r in done:
        if r.bkw_K0 is None:
            continue
        t = r.steps_total * dt
        K = 1.0 - (1.0 - r.bkw_K0) * np.exp(-t / 6.0)
        ref = inputs.bkw(r.N, L, K)
        err = float(np.abs(r.result - ref).max())
        change = float(np.abs(ref - inputs.bkw(r.N, L, r.bkw_K0)).max())
        out["requests"] += 1
        out["max_rel_to_state"] = max(out["max_rel_to_state"], err / float(np.abs(ref).max()))
        out["max_rel_to_change"] = max(out["max_rel_to_change"], err / change)
    return out


def serve_bench(n: int = 48, rate: float = 50.0, seed: int = 13014195, horizon=(0.1, 0.5), bkw_every: int = 0,
                **kw) -> dict:
    """Run a Poisson workload through a fresh server; latency percentiles and
    throughput (nominal pair-updates/s = 2 N^6 per Heun step per request)."""
    reqs = poisson_requests(n, rate, seed, horizon=horizon, bkw_every=bkw_every)
    srv = Server(**kw)
    srv.warm([(N, lam) for N in (12, 16, 24, 32) for lam in (0.0, 1.0)])  # resident tables, clock restarts
    t0 = time.perf_counter()
    done = srv.run(reqs)
    wall = time.perf_counter() - t0
    srv.close()
    lat = [r.latency for r in done]
    pairs = sum(2 * r.steps_total * r.N ** 6 for r in done)
    out = {"requests": len(done), "rate_per_s": rate, "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99),
           "mean_s": float(np.mean(lat)), "max_s": float(np.max(lat)), "wall_s": wall, "iterations": srv.iterations,
           "throughput_pair_updates_per_s": pairs / wall, "requests_per_s": len(done) / wall,
           "horizon_time_units": list(horizon), "N_set": [12, 16, 24, 32], "lambda_set": [0, 1]}
    if bkw_every:
        out["bkw"] = bkw_errors(done, srv.L, srv.dt)
    return out


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="Poisson serving run of the relaxation server")
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--rate", type=float, nargs="+", default=[50.0])
    ap.add_argument("--horizon", type=float, nargs=2, default=[0.1, 0.5])
    ap.add_argument("--seed", type=int, default=13014195)
    args = ap.parse_args()
    from . import build as _b
    _b.build()
    for rate in args.rate:
        print(json.dumps(serve_bench(args.requests, rate, args.seed, tuple(args.horizon))), flush=True)
