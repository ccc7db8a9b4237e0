"""Serving driver for the FFT function block's request server.

The paper offloads a function block of an application that keeps running in
its production environment (Sec. 3.1, Sec. 5.1(c)); here many callers send
transform requests of mixed shapes to one GPU.  The server itself -- FIFO
admission by a device-memory budget, stream slots, resident plans, completion
events -- is native code in the library (``fb_fft_server_*``); this module
builds the request mix, replays an arrival trace against it, and replays the
same trace against the plain per-call path for comparison.

Latency of a request = completion seen by the host - its scheduled arrival,
so host-side queueing counts.  "plain" = one resident ``fb_fft_plan`` per
shape, one call at a time on one stream, each call synchronised before the
next starts (what a caller of the per-call API gets).
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import fbfft, inputs


# -- workload ----------------------------------------------------------------------
def request_mix(count: int, seed: int, max_1d: int = 1 << 22, max_2d: int = 512, max_3d: int = 128):
    """Shapes of `count` requests: 60 % 1-D with N 5-smooth, log-uniform in
    [2^8, max_1d]; 25 % 2-D with each side 5-smooth log-uniform in [16, max_2d];
    15 % 3-D with each side in [8, max_3d].  Shapes the planner rejects (a 1-D
    length with no four-step split) are redrawn."""
    rng = np.random.default_rng(seed)
    kinds = rng.choice(3, size=count, p=[0.60, 0.25, 0.15])
    shapes = []
    for k in kinds:
        while True:
            s = int(rng.integers(1 << 30))
            if k == 0:
                dims = (int(inputs.uneven_lengths(1, 256, max_1d, s)[0]),)
            elif k == 1:
                dims = tuple(int(v) for v in inputs.uneven_lengths(2, 16, max_2d, s))
            else:
                dims = tuple(int(v) for v in inputs.uneven_lengths(3, 8, max_3d, s))
            try:
                fbfft.plan_query(list(dims))
            except fbfft.FFTError:
                continue
            shapes.append(dims)
            break
    return shapes


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate; 0 for rate=inf."""
    if math.isinf(rate_per_s):
        return np.zeros(count)
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


class Workload:
    """Device-resident inputs/outputs (and pinned host copies) of a request list."""

    def __init__(self, shapes, seed: int, directions=None, host: bool = False, device: str = "cuda"):
        import torch
        self.shapes = [tuple(s) for s in shapes]
        self.directions = list(directions) if directions is not None else [fbfft.FORWARD] * len(shapes)
        self.n = [int(np.prod(s)) for s in self.shapes]
        self.x = [torch.from_numpy(inputs.uniform_c64((n,), seed + i)).to(device) for i, n in enumerate(self.n)]
        self.y = [torch.empty_like(v) for v in self.x]
        self.hx = self.hy = None
        if host:
            self.hx = [v.cpu().pin_memory() for v in self.x]
            self.hy = [torch.empty_like(v).pin_memory() for v in self.hx]
        torch.cuda.synchronize()
        self._reqs = {}

    def requests(self, host_io: bool = False):
        """The whole request list as one fb_fft_server_request array (tag = index)."""
        if host_io not in self._reqs:
            xs, ys = (self.hx, self.hy) if host_io else (self.x, self.y)
            self._reqs[host_io] = fbfft.Server.requests(
                [(s, xs[i].data_ptr(), ys[i].data_ptr(), i, self.directions[i], 1, False, host_io)
                 for i, s in enumerate(self.shapes)])
        return self._reqs[host_io]

    def bytes_moved(self) -> int:
        """Algorithmic bytes of all requests: one read and one write of each array."""
        return sum(2 * 8 * n for n in self.n)


# -- replay ------------------------------------------------------------------------
def _stats(lat_s: np.ndarray, wall_s: float, nbytes: int) -> dict:
    lat = lat_s * 1e3
    return {"requests": int(lat.size), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "throughput_req_s": lat.size / wall_s, "throughput_gbs": nbytes / wall_s / 1e9, "wall_s": wall_s}


def run_served(server: fbfft.Server, w: Workload, arrivals: np.ndarray, host_io: bool = False,
               together: bool = True) -> dict:
    """Replay `arrivals` against `server`; returns latency/throughput stats.
    together: every request whose arrival time has passed is handed over in
    one fb_fft_server_submit_many call (what a front end that collects
    requests does); False: one fb_fft_server_submit per request."""
    count = len(w.shapes)
    done_at = np.full(count, np.nan)
    status = np.zeros(count, dtype=np.int64)
    arrivals = np.asarray(arrivals, dtype=np.float64)
    if together and count and np.any(np.diff(arrivals) < 0):
        together = False
    reqs = w.requests(host_io) if together else None

    def take(items):
        for tag, st, _slot, _ts, _ta, td in items:
            done_at[tag] = td
            status[tag] = st

    t0 = server.clock()
    i = 0
    while i < count:
        if together:
            j = int(np.searchsorted(arrivals, server.clock() - t0, side="right"))
            if j > i:
                st = server.submit_many(reqs, i, j - i)
                if any(st):
                    raise RuntimeError(f"requests rejected: {[(i + k, v) for k, v in enumerate(st) if v][:5]}")
                i = j
                take(server.poll())
            else:  # nothing due yet: watch the running requests until the next arrival
                due = t0 + arrivals[i]
                server.wait(due)
                items = server.poll()
                take(items)
                if not items:
                    # the wait ended with nothing finished before `due`:
                    # nothing is running, so no completion can be missed;
                    # spin to the arrival as the plain replay does (a turn
                    # of this loop is several microseconds of Python)
                    while server.clock() < due:
                        pass
            continue
        due = t0 + arrivals[i]
        while server.clock() < due:
            take(server.poll())
        if host_io:
            server.submit_ptr(w.shapes[i], w.hx[i].data_ptr(), w.hy[i].data_ptr(), i, w.directions[i], host_io=True)
        else:
            server.submit_ptr(w.shapes[i], w.x[i].data_ptr(), w.y[i].data_ptr(), i, w.directions[i])
        take(server.poll())
        i += 1
    server.drain()
    take(server.poll())
    if np.isnan(done_at).any() or (status != 0).any():
        bad = [(i, int(status[i])) for i in range(count) if status[i] != 0 or np.isnan(done_at[i])][:5]
        raise RuntimeError(f"requests did not complete: {bad}")
    wall = float(np.nanmax(done_at) - t0)
    return _stats(done_at - (t0 + arrivals), wall, w.bytes_moved())


def plain_plans(w: Workload, stream=None) -> dict:
    """One resident per-call plan for every shape of the workload."""
    plans = {}
    for s in w.shapes:
        if s not in plans:
            plans[s] = fbfft.Plan(list(s), 1, stream=stream)
    return plans


def run_plain(plans: dict, w: Workload, arrivals: np.ndarray, host_io: bool = False) -> dict:
    """Replay `arrivals` through the per-call path: one call at a time, each
    synchronised (exec + stream sync, or exec_host) before the next."""
    import torch
    count = len(w.shapes)
    done_at = np.empty(count)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    for i in range(count):
        due = t0 + arrivals[i]
        while time.perf_counter() < due:
            pass
        p = plans[w.shapes[i]]
        if host_io:
            p.exec_host(w.hx[i].numpy(), w.hy[i].numpy(), w.directions[i])
        else:
            p.set_stream(stream)
            p.exec_ptr(w.x[i].data_ptr(), w.y[i].data_ptr(), w.directions[i])
            stream.synchronize()
        done_at[i] = time.perf_counter()
    wall = float(done_at[-1] - t0) if count else 0.0
    return _stats(done_at - (t0 + arrivals), wall, w.bytes_moved())
