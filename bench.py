"""Benchmark of the FFT function block on GB300.

Headline workload: 3-D complex64 C2C 256x256x128, re/im iid standard normal
from a fixed seed, forward then inverse with 1/N scale; one step = one forward
and one inverse exec of that volume (the whole hot path).  Metric: effective
HBM bandwidth, algorithmic bytes (one read + one write of the volume per exec,
2 * 2 * 8 * N per step) / time, in GB/s; 5 N log2 N flops per exec are reported
beside it.  Four input/output buffer pairs (512 MiB) rotate between steps so
the working set exceeds the 126 MB L2.

The default run (no --workload) prints ONE JSON line: the headline workload's
line, with every other workload's own line under the key ``workloads`` (each
with its time, GB/s, the dominant kernel's event-timed roofline, its error
against the FP64 oracle and its clocks):

  1d4096     1-D N=4096 x 64, uniform
  1d4096L    1-D N=4096 x 16384, uniform (the large batched transform)
  1d2p20     1-D N=2^20 x 32, normal, FP32 path
  1d2p20tc   the same with the radix-16 stages on the tensor cores
  uneven     4096 1-D transforms, lengths 5-smooth log-uniform in [64, 65536]
  serving    2000 requests of mixed 1-D/2-D/3-D shapes, Poisson arrivals
  grid2048   2-D 2048x2048 (the paper's FFT grid), forward then inverse 1/N

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload 3d|1d4096|...]   (one workload alone)

Under torchrun each rank runs its own replica (independent transforms, no
collective on the data path); rank 0 prints the line.  --impl reference times
the CPU oracle (FP64) on this machine's cores on the headline workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2004_09883_gb300 import inputs  # noqa: E402

METRIC = "C2C FFT GB/s vs HBM peak; 5NlogN GFLOP/s; served p50/p99 vs plain path"
WORKLOADS = {
    "3d": dict(name="3d_c2c_256x256x128_fwd_then_inv_scaled", dims=[256, 256, 128], batch=1,
               seed=inputs.seed_for(inputs.WORKLOAD_3D_256x256x128), dist="normal", inverse=True),
    "1d4096": dict(name="1d_c2c_4096_batch64_fwd", dims=[4096], batch=64,
                   seed=inputs.seed_for(inputs.WORKLOAD_1D_4096x64), dist="uniform", inverse=False),
    "1d4096L": dict(name="1d_c2c_4096_batch16384_fwd", dims=[4096], batch=16384,
                    seed=inputs.seed_for(inputs.WORKLOAD_1D_4096x64), dist="uniform", inverse=False),
    "uneven": dict(name="1d_c2c_uneven_4096_lengths_64_to_65536_fwd", dims=None, batch=4096,
                   seed=inputs.seed_for(inputs.WORKLOAD_UNEVEN_4096), dist="uniform", inverse=False,
                   lengths=(4096, 64, 65536)),
    "1d2p20": dict(name="1d_c2c_2p20_batch32_fwd", dims=[1 << 20], batch=32,
                   seed=inputs.seed_for(inputs.WORKLOAD_1D_2P20x32), dist="normal", inverse=False),
    "1d2p20tc": dict(name="1d_c2c_2p20_batch32_fwd_tensor_core_radix16", dims=[1 << 20], batch=32,
                     seed=inputs.seed_for(inputs.WORKLOAD_1D_2P20x32), dist="normal", inverse=False, tc=True),
    "serving": dict(name="serving_mix_2000_requests_1d_2d_3d_poisson", dims=None, batch=1,
                    seed=inputs.seed_for(inputs.WORKLOAD_SERVING), dist="uniform", inverse=False,
                    serving=dict(requests=2000, host_requests=600, slots=8, hbm_cap=40 * 10 ** 9, max_batch=64,
                                 fractions=[0.1, 0.25, 0.5, 0.75, 0.9, 1.1], checked=100)),
    "grid2048": dict(name="2d_c2c_2048x2048_fwd_then_inv_scaled", dims=[2048, 2048], batch=1,
                     seed=inputs.seed_for(inputs.WORKLOAD_GRID_2048x2048), dist="normal", inverse=True),
}
HEADLINE = "3d"
SUITE = ["1d4096", "1d4096L", "1d2p20", "1d2p20tc", "uneven", "serving", "grid2048"]
# error check: every batch item up to this many elements, else the first ERR_ITEMS items
ERR_ALL_ELEMS = 1 << 25
ERR_ITEMS = 64
# sources that decide what the timed kernels do (device code and the planner's launch choices)
KERNEL_SOURCES = sorted(
    os.path.join("paper_2004_09883_gb300", "csrc", f)
    for f in os.listdir(os.path.join(ROOT, "paper_2004_09883_gb300", "csrc"))
    if f.endswith((".cuh", ".h")) or f.startswith(("fft_kernels", "twiddle")) or f == "fb_fft.cu")


def kernel_hash() -> str:
    """Hash of the kernel sources' code: comments and blank lines are left
    out, so documentation edits keep a committed capture valid."""
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for line in text.splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def load_traffic(workload: str, pass_name: str | None = None) -> dict | None:
    """DRAM bytes per launch from a committed ncu capture, valid only while the
    kernel sources are unchanged since the capture.  A workload holds one
    entry, or a list of them (one per pass role, e.g. the batched uneven exec
    in one launch and in two)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(workload)
    for x in (e if isinstance(e, list) else [e] if e else []):
        if x.get("kernel_hash") == kernel_hash() and (pass_name is None or x.get("pass") == pass_name):
            return x
    return None


class ClockSampler:
    """nvidia-smi clock/throttle samples (200 ms) with host timestamps."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.samples = []
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0: float, t1: float) -> dict:
        win = [s for t, s in self.samples if t0 <= t <= t1]
        where = "timed"
        if not win:  # timed region shorter than the sampling period: widen to the pre-roll
            win = [s for t, s in self.samples if t0 - 2.0 <= t <= t1 + 0.5]
            where = "timed+preroll"
        if not win:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "window": where}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(s[1]) for s in win if num(s[1]) is not None]
        mx = [num(s[2]) for s in win if num(s[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in win for i in range(4) if s[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max((num(s[3]) or 0.0) for s in win), "reasons": reasons,
                "samples": len(win), "window": where}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------
# Multi-rank host logic (replicas: each rank transforms its own inputs; no
# collective touches the data path, only the timing reduction below)
# ---------------------------------------------------------------------------
def replica_rep(rank: int, r: int) -> int:
    """Seed repeat index of buffer r on `rank`: distinct data on every rank."""
    return rank * 16 + r


def max_over_ranks(x: float, dist, device) -> float:
    """Largest value of x over all ranks (per-step times: the job is as slow
    as its slowest rank).  dist None = single process."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank_step: float, ms_per_step: float) -> float:
    """Units all ranks processed per second, from the slowest rank's step time."""
    return world * units_per_rank_step / (ms_per_step / 1e3)


def make_input(wl: dict, rep: int) -> np.ndarray:
    shape = [wl["batch"]] + wl["dims"]
    gen = inputs.normal_c64 if wl["dist"] == "normal" else inputs.uniform_c64
    return gen(shape, wl["seed"] + 1000 * rep)


def algorithmic(wl: dict) -> tuple[float, float, int]:
    """(bytes per step, flops per step, execs per step)."""
    n = int(np.prod(wl["dims"]))
    execs = 2 if wl["inverse"] else 1
    return execs * 2 * 8.0 * n * wl["batch"], execs * 5.0 * n * math.log2(n) * wl["batch"], execs


def config_of(wl: dict, world: int) -> dict:
    """The workload's `config` object, the same on the GPU arm and the reference arm."""
    n = int(np.prod(wl["dims"]))
    nbuf = buffers_for(wl)
    return {"workload": wl["name"], "dims": wl["dims"], "batch": wl["batch"], "dtype_storage": "complex64",
            "l2": f"{nbuf} rotating input/output buffer pairs ({nbuf * 2 * 8 * n * wl['batch'] / 2 ** 20:.0f} MiB)"
                  f" > 126 MB L2",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def buffers_for(wl: dict) -> int:
    n = int(np.prod(wl["dims"]))
    return min(8, max(2, int(math.ceil(512 * 2 ** 20 / (2 * 8 * n * wl["batch"])))))


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and the cpu_baseline object)
# ---------------------------------------------------------------------------
def oracle_sample(wl: dict, budget_s: float, threads: int) -> dict:
    """Time the FP64 oracle on the workload.  Runs whole steps (forward, plus
    inverse when the workload has one) until `budget_s` is spent (at least
    one); returns GB/s in the workload's own byte accounting."""
    import oracle

    x = make_input(wl, 0).astype(np.complex128)
    bytes_step, _, _ = algorithmic(wl)
    dims = wl["dims"]
    reps, t_total = 0, 0.0
    while reps == 0 or t_total < budget_s:
        t = time.perf_counter()
        y = oracle.fft(x, dims, -1, False, threads)
        if wl["inverse"]:
            oracle.fft(y, dims, 1, True, threads)
        t_total += time.perf_counter() - t
        reps += 1
    return {"value": bytes_step * reps / t_total / 1e9, "seconds": t_total, "steps": reps}


def workload_shapes(wl: dict) -> list[tuple]:
    """Transform shapes of a many-transform workload, in order."""
    if wl.get("serving"):
        from paper_2004_09883_gb300 import serving
        return serving.request_mix(wl["serving"]["requests"], wl["seed"])
    return [(int(n),) for n in uneven_lengths(wl)]


def oracle_single_thread(wl: dict, budget_s: float) -> dict:
    """The oracle on one host thread, one batch item at a time (forward, plus
    inverse when the workload has one) until `budget_s` is spent (at least
    one item); GB/s in the workload's byte accounting."""
    import oracle

    bytes_step, _, _ = algorithmic(wl)
    per_item = bytes_step / wl["batch"]
    x = make_input(wl, 0)
    done, t_total, k = 0.0, 0.0, 0
    while k == 0 or (t_total < budget_s and k < wl["batch"]):
        item = x[k % wl["batch"]].astype(np.complex128)
        t = time.perf_counter()
        y = oracle.fft(item, wl["dims"], -1, False, 1)
        if wl["inverse"]:
            oracle.fft(y, wl["dims"], 1, True, 1)
        t_total += time.perf_counter() - t
        done += per_item
        k += 1
    return {"value": done / t_total / 1e9, "seconds": t_total, "items": k}


def oracle_uneven_sample(wl: dict, budget_s: float, threads: int) -> dict:
    """Time the oracle on a many-transform workload's transforms, in order,
    until the budget is spent (at least one); GB/s over the transforms done."""
    import oracle

    shapes = workload_shapes(wl)
    done_bytes, t_total, k = 0.0, 0.0, 0
    while k < len(shapes) and (k == 0 or t_total < budget_s):
        dims = list(shapes[k])
        n = int(np.prod(dims))
        x = inputs.uniform_c64((n,), wl["seed"] + k).astype(np.complex128)
        t = time.perf_counter()
        oracle.fft(x, dims, -1, False, threads)
        t_total += time.perf_counter() - t
        done_bytes += 2 * 8.0 * n
        k += 1
    return {"value": done_bytes / t_total / 1e9, "seconds": t_total, "transforms": k}


def oracle_each(items, threads: int, sign: int = -1, scale: bool = False) -> list:
    """The oracle on a list of (array, dims): one transform per worker thread
    (its C routine runs without the interpreter lock)."""
    import oracle

    def one(it):
        x, dims = it
        return oracle.fft(np.asarray(x).astype(np.complex128), list(dims), sign, scale)
    with ThreadPoolExecutor(max(1, threads)) as ex:
        return list(ex.map(one, items))


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def host_threads() -> int:
    return len(os.sched_getaffinity(0))


def run_reference(args, wl: dict) -> None:
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    threads = host_threads()
    if wl.get("lengths") or wl.get("serving"):  # many transforms: each step a bounded sample of them
        per_step = max(0.5, 150.0 / max(1, args.steps + args.warmup))
        for _ in range(args.warmup):
            oracle_uneven_sample(wl, per_step, threads)
        runs = [oracle_uneven_sample(wl, per_step, threads) for _ in range(args.steps)]
        secs = sum(r["seconds"] for r in runs)
        value = sum(r["value"] * r["seconds"] for r in runs) / secs
        total = len(workload_shapes(wl))
        desc = (f"first {runs[0]['transforms']} of {total} transforms of {wl['name']} per step, FP64 oracle, "
                f"{threads} threads on {cpu_model()}")
        line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": wl["name"], "parallelism": "host threads"},
                "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                                 "sample": desc},
                "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    bytes_step, flops_step, _ = algorithmic(wl)
    # one step = one forward(+inverse) of the workload by the oracle; for long
    # runs each step is a bounded sample: a share of the batch items (the
    # 3-D volume is one item, so it always runs whole).
    per_step_budget = max(0.5, 150.0 / max(1, args.steps + args.warmup))
    import oracle

    x = make_input(wl, 0).astype(np.complex128)
    dims = wl["dims"]
    # size the per-step sample (batch items) to the budget
    t = time.perf_counter()
    oracle.fft(x[:1], dims, -1, False, threads)
    one = max(1e-6, time.perf_counter() - t) * (2 if wl["inverse"] else 1)
    items = int(max(1, min(wl["batch"], per_step_budget // one)))
    sample = x[:items]

    def step():
        y = oracle.fft(sample, dims, -1, False, threads)
        if wl["inverse"]:
            oracle.fft(y, dims, 1, True, threads)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    frac = items / wl["batch"]
    value = bytes_step * frac / dt / 1e9
    desc = (f"{items} of {wl['batch']} batch item(s) of {wl['name']} per step, FP64 oracle, "
            f"{threads} threads on {cpu_model()}")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        # the same workload description as the GPU arm's line (the oracle runs on its host cores)
        "config": config_of(wl, world),
        "gflops": flops_step * frac / dt / 1e9,
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
class Ctx:
    """Device, process group and library of one rank (set up once per run)."""

    def __init__(self):
        import torch

        self.world, self.rank, self.local = dist_setup()
        torch.cuda.set_device(self.local)
        self.dev = torch.device("cuda", self.local)
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl", device_id=self.dev)
            self.dist = dist
        from paper_2004_09883_gb300 import build as fbbuild
        fbbuild.build()
        from paper_2004_09883_gb300 import fbfft
        self.fb = fbfft
        self.stream = torch.cuda.current_stream(self.dev)

    def barrier(self):
        import torch
        torch.cuda.synchronize(self.dev)
        if self.dist is not None:
            self.dist.barrier()
        torch.cuda.synchronize(self.dev)

    def max(self, x: float) -> float:
        return max_over_ranks(x, self.dist, self.dev)

    def close(self):
        if self.dist is not None:
            self.dist.barrier()
            self.dist.destroy_process_group()


def event_timed(ctx: Ctx, step, steps: int, warmup: int):
    """(ms per step, max over ranks; library launches) of `steps` calls of
    step(i) between two CUDA events on the launching stream, after `warmup`
    untimed calls."""
    import torch
    for i in range(warmup):
        step(i)
    ctx.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = ctx.fb.launch_count()
    e0.record(ctx.stream)
    for i in range(steps):
        step(i)
    e1.record(ctx.stream)
    ctx.barrier()
    return ctx.max(e0.elapsed_time(e1) / steps), ctx.fb.launch_count() - l0


def roofline_of(passes, prof_steps: int, execs: int, bytes_per_exec: float, wl_name: str, peaks: dict,
                basis: str | None = None):
    """Roofline of the dominant kernel: the pass role with the largest measured
    time.  One launch covers the exec's data divided by the role's launches per
    exec (four-step roles run once per batch chunk); algorithmic bytes = one
    read + one write of that data."""
    dom = max(passes, key=lambda r: r[1]) if passes else None
    if not dom or dom[2] <= 0:
        return None
    per_launch_ms = dom[1] / dom[2]
    launches_per_exec = dom[2] / (prof_steps * execs)
    launch_bytes = bytes_per_exec / launches_per_exec
    achieved = launch_bytes / (per_launch_ms / 1e3) / 1e9
    tr = load_traffic(wl_name, dom[0])
    traffic = tr["dram_bytes_per_launch"] if tr else None
    r = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peaks["hbm_gbs"], "unit": "GB/s",
         "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
         "kernel_pass": dom[0], "launch_ms": round(per_launch_ms, 5), "algorithmic_bytes_per_launch": launch_bytes,
         "peak_source": f"{peaks['source']} (MEASURED_PEAKS.json hbm_gbs, burst copy)"
         if peaks["source"] == "measured" else "fallback 6.8 TB/s"}
    if traffic is not None:
        r["traffic_note"] = ("dram__bytes_read.sum + dram__bytes_write.sum of this kernel's launch in one ncu "
                             "capture: reads plus the write-back that happens during the launch (the rest of "
                             "the output is written back to HBM during later launches)")
    if basis:
        r["basis"] = basis
    return r


def error_items(batch: int, n: int) -> int:
    return batch if batch * n <= ERR_ALL_ELEMS else min(batch, ERR_ITEMS)


def gpu_regular(args, ctx: Ctx, wl: dict, headline: bool) -> dict:
    """A regular plan (rank 1-3, batch): timed steps, per-pass roofline,
    e2e through fb_fft_exec_host, errors against the oracle, CPU baseline."""
    import torch
    fbfft = ctx.fb
    dev, stream, world, rank = ctx.dev, ctx.stream, ctx.world, ctx.rank
    dims, batch = wl["dims"], wl["batch"]
    n = int(np.prod(dims))
    bytes_step, flops_step, execs = algorithmic(wl)
    nbuf = buffers_for(wl)
    host_inputs = [make_input(wl, replica_rep(rank, r)) for r in range(nbuf)]
    xin = [torch.from_numpy(h.reshape(-1)).to(dev) for h in host_inputs]
    xout = [torch.empty_like(xin[0]) for _ in range(nbuf)]
    tc = bool(wl.get("tc"))
    plan = fbfft.Plan(dims, batch, scale_inv_n=wl["inverse"], stream=stream, tensor_cores=tc)
    threads = host_threads()

    def step(i, p=None):
        p = p or plan
        a, b = xin[i % nbuf], xout[i % nbuf]
        p.exec_ptr(a.data_ptr(), b.data_ptr(), fbfft.FORWARD)
        if wl["inverse"]:
            p.exec_ptr(b.data_ptr(), b.data_ptr(), fbfft.INVERSE)

    clocks = ClockSampler(ctx.local) if rank == 0 and not args.quick else None
    for i in range(args.warmup):
        step(i)
    # pre-roll: untimed extra warm-up so the clock samples see a loaded GPU
    t_pre = time.time()
    i = 0
    while not args.quick and time.time() - t_pre < 1.0:
        step(i)
        i += 1
        if i % 64 == 0:
            torch.cuda.synchronize(dev)
    wall0 = time.time()
    ms, launches = event_timed(ctx, step, args.steps, 0)
    wall1 = time.time()
    # per-pass launch times, in a separate run: the event pair around every
    # launch serialises the passes, which the timed loop above lets overlap
    prof_steps = max(3, min(args.steps, 50))
    plan.profile(True)
    for i in range(prof_steps):
        step(i)
    ctx.barrier()
    passes = plan.profile_read()
    plan.profile(False)
    plan.check()
    clk = clocks.summary(wall0, wall1) if clocks else None
    if clocks:
        clocks.stop()

    # tensor-core workload: the plain FP32 plan on the same buffers, the plain
    # per-call FP32 path, and every result of both plans against the oracle
    precision = None
    errors = None
    if tc:
        p32 = fbfft.Plan(dims, batch, scale_inv_n=wl["inverse"], stream=stream)
        ms32, _ = event_timed(ctx, lambda i: step(i, p32), args.steps, args.warmup)
        precision = {"fp32_path": {"value": round(whole_job_rate(world, bytes_step, ms32) / 1e9, 3), "unit": "GB/s",
                                   "ms_per_step": round(ms32, 5)},
                     "speedup_vs_fp32_path": round(ms32 / ms, 3), "tolerance_rel_l2": 5e-5}
        # the plain per-call FP32 path: one exec per transform (a resident
        # batch-1 plan), as the replaced CPU routine is called per transform
        p1 = fbfft.Plan(dims, 1, stream=stream)

        def step_per_call(i):
            a, b = xin[i % nbuf], xout[i % nbuf]
            for k in range(batch):
                p1.exec_ptr(a.data_ptr() + k * n * 8, b.data_ptr() + k * n * 8, fbfft.FORWARD)
        ms1, _ = event_timed(ctx, step_per_call, args.steps, args.warmup)
        p1.check()
        p1.close()
        precision["per_call_fp32_path"] = {"value": round(whole_job_rate(world, bytes_step, ms1) / 1e9, 3),
                                           "unit": "GB/s", "ms_per_step": round(ms1, 5), "calls_per_step": batch}
        precision["speedup_vs_per_call_fp32_path"] = round(ms1 / ms, 3)
        if rank == 0 and not args.quick:
            import oracle
            x = host_inputs[0].reshape(batch, n)
            ref = oracle.fft(x.astype(np.complex128), dims, fbfft.FORWARD, False, threads).reshape(batch, n)
            for name, p in (("tensor_cores", plan), ("fp32", p32)):
                y = p.exec(xin[0], None, fbfft.FORWARD)
                torch.cuda.synchronize(dev)
                e = oracle.rel_l2(y.cpu().numpy().reshape(batch, n), ref)
                precision[f"{name}_max_rel_l2"] = float(e.max())
                precision[f"{name}_median_rel_l2"] = float(np.median(e))
                precision[f"{name}_rel_l2_per_result"] = [float(f"{v:.3e}") for v in e]
                if name == "tensor_cores":
                    errors = {"forward_max_rel_l2": float(e.max()), "forward_median_rel_l2": float(np.median(e)),
                              "tolerance_rel_l2": 5e-5, "items": batch, "pass": bool(e.max() <= 5e-5)}
            precision["errors"] = f"all {batch} results of input buffer 0 against the FP64 oracle"
        p32.close()

    # end to end through the drop-in host-array call: every step copies the
    # input host->device and the result device->host inside the call
    e2e = None
    if not args.quick:
        bufs = pinned_buffers(n * batch, 4)
        hbuf, hres = bufs[:2], bufs[2:]
        for b, h in zip(hbuf, host_inputs[:2]):
            b.copy_(torch.from_numpy(h.reshape(-1)))
        e2e_steps = max(3, min(args.steps, 20 if headline else 10))

        def e2e_step(i):
            src, dst = hbuf[i % 2], hres[i % 2]
            plan.exec_host(src.numpy(), dst.numpy(), fbfft.FORWARD)
            if wl["inverse"]:
                plan.exec_host(dst.numpy(), dst.numpy(), fbfft.INVERSE)

        for i in range(2):
            e2e_step(i)
        ctx.barrier()
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            e2e_step(i)
        ctx.barrier()
        e2e_ms = ctx.max((time.perf_counter() - t0) / e2e_steps * 1e3)
        io = 8 * n * batch * execs
        e2e = {"value": round(whole_job_rate(world, bytes_step, e2e_ms) / 1e9, 3), "unit": "GB/s",
               "h2d_bytes_per_step": io, "d2h_bytes_per_step": io, "ms_per_step": e2e_ms,
               "path": "fb_fft_exec_host (pinned host arrays)" + (", forward then inverse" if wl["inverse"] else ", forward")}

    # error against the oracle: every batch item of input buffer 0 (the first
    # ERR_ITEMS items of very large batches)
    if rank == 0 and not args.quick and not tc:
        import oracle
        k = error_items(batch, n)
        x0 = host_inputs[0].reshape(batch, n)[:k]
        y = plan.exec(xin[0], None, fbfft.FORWARD)
        torch.cuda.synchronize(dev)
        yk = y.cpu().numpy().reshape(batch, n)[:k]
        ref = oracle.fft(x0.astype(np.complex128).reshape([k] + dims), dims, fbfft.FORWARD, False, threads)
        e = oracle.rel_l2(yk, ref.reshape(k, n))
        tol = 2e-6 * math.log2(n)
        errors = {"forward_max_rel_l2": float(e.max()), "forward_median_rel_l2": float(np.median(e)),
                  "tolerance_rel_l2": tol, "items": k, "of_items": batch}
        ok = e.max() <= tol
        if wl["inverse"]:
            z = plan.exec(y, None, fbfft.INVERSE)
            torch.cuda.synchronize(dev)
            zk = z.cpu().numpy().reshape(batch, n)[:k]
            refi = oracle.fft(yk.astype(np.complex128).reshape([k] + dims), dims, fbfft.INVERSE, True, threads)
            ei = oracle.rel_l2(zk, refi.reshape(k, n))
            rt = oracle.rel_l2(zk, x0.astype(np.complex128))
            errors.update({"inverse_max_rel_l2": float(ei.max()), "round_trip_max_rel_l2": float(rt.max())})
            ok = ok and ei.max() <= tol and rt.max() <= tol
        errors["pass"] = bool(ok)

    # library context: cuFFT through torch.fft on the same buffers (not part of the product)
    context = None
    if not args.quick:
        axes = tuple(range(1, len(dims) + 1))

        def lib_step(i):
            yy = torch.fft.fftn(xin[i % nbuf].view([batch] + dims), dim=axes)
            if wl["inverse"]:
                torch.fft.ifftn(yy, dim=axes)

        lib_ms, _ = event_timed(ctx, lib_step, args.steps, args.warmup)
        context = {"library": "cuFFT via torch.fft on the same GPU and buffers (a reference point, not part of "
                              "this product)", "value": round(bytes_step / (lib_ms / 1e3) / 1e9, 3), "unit": "GB/s",
                   "ms_per_step": round(lib_ms, 5)}

    line = None
    if rank == 0:
        peaks = load_peaks()
        value = whole_job_rate(world, bytes_step, ms) / 1e9
        roofline = roofline_of(passes, prof_steps, execs, 2 * 8.0 * n * batch, wl["name"], peaks)
        cpu_baseline = None
        if not args.quick:
            cb = oracle_sample(wl, budget_s=float(args.cpu_budget if headline else args.cpu_budget_sub), threads=threads)
            st1 = oracle_single_thread(wl, budget_s=3.0 if headline else 1.0)
            cpu_baseline = {"value": round(cb["value"], 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                            "sample": f"{cb['steps']} full step(s) of {wl['name']} by the FP64 oracle in "
                                      f"{cb['seconds']:.1f} s on {cpu_model()}",
                            "single_thread": {"value": round(st1["value"], 5), "unit": "GB/s",
                                              "sample": f"{st1['items']} batch item(s), one thread, "
                                                        f"{st1['seconds']:.1f} s"}}
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 5), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16 hi/lo products, f32 accumulate" if tc else "f32", "data": "synthetic",
            "config": config_of(wl, world),
            "gflops": round(whole_job_rate(world, flops_step, ms) / 1e9, 2),
            "hbm_frac_effective": round(value / world / peaks["hbm_gbs"], 4),
            "roofline": roofline,
            "cpu_baseline": cpu_baseline,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk,
            "passes": [{"pass": p[0], "ms_per_launch": round(p[1] / max(1, p[2]), 5), "launches": p[2]}
                       for p in passes],
            "kernel_hash": kernel_hash(),
        }
        if precision:
            line["precision"] = precision
        if errors:
            line["errors_vs_oracle"] = errors
        if context:
            line["context"] = context
    plan.close()
    return line


def uneven_lengths(wl: dict) -> np.ndarray:
    count, lo, hi = wl["lengths"]
    return inputs.uneven_lengths(count, lo, hi, wl["seed"])


def uneven_roofline(passes, prof_steps, lens, bytes_step, ms, launches_per_exec, wl_name, peaks):
    """Roofline of a batched uneven exec.  One-kernel engine: its one launch
    moves one read and one write of every value (the single passes and the
    four-step columns) plus one of every value of a length above 2048 (the
    four-step rows); in its two-launch form, the dominant launch (phase 0 the
    first part, phase 1 the rows).  The per-kernel engine: the whole exec (all
    its launches)."""
    rows = float(sum(16 * int(n) for n in lens if int(n) > 2048))
    phase_bytes = {"many.uneven": bytes_step + rows, "many.uneven.phase0": bytes_step,
                   "many.uneven.phase1": rows}
    dom = max(passes, key=lambda r: r[1]) if passes else None
    if dom and dom[0] in phase_bytes and dom[2] > 0:
        per_launch_ms = dom[1] / dom[2]
        achieved = phase_bytes[dom[0]] / (per_launch_ms / 1e3) / 1e9
        tr = load_traffic(wl_name, dom[0])
        traffic = tr["dram_bytes_per_launch"] if tr else None
        r = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peaks["hbm_gbs"], "unit": "GB/s",
             "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic, "kernel_pass": dom[0],
             "launch_ms": round(per_launch_ms, 5), "algorithmic_bytes_per_launch": phase_bytes[dom[0]],
             "launches_per_exec": round(launches_per_exec, 2),
             "basis": "one read + one write of the values the launch transforms / its event-timed duration"}
        if traffic is not None:
            r["traffic_note"] = ("dram__bytes_read.sum + dram__bytes_write.sum of this launch in one ncu capture "
                                 "(reads plus the write-back during the launch)")
        return r
    return {"bound": "hbm", "achieved": round(bytes_step / (ms / 1e3) / 1e9, 2), "peak": peaks["hbm_gbs"],
            "unit": "GB/s", "frac": round(bytes_step / (ms / 1e3) / 1e9 / peaks["hbm_gbs"], 4), "traffic": None,
            "kernel_pass": "whole exec", "launches_per_exec": round(launches_per_exec, 2),
            "algorithmic_bytes_per_launch": bytes_step,
            "basis": "one read + one write of every transform / exec time (all launches of one exec)"}


def gpu_many(args, ctx: Ctx, wl: dict, headline: bool) -> dict:
    """Batched uneven 1-D lengths: one exec of the autotuned batched plan
    (fb_fft_plan_many) per step against the plain per-call path (one
    fb_fft_exec per transform, plans cached per length) on the same buffers;
    every transform checked against the oracle."""
    import torch
    fbfft = ctx.fb
    dev, stream, world, rank = ctx.dev, ctx.stream, ctx.world, ctx.rank
    lens = uneven_lengths(wl)
    _, total = fbfft.many_layout(lens)
    nbuf = 2
    host_in = [inputs.uniform_c64((total,), wl["seed"] + 1000 * replica_rep(rank, r)) for r in range(nbuf)]
    xin = [torch.from_numpy(h).to(dev) for h in host_in]
    xout = [torch.empty_like(xin[0]) for _ in range(nbuf)]
    # the library's autotuner picks the plan knobs on this workload (untimed;
    # --quick keeps the defaults so profiler runs stay short)
    if args.quick:
        tuned = fbfft.ManyOpts(engine=args.uneven_engine or 0)
    else:
        tuned, _ = fbfft.autotune_many(lens, xin[0], xout[0], fbfft.FORWARD, reps=3)
    default_plan = fbfft.PlanMany(lens, stream=stream)
    plan = fbfft.PlanMany(lens, stream=stream, opts=tuned)
    bytes_step = float(sum(2 * 8 * int(n) for n in lens))
    flops_step = float(sum(5 * int(n) * math.log2(int(n)) for n in lens))

    def batched(i):
        plan.exec_ptr(xin[i % nbuf].data_ptr(), xout[i % nbuf].data_ptr(), fbfft.FORWARD)

    clocks = ClockSampler(ctx.local) if rank == 0 and not args.quick else None
    wall0 = time.time()
    ms, launches = event_timed(ctx, batched, args.steps, args.warmup)
    wall1 = time.time()
    plan.check()
    ms_default, _ = event_timed(ctx, lambda i: default_plan.exec_ptr(
        xin[i % nbuf].data_ptr(), xout[i % nbuf].data_ptr(), fbfft.FORWARD), max(3, min(args.steps, 20)), 3)
    # the plain per-call path: one exec per transform on the same data
    plans = {}
    for n in sorted(set(int(x) for x in lens)):
        plans[n] = fbfft.Plan([n], 1, stream=stream)
    offs = plan.offsets

    def per_call(i):
        a, b = xin[i % nbuf].data_ptr(), xout[i % nbuf].data_ptr()
        for n, o in zip(lens, offs):
            plans[int(n)].exec_ptr(a + 8 * int(o), b + 8 * int(o), fbfft.FORWARD)

    ms_plain, _ = event_timed(ctx, per_call, max(3, min(args.steps, 20)), 3)
    # per-launch times of the batched plan (a separate loop: the event pairs
    # around each launch would serialise the timed loop's launches)
    prof_steps = max(3, min(args.steps, 20))
    plan.profile(True)
    for i in range(prof_steps):
        batched(i)
    ctx.barrier()
    passes = plan.profile_read()
    plan.profile(False)
    clk = clocks.summary(wall0, wall1) if clocks else None
    if clocks:
        clocks.stop()
    # end to end through the host-array call on pinned packed arrays: the
    # packed batch in, one exec, the packed result out, every step
    e2e = None
    if not args.quick:
        hbuf = [torch.from_numpy(h).pin_memory() for h in host_in]
        hres = [torch.empty_like(hbuf[0]).pin_memory() for _ in range(nbuf)]
        e2e_steps = max(3, min(args.steps, 10))
        for i in range(2):
            plan.exec_host(hbuf[i % nbuf].numpy(), hres[i % nbuf].numpy(), fbfft.FORWARD)
        ctx.barrier()
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            plan.exec_host(hbuf[i % nbuf].numpy(), hres[i % nbuf].numpy(), fbfft.FORWARD)
        ctx.barrier()
        e2e_ms = ctx.max((time.perf_counter() - t0) / e2e_steps * 1e3)
        e2e = {"value": round(whole_job_rate(world, bytes_step, e2e_ms) / 1e9, 3), "unit": "GB/s",
               "h2d_bytes_per_step": 8 * total, "d2h_bytes_per_step": 8 * total, "ms_per_step": e2e_ms,
               "path": "fb_fft_exec_host (pinned packed host arrays), forward"}
    errors = None
    if rank == 0 and not args.quick:
        y = plan.exec(xin[0], None, fbfft.FORWARD)
        torch.cuda.synchronize(dev)
        yh = y.cpu().numpy()
        import oracle
        refs = oracle_each([(host_in[0][o:o + n], [int(n)]) for o, n in zip(offs, lens)], host_threads())
        e = np.array([oracle.rel_l2(yh[o:o + n], r)[0] for o, n, r in zip(offs, lens, refs)])
        tols = np.array([2e-6 * math.log2(int(n)) for n in lens])
        errors = {"forward_max_rel_l2": float(e.max()), "forward_median_rel_l2": float(np.median(e)),
                  "max_error_over_tolerance": float((e / tols).max()),
                  "tolerance_rel_l2": "2e-6 log2 N per transform", "items": len(lens), "of_items": len(lens),
                  "pass": bool((e <= tols).all())}
    line = None
    if rank == 0:
        peaks = load_peaks()
        value = whole_job_rate(world, bytes_step, ms) / 1e9
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 5), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["name"], "transforms": len(lens), "distinct_lengths": len(plans),
                       "elements": int(sum(int(n) for n in lens)), "l2": "2 rotating buffer pairs of "
                       f"{total * 8 / 2 ** 20:.0f} MiB each > 126 MB L2", "parallelism": "replicas" if world > 1
                       else "single GPU", "path": "fb_fft_plan_many, autotuned, one exec per step"},
            "gflops": round(whole_job_rate(world, flops_step, ms) / 1e9, 2),
            "hbm_frac_effective": round(value / world / peaks["hbm_gbs"], 4),
            "roofline": uneven_roofline(passes, prof_steps, lens, bytes_step, ms, launches / max(1, args.steps),
                                        wl["name"], peaks),
            "passes": [{"pass": p[0], "ms_per_launch": round(p[1] / max(1, p[2]), 5), "launches": p[2]}
                       for p in passes],
            "plain_per_call": {"value": round(whole_job_rate(world, bytes_step, ms_plain) / 1e9, 3), "unit": "GB/s",
                               "ms_per_step": round(ms_plain, 4), "execs_per_step": len(lens)},
            "speedup_vs_plain_per_call": round(ms_plain / ms, 3),
            "autotuned": tuned.as_dict(), "untuned_plan_ms_per_step": round(ms_default, 4), "e2e": e2e,
            "cpu_baseline": None if args.quick else (lambda cb: {
                "value": round(cb["value"], 4), "unit": "GB/s", "cores": host_threads(),
                "kind": "oracle", "sample": f"first {cb['transforms']} transforms of the workload by the FP64 "
                                            f"oracle in {cb['seconds']:.1f} s on {cpu_model()}"})(
                oracle_uneven_sample(wl, float(args.cpu_budget if headline else args.cpu_budget_sub),
                                     host_threads())),
            "gpu_launches": int(launches), "clocks": clk, "kernel_hash": kernel_hash(),
        }
        if errors:
            line["errors_vs_oracle"] = errors
    for p in plans.values():
        p.close()
    plan.close()
    default_plan.close()
    return line


def gpu_serving(args, ctx: Ctx, wl: dict, headline: bool) -> dict:
    """Request server against the plain per-call path on one arrival trace:
    saturation throughput (all requests queued at t=0), then Poisson arrivals
    at fractions of the plain path's saturation rate, p50/p99 latency of both.
    Device-resident requests (inputs already in HBM, latency = arrival ->
    completion seen by the host), plus a host-array variant (pinned host
    buffers, copies through the server's staging)."""
    import torch
    from paper_2004_09883_gb300 import serving
    fbfft = ctx.fb
    world, rank = ctx.world, ctx.rank

    cfg = wl["serving"]
    seed = wl["seed"] + 1000 * replica_rep(rank, 0)
    shapes = serving.request_mix(cfg["requests"], seed)
    w = serving.Workload(shapes, seed)
    hshapes = shapes[:cfg["host_requests"]]
    wh = serving.Workload(hshapes, seed, host=True)
    srv = fbfft.Server(slots=cfg["slots"], hbm_cap_bytes=cfg["hbm_cap"], max_batch=cfg["max_batch"])
    for s in set(shapes):
        srv.prepare(list(s))
    plans = serving.plain_plans(w)
    zero, zero_h = np.zeros(len(shapes)), np.zeros(len(hshapes))
    for _ in range(args.warmup):  # untimed passes: plans, staging, allocator, caches
        serving.run_served(srv, w, zero)
        serving.run_plain(plans, w, zero)
    serving.run_served(srv, wh, zero_h, host_io=True)
    serving.run_plain(plans, wh, zero_h, host_io=True)

    steps = max(3, min(args.steps, 20))
    clocks = ClockSampler(ctx.local) if rank == 0 else None
    ctx.barrier()
    wall0 = time.time()
    l0 = fbfft.launch_count()
    sat = [serving.run_served(srv, w, zero) for _ in range(steps)]
    launches = (fbfft.launch_count() - l0) // steps
    wall1 = time.time()
    clk = clocks.summary(wall0, wall1) if clocks else None
    if clocks:
        clocks.stop()
    # the served results of the last replay against the oracle
    errors = None
    if rank == 0:
        k = min(cfg["checked"], len(shapes))
        import oracle
        refs = oracle_each([(w.x[i].cpu().numpy(), list(shapes[i])) for i in range(k)], host_threads())
        e = np.array([oracle.rel_l2(w.y[i].cpu().numpy(), refs[i].reshape(-1))[0] for i in range(k)])
        tols = np.array([2e-6 * math.log2(max(2, w.n[i])) for i in range(k)])
        errors = {"forward_max_rel_l2": float(e.max()), "forward_median_rel_l2": float(np.median(e)),
                  "max_error_over_tolerance": float((e / tols).max()),
                  "tolerance_rel_l2": "2e-6 log2 N per request", "items": k, "of_items": len(shapes),
                  "pass": bool((e <= tols).all())}
    sat_plain = [serving.run_plain(plans, w, zero) for _ in range(3)]
    # the same server with batching off: every request alone through its plan
    srv.set_batch(1)
    serving.run_served(srv, w, zero)
    sat_alone = max((serving.run_served(srv, w, zero) for _ in range(3)), key=lambda r: r["throughput_req_s"])
    srv.set_batch(cfg["max_batch"])
    ctx.barrier()
    best = max(sat, key=lambda r: r["throughput_req_s"])
    best_plain = max(sat_plain, key=lambda r: r["throughput_req_s"])
    rate_plain = best_plain["throughput_req_s"]
    sweep = []
    for k, f in enumerate(cfg["fractions"]):
        arr = serving.poisson_arrivals(len(shapes), f * rate_plain, seed + 17 + k)
        a = serving.run_served(srv, w, arr)
        b = serving.run_plain(plans, w, arr)
        sweep.append({"rate_frac_of_plain_saturation": f, "rate_req_s": round(f * rate_plain, 1),
                      "served": {q: round(a[q], 4) for q in ("p50_ms", "p99_ms", "throughput_req_s")},
                      "plain": {q: round(b[q], 4) for q in ("p50_ms", "p99_ms", "throughput_req_s")}})
    host_sat = max((serving.run_served(srv, wh, zero_h, host_io=True) for _ in range(3)),
                   key=lambda r: r["throughput_req_s"])
    host_plain = max((serving.run_plain(plans, wh, zero_h, host_io=True) for _ in range(3)),
                     key=lambda r: r["throughput_req_s"])
    # half the plain path's host-array rate: 600 requests per replay, so one
    # host-side stall can decide a percentile; three replays of each path,
    # the median of each statistic reported
    arr = serving.poisson_arrivals(len(hshapes), 0.5 * host_plain["throughput_req_s"], seed + 99)

    def median_of(runs):
        return {q: float(np.median([r[q] for r in runs])) for q in ("p50_ms", "p99_ms")}
    host_half = median_of([serving.run_served(srv, wh, arr, host_io=True) for _ in range(3)])
    host_half_plain = median_of([serving.run_plain(plans, wh, arr, host_io=True) for _ in range(3)])
    st = srv.stats()
    value = ctx.max(best["throughput_gbs"])
    line = None
    if rank == 0:
        nb = w.bytes_moved()
        kinds = {1: 0, 2: 0, 3: 0}
        for s in shapes:
            kinds[len(s)] += 1
        line = {
            "metric": METRIC, "value": round(value * world, 3), "unit": "GB/s", "n_gpus": world,
            "steps": steps, "warmup": args.warmup,
            "ms_per_step": round(best["wall_s"] * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["name"], "requests": len(shapes), "rank_mix": kinds,
                       "distinct_shapes": len(set(shapes)), "elements": int(sum(w.n)),
                       "slots": cfg["slots"], "hbm_cap_bytes": cfg["hbm_cap"], "max_batch": cfg["max_batch"],
                       "step": "one replay of the whole request list, all arriving at t=0",
                       "l2": f"{nb / 2 / 2 ** 30:.1f} GiB of distinct inputs per step > 126 MB L2",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "saturation": {"served_req_s": round(best["throughput_req_s"], 1),
                           "plain_req_s": round(rate_plain, 1),
                           "served_gbs": round(best["throughput_gbs"], 2),
                           "plain_gbs": round(best_plain["throughput_gbs"], 2),
                           "speedup_vs_plain": round(best["throughput_req_s"] / rate_plain, 3),
                           "unbatched_server_req_s": round(sat_alone["throughput_req_s"], 1),
                           "served_p50_ms": round(best["p50_ms"], 4), "served_p99_ms": round(best["p99_ms"], 4),
                           "plain_p50_ms": round(best_plain["p50_ms"], 4),
                           "plain_p99_ms": round(best_plain["p99_ms"], 4)},
            "sweep_device_resident": sweep,
            "host_arrays": {"requests": len(hshapes),
                            "saturation_req_s": {"served": round(host_sat["throughput_req_s"], 1),
                                                 "plain": round(host_plain["throughput_req_s"], 1)},
                            "half_plain_rate": {"replays": "median of 3 per path",
                                                "served_p50_ms": round(host_half["p50_ms"], 4),
                                                "served_p99_ms": round(host_half["p99_ms"], 4),
                                                "plain_p50_ms": round(host_half_plain["p50_ms"], 4),
                                                "plain_p99_ms": round(host_half_plain["p99_ms"], 4)}},
            "e2e": {"value": round(host_sat["throughput_gbs"] * world, 3), "unit": "GB/s",
                    "h2d_bytes_per_step": wh.bytes_moved() // 2, "d2h_bytes_per_step": wh.bytes_moved() // 2,
                    "ms_per_step": round(host_sat["wall_s"] * 1e3, 3),
                    "path": f"fb_fft_server_submit on pinned host arrays, the first {len(hshapes)} requests of "
                            "the mix at t=0, copies through the server's staging"},
            "server_stats": {k: st[k] for k in ("plans", "plan_builds", "arena_peak", "max_in_flight", "batches",
                                                "batched_requests", "largest_batch", "max_busy_slots")},
            "roofline": None,
            "roofline_note": "a mix of 3000+ shapes: the per-kernel rooflines are those of the other workloads",
            "gpu_launches": int(launches), "clocks": clk, "kernel_hash": kernel_hash(),
            "errors_vs_oracle": errors,
            "cpu_baseline": (lambda cb: {
                "value": round(cb["value"], 4), "unit": "GB/s", "cores": host_threads(),
                "kind": "oracle", "sample": f"first {cb['transforms']} requests of the mix by the FP64 oracle, "
                                            f"one after another, in {cb['seconds']:.1f} s on {cpu_model()}"})(
                oracle_uneven_sample(wl, float(args.cpu_budget if headline else args.cpu_budget_sub),
                                     host_threads())),
        }
    srv.close()
    for p in plans.values():
        p.close()
    return line


def run_workload(args, ctx: Ctx, key: str, headline: bool) -> dict:
    wl = WORKLOADS[key]
    if wl.get("lengths"):
        return gpu_many(args, ctx, wl, headline)
    if wl.get("serving"):
        return gpu_serving(args, ctx, wl, headline)
    return gpu_regular(args, ctx, wl, headline)


# keys a nested workload line repeats from the headline line
_SHARED_KEYS = ("metric", "unit", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "data", "kernel_hash")


_PINNED: dict = {}


def pinned_buffers(nelem: int, count: int) -> list:
    """`count` page-locked host buffers of `nelem` complex64 values for the e2e
    measurements, allocated once per size and reused by later workloads."""
    import torch
    lst = _PINNED.setdefault(nelem, [])
    while len(lst) < count:
        lst.append(torch.empty(nelem, dtype=torch.complex64, pin_memory=True))
    return lst[:count]


def run_gpu(args) -> None:
    ctx = Ctx()
    if not args.quick:
        # the largest e2e buffers (4096 x 16384: 4 x 512 MiB) are pinned first,
        # before the other workloads allocate and free host memory: allocated
        # late in the run they copied at 97-124 GB/s in two of four runs (306
        # GB/s allocated first, and in every run alone)
        wl = WORKLOADS["1d4096L"]
        if args.workload in (None, "1d4096L"):
            pinned_buffers(int(np.prod(wl["dims"])) * wl["batch"], 4)
    if args.workload:
        line = run_workload(args, ctx, args.workload, True)
    else:
        t0 = time.time()
        line = run_workload(args, ctx, HEADLINE, True)
        subs = {}
        for key in SUITE:
            t = time.time()
            sub = run_workload(args, ctx, key, False)
            if ctx.rank == 0:
                sub = {k: v for k, v in sub.items() if k not in _SHARED_KEYS}
                sub["wall_s"] = round(time.time() - t, 1)
                subs[key] = sub
        if ctx.rank == 0:
            line["workloads"] = subs
            line["wall_s_all_workloads"] = round(time.time() - t0, 1)
    if ctx.rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=None, choices=sorted(WORKLOADS),
                    help="one workload alone (default: the headline with every other workload nested)")
    ap.add_argument("--cpu-budget", default=10.0, type=float, help="seconds of oracle time for cpu_baseline")
    ap.add_argument("--cpu-budget-sub", default=3.0, type=float,
                    help="seconds of oracle time for the cpu_baseline of each nested workload")
    ap.add_argument("--quick", action="store_true",
                    help="timed loop only (no pre-roll, e2e, error check or CPU baseline): for profiler runs")
    ap.add_argument("--uneven-engine", type=int, default=None, choices=[0, 1, 2],
                    help="with --quick, the uneven workload's plan takes this engine (0: one launch per exec, "
                         "2: two launches; the default run lets the autotuner choose)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args, WORKLOADS[args.workload or HEADLINE])
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
