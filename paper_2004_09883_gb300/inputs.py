"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no Fourier-transform arithmetic: it only draws random
complex64 data with numpy's PCG64 generator and picks 5-smooth lengths, so both
the CUDA path and the oracle can be fed the same values.

Recipe (per workload): ``numpy.random.default_rng(seed)`` draws ``2*count``
float64 values (uniform in [-1, 1) or standard normal), which are rounded to
float32 and viewed as interleaved (re, im) complex64.  Workload ``i`` uses seed
``BASE_SEED + i`` (``+ 1000*rep`` for repeats).
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 2004_09883

# Workloads, named by what they are (index = seed offset).
WORKLOAD_1D_4096x64 = 0          # 1-D N=4096, batch 64, uniform
WORKLOAD_3D_256x256x128 = 1      # 3-D 256x256x128, standard normal, fwd then inv 1/N
WORKLOAD_UNEVEN_4096 = 2         # 4096 uneven 1-D lengths in [64, 65536], uniform
WORKLOAD_1D_2P20x32 = 3          # 1-D N=2^20, batch 32, standard normal
WORKLOAD_SERVING = 4             # serving mix, uniform
WORKLOAD_GRID_2048x2048 = 5      # 2-D 2048x2048 (the paper's FFT grid), standard normal


def seed_for(workload: int, rep: int = 0) -> int:
    return BASE_SEED + int(workload) + 1000 * int(rep)


def _as_c64(pairs: np.ndarray) -> np.ndarray:
    pairs = np.ascontiguousarray(pairs.astype(np.float32))
    return pairs.view(np.complex64)[..., 0]


def uniform_c64(shape, seed: int) -> np.ndarray:
    """complex64 array, re/im iid uniform[-1, 1)."""
    shape = tuple(int(s) for s in np.atleast_1d(shape))
    rng = np.random.default_rng(seed)
    return _as_c64(rng.uniform(-1.0, 1.0, size=shape + (2,)))


def normal_c64(shape, seed: int) -> np.ndarray:
    """complex64 array, re/im iid standard normal."""
    shape = tuple(int(s) for s in np.atleast_1d(shape))
    rng = np.random.default_rng(seed)
    return _as_c64(rng.standard_normal(size=shape + (2,)))


def smooth_lengths(lo: int, hi: int) -> list[int]:
    """All 2^a * 3^b * 5^c in [lo, hi], ascending."""
    out = []
    p2 = 1
    while p2 <= hi:
        p3 = p2
        while p3 <= hi:
            p5 = p3
            while p5 <= hi:
                if p5 >= lo:
                    out.append(p5)
                p5 *= 5
            p3 *= 3
        p2 *= 2
    return sorted(out)


def uneven_lengths(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """``count`` 5-smooth lengths, log-uniform in [lo, hi]: draw u ~ U[ln lo, ln hi]
    and snap to the 5-smooth length nearest in log (ties go to the smaller)."""
    cands = np.array(smooth_lengths(lo, hi), dtype=np.int64)
    logs = np.log(cands.astype(np.float64))
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(lo), math.log(hi), size=int(count))
    idx = np.searchsorted(logs, u)
    idx = np.clip(idx, 1, len(cands) - 1)
    left, right = logs[idx - 1], logs[idx]
    pick = np.where(u - left <= right - u, idx - 1, idx)
    return cands[pick]


def is_smooth(n: int) -> bool:
    if n < 1:
        return False
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1
