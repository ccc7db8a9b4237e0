"""The seeded input recipe (no GPU): the generators the tests, the benchmark
and the oracle share draw what the workload definitions say -- value
distributions, 5-smooth log-uniform lengths, the serving request mix and
Poisson arrivals -- and draw it again bit for bit from the same seed."""
import math

import numpy as np
import pytest

from paper_2004_09883_gb300 import inputs


def test_values_are_seeded_complex64_with_the_stated_distributions():
    u = inputs.uniform_c64((64, 4096), inputs.seed_for(inputs.WORKLOAD_1D_4096x64))
    assert u.dtype == np.complex64 and u.shape == (64, 4096)
    assert np.array_equal(u, inputs.uniform_c64((64, 4096), inputs.seed_for(inputs.WORKLOAD_1D_4096x64)))
    assert not np.array_equal(u, inputs.uniform_c64((64, 4096), inputs.seed_for(inputs.WORKLOAD_1D_4096x64, 1)))
    for part in (u.real, u.imag):
        assert part.min() >= -1.0 and part.max() < 1.0
        assert abs(part.mean()) < 0.01 and abs(part.var() - 1 / 3) < 0.01
    assert abs(np.corrcoef(u.real.ravel(), u.imag.ravel())[0, 1]) < 0.01  # re and im independent
    g = inputs.normal_c64((256, 1024), inputs.seed_for(inputs.WORKLOAD_3D_256x256x128))
    for part in (g.real, g.imag):
        assert abs(part.mean()) < 0.01 and abs(part.var() - 1.0) < 0.01
    # float32 rounding of the float64 draws, interleaved (re, im)
    rng = np.random.default_rng(7)
    raw = rng.uniform(-1.0, 1.0, size=(5, 2)).astype(np.float32)
    x = inputs.uniform_c64(5, 7)
    assert np.array_equal(x.real, raw[:, 0]) and np.array_equal(x.imag, raw[:, 1])


@pytest.mark.parametrize("lo,hi", [(1, 1), (1, 100), (64, 65536), (4097, 1 << 24)])
def test_smooth_lengths_are_exactly_the_5_smooth_numbers(lo, hi):
    got = inputs.smooth_lengths(lo, hi)
    assert got == sorted(set(got))
    if hi <= 70000:
        assert got == [n for n in range(lo, hi + 1) if inputs.is_smooth(n)]
    else:
        assert all(inputs.is_smooth(n) and lo <= n <= hi for n in got)
        assert len(got) == sum(1 for a in range(25) for b in range(16) for c in range(11)
                               if lo <= 2 ** a * 3 ** b * 5 ** c <= hi)


def test_uneven_lengths_are_log_uniform_and_snap_to_the_nearest_in_log():
    lens = inputs.uneven_lengths(4096, 64, 65536, inputs.seed_for(inputs.WORKLOAD_UNEVEN_4096))
    assert np.array_equal(lens, inputs.uneven_lengths(4096, 64, 65536, inputs.seed_for(inputs.WORKLOAD_UNEVEN_4096)))
    assert all(inputs.is_smooth(int(n)) for n in lens) and lens.min() >= 64 and lens.max() <= 65536
    logs = np.log(lens.astype(np.float64))
    # log-uniform on [ln 64, ln 65536]: quartiles of ln n at a quarter, half and
    # three quarters of that range (the median at the geometric mean, 2048)
    a, b = math.log(64), math.log(65536)
    q1, med, q3 = np.percentile(logs, [25, 50, 75])
    assert abs(med - math.log(2048)) < 0.15
    assert abs(q1 - (a + (b - a) / 4)) < 0.15 and abs(q3 - (a + 3 * (b - a) / 4)) < 0.15
    # each drawn length is the candidate nearest in log to the uniform draw (ties to the smaller)
    cands = np.array(inputs.smooth_lengths(64, 65536), dtype=np.float64)
    rng = np.random.default_rng(99)
    u = rng.uniform(math.log(64), math.log(65536), size=500)
    got = inputs.uneven_lengths(500, 64, 65536, 99)
    for ui, n in zip(u, got):
        d = np.abs(np.log(cands) - ui)
        best = cands[d <= d.min() + 1e-12]
        assert n == best.min()


def test_serving_mix_and_arrivals():
    serving = pytest.importorskip("paper_2004_09883_gb300.serving")  # needs the library for its planner query
    shapes = serving.request_mix(2000, inputs.seed_for(inputs.WORKLOAD_SERVING))
    assert shapes == serving.request_mix(2000, inputs.seed_for(inputs.WORKLOAD_SERVING))
    ranks = np.array([len(s) for s in shapes])
    frac = [np.mean(ranks == r) for r in (1, 2, 3)]
    assert abs(frac[0] - 0.60) < 0.03 and abs(frac[1] - 0.25) < 0.03 and abs(frac[2] - 0.15) < 0.03
    for s in shapes:
        assert all(inputs.is_smooth(d) for d in s)
        lo, hi = {1: (256, 1 << 22), 2: (16, 512), 3: (8, 128)}[len(s)]
        assert all(lo <= d <= hi for d in s), s
    t = serving.poisson_arrivals(20000, 5000.0, 3)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() * 5000.0 - 1.0) < 0.03  # rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.03  # exponential gaps: coefficient of variation 1
    assert np.array_equal(serving.poisson_arrivals(5, math.inf, 0), np.zeros(5))
