"""Full-size parity: the workloads at the sizes the benchmark times, every
result compared element by element with the FP64 oracle.

* batched uneven lengths: all 4096 transforms (lengths 5-smooth, log-uniform
  in [64, 65536]) through the autotuned batched plan, on the benchmark's own
  packed input buffer;
* 1-D N = 2^20, batch 32: all 32 results, FP32 path and tensor-core path;
* 1-D N = 4096, batch 64: all 64 results;
* the paper's FFT grid, 2-D 2048 x 2048 (Sec. 5.1(b)), forward and inverse.

Bars: relative L2 error per transform <= 2e-6 log2 N for the FP32 path and
<= 5e-5 for the tensor-core path."""
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2004_09883_gb300 import inputs

pytestmark = pytest.mark.gpu
THREADS = max(1, min(16, len(os.sched_getaffinity(0))))
TOL_TC = 5e-5


def tol(n: int) -> float:
    return 2e-6 * math.log2(n) if n > 1 else 1e-7


def oracle_each(items, sign=-1):
    """The oracle on a list of 1-D arrays, one transform per worker thread
    (the oracle's C routine runs without the interpreter lock)."""
    def one(x):
        return oracle.fft(np.asarray(x).astype(np.complex128), [len(x)], sign)
    with ThreadPoolExecutor(THREADS) as ex:
        return list(ex.map(one, items))


def test_uneven_4096_transforms_autotuned_all_results(fb):
    import torch
    seed = inputs.seed_for(inputs.WORKLOAD_UNEVEN_4096)
    lens = inputs.uneven_lengths(4096, 64, 65536, seed)
    offs, total = fb.many_layout(lens)
    packed = inputs.uniform_c64((total,), seed)  # the benchmark's input buffer 0
    x = torch.from_numpy(packed).cuda()
    out = torch.empty_like(x)
    tuned, ms = fb.autotune_many(lens, x, out, fb.FORWARD, reps=3)
    assert ms > 0
    with fb.PlanMany(lens, opts=tuned) as p:
        y = p.exec(x, None, fb.FORWARD)
        y2 = p.exec(x, None, fb.FORWARD)  # the replayed graph gives the same bits
        p.check()
        yh, y2h = y.cpu().numpy(), y2.cpu().numpy()
    items = [packed[o:o + n] for o, n in zip(offs, lens)]
    refs = oracle_each(items)
    worst = 0.0
    for i, (o, n, ref) in enumerate(zip(offs, lens, refs)):
        got = yh[o:o + n]
        assert np.array_equal(got, y2h[o:o + n]), f"transform {i}: replay differs"
        err = oracle.rel_l2(got, ref)[0]
        assert err <= tol(int(n)), f"transform {i} (n={n}): rel L2 {err:.3e} > {tol(int(n)):.3e}"
        worst = max(worst, err / tol(int(n)))
    assert len(refs) == 4096 and worst <= 1.0


@pytest.mark.parametrize("tensor_cores", [False, True])
def test_precision_2p20_batch32_all_results(fb, tensor_cores):
    import torch
    n, batch = 1 << 20, 32
    x = inputs.normal_c64((batch, n), inputs.seed_for(inputs.WORKLOAD_1D_2P20x32))
    with fb.Plan([n], batch, tensor_cores=tensor_cores) as p:
        info = p.info()
        y = p.exec(torch.from_numpy(x.reshape(-1)).cuda(), None, fb.FORWARD)
        p.check()
        yh = y.cpu().numpy().reshape(batch, n)
    assert (info["tc_passes"] > 0) == tensor_cores
    ref = oracle.fft(x.astype(np.complex128), [n], -1, False, THREADS).reshape(batch, n)
    err = oracle.rel_l2(yh, ref)
    bar = TOL_TC if tensor_cores else tol(n)
    assert err.shape == (batch,)
    assert err.max() <= bar, f"max rel L2 {err.max():.3e} (item {int(err.argmax())}) > {bar:.1e}"


def test_plain_4096_batch64_all_results(fb):
    import torch
    n, batch = 4096, 64
    x = inputs.uniform_c64((batch, n), inputs.seed_for(inputs.WORKLOAD_1D_4096x64))
    with fb.Plan([n], batch) as p:
        y = p.exec(torch.from_numpy(x.reshape(-1)).cuda(), None, fb.FORWARD)
        p.check()
        yh = y.cpu().numpy().reshape(batch, n)
    ref = oracle.fft(x.astype(np.complex128), [n], -1, False, THREADS).reshape(batch, n)
    assert oracle.rel_l2(yh, ref).max() <= tol(n)


def test_paper_grid_2048x2048_forward_and_inverse(fb):
    """The 2048 x 2048 grid of the paper's FFT application (Sec. 5.1(b))."""
    import torch
    dims = [2048, 2048]
    n = 2048 * 2048
    x = inputs.normal_c64((n,), inputs.seed_for(inputs.WORKLOAD_GRID_2048x2048))
    with fb.Plan(dims, 1, scale_inv_n=True) as p:
        d = torch.from_numpy(x).cuda()
        y = p.exec(d, None, fb.FORWARD)
        z = p.exec(y, None, fb.INVERSE)
        p.check()
        yh, zh = y.cpu().numpy(), z.cpu().numpy()
    ref = oracle.fft(x.astype(np.complex128), dims, -1, False, THREADS)
    assert oracle.rel_l2(yh, ref)[0] <= tol(n)
    refi = oracle.fft(yh.astype(np.complex128), dims, 1, True, THREADS)
    assert oracle.rel_l2(zh, refi)[0] <= tol(n)
    assert oracle.rel_l2(zh, x.astype(np.complex128))[0] <= tol(n)
