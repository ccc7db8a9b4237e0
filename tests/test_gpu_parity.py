"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Bar: per-transform relative L2 error <= 2e-6 * log2(N)
(N = elements of one transform), the FP32 tolerance the workload definition
states; exact for N = 1."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2004_09883_gb300 import inputs

pytestmark = pytest.mark.gpu
THREADS = max(1, min(16, len(os.sched_getaffinity(0))))


def tol(n: int) -> float:
    return 2e-6 * math.log2(n) if n > 1 else 1e-7


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex64).reshape(-1)).cuda()


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def gpu_fft(fb, x, dims, direction=-1, scale=False, inplace=False, batch=None):
    n = int(np.prod(dims))
    b = x.size // n if batch is None else batch
    with fb.Plan(dims, b, scale_inv_n=scale) as p:
        d = to_dev(x)
        out = p.exec(d, d if inplace else None, direction)
        p.check()
        return to_host(out)


def ref_fft(x, dims, direction=-1, scale=False):
    return oracle.fft(np.asarray(x, np.complex64).astype(np.complex128), dims, direction, scale, THREADS)


def assert_close(y, ref, dims, what=""):
    n = int(np.prod(dims))
    err = oracle.rel_l2(np.asarray(y).reshape(-1, n), np.asarray(ref).reshape(-1, n))
    assert err.max() <= tol(n), f"{what} dims={dims}: max rel L2 {err.max():.3e} > {tol(n):.3e}"
    return err


# --------------------------------------------------------------------------
# Twiddle tables (FP64 on the GPU, rounded to FP32)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("d", [16, 1000, 4096, 1 << 20, 3 * 5 ** 7])
def test_twiddles_round_to_nearest(fb, d):
    count = min(d, 4096)
    got = fb.twiddles(d, count)
    want = np.array([oracle.twiddle(m, d) for m in range(count)]).astype(np.complex64)
    assert np.all(np.abs(got - want) <= 2 * np.finfo(np.float32).eps)
    for g, w in ((got.real, want.real), (got.imag, want.imag)):
        # Where the exact value is 0 (e.g. sin(pi)) the GPU's sincospi returns
        # 0 while the oracle's long-double sinl(pi_L) is ~1e-19: compare those
        # by value; elsewhere the float32 results must be within 1 ulp and
        # nearly always identical (round to nearest of an FP64 evaluation).
        big = np.abs(w) > 1e-12
        assert np.all(np.abs(g[~big]) <= 1e-12)
        gi = g[big].view(np.int32).astype(np.int64)
        wi = w[big].view(np.int32).astype(np.int64)
        assert np.all(np.sign(g[big]) == np.sign(w[big]))
        assert np.all(np.abs(gi - wi) <= 1)
        assert np.mean(gi == wi) > 0.99


# --------------------------------------------------------------------------
# 1-D, one pass in shared memory
# --------------------------------------------------------------------------
POW2 = [2 ** k for k in range(1, 13)]
MIXED = [3, 5, 6, 9, 10, 12, 15, 25, 27, 30, 45, 60, 81, 96, 100, 125, 243, 360, 375, 625, 729,
         1000, 1536, 2187, 2400, 3125, 3645, 4000]


@pytest.mark.parametrize("n", POW2 + MIXED)
@pytest.mark.parametrize("direction", [-1, 1])
def test_1d_single_pass(fb, n, direction):
    batch = 37  # not a multiple of any tile width: ragged last tile
    x = inputs.uniform_c64((batch, n), inputs.seed_for(0, n))
    y = gpu_fft(fb, x, [n], direction)
    assert_close(y, ref_fft(x, [n], direction), [n])


@pytest.mark.parametrize("n", [16, 128, 1000, 4096])
def test_1d_in_place_and_scaled_inverse(fb, n):
    x = inputs.normal_c64((5, n), 11)
    y = gpu_fft(fb, x, [n], 1, scale=True, inplace=True)
    assert_close(y, ref_fft(x, [n], 1, scale=True), [n])
    y = gpu_fft(fb, x, [n], -1, scale=True)  # the flag only scales inverse execs
    assert_close(y, ref_fft(x, [n], -1), [n])


# --------------------------------------------------------------------------
# 1-D four-step (two passes through the plan's scratch)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,batch", [(8192, 3), (65536, 2), (3 * 5 ** 7, 1), (1 << 20, 2),
                                     (6000, 5), (2 * 3 ** 9, 1), (1 << 22, 1), (1 << 23, 1)])
@pytest.mark.parametrize("direction", [-1, 1])
def test_1d_fourstep(fb, n, batch, direction):
    x = inputs.normal_c64((batch, n), 3 + n)
    y = gpu_fft(fb, x, [n], direction)
    assert_close(y, ref_fft(x, [n], direction), [n])


def test_fourstep_largest_length(fb):
    """FB_FFT_MAX_1D_LEN = 4096 x 4096: both passes take 4096-point lines
    (columns strided with the post-twiddle fused, rows transposed out)."""
    n = 1 << 24
    x = inputs.normal_c64((1, n), 24)
    y = gpu_fft(fb, x, [n], -1)
    assert_close(y, ref_fft(x, [n], -1), [n])


def test_fourstep_in_place_one_chunk(fb):
    n, batch = 1 << 16, 70
    x = inputs.uniform_c64((batch, n), 5)
    y = gpu_fft(fb, x, [n], -1, inplace=True)
    assert_close(y, ref_fft(x, [n], -1), [n])


def test_fourstep_batch_in_several_chunks(fb):
    """1100 x 2^16 values = 550 MiB of intermediate: a 512 MiB chunk of 1024
    transforms, then a ragged chunk of 76; items at both chunk edges are checked."""
    import torch
    n, batch = 1 << 16, 1100
    x = torch.from_numpy(inputs.uniform_c64((batch, n), 6)).cuda()
    with fb.Plan([n], batch) as p:
        assert p.info()["scratch_bytes"] == 1024 * n * 8
        y = p.exec(x, x, -1)  # in place
        torch.cuda.synchronize()
        p.check()
    x0 = inputs.uniform_c64((batch, n), 6)
    for i in (0, 1023, 1024, 1099):
        assert_close(y[i].cpu().numpy(), ref_fft(x0[i], [n], -1), [n], f"item {i}")


# --------------------------------------------------------------------------
# Multi-dimensional
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dims,batch", [([16, 12], 3), ([256, 256], 2), ([512, 512], 1), ([100, 30], 4),
                                        ([8, 8, 8], 5), ([30, 20, 12], 2), ([128, 128, 128], 1),
                                        ([6, 250, 18], 1), ([3, 5, 4096], 1), ([4096, 2, 3], 1),
                                        ([2048, 3, 5], 1), ([5, 2048], 2)])
@pytest.mark.parametrize("direction", [-1, 1])
def test_multi_d(fb, dims, batch, direction):
    x = inputs.uniform_c64([batch] + dims, 21)
    y = gpu_fft(fb, x, dims, direction)
    assert_close(y, ref_fft(x, dims, direction), dims)


# --------------------------------------------------------------------------
# The workloads at full size, in the configuration the benchmark times
# --------------------------------------------------------------------------
def test_workload_1d_4096x64(fb):
    x = inputs.uniform_c64((64, 4096), inputs.seed_for(inputs.WORKLOAD_1D_4096x64))
    y = gpu_fft(fb, x, [4096], -1)
    err = assert_close(y, ref_fft(x, [4096], -1), [4096])
    assert err.max() < 1e-6  # far inside the bound: accurate twiddles


def test_workload_3d_256x256x128_fwd_inv(fb):
    import torch
    dims = [256, 256, 128]
    x = inputs.normal_c64(dims, inputs.seed_for(inputs.WORKLOAD_3D_256x256x128))
    with fb.Plan(dims, 1, scale_inv_n=True) as p:
        d = to_dev(x)
        y = p.exec(d, None, -1)
        z = p.exec(y, torch.empty_like(y), 1)
        p.check()
        yh, zh = to_host(y), to_host(z)
    assert_close(yh, ref_fft(x, dims, -1), dims, "forward")
    assert_close(zh, ref_fft(yh, dims, 1, scale=True), dims, "inverse")
    rt = np.linalg.norm(zh - x.reshape(-1)) / np.linalg.norm(x)
    assert rt <= tol(int(np.prod(dims))), f"round trip {rt:.3e}"


def test_workload_1d_2p20x32_sampled(fb):
    n, batch = 1 << 20, 32
    x = inputs.normal_c64((batch, n), inputs.seed_for(inputs.WORKLOAD_1D_2P20x32))
    y = gpu_fft(fb, x, [n], -1).reshape(batch, n)
    for b in (0, 13, 31):
        assert_close(y[b], ref_fft(x[b], [n], -1), [n], f"item {b}")
    # every item: Parseval against its own input (any size)
    e_in = np.sum(np.abs(x.astype(np.complex128)) ** 2, axis=1) * n
    e_out = np.sum(np.abs(y.astype(np.complex128)) ** 2, axis=1)
    assert np.max(np.abs(e_out - e_in) / e_in) < 4 * tol(n)


def test_workload_uneven_lengths_sample(fb):
    lens = inputs.uneven_lengths(24, 64, 65536, inputs.seed_for(inputs.WORKLOAD_UNEVEN_4096))
    for i, n in enumerate(lens):
        x = inputs.uniform_c64((1, int(n)), 100 + i)
        assert_close(gpu_fft(fb, x, [int(n)], -1), ref_fft(x, [int(n)], -1), [int(n)], f"n={n}")


# --------------------------------------------------------------------------
# Edge cases
# --------------------------------------------------------------------------
def test_batch_zero_and_length_one(fb):
    import torch
    with fb.Plan([64], 0) as p:
        p.exec_ptr(0, 0, -1)
        assert p.info()["passes"] == 1
    x = inputs.uniform_c64((7,), 1)
    for dims in ([1], [1, 1], [1, 1, 1]):
        assert np.array_equal(gpu_fft(fb, x, dims, -1), x)
    x = inputs.uniform_c64((2, 1, 64), 2)
    assert_close(gpu_fft(fb, x, [1, 64], 1), ref_fft(x, [1, 64], 1), [1, 64])
    x = inputs.uniform_c64((2, 64, 1), 3)
    assert_close(gpu_fft(fb, x, [64, 1], 1), ref_fft(x, [64, 1], 1), [64, 1])
    del torch


@pytest.mark.parametrize("dims", [[4096], [1 << 16], [64, 256]])
def test_misaligned_buffers_take_the_plain_path(fb, dims):
    import torch
    n = int(np.prod(dims))
    x = inputs.uniform_c64((3, n), 9)
    buf = torch.zeros(3 * n + 2, dtype=torch.complex64, device="cuda")
    src = buf[1:1 + 3 * n]  # 8-byte but not 16-byte aligned
    src.copy_(to_dev(x))
    out = torch.zeros(3 * n + 2, dtype=torch.complex64, device="cuda")[1:1 + 3 * n]
    with fb.Plan(dims, 3) as p:
        p.exec(src, out, -1)
        p.check()
    assert_close(to_host(out), ref_fft(x, dims, -1), dims)


def test_exec_argument_errors(fb):
    import torch
    with fb.Plan([256], 4) as p:
        x = torch.zeros(1024 + 8, dtype=torch.complex64, device="cuda")
        with pytest.raises(fb.FFTError) as e:
            p.exec_ptr(x.data_ptr(), x.data_ptr(), 0)
        assert e.value.status == -1
        with pytest.raises(fb.FFTError) as e:  # partial overlap
            p.exec_ptr(x.data_ptr(), x.data_ptr() + 8 * 8, -1)
        assert e.value.status == -1
        with pytest.raises(fb.FFTError) as e:  # not 8-byte aligned
            p.exec_ptr(x.data_ptr() + 4, x.data_ptr() + 4, -1)
        assert e.value.status == -1


def test_exec_host_matches_device(fb):
    dims = [64, 48]
    x = inputs.uniform_c64((3, 64, 48), 4)
    with fb.Plan(dims, 3, scale_inv_n=True) as p:
        y = p.exec_host(x.reshape(-1), direction=1)
        y2 = x.reshape(-1).copy()
        p.exec_host(y2, y2, 1)  # in place on the host array
    assert_close(y, ref_fft(x, dims, 1, scale=True), dims)
    assert np.array_equal(y, y2)


def test_timeout_hook_reports_and_recovers(fb):
    dims = [256, 256]
    x = inputs.uniform_c64(dims, 6)
    with fb.Plan(dims, 1) as p:
        d = to_dev(x)
        p.debug_inject_timeout(True)
        p.exec(d, None, -1)
        with pytest.raises(fb.FFTError) as e:
            p.check()
        assert e.value.status == -5
        p.debug_inject_timeout(False)
        y = p.exec(d, None, -1)
        p.check()
        assert_close(to_host(y), ref_fft(x, dims, -1), dims)


def test_profile_and_launch_count(fb):
    dims = [64, 64, 32]
    with fb.Plan(dims, 2) as p:
        d = to_dev(inputs.uniform_c64((2, 64, 64, 32), 1))
        n0 = fb.launch_count()
        p.profile(True)
        for _ in range(3):
            p.exec(d, None, -1)
        rows = p.profile_read()
        assert fb.launch_count() - n0 == 3 * p.info()["passes"]
        assert [r[0] for r in rows] == ["axis2", "axis1", "axis0"]
        assert all(r[2] == 3 and r[1] > 0 for r in rows)


def test_gpu_linearity_and_parseval_large(fb):
    import torch
    n = 1 << 22
    x = inputs.normal_c64((1, n), 31)
    y = inputs.normal_c64((1, n), 32)
    a, b = 0.75 - 0.5j, -1.25 + 2.0j
    with fb.Plan([n], 1) as p:
        fx = p.exec(to_dev(x), None, -1)
        fy = p.exec(to_dev(y), None, -1)
        fz = p.exec(to_dev((a * x + b * y).astype(np.complex64)), None, -1)
        lhs = fz
        rhs = torch.tensor(a, dtype=torch.complex64) * fx + torch.tensor(b, dtype=torch.complex64) * fy
        rel = (torch.linalg.vector_norm(lhs - rhs) / torch.linalg.vector_norm(rhs)).item()
        e_in = float(np.sum(np.abs(x.astype(np.complex128)) ** 2)) * n
        e_out = float(np.sum(np.abs(to_host(fx).astype(np.complex128)) ** 2))
    assert rel < 4 * tol(n)
    assert abs(e_out - e_in) / e_in < 4 * tol(n)


@pytest.mark.parametrize("dims,batch,tc", [([256, 256, 128], 1, False), ([1 << 20], 8, False), ([1 << 20], 8, True),
                                           ([4096], 8192, False), ([128], 32768, False), ([1024], 8192, True)])
def test_launch_configuration_fits_the_gpu(fb, dims, batch, tc):
    """Every pass's grid is a whole number of CTAs per SM (persistent CTAs),
    its CTA a whole number of warps, its shared memory within the opt-in limit;
    tensor-core passes run two CTAs per SM once there are enough tiles."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    with fb.Plan(dims, batch, tensor_cores=tc) as p:
        cfg = p.launch_config()
        info = p.info()
    assert len(cfg) == info["passes"]
    for grid, block, smem in cfg:
        assert grid >= 1 and block % 32 == 0 and 0 < smem <= 227 * 1024
        assert grid % sms == 0 or grid < sms, (grid, sms)
    if tc and batch * int(np.prod(dims)) >= 1 << 23:
        assert all(g == 2 * sms for g, _, _ in cfg), cfg
