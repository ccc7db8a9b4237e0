"""Out-of-bounds writes, caught without a sanitizer: every output sits between
two guard bands of a sentinel pattern in one device allocation, and after the
exec the bands must hold the pattern bit for bit (and an out-of-place input
must be untouched).  Covers single-pass, four-step, multi-D, plane-pass and
batched-uneven plans, aligned and 8-byte-aligned (plain-copy) buffers, and the
pipelined host-array path with bands around pinned host arrays."""
import numpy as np
import pytest

from paper_2004_09883_gb300 import inputs
from test_gpu_parity import assert_close, ref_fft, to_dev

pytestmark = pytest.mark.gpu

GUARD = 4096  # values per band: wider than any tile row a pass writes
SENTINEL = np.complex64(12345.678 - 9876.5j)


def banded(n, shift):
    """Device buffer with bands; returns (whole buffer, view of n values)."""
    import torch
    buf = torch.full((n + 2 * GUARD + 1,), complex(SENTINEL), dtype=torch.complex64, device="cuda")
    return buf, buf[GUARD + shift:GUARD + shift + n]


def check_bands(buf, n, shift):
    h = buf.cpu().numpy()
    lo, hi = h[:GUARD + shift], h[GUARD + shift + n:]
    assert np.array_equal(lo, np.full_like(lo, SENTINEL)), "write below the output"
    assert np.array_equal(hi, np.full_like(hi, SENTINEL)), "write above the output"


@pytest.mark.parametrize("dims,batch", [([4096], 7), ([1000], 5), ([1 << 20], 3), ([3 * 5 ** 6], 2),
                                        ([256, 256, 128], 1), ([30, 20, 12], 2), ([64, 1], 3), ([2048, 3, 5], 1)])
@pytest.mark.parametrize("shift", [0, 1])  # 1: 8-byte aligned only, the plain-copy paths
@pytest.mark.parametrize("direction", [-1, 1])
def test_no_write_outside_the_output(fb, dims, batch, shift, direction):
    import torch
    n = int(np.prod(dims)) * batch
    x = inputs.uniform_c64([batch] + dims, 71)
    xin = to_dev(x)
    ibuf, src = banded(n, shift)
    src.copy_(xin)
    obuf, dst = banded(n, shift)
    with fb.Plan(dims, batch, scale_inv_n=True) as p:
        p.exec_ptr(src.data_ptr(), dst.data_ptr(), direction)
        p.check()
    torch.cuda.synchronize()
    check_bands(obuf, n, shift)
    check_bands(ibuf, n, shift)
    assert torch.equal(src, xin), "out-of-place exec changed its input"
    m = int(np.prod(dims))
    y = dst.cpu().numpy().reshape(batch, m)
    # the plan scales inverse execs only (FB_FFT_SCALE_INV_N)
    assert_close(y[-1], ref_fft(x.reshape(batch, m)[-1], dims, direction, scale=direction == 1), dims)


def test_plane_pass_and_in_place_stay_inside(fb, monkeypatch):
    monkeypatch.setenv("FB_FFT_PLANE", "1")
    dims, batch = [3, 256, 128], 2
    n = int(np.prod(dims)) * batch
    x = inputs.uniform_c64([batch] + dims, 72)
    buf, v = banded(n, 0)
    v.copy_(to_dev(x))
    with fb.Plan(dims, batch) as p:
        assert p.pass_names()[0] == "plane"
        p.exec_ptr(v.data_ptr(), v.data_ptr(), -1)  # in place
        p.check()
    check_bands(buf, n, 0)
    m = int(np.prod(dims))
    assert_close(v.cpu().numpy().reshape(batch, m)[1], ref_fft(x.reshape(batch, m)[1], dims, -1), dims)


def test_batched_uneven_stays_inside(fb):
    lens = [64, 75, 4096, 3 * 5 ** 5, 1 << 16, 6000, 128, 2048]
    offs, total = fb.many_layout(lens)
    x = inputs.uniform_c64((total,), 73)
    with fb.PlanMany(lens) as p:
        ibuf, src = banded(total, 0)
        src.copy_(to_dev(x))
        obuf, dst = banded(total, 0)
        p.exec_ptr(src.data_ptr(), dst.data_ptr(), -1)
        p.check()
    check_bands(obuf, total, 0)
    check_bands(ibuf, total, 0)
    y = dst.cpu().numpy()
    for o, n in zip(offs, lens):
        assert_close(y[o:o + n], ref_fft(x[o:o + n], [n], -1), [n], f"n={n}")


def test_pipelined_host_exec_stays_inside(fb):
    import torch
    dims, batch = [4096], 4096  # four 32 MiB chunks
    n = int(np.prod(dims)) * batch
    x = inputs.uniform_c64([batch] + dims, 74)
    t = torch.full((n + 2 * GUARD,), complex(SENTINEL), dtype=torch.complex64, pin_memory=True)
    h = t.numpy()
    h[GUARD:GUARD + n] = x.reshape(-1)
    with fb.Plan(dims, batch) as p:
        p.exec_host(h[GUARD:GUARD + n], h[GUARD:GUARD + n], -1)  # in place on a pinned slice
    assert np.array_equal(h[:GUARD], np.full(GUARD, SENTINEL)) and np.array_equal(h[GUARD + n:], np.full(GUARD, SENTINEL))
    y = h[GUARD:GUARD + n].reshape(batch, -1)
    assert_close(y[-1], ref_fft(x.reshape(batch, -1)[-1], dims, -1), dims)
