"""fb_fft_exec_host on pinned host arrays: a batch of at least two 32 MiB
chunks moves chunk by chunk, its copy in, transform and copy out overlapping
on three streams.  Each chunk runs a plan of its own batch size with the same
kernels, so the result must equal, bit for bit, the device exec of the whole
batch; pageable arrays and FB_FFT_HOST_PIPELINE=0 take the whole-array path
and must agree too."""
import numpy as np
import pytest

from paper_2004_09883_gb300 import inputs
from test_gpu_parity import assert_close, ref_fft, to_dev, to_host

pytestmark = pytest.mark.gpu


def pinned_like(x):
    import torch
    t = torch.empty(x.size, dtype=torch.complex64, pin_memory=True)
    a = t.numpy()
    a[:] = x.reshape(-1)
    return t, a


@pytest.mark.parametrize("dims,batch,direction,scale", [
    ([4096], 4096, -1, False),       # 128 MiB: four chunks
    ([1 << 20], 12, -1, False),      # four-step plans per chunk: three chunks of 4
    ([9375], 1000, 1, True),         # odd N: even chunks of 446, a tail of 108
    ([64, 48], 3000, 1, True),       # multi-D: chunks of 1365, a tail of 270
])
@pytest.mark.parametrize("inplace", [False, True])
def test_pipelined_host_exec_equals_device_exec(fb, dims, batch, direction, scale, inplace):
    x = inputs.uniform_c64([batch] + dims, 61)
    with fb.Plan(dims, batch, scale_inv_n=scale) as p:
        want = to_host(p.exec(to_dev(x), None, direction))
        tin, a = pinned_like(x)
        if inplace:
            got = p.exec_host(a, a, direction)
        else:
            tout, b = pinned_like(np.zeros_like(x))
            got = p.exec_host(a, b, direction)
        assert np.array_equal(got.reshape(-1), want)
    n = int(np.prod(dims))
    for i in (0, batch // 2, batch - 1):  # and against the oracle on samples
        assert_close(got.reshape(batch, n)[i], ref_fft(x.reshape(batch, n)[i], dims, direction, scale), dims)


def test_pageable_and_switched_off_paths_agree(fb, monkeypatch):
    dims, batch = [4096], 4096
    x = inputs.uniform_c64([batch] + dims, 62)
    with fb.Plan(dims, batch) as p:
        want = to_host(p.exec(to_dev(x), None, -1))
        assert np.array_equal(p.exec_host(x.reshape(-1)).reshape(-1), want)  # pageable numpy array
        monkeypatch.setenv("FB_FFT_HOST_PIPELINE", "0")
        _, a = pinned_like(x)
        assert np.array_equal(p.exec_host(a).reshape(-1), want)
        monkeypatch.delenv("FB_FFT_HOST_PIPELINE")
        assert np.array_equal(p.exec_host(a).reshape(-1), want)  # pipelined again, same plan
