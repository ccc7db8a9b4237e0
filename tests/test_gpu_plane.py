"""GPU parity of the plane pass: the two trailing axes of a multi-D transform
in one pass, one thread-block cluster per plane exchanging the plane through
distributed shared memory.  Every compiled plane shape, both directions, the
1/N scale, in place, misaligned buffers (plain copies instead of TMA), fewer
planes than clusters and a ragged last round of planes, each against the FP64
oracle with the FP32 bound 2e-6 log2(N), and against the per-axis passes."""
import numpy as np
import pytest

from paper_2004_09883_gb300 import inputs
from test_gpu_parity import assert_close, ref_fft, to_dev, to_host, tol

pytestmark = pytest.mark.gpu


def run(fb, x, dims, batch, direction, scale=False, inplace=False, misalign=False):
    import torch
    n = int(np.prod(dims)) * batch
    with fb.Plan(dims, batch, scale_inv_n=scale) as p:
        names = p.pass_names()
        if misalign:  # 8-byte but not 16-byte aligned: the kernel's plain copies
            src = torch.zeros(n + 2, dtype=torch.complex64, device="cuda")[1:1 + n]
            src.copy_(to_dev(x))
            out = src if inplace else torch.zeros(n + 2, dtype=torch.complex64, device="cuda")[1:1 + n]
        else:
            src = to_dev(x)
            out = src if inplace else torch.empty_like(src)
        p.exec(src, out, direction)
        p.check()
        return to_host(out), names


@pytest.mark.parametrize("dims,batch", [([256, 128], 3), ([128, 128], 2), ([256, 256], 1), ([128, 256], 2),
                                        ([5, 256, 128], 1), ([3, 128, 128], 3), ([2, 256, 256], 2),
                                        ([6, 128, 256], 1)])
@pytest.mark.parametrize("direction", [-1, 1])
@pytest.mark.parametrize("threads", ["512", "256"])
def test_plane_pass_matches_oracle(fb, monkeypatch, dims, batch, direction, threads):
    monkeypatch.setenv("FB_FFT_PLANE", "1")
    monkeypatch.setenv("FB_FFT_PLANE_THREADS", threads)  # 256 x 256 planes: 512 only
    x = inputs.uniform_c64([batch] + dims, 51)
    y, names = run(fb, x, dims, batch, direction)
    assert names[0] == "plane" and len(names) == len([d for d in dims if d > 1]) - 1
    assert_close(y, ref_fft(x, dims, direction), dims)


@pytest.mark.parametrize("inplace,misalign", [(True, False), (False, True), (True, True)])
@pytest.mark.parametrize("threads", ["512", "256"])
def test_plane_pass_in_place_and_misaligned(fb, monkeypatch, inplace, misalign, threads):
    monkeypatch.setenv("FB_FFT_PLANE", "1")
    monkeypatch.setenv("FB_FFT_PLANE_THREADS", threads)
    dims, batch = [3, 256, 128], 2
    x = inputs.normal_c64([batch] + dims, 52)
    y, names = run(fb, x, dims, batch, 1, scale=True, inplace=inplace, misalign=misalign)
    assert names == ["plane", "axis0"]
    assert_close(y, ref_fft(x, dims, 1, scale=True), dims)


@pytest.mark.parametrize("threads", ["512", "256"])
def test_plane_pass_many_rounds_of_planes(fb, monkeypatch, threads):
    """More planes than clusters that fit (several rounds through the three
    buffers per CTA) with a ragged last round: the bench's 256 x 256 x 128
    volume plus 3 planes, every plane against the oracle at sampled planes
    and by Parseval overall."""
    monkeypatch.setenv("FB_FFT_PLANE", "1")
    monkeypatch.setenv("FB_FFT_PLANE_THREADS", threads)
    dims = [259, 256, 128]
    x = inputs.normal_c64([1] + dims, 53)
    with fb.Plan(dims[1:], dims[0]) as p:
        assert p.pass_names() == ["plane"]
        d = to_dev(x)
        y = p.exec(d, None, -1)
        p.check()
        yh = to_host(y).reshape(dims[0], -1)
    plane = dims[1] * dims[2]
    xs = x.reshape(dims[0], plane)
    for i in (0, 1, 75, 151, 152, 257, 258):
        assert_close(yh[i], ref_fft(xs[i], dims[1:], -1), dims[1:], f"plane {i}")
    e_in = np.sum(np.abs(xs.astype(np.complex128)) ** 2, axis=1) * plane
    e_out = np.sum(np.abs(yh.astype(np.complex128)) ** 2, axis=1)
    assert np.max(np.abs(e_out - e_in) / e_in) < 4 * tol(plane)


def test_plane_pass_agrees_with_axis_passes(fb, monkeypatch):
    """The bench's 3-D volume both ways: the fused plan and one pass per
    axis (the default) give the same transform within twice the bound of
    each other."""
    dims = [256, 256, 128]
    x = inputs.normal_c64(dims, 54)
    monkeypatch.setenv("FB_FFT_PLANE", "1")
    y1, names1 = run(fb, x, dims, 1, -1)
    monkeypatch.delenv("FB_FFT_PLANE")
    y0, names0 = run(fb, x, dims, 1, -1)
    assert names1 == ["plane", "axis0"] and names0 == ["axis2", "axis1", "axis0"]
    n = int(np.prod(dims))
    rel = np.linalg.norm(y1.astype(np.complex128) - y0) / np.linalg.norm(y0.astype(np.complex128))
    assert rel <= 2 * tol(n)
