"""Radix-16 stages on the tensor cores (FB_FFT_TENSOR_CORES): every layout of
the power-of-two line pass against the FP64 oracle within 5e-5 relative L2
per result, next to the FP32 path's error on the same data."""
import numpy as np
import pytest

import oracle
from paper_2004_09883_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_TC = 5e-5


def _run(fb, dims, batch, direction, scale, x, tc):
    import torch
    with fb.Plan(dims, batch, scale_inv_n=scale, tensor_cores=tc) as p:
        info = p.info()
        y = p.exec(torch.from_numpy(x).cuda(), None, direction)
        torch.cuda.synchronize()
        p.check()
    return y.cpu().numpy(), info


def _errs(y, ref, batch):
    return oracle.rel_l2(y.reshape(batch, -1), ref.reshape(batch, -1))


CASES = [
    ([256], 64), ([512], 32), ([1024], 16), ([2048], 8), ([4096], 4),  # contiguous lines (NN)
    ([1 << 16], 2), ([1 << 20], 2), ([4096 * 1024], 1),               # four-step: strided columns + transposed rows
    ([256, 256], 2), ([512, 1024], 1), ([64, 4096], 1), ([256, 256, 16], 1), ([16, 2048, 8], 1),  # strided axes
    ([300, 256], 2), ([3, 1024], 5),                                   # ragged tiles, mixed with FP32 passes
]


@pytest.mark.parametrize("dims,batch", CASES)
@pytest.mark.parametrize("direction,scale", [(-1, False), (1, True)])
def test_tensor_core_path_matches_oracle(fb, dims, batch, direction, scale):
    n = int(np.prod(dims))
    x = inputs.normal_c64((batch, n), 3300 + n % 997 + batch)
    ref = oracle.fft(x.astype(np.complex128), dims, direction, scale, 8)
    y_tc, info = _run(fb, dims, batch, direction, scale, x, True)
    assert info["tc_passes"] > 0
    e_tc = _errs(y_tc, ref, batch)
    assert e_tc.max() <= TOL_TC, f"{dims} x {batch}: tensor-core rel L2 {e_tc.max():.3e}"
    y32, info32 = _run(fb, dims, batch, direction, scale, x, False)
    assert info32["tc_passes"] == 0
    e32 = _errs(y32, ref, batch)
    # both paths solve the same transform; the split products keep ~22 bits
    assert e_tc.max() <= max(50 * e32.max(), 2e-6), (e_tc.max(), e32.max())


def test_short_lines_keep_fp32_butterflies(fb):
    """Lengths below 256 have no tensor-core pass; results equal the FP32 plan's bit for bit."""
    x = inputs.uniform_c64((8, 128), 41)
    y_tc, info = _run(fb, [128], 8, -1, False, x, True)
    y32, _ = _run(fb, [128], 8, -1, False, x, False)
    assert info["tc_passes"] == 0
    assert np.array_equal(y_tc, y32)


def test_tensor_core_precision_workload_sample(fb):
    """The precision workload's shape (N = 2^20, standard normal): every result
    of a batch of 4 within 5e-5, and the round trip close to the identity."""
    import torch
    n, b = 1 << 20, 4
    x = inputs.normal_c64((b, n), inputs.seed_for(inputs.WORKLOAD_1D_2P20x32))
    ref = oracle.fft(x.astype(np.complex128), [n], -1, False, 16)
    with fb.Plan([n], b, tensor_cores=True) as pf, fb.Plan([n], b, scale_inv_n=True, tensor_cores=True) as pi:
        d = torch.from_numpy(x).cuda()
        y = pf.exec(d, None, -1)
        z = pi.exec(y, None, 1)
        torch.cuda.synchronize()
        pf.check()
        pi.check()
    e = _errs(y.cpu().numpy(), ref, b)
    assert e.max() <= TOL_TC, e
    rt = _errs(z.cpu().numpy(), x.astype(np.complex128), b)
    assert rt.max() <= 2 * TOL_TC, rt


def test_tensor_core_plans_through_the_server(fb):
    import torch
    x = torch.from_numpy(inputs.normal_c64((1024,), 5)).cuda()
    y = torch.empty_like(x)
    with fb.Server(slots=2, hbm_cap_bytes=1 << 20) as srv:
        srv.submit_ptr([1024], x.data_ptr(), y.data_ptr(), 7, -1, tensor_cores=True)
        srv.drain()
        assert [d[:2] for d in srv.poll()] == [(7, 0)]
    ref = oracle.fft(x.cpu().numpy().astype(np.complex128), [1024], -1)
    assert oracle.rel_l2(y.cpu().numpy().reshape(1, -1), ref.reshape(1, -1))[0] <= TOL_TC
