"""fb_fft_exec_1d_noalloc: the entry point for callers that cannot allocate
device memory (code running during a CUDA graph capture, real-time code that
must stay out of allocators, embedders whose memory belongs to another
allocator).  It must give the same results as the plan-based entry point,
call after call, although every call reuses one static workspace.

This file is named so pytest collects it last."""
import math

import numpy as np
import pytest

import oracle
from paper_2004_09883_gb300 import inputs

pytestmark = pytest.mark.gpu


def tol(n: int) -> float:  # the parity tolerance used throughout the tests
    return 2e-6 * math.log2(n) if n > 1 else 1e-7


def _plan_result(fb, x, n, batch, direction, scale):
    with fb.Plan([n], batch, scale_inv_n=scale) as p:
        y = p.exec(x, None, direction)
        p.check()
        return y


@pytest.mark.parametrize("n,batch", [(1 << 20, 3), (4096, 5), (3 * 5 ** 7, 2), (6000, 4), (65536, 70)])
@pytest.mark.parametrize("direction,scale", [(-1, False), (1, True)])
def test_noalloc_matches_plan_api_on_two_calls_in_a_row(fb, n, batch, direction, scale):
    import torch
    x = torch.from_numpy(inputs.normal_c64((batch, n), 77 + n).reshape(-1)).cuda()
    want = _plan_result(fb, x, n, batch, direction, scale).cpu().numpy().reshape(batch, n)
    for call in range(2):
        out = torch.full_like(x, complex(float("nan"), 0.0))
        fb.exec_1d_noalloc(x, out, n, batch, direction, scale)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(batch, n)
        err = oracle.rel_l2(got, want)
        assert np.all(np.isfinite(got)), f"call {call}: non-finite output"
        assert err.max() <= tol(n), f"call {call}: rel L2 {err.max():.3e} > {tol(n):.3e}"


def test_noalloc_in_place_and_limits(fb):
    import torch
    n, batch = 1 << 16, 3
    x = torch.from_numpy(inputs.uniform_c64((batch, n), 5).reshape(-1)).cuda()
    want = _plan_result(fb, x, n, batch, -1, False).cpu().numpy()
    y = x.clone()
    fb.exec_1d_noalloc(y, y, n, batch, -1)
    torch.cuda.synchronize()
    assert oracle.rel_l2(y.cpu().numpy().reshape(batch, n), want.reshape(batch, n)).max() <= tol(n)
    big = 1 << 23  # one transform larger than the static workspace
    with pytest.raises(fb.FFTError) as e:
        fb.exec_1d_noalloc(x, x, big, 1, -1)
    assert e.value.status == -2
    with pytest.raises(fb.FFTError) as e:
        fb.exec_1d_noalloc(x, x, 14, 1, -1)
    assert e.value.status == -2
