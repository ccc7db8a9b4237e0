"""fb_fft_exec_1d_noalloc: the entry point for callers that cannot allocate
device memory (a library embedded in a host application that owns all device
memory, real-time code that must stay out of allocators, code held to a fixed
memory budget).  Every call reuses one static workspace, so each result is
checked on two calls in a row: against the plan-based entry point's result
and against the FP64 oracle, within the parity tolerance of the other tests.

This file is named so pytest collects it last."""
import math
import os

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


@pytest.mark.parametrize("n,batch", [(1, 5), (2, 9), (64, 33), (256, 7), (4096, 5), (6000, 4), (3 * 5 ** 7, 2),
                                     (65536, 70), (1 << 20, 3)])
@pytest.mark.parametrize("direction,scale", [(-1, False), (1, True)])
def test_noalloc_matches_plan_api_and_oracle_on_two_calls_in_a_row(fb, n, batch, direction, scale):
    import torch
    x_h = inputs.normal_c64((batch, n), 77 + n)
    x = torch.from_numpy(x_h.reshape(-1)).cuda()
    want = _plan_result(fb, x, n, batch, direction, scale).cpu().numpy().reshape(batch, n)
    ref = oracle.fft(x_h.astype(np.complex128), [n], direction, scale, 8).reshape(batch, n)
    for call in range(2):
        out = torch.full_like(x, complex(float("nan"), 0.0))
        fb.exec_1d_noalloc(x, out, n, batch, direction, scale, check=(call == 1))
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(batch, n)
        assert np.all(np.isfinite(got)), f"call {call}: non-finite output"
        e_plan = oracle.rel_l2(got, want)
        e_ref = oracle.rel_l2(got, ref)
        assert e_plan.max() <= tol(n), f"call {call}: vs plan API rel L2 {e_plan.max():.3e} > {tol(n):.3e}"
        assert e_ref.max() <= tol(n), f"call {call}: vs oracle rel L2 {e_ref.max():.3e} > {tol(n):.3e}"


def test_noalloc_in_place_and_limits(fb):
    import torch
    n, batch = 1 << 16, 3
    x_h = inputs.uniform_c64((batch, n), 5)
    x = torch.from_numpy(x_h.reshape(-1)).cuda()
    ref = oracle.fft(x_h.astype(np.complex128), [n], -1, False, 8).reshape(batch, n)
    y = x.clone()
    fb.exec_1d_noalloc(y, y, n, batch, -1)
    torch.cuda.synchronize()
    assert oracle.rel_l2(y.cpu().numpy().reshape(batch, n), ref).max() <= tol(n)
    big = 1 << 23  # one transform larger than the static workspace
    with pytest.raises(fb.FFTError) as e:
        fb.exec_1d_noalloc(x, x, big, 1, -1)
    assert e.value.status == -2
    with pytest.raises(fb.FFTError) as e:
        fb.exec_1d_noalloc(x, x, 14, 1, -1)  # not 5-smooth
    assert e.value.status == -2


def test_noalloc_reports_a_timed_out_wait_when_asked(fb):
    """The library's test hook makes every TMA wait of the no-allocation path
    run out (after about a second; nothing faults).  With the check flag the
    call reports FB_FFT_ERR_TIMEOUT; the next call, without the hook, is
    correct again."""
    import torch
    n, batch = 4096, 8
    x_h = inputs.uniform_c64((batch, n), 6)
    x = torch.from_numpy(x_h.reshape(-1)).cuda()
    out = torch.empty_like(x)
    os.environ["FB_FFT_NOALLOC_DEBUG_TIMEOUT"] = "1"
    try:
        with pytest.raises(fb.FFTError) as e:
            fb.exec_1d_noalloc(x, out, n, batch, -1, check=True)
        assert e.value.status == -5
    finally:
        del os.environ["FB_FFT_NOALLOC_DEBUG_TIMEOUT"]
    fb.exec_1d_noalloc(x, out, n, batch, -1, check=True)
    ref = oracle.fft(x_h.astype(np.complex128), [n], -1).reshape(batch, n)
    assert oracle.rel_l2(out.cpu().numpy().reshape(batch, n), ref).max() <= tol(n)
