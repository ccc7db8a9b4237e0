"""The offload decision (the paper's verification step): the library times
the caller's CPU block against its own host-array GPU call and picks the
faster.  Here the caller's CPU block is the oracle (test infrastructure)."""
import numpy as np
import pytest

import oracle
from paper_2004_09883_gb300 import inputs

pytestmark = pytest.mark.gpu


def _oracle_block(dims):
    def block(x, out, direction):
        out[:] = oracle.fft(x.astype(np.complex128), dims, direction).astype(np.complex64).reshape(-1)
    return block


def test_decision_follows_the_measured_times(fb):
    tiny = inputs.uniform_c64((1, 8), 1)
    with fb.Plan([8], 1) as p:
        r = p.offload_decide(_oracle_block([8]), tiny, -1, reps=5)
    assert r["use_gpu"] == (r["gpu_ms"] < r["cpu_ms"])
    big = inputs.uniform_c64((4, 1 << 18), 2)
    with fb.Plan([1 << 18], 4) as p:
        r2 = p.offload_decide(_oracle_block([1 << 18]), big, -1, reps=2)
    assert r2["use_gpu"] == (r2["gpu_ms"] < r2["cpu_ms"])
    assert r2["use_gpu"], f"a 4 x 2^18 transform should offload: {r2}"
    assert r2["cpu_ms"] > 10 * r2["gpu_ms"]


def test_decide_rejects_bad_arguments(fb):
    x = inputs.uniform_c64((1, 16), 3)
    with fb.Plan([16], 1) as p:
        with pytest.raises(fb.FFTError):
            p.offload_decide(_oracle_block([16]), x, 0)
