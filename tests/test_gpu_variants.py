"""Launch variants that change scheduling, not arithmetic, give the same bits:
programmatic dependent launch off (FB_FFT_PDL=0), the CTA size of passes
over short contiguous lines (FB_FFT_NN_SMALL_THREADS=64/128/256), and the L2
policies of the first pass's loads and the intermediate passes' stores
(FB_FFT_EVICT_FIRST=0, FB_FFT_EVICT_LAST=0).  Each runs in a subprocess (the
library reads the variables once)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2004_09883_gb300 import fbfft, inputs
out = []
for dims, b in [([256, 256, 128], 1), ([128], 512), ([64, 100], 3), ([1 << 20], 2), ([4096], 16), ([256], 300),
                ([32], 999)]:
    x = torch.from_numpy(inputs.uniform_c64([b] + dims, 4242)).cuda()
    with fbfft.Plan(dims, b, scale_inv_n=True) as p:
        y = p.exec(x, None, -1)
        z = p.exec(y, None, 1)
        torch.cuda.synchronize()
        p.check()
    out.append(y.cpu().numpy().ravel())
    out.append(z.cpu().numpy().ravel())
np.save(sys.argv[2], np.concatenate(out))
"""


def _run(tmp_path, name, env_extra):
    path = tmp_path / f"{name}.npy"
    env = dict(os.environ, **env_extra)
    subprocess.run([sys.executable, "-c", SCRIPT, ROOT, str(path)], check=True, env=env, timeout=600)
    return np.load(path)


def test_launch_variants_give_identical_bits(fb, tmp_path):
    base = _run(tmp_path, "base", {})
    for name, env in [("no_pdl", {"FB_FFT_PDL": "0"}), ("nn256", {"FB_FFT_NN_SMALL_THREADS": "256"}),
                      ("nn128", {"FB_FFT_NN_SMALL_THREADS": "128"}), ("nn64", {"FB_FFT_NN_SMALL_THREADS": "64"}),
                      ("no_evict_first", {"FB_FFT_EVICT_FIRST": "0"}), ("no_evict_last", {"FB_FFT_EVICT_LAST": "0"})]:
        got = _run(tmp_path, name, env)
        assert np.array_equal(base, got), name
