"""The butterflies of the line-pass kernels (dft<R> for R = 2, 3, 4, 5, 8, 16,
both directions), compiled for the host and checked against the DFT sum in
double on random inputs: relative L2 error at FP32 rounding level."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_butterflies_match_the_dft_sum(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "bfly"
    subprocess.run([nvcc, "-std=c++17", "-O2", f"-I{ROOT}/include", f"-I{ROOT}/paper_2004_09883_gb300/csrc",
                    os.path.join(ROOT, "tests", "butterfly_host.cu"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    seen = set()
    for line in filter(None, out):
        r, ef, ei = line.split()
        seen.add(int(r))
        assert float(ef) < 5e-7 and float(ei) < 5e-7, line
    assert seen == {2, 3, 4, 5, 8, 16}
