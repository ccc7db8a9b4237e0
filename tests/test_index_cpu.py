"""Index arithmetic of the line-pass kernels, compiled for the host from the
kernels' own headers: j mod Ns by multiply-high reciprocals (exact for every
case the kernels meet), and the split last-stage twiddle tables of the 2048-
and 4096-point schedules (their products equal exp(-2 pi i k r / L)), the
swizzled first work generation, and the bank placement of work and landing
rows."""
import math
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_index_arithmetic(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "idx"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                    f"-I{ROOT}/include", f"-I{ROOT}/paper_2004_09883_gb300/csrc",
                    os.path.join(ROOT, "tests", "index_host.cu"), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    rows = {ln.split()[0]: ln.split()[1:] for ln in lines if ln}
    cases, bad = map(int, rows["mod_by_reciprocal"])
    assert cases > 100_000 and bad == 0
    # 2048 and 4096 points split their last stage; 512 and 1024 keep one table
    assert rows["split_lg9"][0] == "none" and rows["split_lg10"][0] == "none"
    for lg in (11, 12):
        n, worst, sizes_ok = rows[f"split_lg{lg}"]
        assert int(n) == (1 << lg) // 16 * 15 and float(worst) < 1e-13 and sizes_ok == "1"
        # the kernel's FP32 factors (two table products, the rest stepped):
        # within a few ulp of 1 (at most seven products in a row)
        n, worst = rows[f"split_step_lg{lg}"]
        assert int(n) == (1 << lg) // 16 * 15 and float(worst) < 1e-6
    # the batched-uneven kernel's stage twiddles formed as powers (at most
    # three products deep): within a few ulp of 1
    n, worst = rows["uneven_step"]
    assert int(n) > 10_000 and float(worst) < 5e-7
    # the swizzled first work generation: one-to-one, inside the row, and
    # the second stage's shortcut reads the slots the first stage wrote
    n, bad, configs = map(int, rows["swizzle"])
    assert configs >= 3 and n > 10_000 and bad == 0
    # work-row strides: half-warps of lines-fast stages on 16 distinct banks
    n, bad = map(int, rows["p2_rows"])
    assert n > 1000 and bad == 0
    n, bad = map(int, rows["uneven_rows"])
    assert n > 10_000 and bad == 0
    n, bad = map(int, rows["uneven_land"])
    assert n > 100 and bad == 0


def test_plane_pass_emulation(tmp_path):
    """The plane pass (two trailing axes, one cluster of CTAs per plane) run
    on the host thread by thread and phase by phase with the kernel's own
    index functions and butterflies: every shared-memory slot, owner CTA and
    row in range, no slot written twice in a phase, and the result equal to
    the 2-D DFT summed in double for every compiled plane shape; and every
    shared-memory access pattern of every phase free of bank conflicts (each
    half-warp's 16 eight-byte slots in 16 different bank pairs)."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "plane"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                    f"-I{ROOT}/include", f"-I{ROOT}/paper_2004_09883_gb300/csrc",
                    os.path.join(ROOT, "tests", "plane_host.cu"), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    banks = [ln.split() for ln in lines if ln.startswith("banks")]
    assert len(banks) == 7
    for row in banks:  # every shared-memory access of every phase: one wavefront per half-warp
        assert all(int(v) == 1 for v in row[4:]), row
    rows = [ln.split() for ln in lines if ln.startswith("plane")]
    shapes = {(int(r[1]), int(r[2]), int(r[3])) for r in rows}
    assert shapes == {(256, 128, 512), (128, 128, 512), (256, 256, 512), (128, 256, 512),
                      (256, 128, 256), (128, 128, 256), (128, 256, 256)}
    assert len(rows) == 14
    for _, l1, l2, threads, direction, err, bad in rows:
        assert int(bad) == 0, (l1, l2, threads, direction)
        assert float(err) < 2e-6 * math.log2(int(l1) * int(l2)), (l1, l2, threads, direction, err)
