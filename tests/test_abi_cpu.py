"""Host-side checks of the C ABI library that need no GPU: it builds, loads,
exports every entry point the header declares, and its planner logic (radix
schedules, four-step splits, argument validation) behaves as documented."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2004_09883_gb300 import build as fbbuild
from paper_2004_09883_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def fb():
    fbbuild.build()
    from paper_2004_09883_gb300 import fbfft
    return fbfft


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(fb_fft_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_core_calls():
    names = declared_functions()
    for core in ("fb_fft_plan", "fb_fft_exec", "fb_fft_destroy", "fb_fft_exec_host", "fb_fft_status_string"):
        assert core in names


def test_library_exports_every_declared_symbol(fb):
    nm = subprocess.run(["nm", "-D", "--defined-only", fb.LIB_PATH], capture_output=True, text=True,
                        check=True).stdout
    exported = set(re.findall(r"\bT\s+(fb_fft_\w+)", nm))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for n in declared_functions():
        assert hasattr(fb.lib, n)


def test_header_compiles_as_plain_c(tmp_path):
    src = tmp_path / "use.c"
    src.write_text('#include "fb_fft.h"\nint main(void){ fb_fft_plan_t p = 0; (void)p; '
                   'return fb_fft_destroy(0); }\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-c", f"-I{ROOT}/include", str(src),
                    "-o", str(tmp_path / "use.o")], check=True)


def test_status_strings(fb):
    for code in range(-9, 1):
        assert fb.lib.fb_fft_status_string(code)
    assert b"unknown" in fb.lib.fb_fft_status_string(-99)


@pytest.mark.parametrize("n", inputs.smooth_lengths(1, 4096))
def test_factorize_every_smooth_length(fb, n):
    r = fb.factorize(n)
    assert int(np.prod(r)) == n
    assert all(x in (2, 3, 4, 5, 8, 16) for x in r)
    assert len(r) <= 8
    # power-of-two radices (16s and at most one 8/4/2) before 5s before 3s
    p2 = [x for x in r if x in (2, 4, 8)]
    assert len(p2) <= 1
    assert r == sorted(r, key=lambda x: {8: 0, 4: 0, 2: 0, 16: 0, 5: 2, 3: 3}[x])
    pw = [x for x in r if x in (2, 4, 8, 16)]
    if p2 and len(pw) == 2:
        assert pw == [16, p2[0]]       # two stages: radix 16 first
    elif p2:
        assert pw[0] == p2[0]          # three or more: the small radix first


@pytest.mark.parametrize("n", [0, -4, 7, 14, 4097 * 2, 8192, 11 * 16])
def test_factorize_rejects(fb, n):
    with pytest.raises(fb.FFTError):
        fb.factorize(n)


@pytest.mark.parametrize("n", [4097 * 0 + 4096, 5000, 8192, 65536, 1 << 20, 3 * 5 ** 7, 1 << 22, 1 << 24, 2 * 3 ** 9])
def test_split(fb, n):
    n1, n2 = fb.split(n)
    assert n1 * n2 == n
    assert n1 <= fb.MAX_SMEM_LEN and n2 <= fb.MAX_SMEM_LEN
    if n <= fb.MAX_SMEM_LEN:
        assert (n1, n2) == (n, 1)
    else:
        assert n1 <= n2  # the column pass takes the shorter factor


@pytest.mark.parametrize("n", [(1 << 24) * 2, 7 * 4096, 4099])
def test_split_rejects(fb, n):
    with pytest.raises(fb.FFTError):
        fb.split(n)


def _plan_rc(fb, dims, batch=1, flags=0):
    h = ctypes.c_void_p()
    cd = (ctypes.c_longlong * max(1, len(dims)))(*dims)
    return fb.lib.fb_fft_plan(ctypes.byref(h), len(dims), cd, batch, flags, None), h


@pytest.mark.parametrize("dims,batch,flags,rc", [
    ([], 1, 0, -1),            # rank 0
    ([4, 4, 4, 4], 1, 0, -1),  # rank 4
    ([0], 1, 0, -1),           # zero length
    ([8], -1, 0, -1),          # negative batch
    ([8], 1, 0x100, -1),       # unknown flag
    ([14], 1, 0, -2),          # 7 is not a supported prime
    ([8192, 2], 1, 0, -2),     # axis longer than one pass
    ([1 << 25], 1, 0, -2),     # longer than the four-step limit
])
def test_plan_argument_errors_need_no_device(fb, dims, batch, flags, rc):
    got, h = _plan_rc(fb, dims, batch, flags)
    assert got == rc
    assert not h.value


def test_plan_without_device_reports_no_device(fb):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    got, h = _plan_rc(fb, [64], 2)
    assert got == -7
    assert not h.value
    out = np.zeros(8, np.float32)
    assert fb.lib.fb_fft_twiddles(8, 4, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))) == -7


def test_null_plan_handling(fb):
    assert fb.lib.fb_fft_destroy(None) == 0
    assert fb.lib.fb_fft_exec(None, None, None, -1) == -6
    assert fb.lib.fb_fft_exec_host(None, None, None, -1) == -6
    assert fb.lib.fb_fft_check(None) == -6
    assert fb.lib.fb_fft_pass_name(None, 0) is None
    assert fb.lib.fb_fft_plan(None, 1, None, 1, 0, None) == -1


def test_struct_layouts_match_the_binding(fb, tmp_path):
    """Sizes and field offsets of the ABI structs, from a C compile of the
    header, equal those of the ctypes mirrors."""
    structs = {"fb_fft_info": fb.Info, "fb_fft_many_opts": fb.ManyOpts, "fb_fft_server_done": fb.ServerDone,
               "fb_fft_server_stats": fb.ServerStats, "fb_fft_server_request": fb.ServerRequest}
    cfield = {"in_ptr": "in", "out_ptr": "out"}  # C names that are Python keywords
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fb_fft.h"', 'int main(void){']
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {cfield.get(f, f)}));')
    lines.append('return 0; }')
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", f"-I{ROOT}/include", str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        cname, f, v = line.split()
        got[(cname, f)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_server_calls_without_device(fb):
    import torch
    assert fb.lib.fb_fft_server_destroy(None) == 0
    assert fb.lib.fb_fft_server_drain(None) == -6
    assert fb.lib.fb_fft_server_cancel(None, 0) == -6
    assert fb.lib.fb_fft_server_clock(None) == -1.0
    assert fb.lib.fb_fft_server_stats_get(None, None) == -6
    h = ctypes.c_void_p()
    assert fb.lib.fb_fft_server_create(None, 1, 0, 1) == -1
    assert fb.lib.fb_fft_server_create(ctypes.byref(h), 0, 0, 1) == -1
    assert fb.lib.fb_fft_server_create(ctypes.byref(h), 1, 0, 0) == -1
    if not torch.cuda.is_available():
        assert fb.lib.fb_fft_server_create(ctypes.byref(h), 1, 0, 1) == -7
        assert not h.value


def test_server_request_packing(fb):
    """Server.requests fills the request array the way submit_many reads it."""
    arr = fb.Server.requests([((64,), 0x1000, 0x2000, 7, -1), ((8, 12, 20), 0x3000, 0x3000, 8, 1, 2, True, True)])
    a, b = arr[0], arr[1]
    assert (a.rank, a.dims[0], a.batch, a.tag, a.in_ptr, a.out_ptr, a.direction, a.flags, a.host_io) == \
        (1, 64, 1, 7, 0x1000, 0x2000, -1, 0, 0)
    assert (b.rank, list(b.dims), b.batch, b.tag, b.in_ptr, b.out_ptr, b.direction, b.host_io) == \
        (3, [8, 12, 20], 2, 8, 0x3000, 0x3000, 1, 1)
    assert b.flags == fb.SCALE_INV_N
    assert fb.lib.fb_fft_server_submit_many(None, None, 0, None) == -6
    assert fb.lib.fb_fft_server_wait(None, 0.0) == -6


def test_launch_counter_starts_at_zero_without_gpu(fb):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    assert fb.launch_count() == 0


GPU_TEST_SHAPES = (
    [([n], 37) for n in [2 ** k for k in range(1, 13)]]
    + [([n], 37) for n in [3, 5, 6, 9, 10, 12, 15, 25, 27, 30, 45, 60, 81, 96, 100, 125, 243, 360, 375, 625,
                           729, 1000, 1536, 2187, 2400, 3125, 3645, 4000]]
    + [([n], b) for n, b in [(8192, 3), (65536, 2), (3 * 5 ** 7, 1), (1 << 20, 2), (6000, 5), (2 * 3 ** 9, 1),
                             (1 << 22, 1), (1 << 16, 70), (1 << 20, 32), (1 << 14, 3)]]
    + [(d, b) for d, b in [([16, 12], 3), ([256, 256], 2), ([512, 512], 1), ([100, 30], 4), ([8, 8, 8], 5),
                           ([30, 20, 12], 2), ([128, 128, 128], 1), ([6, 250, 18], 1), ([3, 5, 4096], 1),
                           ([4096, 2, 3], 1), ([256, 256, 128], 1), ([32, 32, 16], 2), ([60, 45], 2),
                           ([64, 48], 3), ([64, 64, 32], 2), ([1, 64], 2), ([64, 1], 2), ([1, 1, 1], 7)]]
)


@pytest.mark.parametrize("dims,batch", GPU_TEST_SHAPES)
def test_planner_accepts_every_tested_shape(fb, dims, batch):
    info = fb.plan_query(dims, batch, scale_inv_n=True)
    assert info["elements"] == int(np.prod(dims))
    n = info["elements"]
    nontrivial = [d for d in dims if d > 1]
    if len(dims) == 1 and n > fb.MAX_SMEM_LEN:
        assert info["passes"] % 2 == 0 and info["scratch_bytes"] > 0
    else:
        assert info["passes"] == len(nontrivial)  # one per axis (the plane pass is opt-in)
        assert info["scratch_bytes"] == 0


@pytest.mark.parametrize("dims,batch", [([256, 256, 128], 1), ([4, 256, 128], 2), ([256, 128], 3),
                                        ([128, 128], 1), ([2, 256, 256], 1), ([128, 256], 5)])
def test_plane_pass_switch(fb, dims, batch, monkeypatch):
    """FB_FFT_PLANE=1 fuses the two trailing axes into one plane pass;
    unset or 0, one pass per axis."""
    axes = len([d for d in dims if d > 1])
    monkeypatch.setenv("FB_FFT_PLANE", "0")
    assert fb.plan_query(dims, batch)["passes"] == axes
    monkeypatch.setenv("FB_FFT_PLANE", "1")
    assert fb.plan_query(dims, batch)["passes"] == axes - 1
    monkeypatch.setenv("FB_FFT_PLANE", "1")
    assert fb.plan_query(dims, batch, tensor_cores=True)["passes"] == axes  # FP32 butterflies only
    monkeypatch.delenv("FB_FFT_PLANE")
    assert fb.plan_query(dims, batch)["passes"] == axes
    # planes of other shapes always run per axis
    monkeypatch.setenv("FB_FFT_PLANE", "1")
    assert fb.plan_query([64, 128], 4)["passes"] == 2
    assert fb.plan_query([512, 128], 4)["passes"] == 2


@pytest.mark.parametrize("n", inputs.smooth_lengths(4097, 1 << 24)[::7])
def test_planner_accepts_long_1d(fb, n):
    # plannable exactly when n = n1 * n2 with both factors <= 4096
    splittable = any(n % d == 0 and n // d <= fb.MAX_SMEM_LEN for d in range(1, fb.MAX_SMEM_LEN + 1))
    if not splittable:
        with pytest.raises(fb.FFTError):
            fb.plan_query([n], 2)
        return
    info = fb.plan_query([n], 2)
    assert info["passes"] % 2 == 0 and info["passes"] >= 2 and info["scratch_bytes"] >= 8 * n


def test_many_layout_is_packed_and_16_byte_aligned(fb):
    lens = [3, 4, 5, 8, 1, 64, 75]
    offs, total = fb.many_layout(lens)
    assert offs[0] == 0
    for i in range(1, len(lens)):
        assert offs[i] == offs[i - 1] + lens[i - 1] + (lens[i - 1] & 1)
        assert offs[i] % 2 == 0
    assert total == offs[-1] + lens[-1] + (lens[-1] & 1)
    assert fb.many_layout([])[1] == 0
    with pytest.raises(ValueError):
        fb.many_layout([4, 0])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_many_planner_schedules_pass_host_checks(fb, seed):
    lens = list(inputs.uneven_lengths(300, 64, 65536, inputs.seed_for(inputs.WORKLOAD_UNEVEN_4096, seed)))
    lens += [2, 3, 4096, 4096, 65536, 1 << 20, 6000, 45000, 75]
    info = fb.plan_many_query(lens)
    offs, total = fb.many_layout(lens)
    assert info["elements"] == total and info["batch"] == len(lens)
    # the one-kernel engine (every length fits it here): every pass of the batch in one launch
    assert info["passes"] == 1
    # every four-step transform owns its scratch (the merged launches run them together)
    assert info["scratch_bytes"] >= 8 * sum(int(n) for n in lens if n > fb.MAX_SMEM_LEN)


@pytest.mark.parametrize("dims,tc", [([128], 0), ([256], 1), ([1024], 1), ([4096], 1), ([1 << 20], 2), ([1 << 13], 0), ([1 << 16], 2),
                                     ([256, 256], 2), ([16, 2048, 8], 1), ([300, 256], 1), ([60, 45], 0),
                                     ([3 * 1024], 0)])
def test_tensor_core_flag_planning(fb, dims, tc):
    """Passes over power-of-two lines of length >= 256 take the tensor-core
    kernels; the pass list is otherwise the FP32 plan's."""
    q = fb.plan_query(dims, 2, tensor_cores=True)
    q32 = fb.plan_query(dims, 2)
    assert q["tc_passes"] == tc and q32["tc_passes"] == 0
    assert q["passes"] == q32["passes"] and q["scratch_bytes"] == q32["scratch_bytes"]


def test_tensor_core_flag_rejected_where_unsupported(fb):
    lens = (ctypes.c_longlong * 2)(256, 512)
    inf = fb.Info()
    assert fb.lib.fb_fft_plan_many_query(2, lens, fb.TENSOR_CORES, ctypes.byref(inf)) == -1
    assert fb.lib.fb_fft_exec_1d_noalloc(None, None, 256, 0, -1, fb.TENSOR_CORES, None) == -1
    assert fb.lib.fb_fft_plan_query(1, (ctypes.c_longlong * 1)(256), 1, 0x4, ctypes.byref(inf)) == -1
