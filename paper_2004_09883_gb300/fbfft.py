"""ctypes binding of ``libfbfft.so`` (the C ABI in ``include/fb_fft.h``).

Argument marshalling only: every transform runs in the library's CUDA kernels.
Device buffers are torch tensors (complex64, contiguous, on the plan's device);
host buffers for :meth:`Plan.exec_host` are numpy complex64 arrays.  Importing
this module raises if the compiled library is missing -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfbfft.so")

FORWARD = -1
INVERSE = 1
SCALE_INV_N = 0x1
TENSOR_CORES = 0x2
NOALLOC_CHECK = 0x100  # fb_fft_exec_1d_noalloc: wait and report a timed-out device wait
MAX_SMEM_LEN = 4096
MAX_1D_LEN = 4096 * 4096

STATUS = {
    0: "FB_FFT_OK", -1: "FB_FFT_ERR_INVALID_ARG", -2: "FB_FFT_ERR_UNSUPPORTED_SIZE",
    -3: "FB_FFT_ERR_ALLOC", -4: "FB_FFT_ERR_CUDA", -5: "FB_FFT_ERR_TIMEOUT",
    -6: "FB_FFT_ERR_BAD_PLAN", -7: "FB_FFT_ERR_NO_DEVICE", -8: "FB_FFT_ERR_CANCELLED",
    -9: "FB_FFT_ERR_OVER_BUDGET",
}


class FFTError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        detail = lib.fb_fft_last_error().decode() if status == -4 else ""
        super().__init__(f"{what}: {STATUS.get(status, status)} ({_text(status)})"
                         + (f" [{detail}]" if detail else ""))


class Info(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int), ("tc_passes", ctypes.c_int),
                ("smem_len_max", ctypes.c_longlong), ("scratch_bytes", ctypes.c_longlong),
                ("twiddle_bytes", ctypes.c_longlong), ("elements", ctypes.c_longlong),
                ("batch", ctypes.c_longlong)]


class ManyOpts(ctypes.Structure):
    """Knobs of a batched uneven plan (0 = default)."""
    _fields_ = [("streams", ctypes.c_int), ("use_graph", ctypes.c_int), ("chunk_bytes", ctypes.c_longlong),
                ("odd_radices_first", ctypes.c_int), ("max_lines", ctypes.c_int), ("per_length", ctypes.c_int),
                ("engine", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerDone(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_longlong), ("status", ctypes.c_int), ("slot", ctypes.c_int),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("t_dev_start", ctypes.c_double), ("t_dev_end", ctypes.c_double)]


class ServerRequest(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_longlong * 3), ("batch", ctypes.c_longlong), ("tag", ctypes.c_longlong),
                ("in_ptr", ctypes.c_void_p), ("out_ptr", ctypes.c_void_p), ("rank", ctypes.c_int),
                ("flags", ctypes.c_uint), ("direction", ctypes.c_int), ("host_io", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_longlong) for f in (
        "submitted", "completed", "rejected", "cancelled", "pending", "in_flight", "plans", "plan_builds",
        "plan_bytes", "arena_bytes", "arena_in_use", "arena_peak", "max_in_flight")] + [
        ("slots", ctypes.c_int), ("reserved", ctypes.c_int)] + [
        (f, ctypes.c_longlong) for f in ("batches", "batched_requests", "largest_batch", "max_busy_slots")]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


CPU_BLOCK = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int)


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                      "(python -m paper_2004_09883_gb300.build)")

lib = ctypes.CDLL(LIB_PATH)
_vp, _ll, _int = ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int
_sig = {
    "fb_fft_plan": (_int, [ctypes.POINTER(_vp), _int, ctypes.POINTER(_ll), _ll, ctypes.c_uint, _vp]),
    "fb_fft_exec": (_int, [_vp, _vp, _vp, _int]),
    "fb_fft_exec_host": (_int, [_vp, _vp, _vp, _int]),
    "fb_fft_check": (_int, [_vp]),
    "fb_fft_set_stream": (_int, [_vp, _vp]),
    "fb_fft_destroy": (_int, [_vp]),
    "fb_fft_status_string": (ctypes.c_char_p, [_int]),
    "fb_fft_last_error": (ctypes.c_char_p, []),
    "fb_fft_plan_info": (_int, [_vp, ctypes.POINTER(Info)]),
    "fb_fft_plan_query": (_int, [_int, ctypes.POINTER(_ll), _ll, ctypes.c_uint, ctypes.POINTER(Info)]),
    "fb_fft_factorize": (_int, [_ll, ctypes.POINTER(_int), _int, ctypes.POINTER(_int)]),
    "fb_fft_split": (_int, [_ll, ctypes.POINTER(_ll), ctypes.POINTER(_ll)]),
    "fb_fft_profile": (_int, [_vp, _int]),
    "fb_fft_profile_read": (_int, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_ll), _int,
                                   ctypes.POINTER(_int)]),
    "fb_fft_pass_name": (ctypes.c_char_p, [_vp, _int]),
    "fb_fft_pass_launch": (_int, [_vp, _int, ctypes.POINTER(_ll), ctypes.POINTER(_int), ctypes.POINTER(_ll)]),
    "fb_fft_launch_count": (_ll, []),
    "fb_fft_twiddles": (_int, [_ll, _ll, ctypes.POINTER(ctypes.c_float)]),
    "fb_fft_debug_inject_timeout": (_int, [_vp, _int]),
    "fb_fft_exec_1d_noalloc": (_int, [_vp, _vp, _ll, _ll, _int, ctypes.c_uint, _vp]),
    "fb_fft_many_layout": (_ll, [_int, ctypes.POINTER(_ll), ctypes.POINTER(_ll)]),
    "fb_fft_plan_many": (_int, [ctypes.POINTER(_vp), _int, ctypes.POINTER(_ll), ctypes.c_uint, _vp]),
    "fb_fft_set_graph": (_int, [_vp, _int]),
    "fb_fft_offload_decide": (_int, [_vp, CPU_BLOCK, _vp, _vp, _vp, _int, _int, ctypes.POINTER(_int),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "fb_fft_server_create": (_int, [ctypes.POINTER(_vp), _int, _ll, _int]),
    "fb_fft_server_submit": (_int, [_vp, _int, ctypes.POINTER(_ll), _ll, ctypes.c_uint, _int, _vp, _vp, _int, _ll]),
    "fb_fft_server_prepare": (_int, [_vp, _int, ctypes.POINTER(_ll), _ll, ctypes.c_uint]),
    "fb_fft_server_poll": (_int, [_vp, _int, ctypes.POINTER(ServerDone), _int, ctypes.POINTER(_int)]),
    "fb_fft_server_drain": (_int, [_vp]),
    "fb_fft_server_cancel": (_int, [_vp, _ll]),
    "fb_fft_server_clock": (ctypes.c_double, [_vp]),
    "fb_fft_server_stats_get": (_int, [_vp, ctypes.POINTER(ServerStats)]),
    "fb_fft_server_set_batch": (_int, [_vp, _int]),
    "fb_fft_server_wait": (_int, [_vp, ctypes.c_double]),
    "fb_fft_server_submit_many": (_int, [_vp, ctypes.POINTER(ServerRequest), _int, ctypes.POINTER(_int)]),
    "fb_fft_server_destroy": (_int, [_vp]),
    "fb_fft_plan_many_query": (_int, [_int, ctypes.POINTER(_ll), ctypes.c_uint, ctypes.POINTER(Info)]),
    "fb_fft_plan_many_ex": (_int, [ctypes.POINTER(_vp), _int, ctypes.POINTER(_ll), ctypes.c_uint, _vp,
                                   ctypes.POINTER(ManyOpts)]),
    "fb_fft_autotune_many": (_int, [_int, ctypes.POINTER(_ll), ctypes.c_uint, _vp, _vp, _int, _vp, _int,
                                    ctypes.POINTER(ManyOpts), ctypes.POINTER(ctypes.c_float)]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _text(status: int) -> str:
    return lib.fb_fft_status_string(int(status)).decode()


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise FFTError(rc, what)


def factorize(n: int) -> list[int]:
    """Radix schedule the planner uses for an in-shared-memory line of length n."""
    buf = (_int * 32)()
    cnt = _int()
    _check(lib.fb_fft_factorize(int(n), buf, 32, ctypes.byref(cnt)), "fb_fft_factorize")
    return list(buf[: cnt.value])


def split(n: int) -> tuple[int, int]:
    """Four-step split n = n1 * n2 of a rank-1 length (n2 == 1: one pass)."""
    n1, n2 = _ll(), _ll()
    _check(lib.fb_fft_split(int(n), ctypes.byref(n1), ctypes.byref(n2)), "fb_fft_split")
    return n1.value, n2.value


def _flags(scale_inv_n: bool, tensor_cores: bool) -> int:
    return (SCALE_INV_N if scale_inv_n else 0) | (TENSOR_CORES if tensor_cores else 0)


def plan_query(dims, batch: int = 1, scale_inv_n: bool = False, tensor_cores: bool = False) -> dict:
    """Host-only planner run: what fb_fft_plan would build (no GPU needed)."""
    dims = [int(d) for d in dims]
    cd = (_ll * len(dims))(*dims)
    inf = Info()
    _check(lib.fb_fft_plan_query(len(dims), cd, int(batch), _flags(scale_inv_n, tensor_cores),
                                 ctypes.byref(inf)), "fb_fft_plan_query")
    return {f: getattr(inf, f) for f, _ in Info._fields_ if f != "reserved"}


def many_layout(lengths) -> tuple[np.ndarray, int]:
    """(offsets, total) of the packed layout of a batch of uneven transforms."""
    lens = np.ascontiguousarray(np.asarray(lengths, dtype=np.int64))
    offs = np.empty_like(lens)
    total = lib.fb_fft_many_layout(len(lens), lens.ctypes.data_as(ctypes.POINTER(_ll)),
                                   offs.ctypes.data_as(ctypes.POINTER(_ll)))
    if total < 0:
        raise ValueError("bad lengths")
    return offs, int(total)


def plan_many_query(lengths, scale_inv_n: bool = False) -> dict:
    """Host-only planner run for a batched uneven plan (no GPU needed)."""
    lens = np.ascontiguousarray(np.asarray(lengths, dtype=np.int64))
    inf = Info()
    _check(lib.fb_fft_plan_many_query(len(lens), lens.ctypes.data_as(ctypes.POINTER(_ll)),
                                      SCALE_INV_N if scale_inv_n else 0, ctypes.byref(inf)), "fb_fft_plan_many_query")
    return {f: getattr(inf, f) for f, _ in Info._fields_ if f != "reserved"}


def launch_count() -> int:
    return int(lib.fb_fft_launch_count())


def twiddles(d: int, count: int) -> np.ndarray:
    """exp(-2*pi*i*m/d), m = 0..count-1, from the library's FP64 twiddle kernel."""
    out = np.empty(2 * int(count), dtype=np.float32)
    _check(lib.fb_fft_twiddles(int(d), int(count), out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
           "fb_fft_twiddles")
    return out.view(np.complex64)


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        if not torch.cuda.is_available():
            return 0
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """A planned complex64 C2C transform: ``dims`` (row-major) x ``batch``."""

    def __init__(self, dims, batch: int = 1, scale_inv_n: bool = False, stream=None, tensor_cores: bool = False):
        dims = [int(d) for d in (dims if hasattr(dims, "__len__") else [dims])]
        self.dims = dims
        self.batch = int(batch)
        self.flags = _flags(scale_inv_n, tensor_cores)
        self.n = int(np.prod(dims))
        self._h = _vp()
        cd = (_ll * len(dims))(*dims)
        self._stream = _stream_handle(stream)
        _check(lib.fb_fft_plan(ctypes.byref(self._h), len(dims), cd, self.batch, self.flags,
                               _vp(self._stream)), "fb_fft_plan")

    # -- lifetime -----------------------------------------------------------
    def close(self) -> None:
        if self._h:
            rc = lib.fb_fft_destroy(self._h)
            self._h = _vp()
            _check(rc, "fb_fft_destroy")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> int:
        return self._h.value or 0

    # -- execution ----------------------------------------------------------
    def set_stream(self, stream) -> None:
        self._stream = _stream_handle(stream)
        _check(lib.fb_fft_set_stream(self._h, _vp(self._stream)), "fb_fft_set_stream")

    def exec_ptr(self, in_ptr: int, out_ptr: int, direction: int = FORWARD) -> None:
        """Run on raw device pointers (asynchronous on the plan's stream)."""
        _check(lib.fb_fft_exec(self._h, _vp(in_ptr), _vp(out_ptr), int(direction)), "fb_fft_exec")

    def exec(self, x, out=None, direction: int = FORWARD):
        """Transform torch complex64 CUDA tensor ``x`` (batch*prod(dims) values)
        into ``out`` (new tensor if None; ``out is x`` runs in place)."""
        import torch
        if x.dtype != torch.complex64 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("x must be a contiguous complex64 CUDA tensor")
        if x.numel() != self.n * self.batch:
            raise ValueError(f"x has {x.numel()} values, plan expects {self.n * self.batch}")
        if out is None:
            out = torch.empty_like(x)
        elif out.dtype != torch.complex64 or not out.is_contiguous() or out.numel() != x.numel():
            raise ValueError("out must be a contiguous complex64 tensor like x")
        s = torch.cuda.current_stream(x.device).cuda_stream
        if s != self._stream:
            self.set_stream(s)
        self.exec_ptr(x.data_ptr(), out.data_ptr(), direction)
        return out

    def exec_host(self, x: np.ndarray, out: np.ndarray | None = None, direction: int = FORWARD):
        """Drop-in CPU-array form: host in, host out, synchronous."""
        x = np.ascontiguousarray(x, dtype=np.complex64)
        if x.size != self.n * self.batch:
            raise ValueError("size mismatch")
        if out is None:
            out = np.empty_like(x)
        if out.dtype != np.complex64 or not out.flags.c_contiguous or out.size != x.size:
            raise ValueError("out must be a contiguous complex64 array like x")
        _check(lib.fb_fft_exec_host(self._h, _vp(x.ctypes.data), _vp(out.ctypes.data), int(direction)),
               "fb_fft_exec_host")
        return out

    def offload_decide(self, cpu_block, x: np.ndarray, direction: int = FORWARD, reps: int = 3) -> dict:
        """Time the caller's CPU routine ``cpu_block(x_in, x_out, direction)``
        (numpy complex64 arrays) against this plan's host-array GPU call and
        say which is faster (the verification step)."""
        x = np.ascontiguousarray(x, dtype=np.complex64)
        out = np.empty_like(x)
        n = x.size

        def tramp(_ctx, src, dst, d):
            a = np.ctypeslib.as_array(ctypes.cast(src, ctypes.POINTER(ctypes.c_float)), shape=(2 * n,))
            b = np.ctypeslib.as_array(ctypes.cast(dst, ctypes.POINTER(ctypes.c_float)), shape=(2 * n,))
            cpu_block(a.view(np.complex64), b.view(np.complex64), d)

        cb = CPU_BLOCK(tramp)
        use, cms, gms = _int(), ctypes.c_double(), ctypes.c_double()
        _check(lib.fb_fft_offload_decide(self._h, cb, None, _vp(x.ctypes.data), _vp(out.ctypes.data), int(direction),
                                         int(reps), ctypes.byref(use), ctypes.byref(cms), ctypes.byref(gms)),
               "fb_fft_offload_decide")
        return {"use_gpu": bool(use.value), "cpu_ms": cms.value, "gpu_ms": gms.value}

    def debug_inject_timeout(self, enable: bool = True) -> None:
        """Test hook: make the plan's bounded device waits run out."""
        _check(lib.fb_fft_debug_inject_timeout(self._h, 1 if enable else 0), "fb_fft_debug_inject_timeout")

    def check(self) -> None:
        """Synchronise and raise if a kernel reported a bounded-wait timeout."""
        _check(lib.fb_fft_check(self._h), "fb_fft_check")

    # -- introspection ------------------------------------------------------
    def info(self) -> dict:
        inf = Info()
        _check(lib.fb_fft_plan_info(self._h, ctypes.byref(inf)), "fb_fft_plan_info")
        return {f: getattr(inf, f) for f, _ in Info._fields_ if f != "reserved"}

    def launch_config(self) -> list[tuple[int, int, int]]:
        """(grid, threads per CTA, dynamic shared bytes) of every pass, in launch order."""
        out = []
        for i in range(self.info()["passes"]):
            g, b, m = _ll(), _int(), _ll()
            _check(lib.fb_fft_pass_launch(self._h, i, ctypes.byref(g), ctypes.byref(b), ctypes.byref(m)),
                   "fb_fft_pass_launch")
            out.append((g.value, b.value, m.value))
        return out

    def pass_names(self) -> list[str]:
        names = []
        i = 0
        while True:
            nm = lib.fb_fft_pass_name(self._h, i)
            if not nm:
                return names
            names.append(nm.decode())
            i += 1

    def profile(self, enable: bool = True) -> None:
        _check(lib.fb_fft_profile(self._h, 1 if enable else 0), "fb_fft_profile")

    def profile_read(self) -> list[tuple[str, float, int]]:
        """Per pass role: (name, total ms, launches) since the last read."""
        cap = 16
        ms = (ctypes.c_double * cap)()
        cnt = (_ll * cap)()
        n = _int()
        _check(lib.fb_fft_profile_read(self._h, ms, cnt, cap, ctypes.byref(n)), "fb_fft_profile_read")
        names = self.pass_names()
        return [(names[i], ms[i], cnt[i]) for i in range(min(n.value, cap))]


class PlanMany(Plan):
    """Batched 1-D transforms of uneven lengths in the packed layout of
    :func:`many_layout` (one graph launch per exec)."""

    def __init__(self, lengths, scale_inv_n: bool = False, stream=None, opts: "ManyOpts | dict | None" = None):
        lens = np.ascontiguousarray(np.asarray(lengths, dtype=np.int64))
        self.lengths = lens
        self.offsets, self.total = many_layout(lens)
        self.dims = None
        self.batch = len(lens)
        self.flags = SCALE_INV_N if scale_inv_n else 0
        self._h = _vp()
        self._stream = _stream_handle(stream)
        if isinstance(opts, dict):
            opts = ManyOpts(**opts)
        self.opts = opts
        _check(lib.fb_fft_plan_many_ex(ctypes.byref(self._h), len(lens), lens.ctypes.data_as(ctypes.POINTER(_ll)),
                                       self.flags, _vp(self._stream), ctypes.byref(opts) if opts else None),
               "fb_fft_plan_many_ex")
        self.n = self.total  # exec() checks numel == n * batch
        self.batch_for_size = 1

    def exec(self, x, out=None, direction: int = FORWARD):
        import torch
        if x.dtype != torch.complex64 or not x.is_cuda or not x.is_contiguous() or x.numel() != self.total:
            raise ValueError(f"x must be a contiguous complex64 CUDA tensor of {self.total} values")
        if out is None:
            out = torch.empty_like(x)
        s = torch.cuda.current_stream(x.device).cuda_stream
        if s != self._stream:
            self.set_stream(s)
        self.exec_ptr(x.data_ptr(), out.data_ptr(), direction)
        return out

    def exec_host(self, x, out=None, direction: int = FORWARD):
        x = np.ascontiguousarray(x, dtype=np.complex64)
        if x.size != self.total:
            raise ValueError("size mismatch")
        out = np.empty_like(x) if out is None else out
        _check(lib.fb_fft_exec_host(self._h, _vp(x.ctypes.data), _vp(out.ctypes.data), int(direction)),
               "fb_fft_exec_host")
        return out

    def set_graph(self, enable: bool) -> None:
        _check(lib.fb_fft_set_graph(self._h, 1 if enable else 0), "fb_fft_set_graph")

    def pack(self, items) -> np.ndarray:
        """Host helper: pack a list of 1-D arrays into the plan's layout."""
        buf = np.zeros(self.total, dtype=np.complex64)
        for o, a in zip(self.offsets, items):
            buf[o:o + len(a)] = a
        return buf

    def unpack(self, buf):
        return [np.asarray(buf[o:o + n]) for o, n in zip(self.offsets, self.lengths)]


def autotune_many(lengths, x, out, direction: int = FORWARD, scale_inv_n: bool = False, reps: int = 5):
    """Run the library's autotuner on device buffers x/out (packed layout);
    returns (ManyOpts, ms per exec).  `out` is overwritten."""
    import torch
    lens = np.ascontiguousarray(np.asarray(lengths, dtype=np.int64))
    best = ManyOpts()
    ms = ctypes.c_float()
    s = torch.cuda.current_stream(x.device).cuda_stream
    _check(lib.fb_fft_autotune_many(len(lens), lens.ctypes.data_as(ctypes.POINTER(_ll)),
                                    SCALE_INV_N if scale_inv_n else 0, _vp(x.data_ptr()), _vp(out.data_ptr()),
                                    int(direction), _vp(s), int(reps), ctypes.byref(best), ctypes.byref(ms)),
           "fb_fft_autotune_many")
    return best, ms.value


def exec_1d_noalloc(x, out, n: int, batch: int, direction: int = FORWARD, scale_inv_n: bool = False,
                    check: bool = False):
    """Batched 1-D transform through fb_fft_exec_1d_noalloc: no plan, no
    device allocation (the library's static workspace is used), on the
    current torch stream.  ``x`` and ``out`` are complex64 CUDA tensors.
    ``check`` waits for the transform and raises FFTError (status
    FB_FFT_ERR_TIMEOUT) if one of its device-side waits gave up."""
    import torch
    s = torch.cuda.current_stream(x.device).cuda_stream
    flags = (SCALE_INV_N if scale_inv_n else 0) | (NOALLOC_CHECK if check else 0)
    _check(lib.fb_fft_exec_1d_noalloc(_vp(x.data_ptr()), _vp(out.data_ptr()), int(n), int(batch), int(direction),
                                      flags, _vp(s)), "fb_fft_exec_1d_noalloc")
    return out


def fft(x, dims, direction: int = FORWARD, scale_inv_n: bool = False, out=None):
    """One-shot convenience: plan, run, destroy (plans should be reused in hot loops)."""
    n = int(np.prod(dims))
    with Plan(dims, x.numel() // n, scale_inv_n=scale_inv_n) as p:
        return p.exec(x, out, direction)


class Server:
    """Continuous-batching request server (``fb_fft_server_*``): ``slots``
    concurrent requests or batches, ``hbm_cap_bytes`` of device memory for
    their scratch and staging, resident plans (at most ``max_plans``); up to
    ``max_batch`` queued requests run as one batch (1: each alone through its
    plan)."""

    def __init__(self, slots: int = 8, hbm_cap_bytes: int = 40 * 10**9, max_plans: int = 4096,
                 max_batch: int = 64):
        self._h = _vp()
        _check(lib.fb_fft_server_create(ctypes.byref(self._h), int(slots), int(hbm_cap_bytes), int(max_plans)),
               "fb_fft_server_create")
        self._buf = (ServerDone * 256)()
        self._shape_args = {}
        self.set_batch(max_batch)

    def set_batch(self, max_requests: int) -> None:
        _check(lib.fb_fft_server_set_batch(self._h, int(max_requests)), "fb_fft_server_set_batch")

    def close(self) -> None:
        if self._h:
            rc = lib.fb_fft_server_destroy(self._h)
            self._h = _vp()
            _check(rc, "fb_fft_server_destroy")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def _dims(dims):
        dims = [int(d) for d in (dims if hasattr(dims, "__len__") else [dims])]
        return len(dims), (_ll * len(dims))(*dims)

    def prepare(self, dims, batch: int = 1, scale_inv_n: bool = False, tensor_cores: bool = False) -> None:
        r, cd = self._dims(dims)
        _check(lib.fb_fft_server_prepare(self._h, r, cd, int(batch), _flags(scale_inv_n, tensor_cores)),
               "fb_fft_server_prepare")

    def submit_ptr(self, dims, in_ptr: int, out_ptr: int, tag: int, direction: int = FORWARD, batch: int = 1,
                   scale_inv_n: bool = False, host_io: bool = False, tensor_cores: bool = False) -> None:
        """Queue one transform on raw pointers (device, or host when host_io)."""
        key = dims if isinstance(dims, tuple) else None
        rc = self._shape_args.get(key) if key is not None else None
        if rc is None:
            rc = self._dims(dims)
            if key is not None:
                self._shape_args[key] = rc
        r, cd = rc
        _check(lib.fb_fft_server_submit(self._h, r, cd, int(batch), _flags(scale_inv_n, tensor_cores),
                                        int(direction), _vp(in_ptr), _vp(out_ptr), 1 if host_io else 0, int(tag)),
               "fb_fft_server_submit")

    @staticmethod
    def requests(items) -> "ctypes.Array":
        """Pack (dims, in_ptr, out_ptr, tag, direction[, batch, scale_inv_n,
        host_io, tensor_cores]) tuples into a request array for submit_many."""
        arr = (ServerRequest * len(items))()
        for k, it in enumerate(items):
            dims, in_ptr, out_ptr, tag, direction = it[:5]
            batch, scale, host_io, tc = (tuple(it[5:]) + (1, False, False, False)[len(it) - 5:])[:4]
            dims = [int(d) for d in (dims if hasattr(dims, "__len__") else [dims])]
            q = arr[k]
            q.rank = len(dims)
            for e, d in enumerate(dims):
                q.dims[e] = d
            q.batch, q.tag, q.in_ptr, q.out_ptr = int(batch), int(tag), int(in_ptr), int(out_ptr)
            q.flags, q.direction, q.host_io = _flags(scale, tc), int(direction), 1 if host_io else 0
        return arr

    def submit_many(self, reqs, first: int = 0, count: int | None = None) -> list[int]:
        """Queue reqs[first:first+count] (an array from ``requests``) in one
        call; returns each request's status (0 = queued)."""
        n = len(reqs) - first if count is None else int(count)
        if first < 0 or n < 0 or first + n > len(reqs):
            raise ValueError("request range out of bounds")
        st = (_int * max(1, n))()
        base = ctypes.cast(ctypes.byref(reqs, first * ctypes.sizeof(ServerRequest)), ctypes.POINTER(ServerRequest))
        _check(lib.fb_fft_server_submit_many(self._h, base, n, st), "fb_fft_server_submit_many")
        return list(st[:n])

    def poll(self, wait: bool = False, device_times: bool = False) -> list[tuple]:
        """Finished requests as (tag, status, slot, t_submit, t_admit, t_done),
        plus (t_dev_start, t_dev_end) with ``device_times``."""
        out = []
        while True:
            n = _int(0)
            _check(lib.fb_fft_server_poll(self._h, 1 if wait else 0, self._buf, len(self._buf), ctypes.byref(n)),
                   "fb_fft_server_poll")
            for i in range(n.value):
                d = self._buf[i]
                rec = (d.tag, d.status, d.slot, d.t_submit, d.t_admit, d.t_done)
                out.append(rec + (d.t_dev_start, d.t_dev_end) if device_times else rec)
            if n.value < len(self._buf):
                return out
            wait = False

    def wait(self, until_s: float) -> None:
        """Spin until a request finishes, nothing runs, or the server clock
        reaches ``until_s`` (see fb_fft_server_wait)."""
        _check(lib.fb_fft_server_wait(self._h, float(until_s)), "fb_fft_server_wait")

    def drain(self) -> None:
        _check(lib.fb_fft_server_drain(self._h), "fb_fft_server_drain")

    def cancel(self, tag: int) -> None:
        _check(lib.fb_fft_server_cancel(self._h, int(tag)), "fb_fft_server_cancel")

    def clock(self) -> float:
        return lib.fb_fft_server_clock(self._h)

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib.fb_fft_server_stats_get(self._h, ctypes.byref(st)), "fb_fft_server_stats_get")
        return st.as_dict()
