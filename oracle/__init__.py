"""Oracle: a plain FP64 CPU discrete Fourier transform.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this package.  The product library
never imports, links or calls it, and it shares no code with the CUDA path.

Definition followed (Sec. 3.3 and Sec. 5.1(a) of the paper name the Fourier
transform function block; the paper gives no formula, so the textbook complex
DFT is used):  X[k] = c * sum_n x[n] exp(s*2*pi*i*n*k/N), s = -1 forward,
s = +1 inverse, c = 1 or 1/N; multi-dimensional transforms apply it along every
axis; batches are independent.

The arithmetic lives in ``oracle_fft.c`` (plain C, compiled with gcc, no
fast-math, no FMA contraction); this module marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle_fft.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_fft.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle_fft.c`` into ``liboracle_fft.so`` beside it."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ll = ctypes.c_longlong
            lib.oracle_dft_naive.argtypes = [dp, dp, ll, ctypes.c_int]
            lib.oracle_dft_naive.restype = ctypes.c_int
            lib.oracle_fft_1d.argtypes = [dp, dp, ll, ctypes.c_int]
            lib.oracle_fft_1d.restype = ctypes.c_int
            lib.oracle_fft_nd.argtypes = [dp, dp, ctypes.c_int, ctypes.POINTER(ll), ll,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.oracle_fft_nd.restype = ctypes.c_int
            lib.oracle_twiddle.argtypes = [ll, ll, ctypes.c_int, dp, dp]
            lib.oracle_twiddle.restype = None
            _lib = lib
    return _lib


def _c128(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x), dtype=np.complex128)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def dft_naive(x, sign: int = -1) -> np.ndarray:
    """O(N^2) DFT of a 1-D sequence, summed in long double (tiny N only)."""
    x = _c128(x).reshape(-1)
    out = np.empty_like(x)
    rc = _load().oracle_dft_naive(_dptr(x), _dptr(out), x.size, int(sign))
    if rc != 0:
        raise ValueError(f"oracle_dft_naive failed ({rc})")
    return out


def fft1d(x, sign: int = -1) -> np.ndarray:
    """Recursive mixed-radix FFT of one 1-D sequence (any length >= 1)."""
    x = _c128(x).reshape(-1)
    out = np.empty_like(x)
    rc = _load().oracle_fft_1d(_dptr(x), _dptr(out), x.size, int(sign))
    if rc != 0:
        raise ValueError(f"oracle_fft_1d failed ({rc})")
    return out


def fft(x, dims, sign: int = -1, scale_inv_n: bool = False, threads: int = 1) -> np.ndarray:
    """Batched multi-dimensional DFT.

    ``x`` holds ``batch * prod(dims)`` complex values (any shape, C order);
    ``dims`` are the transform dims, row-major, last fastest.  Returns a
    complex128 array of the same shape.  ``scale_inv_n`` multiplies by
    1/prod(dims).  ``threads`` worker threads split each axis' lines.
    """
    a = _c128(x)
    dims = [int(d) for d in dims]
    n = int(np.prod(dims))
    if n <= 0 or a.size % n:
        raise ValueError("size is not a multiple of prod(dims)")
    batch = a.size // n
    out = np.empty_like(a)
    cd = (ctypes.c_longlong * len(dims))(*dims)
    rc = _load().oracle_fft_nd(_dptr(a), _dptr(out), len(dims), cd, batch, int(sign),
                               1 if scale_inv_n else 0, int(threads))
    if rc != 0:
        raise ValueError(f"oracle_fft_nd failed ({rc})")
    return out


def twiddle(m: int, d: int, sign: int = -1) -> complex:
    """exp(sign*2*pi*i*m/d) evaluated in long double and rounded to double."""
    re, im = ctypes.c_double(), ctypes.c_double()
    _load().oracle_twiddle(int(m), int(d), int(sign), ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def rel_l2(y, ref) -> np.ndarray:
    """Per-transform relative L2 error ||y - ref||_2 / ||ref||_2 in FP64, the
    error measure of every parity check.

    ``y`` and ``ref`` have the same shape: 1-D (one transform) or 2-D with one
    transform per row (``(batch, n)``; reshape multi-dimensional transforms to
    that first).  Other shapes raise ValueError, so a volume passed unreshaped
    cannot be split into per-row errors by accident.  A row whose reference
    is all zero reports the absolute norm ||y||_2.  Returns a float64 array
    of one error per transform.
    """
    y = np.asarray(y, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    if y.shape != ref.shape:
        raise ValueError(f"rel_l2: shapes differ {y.shape} vs {ref.shape}")
    if y.ndim not in (1, 2):
        raise ValueError(f"rel_l2: want 1-D or (batch, n) arrays, got shape {y.shape}")
    y2 = y.reshape(1, -1) if y.ndim == 1 else y
    r2 = ref.reshape(y2.shape)
    num = np.sqrt(np.sum(np.abs(y2 - r2) ** 2, axis=1))
    den = np.sqrt(np.sum(np.abs(r2) ** 2, axis=1))
    den = np.where(den == 0, 1.0, den)
    return num / den
