"""Pins for the FP64 oracle against facts fixed by mathematics, not by itself.

Each check is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a wrong index or stride, a transposed axis) fails at least one of
them; ``test_planted_mistakes_are_caught`` proves that for a set of such slips
by compiling mutated copies of the oracle source.
"""
import cmath
import ctypes
import json
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2004_09883_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dft_textbook.json")
TOL = 1e-13  # FP64 oracle vs exact / long-double values (relative L2)


def _eval(expr: str) -> complex:
    env = {"sqrt": math.sqrt, "pi": math.pi, "cos": math.cos, "sin": math.sin}
    return complex(eval(expr, {"__builtins__": {}}, env))


def _rel(a, b) -> float:
    a = np.asarray(a, dtype=np.complex128).ravel()
    b = np.asarray(b, dtype=np.complex128).ravel()
    d = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (d if d else 1.0))


def _rng_c128(n, seed):
    return inputs.uniform_c64((n,), seed).astype(np.complex128)


# --------------------------------------------------------------------------
# Golden, hand-derived values
# --------------------------------------------------------------------------
def _golden_cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_golden_textbook_values(case):
    x = np.array([_eval(v) for v in case["x"]])
    want = np.array([_eval(v) for v in case["X"]])
    dims = case["dims"]
    got = oracle.fft(x, dims, sign=case["sign"])
    assert np.max(np.abs(got - want)) < 1e-14 * len(x)
    if len(dims) == 1:
        got_naive = oracle.dft_naive(x, case["sign"])
        assert np.max(np.abs(got_naive - want)) < 1e-14 * len(x)


# --------------------------------------------------------------------------
# The naive DFT itself against closed forms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 12, 16, 17, 30, 64])
@pytest.mark.parametrize("sign", [-1, 1])
def test_naive_closed_forms(n, sign):
    # impulse -> all ones
    x = np.zeros(n, complex)
    x[0] = 1
    assert np.max(np.abs(oracle.dft_naive(x, sign) - 1)) < 1e-15
    # delayed impulse -> exp(s*2*pi*i*k*n0/N)
    n0 = (n * 2) // 3
    x = np.zeros(n, complex)
    x[n0] = 1
    k = np.arange(n)
    want = np.exp(sign * 2j * np.pi * ((k * n0) % n) / n)
    assert np.max(np.abs(oracle.dft_naive(x, sign) - want)) < 1e-15
    # single tone exp(-s*2*pi*i*m*n/N) -> N * delta[k - m]
    m = (n * 3) // 5
    x = np.exp(-sign * 2j * np.pi * ((k * m) % n) / n)
    want = np.zeros(n, complex)
    want[m] = n
    assert np.max(np.abs(oracle.dft_naive(x, sign) - want)) < 1e-13 * n
    # constant -> N * delta[k]
    want = np.zeros(n, complex)
    want[0] = n
    assert np.max(np.abs(oracle.dft_naive(np.ones(n), sign) - want)) < 1e-13 * n


# --------------------------------------------------------------------------
# Fast oracle against the naive sum (brute force on small sizes)
# --------------------------------------------------------------------------
SMALL = list(range(1, 65)) + [81, 96, 97, 100, 125, 127, 128, 150, 243, 250, 251, 256,
                              360, 384, 486, 500, 509, 512]


@pytest.mark.parametrize("n", SMALL)
def test_fft1d_matches_naive(n):
    x = _rng_c128(n, 17 + n)
    for sign in (-1, 1):
        assert _rel(oracle.fft1d(x, sign), oracle.dft_naive(x, sign)) < TOL


def test_fft1d_matches_naive_random_lengths():
    rng = np.random.default_rng(5)
    for n in rng.integers(513, 2049, size=4):
        x = _rng_c128(int(n), int(n))
        assert _rel(oracle.fft1d(x, -1), oracle.dft_naive(x, -1)) < TOL


# --------------------------------------------------------------------------
# Independent library routine (numpy pocketfft, FP64) as a cross-check
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1000, 1024, 1536, 3125, 4096, 6561, 11025, 65536])
def test_fft1d_vs_numpy(n):
    x = _rng_c128(n, n)
    assert _rel(oracle.fft1d(x, -1), np.fft.fft(x)) < TOL
    assert _rel(oracle.fft1d(x, 1), np.fft.ifft(x) * n) < TOL


@pytest.mark.parametrize("dims,batch", [([4, 6], 3), ([16, 5, 9], 2), ([8, 8, 8], 1),
                                         ([3, 1, 7], 2), ([1], 4), ([128], 5)])
def test_fft_nd_vs_numpy(dims, batch):
    n = int(np.prod(dims))
    x = _rng_c128(n * batch, n + batch).reshape([batch] + dims)
    axes = tuple(range(1, len(dims) + 1))
    assert _rel(oracle.fft(x, dims, -1), np.fft.fftn(x, axes=axes)) < TOL
    assert _rel(oracle.fft(x, dims, 1, scale_inv_n=True), np.fft.ifftn(x, axes=axes)) < TOL


def test_threads_do_not_change_result():
    dims = [16, 12, 10]
    x = _rng_c128(2 * 1920, 3).reshape(2, *dims)
    a = oracle.fft(x, dims, -1, threads=1)
    b = oracle.fft(x, dims, -1, threads=7)
    assert np.array_equal(a, b)


# --------------------------------------------------------------------------
# Identities of the transform
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [60, 256, 243, 625, 1000, 4096])
def test_parseval(n):
    x = _rng_c128(n, n + 1)
    X = oracle.fft1d(x, -1)
    lhs = np.sum(np.abs(X) ** 2)
    rhs = n * np.sum(np.abs(x) ** 2)
    assert abs(lhs - rhs) / rhs < TOL


@pytest.mark.parametrize("n", [48, 125, 2048])
def test_linearity(n):
    x, y = _rng_c128(n, 1), _rng_c128(n, 2)
    a, b = 0.3 - 1.7j, -2.2 + 0.4j
    lhs = oracle.fft1d(a * x + b * y, -1)
    rhs = a * oracle.fft1d(x, -1) + b * oracle.fft1d(y, -1)
    assert _rel(lhs, rhs) < TOL


@pytest.mark.parametrize("dims", [[4096], [30, 32], [16, 16, 8], [5, 27, 8]])
def test_round_trip(dims):
    n = int(np.prod(dims))
    x = _rng_c128(n, 9).reshape(dims)
    y = oracle.fft(oracle.fft(x, dims, -1), dims, 1, scale_inv_n=True)
    assert _rel(y, x) < 1e-14


@pytest.mark.parametrize("n", [36, 256, 400])
def test_shift_theorem(n):
    x = _rng_c128(n, 4)
    n0 = n // 3 + 1
    k = np.arange(n)
    for sign in (-1, 1):
        lhs = oracle.fft1d(np.roll(x, n0), sign)
        rhs = np.exp(sign * 2j * np.pi * ((k * n0) % n) / n) * oracle.fft1d(x, sign)
        assert _rel(lhs, rhs) < TOL


@pytest.mark.parametrize("n", [64, 90, 1024])
def test_real_input_symmetry(n):
    x = inputs.uniform_c64((n,), 8).real.astype(np.float64).astype(np.complex128)
    X = oracle.fft1d(x, -1)
    k = np.arange(1, n)
    assert np.max(np.abs(X[n - k] - np.conj(X[k]))) < 1e-12 * n


def test_tone_closed_form_large():
    n, m = 1 << 16, 12345
    k = np.arange(n)
    x = np.exp(2j * np.pi * ((k * m) % n) / n)  # exp(-s*...) with s = -1
    X = oracle.fft1d(x, -1)
    want = np.zeros(n, complex)
    want[m] = n
    assert np.max(np.abs(X - want)) < 1e-9 * n


def test_separability_axis_order():
    """3-D transform == 1-D transforms along each axis in another order."""
    dims = [6, 10, 8]
    x = _rng_c128(480, 11).reshape(dims)
    want = oracle.fft(x, dims, -1)
    y = x.copy()
    for ax in (0, 1, 2):  # the oracle itself goes last axis first
        moved = np.moveaxis(y, ax, -1)
        shp = moved.shape
        moved = oracle.fft(moved.reshape(-1, shp[-1]), [shp[-1]], -1).reshape(shp)
        y = np.moveaxis(moved, -1, ax)
    assert _rel(y, want) < TOL


def test_batch_items_are_independent():
    dims = [12, 20]
    x = _rng_c128(3 * 240, 21).reshape(3, *dims)
    whole = oracle.fft(x, dims, -1)
    for b in range(3):
        assert np.array_equal(whole[b], oracle.fft(x[b], dims, -1))


def test_twiddle_closed_forms():
    assert oracle.twiddle(0, 7) == 1
    assert abs(oracle.twiddle(4, 16) - (-1j)) < 1e-19
    assert abs(oracle.twiddle(8, 16) - (-1)) < 1e-19
    assert abs(oracle.twiddle(1, 8) - (math.sqrt(0.5) - 1j * math.sqrt(0.5))) < 2e-16
    assert abs(oracle.twiddle(1, 8, 1) - (math.sqrt(0.5) + 1j * math.sqrt(0.5))) < 2e-16
    assert abs(oracle.twiddle(1000003, 1000000) - oracle.twiddle(3, 1000000)) == 0
    for m, d in [(1, 3), (2, 5), (7, 1 << 20), (999, 1000)]:
        r = m if 2 * m <= d else m - d  # keep the library's angle small
        assert abs(oracle.twiddle(m, d) - cmath.exp(-2j * math.pi * r / d)) < 4e-16


def test_rejects_bad_arguments():
    with pytest.raises(ValueError):
        oracle.fft(np.zeros(10, complex), [3])
    with pytest.raises(ValueError):
        oracle.fft1d(np.zeros(4, complex), sign=0)


# --------------------------------------------------------------------------
# Planted mistakes: mutated copies of the oracle must fail the pins above
# --------------------------------------------------------------------------
MUTATIONS = {
    "combine_sign": ("ai += y.re * w.im + y.im * w.re;", "ai -= y.re * w.im + y.im * w.re;"),
    "dropped_term": ("for (long long q = 0; q < p; ++q) {\n            const cplx w = c->tab[((q * k) % N) * tstep];\n            const cplx y",
                     "for (long long q = 1; q < p; ++q) {\n            const cplx w = c->tab[((q * k) % N) * tstep];\n            const cplx y"),
    "twiddle_index": ("c->tab[((q * k) % N) * tstep];\n            const cplx y", "c->tab[((q * km) % N) * tstep];\n            const cplx y"),
    "sub_stride": ("ct_rec(c, x + q * stride, stride * p, X + q * M, M, work);",
                   "ct_rec(c, x + q * M * stride, stride, X + q * M, M, work);"),
    "prime_conj": ("ai += v.re * w.im + v.im * w.re;", "ai += v.im * w.re - v.re * w.im;"),
    "axis_stride": ("line[n] = base[n * j->S];", "line[n] = base[n];"),
    "table_sign": ("w.im = (double)((long double)sign * sinl(ang));", "w.im = (double)sinl(ang);"),
    "scale_missing": ("data[i].re *= inv;\n            data[i].im *= inv;", "data[i].re *= inv;"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle_fft.c")).read()
    assert src.count(old) >= 1, f"mutation {name} no longer applies"
    mut = src.replace(old, new, 1)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(mut)
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-o", str(so), str(c), "-lm", "-lpthread"],
                   check=True)
    lib = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    ll = ctypes.c_longlong
    lib.oracle_fft_nd.argtypes = [dp, dp, ctypes.c_int, ctypes.POINTER(ll), ll,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_int]
    return lib


def _mutant_passes_pins(lib) -> bool:
    dp = ctypes.POINTER(ctypes.c_double)

    def run(x, dims, sign, scale=0):
        x = np.ascontiguousarray(x, dtype=np.complex128)
        out = np.empty_like(x)
        cd = (ctypes.c_longlong * len(dims))(*dims)
        lib.oracle_fft_nd(x.ctypes.data_as(dp), out.ctypes.data_as(dp), len(dims), cd,
                          x.size // int(np.prod(dims)), sign, scale, 1)
        return out

    for case in _golden_cases():
        x = np.array([_eval(v) for v in case["x"]])
        want = np.array([_eval(v) for v in case["X"]])
        if np.max(np.abs(run(x, case["dims"], case["sign"]) - want)) > 1e-12:
            return False
    for n in (12, 30, 49, 64, 97):
        x = _rng_c128(n, n)
        for s in (-1, 1):
            if _rel(run(x, [n], s), oracle.dft_naive(x, s)) > TOL:
                return False
    x = _rng_c128(240, 1).reshape(2, 8, 15)
    if _rel(run(x, [8, 15], 1, 1), np.fft.ifftn(x, axes=(1, 2))) > TOL:
        return False
    return True


def test_unmutated_source_passes_the_same_pins(tmp_path):
    lib = _build_mutant(tmp_path, "identity", "int oracle_fft_1d", "int oracle_fft_1d")
    assert _mutant_passes_pins(lib)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistakes_are_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    lib = _build_mutant(tmp_path, name, old, new)
    assert not _mutant_passes_pins(lib), f"mutation {name} slipped through the pins"
