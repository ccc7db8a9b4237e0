"""Pins of oracle.rel_l2, the error measure every parity check decides by.

The values below are worked out by hand (no call to a norm routine), so a
slip in rel_l2 -- a norm over the wrong axis, a missing square root or
modulus, the ratio upside down, the denominator taken from y -- fails one of
them.  test_planted_mistakes_in_rel_l2_are_caught makes each of those slips in
a copy of rel_l2's own source and checks that the pins reject it.
"""
import inspect
import textwrap

import numpy as np
import pytest

import oracle


def _pins(f):
    """Run every pin against the candidate f; raises AssertionError on the
    first one it fails."""
    # 1. ref scaled by (1 + 1e-3): error 1e-3 for any nonzero ref
    ref = np.array([[1 + 2j, -3 + 0.5j, 0.25 - 1j], [2, 0, -1j]], dtype=np.complex128)
    got = f(ref * (1 + 1e-3), ref)
    assert got.shape == (2,), got.shape
    assert np.allclose(got, 1e-3, rtol=1e-9, atol=0), got
    # 2. hand-computed: ref = [3+4i, 0] (norm 5), y differs by 1 in the second slot -> 1/5
    got = f(np.array([3 + 4j, 1]), np.array([3 + 4j, 0]))
    assert got.shape == (1,) and abs(got[0] - 0.2) < 1e-15, got
    # 3. a purely imaginary difference: ref = [1, 0, 0, 0], y = [1, i, 0, 0] -> 1
    got = f(np.array([1, 1j, 0, 0]), np.array([1, 0, 0, 0]))
    assert abs(got[0] - 1.0) < 1e-15, got
    # 4. a complex difference 3 - 4i against ref norm 10 (6 + 8i) -> 5/10
    got = f(np.array([9 + 4j]), np.array([6 + 8j]))
    assert abs(got[0] - 0.5) < 1e-15, got
    # 5. all-zero reference row: the absolute norm of y, here |3| + |4i| -> 5
    got = f(np.array([[3, 4j], [1, 1]]), np.array([[0, 0], [1, 1]]))
    assert np.allclose(got, [5.0, 0.0], rtol=0, atol=1e-15), got
    # 6. rows are independent: errors 0.1, 0 and 2 in a (3, 4) batch (not square,
    #    so a norm down the columns has the wrong length)
    ref = np.array([[2, 0, 0, 0], [1, 1, 1, 1], [0, 0, 0, 0.5j]], dtype=np.complex128)
    y = ref.copy()
    y[0, 3] += 0.2          # |d| = 0.2, |ref| = 2   -> 0.1
    y[2, 1] += 1.0          # |d| = 1,   |ref| = 0.5 -> 2
    got = f(y, ref)
    assert got.shape == (3,) and np.allclose(got, [0.1, 0.0, 2.0], rtol=1e-14, atol=1e-15), got
    # 7. a 1-D transform is one result; a (1, n) batch gives the same number
    a, b = np.array([1, 2, 3, 4j]), np.array([1, 2, 3, 5j])
    assert np.array_equal(f(a, b), f(a.reshape(1, -1), b.reshape(1, -1)))
    # 8. a (batch, n) view of a batch of 2-D transforms: one error per transform,
    #    equal to the error of each transform on its own
    rng = np.random.default_rng(3)
    r = rng.standard_normal((3, 4, 5)) + 1j * rng.standard_normal((3, 4, 5))
    e = r + 1e-2 * (rng.standard_normal((3, 4, 5)) + 1j * rng.standard_normal((3, 4, 5)))
    whole = f(e.reshape(3, -1), r.reshape(3, -1))
    each = [f(e[i].reshape(-1), r[i].reshape(-1))[0] for i in range(3)]
    assert whole.shape == (3,) and np.allclose(whole, each, rtol=1e-15, atol=0)
    # and by hand for item 0: sqrt(sum |e-r|^2 / sum |r|^2), the sums written out
    num = sum(abs(complex(v)) ** 2 for v in (e[0] - r[0]).reshape(-1))
    den = sum(abs(complex(v)) ** 2 for v in r[0].reshape(-1))
    assert abs(whole[0] - (num / den) ** 0.5) < 1e-14


def test_rel_l2_pins():
    _pins(oracle.rel_l2)


def test_rel_l2_rejects_ambiguous_shapes():
    vol = np.ones((4, 4, 2), dtype=np.complex128)
    with pytest.raises(ValueError):
        oracle.rel_l2(vol, vol)  # a volume must be reshaped to (batch, n) first
    with pytest.raises(ValueError):
        oracle.rel_l2(np.ones((2, 3)), np.ones((3, 2)))
    with pytest.raises(ValueError):
        oracle.rel_l2(np.ones(6), np.ones((1, 6)))


MUTATIONS = [
    ("norm down the wrong axis", "axis=1", "axis=0"),
    ("no square root", "num = np.sqrt(np.sum(np.abs(y2 - r2) ** 2, axis=1))",
     "num = np.sum(np.abs(y2 - r2) ** 2, axis=1)"),
    ("no square root in either norm", "np.sqrt(", "("),
    ("ratio upside down", "return num / den", "return den / num"),
    ("modulus dropped", "np.abs(y2 - r2) ** 2", "(y2 - r2) ** 2"),
    ("denominator from y", "np.abs(r2) ** 2", "np.abs(y2) ** 2"),
    ("zero-reference rule dropped", "den = np.where(den == 0, 1.0, den)", "pass"),
    ("first row only", "y2 = y.reshape(1, -1) if y.ndim == 1 else y", "y2 = y.reshape(1, -1)[:, :y.shape[-1]]"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistakes_in_rel_l2_are_caught(name, old, new):
    src = textwrap.dedent(inspect.getsource(oracle.rel_l2))
    assert old in src, f"mutation site for '{name}' not found"
    ns = {"np": np}
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    mutant = ns["rel_l2"]
    with np.errstate(all="ignore"):
        with pytest.raises((AssertionError, ValueError)):
            _pins(mutant)
