"""Pins of the oracle's axis reductions (x.sum(axis=a) and friends, the
write-conflict resolution of Sec. 2.3 with one result per remaining index)
against closed forms, brute-force loops written here, permutation
invariants, NumPy's own reductions, and the exactly rounded sum."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import Program


def test_closed_form_row_and_column_sums():
    m, n = 37, 45
    A = np.tile(np.arange(1, n + 1, dtype=np.float64), (m, 1))      # A[i, j] = j + 1
    s, fs, ab = oracle.reduce_axis("sum", A, 1)
    assert np.all(s == n * (n + 1) / 2) and np.all(fs == s) and np.all(ab == s)
    B = np.tile(np.arange(1, m + 1, dtype=np.float64)[:, None], (1, n))  # B[i, j] = i + 1
    s0, _, _ = oracle.reduce_axis("sum", B, 0)
    assert s0.shape == (n,) and np.all(s0 == m * (m + 1) / 2)
    s_neg, _, _ = oracle.reduce_axis("sum", B, -2)
    assert np.array_equal(s_neg, s0)


@pytest.mark.parametrize("shape", [(2, 3, 4), (1, 5, 1), (4, 1, 3), (3,)])
def test_brute_force_every_axis(shape):
    rng = np.random.default_rng(3)
    x = rng.normal(size=shape)
    for axis in range(len(shape)):
        s, fs, ab = oracle.reduce_axis("sum", x, axis)
        mx = oracle.reduce_axis("max", x, axis)
        mn = oracle.reduce_axis("min", x, axis)
        ma = oracle.reduce_axis("maxabs", x, axis)
        oshape = tuple(d for k, d in enumerate(shape) if k != axis)
        assert s.shape == oshape
        for idx in itertools.product(*[range(d) for d in oshape]):
            acc, best, least, big, mag = 0.0, -np.inf, np.inf, 0.0, 0.0
            for r in range(shape[axis]):
                full = list(idx)
                full.insert(axis, r)
                v = float(x[tuple(full)])
                acc += v
                mag += abs(v)
                best = v if v > best else best
                least = v if v < least else least
                big = abs(v) if abs(v) > big else big
            assert s[idx] == acc and ab[idx] == mag
            assert mx[idx] == best and mn[idx] == least and ma[idx] == big


def test_permutation_columns_and_against_numpy():
    rng = np.random.default_rng(4)
    R, C = 50, 30
    P = np.stack([rng.permutation(R) for _ in range(C)], axis=1).astype(np.float64)
    assert np.all(oracle.reduce_axis("max", P, 0) == R - 1)
    assert np.all(oracle.reduce_axis("min", P, 0) == 0)
    assert np.all(oracle.reduce_axis("maxabs", -P, 0) == R - 1)
    s, fs, _ = oracle.reduce_axis("sum", P, 0)
    assert np.all(s == R * (R - 1) / 2) and np.all(fs == s)
    # random data: NumPy's (pairwise) sums agree to rounding, maxima exactly
    x = rng.normal(size=(64, 200))
    for axis in (0, 1):
        s, fs, ab = oracle.reduce_axis("sum", x, axis)
        ref = np.sum(x, axis=axis)
        assert np.all(np.abs(s - ref) <= 1e-13 * ab)
        assert np.all(np.abs(fs - ref) <= 1e-13 * ab)
        assert np.array_equal(oracle.reduce_axis("max", x, axis), np.max(x, axis=axis))
        assert np.array_equal(oracle.reduce_axis("min", x, axis), np.min(x, axis=axis))


def test_exact_sum_per_output_and_nan():
    # each column cancels to 1 exactly; the sequential sum loses it
    x = np.array([[1e16, 2.0], [1.0, 3.0], [-1e16, 4.0]])
    s, fs, _ = oracle.reduce_axis("sum", x, 0)
    assert fs[0] == 1.0 and s[0] == 0.0 and fs[1] == 9.0
    y = np.ones((4, 3))
    y[2, 1] = np.nan
    mx = oracle.reduce_axis("max", y, 0)
    assert np.isnan(mx[1]) and mx[0] == 1.0 and mx[2] == 1.0
    s, _, _ = oracle.reduce_axis("sum", y, 0)
    assert np.isnan(s[1]) and s[0] == 4.0


def test_integer_wrap_along_axis():
    x = np.full((3, 4), 2 ** 30, dtype=np.int64)
    got = oracle.reduce_axis_i("sum", 32, x, 0)
    ref = np.sum(x.astype(np.int32), axis=0, dtype=np.int32)
    assert np.array_equal(got, ref.astype(np.int64))
    assert np.all(oracle.reduce_axis_i("max", 64, np.arange(12).reshape(3, 4), 1) == [3, 7, 11])


def test_empty_axis_and_program_form():
    x = np.zeros((0, 5))
    s, fs, ab = oracle.reduce_axis("sum", x, 0)
    assert s.shape == (5,) and np.all(s == 0) and np.all(fs == 0)
    with pytest.raises(Exception):
        oracle.reduce_axis("max", x, 0)
    p = Program()
    v = p.input("f64", (3, 4))
    r = p.output(p.reduce(p.map("square", [v]), "sum", axis=1))
    a = np.arange(12, dtype=np.float64).reshape(3, 4)
    vals, extra = oracle.run(p, [a], detail=True)
    assert vals[r].shape == (3,)
    assert np.array_equal(vals[r], (a * a).sum(axis=1))
    assert np.array_equal(extra[r]["fsum"], vals[r])
