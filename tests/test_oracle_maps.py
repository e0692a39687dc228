"""Pins for the oracle's elementwise maps (Sec. 2.3, Table 1).

Nothing here re-calls the oracle's own formula: values come from a
hand-derived golden table, algebraic identities, an extended-precision
evaluation, Python's arbitrary-precision integers, and special cases of the
fused map+reduce workload that reduce to simpler closed forms.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "maps_f64.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        op, a, b, imm, exp = line.split()
        approx = exp.startswith("~")
        rows.append((op, float(a), None if b == "-" else float(b), float(imm),
                     float(exp.lstrip("~")), approx))
    return rows


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: r[0])
def test_golden_values(row):
    op, a, b, imm, expected, approx = row
    y = oracle.map_f(op, np.array([a]), None if b is None else np.array([b]), imm)[0]
    if approx:
        assert abs(y - expected) <= 2.0 * math.ulp(expected) + 1e-300
    else:
        assert y == expected


def test_every_op_has_a_golden_row():
    ops = {r[0] for r in _golden_rows()}
    assert ops == set(oracle.OPS)


def test_identities():
    rng = np.random.default_rng(5)
    x = rng.uniform(-3, 3, 4096)
    z = rng.uniform(-3, 3, 4096)
    e = lambda v: oracle.map_f("exp", v)
    # exp(x + z) = exp(x) exp(z)
    lhs = e(oracle.map_f("add", x, z))
    rhs = oracle.map_f("mul", e(x), e(z))
    assert np.max(np.abs(lhs - rhs) / rhs) < 1e-14
    # sin^2 + cos^2 = 1
    s = oracle.map_f("sin", x)
    c = oracle.map_f("cos", x)
    assert np.max(np.abs(oracle.map_f("add", oracle.map_f("square", s),
                                      oracle.map_f("square", c)) - 1.0)) < 1e-15
    # sin(x) = cos(pi/2 - x)
    assert np.max(np.abs(s - oracle.map_f("cos", oracle.map_f("rsub_s", x, imm=math.pi / 2)))) < 1e-15
    # tanh(x) = (e^{2x} - 1) / (e^{2x} + 1)
    e2 = e(oracle.map_f("mul_s", x, imm=2.0))
    t = oracle.map_f("div", oracle.map_f("sub_s", e2, imm=1.0), oracle.map_f("add_s", e2, imm=1.0))
    assert np.max(np.abs(oracle.map_f("tanh", x) - t)) < 1e-14
    # sqrt(x^2) = |x| exactly for these magnitudes (correctly rounded sqrt of an exact square
    # is not guaranteed, so allow one ulp)
    r = oracle.map_f("sqrt", oracle.map_f("square", x))
    assert np.all(np.abs(r - np.abs(x)) <= np.spacing(np.abs(x)))
    # neg/abs/sub relations
    assert np.array_equal(oracle.map_f("sub", x, z), -oracle.map_f("sub", z, x))
    assert np.array_equal(oracle.map_f("neg", x), oracle.map_f("rsub_s", x, imm=0.0) * 1.0 + 0.0)
    assert np.array_equal(oracle.map_f("max", x, z), -oracle.map_f("min", -x, -z))


def test_against_extended_precision():
    """Oracle libm results within 2 ulp of a long-double evaluation."""
    if np.finfo(np.longdouble).eps >= np.finfo(np.float64).eps:
        pytest.skip("no extended long double on this host")
    rng = np.random.default_rng(11)
    x = rng.normal(0, 2, 2000)
    xl = x.astype(np.longdouble)
    for op, f in [("exp", np.exp), ("sin", np.sin), ("cos", np.cos), ("tanh", np.tanh)]:
        ref = f(xl)
        got = oracle.map_f(op, x).astype(np.longdouble)
        err = np.abs(got - ref) / np.maximum(np.abs(ref), np.longdouble(1e-300))
        assert float(np.max(err)) < 4.5e-16, op  # within 2 ulp


def test_nan_propagation_in_max_min():
    a = np.array([np.nan, 1.0, 2.0])
    b = np.array([0.0, np.nan, 1.0])
    assert np.isnan(oracle.map_f("max", a, b)[:2]).all()
    assert np.isnan(oracle.map_f("min", a, b)[:2]).all()
    assert oracle.map_f("max", a, b)[2] == 2.0


def _cfg2_map(x, a, b):
    """y = exp(a*x + b) * sin(x) - 0.5*x*x through single oracle ops."""
    ax = oracle.map_f("mul", a, x)
    t = oracle.map_f("add", ax, b)
    e = oracle.map_f("exp", t)
    s = oracle.map_f("sin", x)
    p = oracle.map_f("mul", e, s)
    xx = oracle.map_f("mul", x, x)
    h = oracle.map_f("mul_s", xx, imm=0.5)
    return oracle.map_f("sub", p, h)


def test_fused_workload_special_cases():
    rng = np.random.default_rng(3)
    a = rng.normal(size=512)
    b = rng.normal(size=512)
    # x = 0  =>  y = 0 exactly
    assert np.all(_cfg2_map(np.zeros(512), a, b) == 0.0)
    # a = b = 0  =>  y = sin x - x^2/2
    x = rng.normal(size=512)
    y = _cfg2_map(x, np.zeros(512), np.zeros(512))
    assert np.max(np.abs(y - (np.sin(x.astype(np.longdouble)) - x.astype(np.longdouble) ** 2 / 2)
                         .astype(np.float64))) < 1e-15


@pytest.mark.parametrize("bits", [32, 64])
def test_integer_maps_wrap_like_python_ints(bits):
    rng = np.random.default_rng(bits)
    lo, hi = -(1 << (bits - 1)), (1 << (bits - 1))
    a = rng.integers(lo, hi, 300, dtype=np.int64)
    b = rng.integers(lo, hi, 300, dtype=np.int64)
    a[:4] = [lo, hi - 1, 0, -1]
    b[:4] = [-1, hi - 1, lo, lo]
    imm = 123456789 if bits == 32 else (1 << 40) + 7

    def wrap(v):
        v &= (1 << bits) - 1
        return v - (1 << bits) if v >= (1 << (bits - 1)) else v

    ref = {
        "neg": lambda p, q: -p, "abs": lambda p, q: abs(p), "square": lambda p, q: p * p,
        "add": lambda p, q: p + q, "sub": lambda p, q: p - q, "mul": lambda p, q: p * q,
        "max": lambda p, q: max(p, q), "min": lambda p, q: min(p, q),
        "add_s": lambda p, q: p + imm, "mul_s": lambda p, q: p * imm,
        "sub_s": lambda p, q: p - imm, "rsub_s": lambda p, q: imm - p,
    }
    for op, f in ref.items():
        got = oracle.map_i(op, bits, a, b if op in oracle.BINARY else None, imm)
        exp = [wrap(f(int(p), int(q))) for p, q in zip(a, b)]
        assert got.tolist() == exp, op


def test_integer_rejects_float_only_ops():
    with pytest.raises(ValueError):
        oracle.map_i("exp", 32, np.array([1]))
