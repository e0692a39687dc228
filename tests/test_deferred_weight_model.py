"""The deferred common weight of the binary64 stencil kernels, replayed on the
host.

A step whose weights are all exact multiples w_k = f r_k of one weight f sums
the ratios on the state scaled by 1/f^t (the first point of ratio 1 with no
multiply, then the other points in the listed order: an add for ratio 1, an
exact r x plus one rounding for the power-of-two ratios used here), and f^m
is applied after every chunk of m <= D steps.  D comes from the planner
itself (dcp_plan_info's per-step factors): (sum |r_k|)^D <= 2^32.  Against
the oracle's plain weighted sum this keeps long runs within the f64
tolerance, and the scaled state stays finite for inputs up to the bound the
chunk length gives.  Each operation of the model is one IEEE rounding
(numpy float64 adds; f^m is the product of m roundings of f)."""
import math

import numpy as np
import pytest

import oracle
from oracle import programs as OP
from paper_2107_00555_gb300 import Graph, inputs
from paper_2107_00555_gb300 import _capi as C

SEVEN = OP.SEVEN   # centre first, then x-, x+, y-, y+, z-, z+
FIVE = OP.FIVE     # centre, west, east, south, north

# (name, offsets, weights): the heat step (ratios 4 and 1, sum 10), the 0.2
# average (all ratios 1, sum 5), and a negative common weight (f = -0.125:
# ratios -4 and 1, sum 8)
SETS = [
    ("heat", SEVEN, [0.4] + [0.1] * 6),
    ("average", FIVE, [0.2] * 5),
    ("negative", FIVE, [0.5, -0.125, -0.125, -0.125, -0.125]),
]


def _planner_scales(shape, offs, w, bc, T):
    g = Graph()
    x = g.input("f64", shape)
    g.output(g.stencil(x, offs, w, bc, T))
    g.fuse(C.DCP_FUSE_ALL)
    out = []
    for l in g.plan()["launches"]:
        out += l.get("deferred_scales", [None] * (l["steps"][1] - l["steps"][0]))
    return out


def _shift(a, off, bc):
    """a[p + off] for every p (periodic wrap, or zero outside)."""
    if bc == "periodic":
        return np.roll(a, tuple(-o for o in off), axis=tuple(range(a.ndim)))
    out = np.zeros_like(a)
    src, dst = [], []
    for o, n in zip(off, a.shape):
        src.append(slice(max(0, o), n + min(0, o)))
        dst.append(slice(max(0, -o), n - max(0, o)))
    out[tuple(dst)] = a[tuple(src)]
    return out


def _deferred_run(u0, offs, w, bc, T, D):
    f = max(set(w), key=w.count)
    r = [x / f for x in w]
    assert all(x * f == y for x, y in zip(r, w))
    first = r.index(1.0)
    order = [first] + [k for k in range(len(r)) if k != first]
    s = u0.astype(np.float64)
    for t in range(T):
        nb = [_shift(s, offs[k], bc) for k in range(len(offs))]
        acc = nb[order[0]].copy()
        for k in order[1:]:
            if r[k] == 1.0:
                acc = acc + nb[k]
            else:  # power-of-two ratio: r x exact, one rounding
                assert math.frexp(abs(r[k]))[0] == 0.5
                acc = r[k] * nb[k] + acc
        i = t + 1
        m = D if i % D == 0 else (T % D if i == T else 0)
        if m:
            F = 1.0
            for _ in range(m):
                F *= f
            acc = F * acc
        s = acc
    return s


def _chunk(scales):
    """D: the first chunk end in the planner's per-step factors."""
    for i, x in enumerate(scales):
        if x is not None and x != 1:
            return i + 1
    return None


@pytest.mark.parametrize("name,offs,w", SETS)
@pytest.mark.parametrize("bc", ["periodic", "zero"])
def test_long_runs_within_tolerance(name, offs, w, bc):
    if name == "heat":
        shape = (9, 10, 11)
        Ts = (9, 50, 121)
    else:
        shape = (23, 29)
        Ts = (13, 60, 301)
    f = max(set(w), key=w.count)
    D = int(math.floor(32 / math.log2(sum(abs(x / f) for x in w))))
    u0 = inputs.uniform(shape, -1.0, 1.0, 31)
    for T in Ts:
        sc = _planner_scales(shape, offs, w, bc, T)
        assert len(sc) == T and all(x is not None for x in sc), (name, T)
        if T > D:
            assert _chunk(sc) == D, (name, T, sc[:D + 1])
        ref = oracle.stencil(u0, offs, w, bc, T)
        got = _deferred_run(u0, offs, w, bc, T, D)
        scale = float(np.max(np.abs(u0)))
        # the negative-weight step amplifies the state: compare relative to the
        # largest reference value
        if name == "negative":
            scale = max(scale, float(np.max(np.abs(ref))))
        assert np.all(np.abs(got - ref) <= 1e-12 * np.maximum(np.abs(ref), scale)), (name, T)


def test_scaled_state_stays_finite_up_to_the_bound():
    name, offs, w = SETS[0]
    u0 = inputs.uniform((6, 7, 8), -1.0, 1.0, 32)
    u0[0, 0, 0] = 1e298
    D = _chunk(_planner_scales(u0.shape, offs, w, "periodic", 18))
    got = _deferred_run(u0, offs, w, "periodic", 18, D)
    assert np.isfinite(got).all()
    ref = oracle.stencil(u0, offs, w, "periodic", 18)
    assert np.max(np.abs(got - ref)) <= 1e-12 * 1e298
