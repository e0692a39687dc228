"""The deferred common weight of the stencil kernels, replayed on the host.

A step whose weights are all exact multiples w_k = f r_k of one weight f sums
the ratios on the state scaled by 1/f^t (the first point of ratio 1 with no
multiply, then the other points in the listed order: an add for ratio 1, an
exact r x plus one rounding for the power-of-two ratios used here), and f^m
is applied after every chunk of m <= D steps.  D comes from the planner
itself (dcp_plan_info's per-step factors): (sum |r_k|)^D <= 2^32 for
binary64, 2^16 for binary32.  Against the oracle's plain weighted sum this
keeps long runs within the dtype's tolerance, and the scaled state stays
finite for inputs up to the bound the chunk length gives.  Each operation of
the model is one IEEE rounding in the step's dtype (numpy float32 / float64
adds; f^m is the product of m binary64 roundings, rounded once to float32
for binary32)."""
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


def _planner_scales(shape, offs, w, bc, T, dtype):
    g = Graph()
    x = g.input(dtype, shape)
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


def _deferred_run(u0, offs, w, bc, T, dtype, D):
    np_t = np.float32 if dtype == "f32" else np.float64
    wt = [float(np_t(x)) for x in w]
    f = max(set(wt), key=wt.count)
    r = [x / f for x in wt]
    assert all(x * f == y for x, y in zip(r, wt))
    first = r.index(1.0)
    order = [first] + [k for k in range(len(r)) if k != first]
    s = u0.astype(np_t)
    for t in range(T):
        nb = [_shift(s, offs[k], bc) for k in range(len(offs))]
        acc = nb[order[0]].copy()
        for k in order[1:]:
            if r[k] == 1.0:
                acc = acc + nb[k]
            else:  # power-of-two ratio: r x exact, one rounding
                assert math.frexp(abs(r[k]))[0] == 0.5
                acc = np_t(r[k]) * nb[k] + acc
        i = t + 1
        m = D if i % D == 0 else (T % D if i == T else 0)
        if m:
            F = 1.0
            for _ in range(m):
                F *= f
            acc = np_t(F) * acc
        s = acc
    return s


def _chunk(scales):
    """D: the first chunk end in the planner's per-step factors."""
    for i, x in enumerate(scales):
        if x is not None and x != 1:
            return i + 1
    return None


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("name,offs,w", SETS)
@pytest.mark.parametrize("bc", ["periodic", "zero"])
def test_long_runs_within_tolerance(dtype, name, offs, w, bc):
    if name == "heat":
        shape = (9, 10, 11)
        Ts = (9, 50, 121)
    else:
        shape = (23, 29)
        Ts = (13, 60, 301)
    gsum = sum(abs(x / w[-1]) if name != "heat" else abs(x / 0.1) for x in w)
    bits = 16 if dtype == "f32" else 32
    D = int(math.floor(bits / math.log2(gsum)))
    u0 = inputs.uniform(shape, -1.0, 1.0, 31)
    if dtype == "f32":
        u0 = u0.astype(np.float32)
    for T in Ts:
        sc = _planner_scales(shape, offs, w, bc, T, dtype)
        assert len(sc) == T and all(x is not None for x in sc), (name, dtype, T)
        if T > D:
            assert _chunk(sc) == D, (name, dtype, T, sc[:D + 1])
        ref = oracle.stencil(u0.astype(np.float64), offs,
                             [float(np.float32(x)) for x in w] if dtype == "f32" else w, bc, T)
        got = _deferred_run(u0, offs, w, bc, T, dtype, D).astype(np.float64)
        scale = float(np.max(np.abs(u0)))
        # the negative-weight step amplifies the state: compare relative to the
        # largest reference value
        if name == "negative":
            scale = max(scale, float(np.max(np.abs(ref))))
        tol = 1e-5 if dtype == "f32" else 1e-12
        assert np.all(np.abs(got - ref) <= tol * np.maximum(np.abs(ref), scale)), (name, dtype, T)


@pytest.mark.parametrize("dtype,big", [("f64", 1e298), ("f32", 5e33)])
def test_scaled_state_stays_finite_up_to_the_bound(dtype, big):
    name, offs, w = SETS[0]
    np_t = np.float32 if dtype == "f32" else np.float64
    u0 = inputs.uniform((6, 7, 8), -1.0, 1.0, 32).astype(np_t)
    u0[0, 0, 0] = big
    D = _chunk(_planner_scales(u0.shape, offs, w, "periodic", 18, dtype))
    got = _deferred_run(u0, offs, w, "periodic", 18, dtype, D)
    assert np.isfinite(got).all()
    wts = [float(np.float32(x)) for x in w] if dtype == "f32" else w
    ref = oracle.stencil(u0.astype(np.float64), offs, wts, "periodic", 18)
    tol = 1e-5 if dtype == "f32" else 1e-12
    assert np.max(np.abs(got.astype(np.float64) - ref)) <= tol * big
