"""The deferred common weight of the binary64 stencil kernels, replayed on
the host: a step with weights w_k = f r_k sums the ratios (the first point
of ratio 1 with no multiply, the heat stencil's centre as 4 c, exact) on the
state scaled by 1/f^t, and f^m is applied after every chunk of m <= D steps,
(sum |r_k|)^D <= 2^32.  Against the oracle's plain weighted sum this keeps
long runs within the f64 tolerance, and the scaled state stays finite for
inputs up to 1e298 (the bound the planner's chunk length gives).  The model
follows the kernels' operation order; each operation is one IEEE rounding
(numpy's add, and 4 c + acc as one rounding because 4 c is exact)."""
import math

import numpy as np

import oracle
from oracle import programs as OP
from paper_2107_00555_gb300 import inputs

SEVEN = OP.SEVEN          # centre first, then x-, x+, y-, y+, z-, z+
RATIOS = [4.0] + [1.0] * 6
F = 0.1


def _chunk_length(ratios):
    g = sum(abs(r) for r in ratios)
    return int(math.floor(32.0 / math.log2(g)))


def _deferred_heat(u0, T):
    D = _chunk_length(RATIOS)
    assert D == 9
    w = u0.copy()
    for t in range(T):
        nb = [np.roll(w, (-dz, -dy, -dx), axis=(0, 1, 2)) for dz, dy, dx in SEVEN]
        acc = nb[1].copy()                # x-: ratio 1, no multiply
        acc = 4.0 * nb[0] + acc           # centre: fma(4, c, acc), 4 c exact
        for k in range(2, 7):
            acc = acc + nb[k]             # ratio 1: add
        i = t + 1
        m = D if i % D == 0 else (T % D if i == T else 0)
        if m:
            scale = 1.0
            for _ in range(m):
                scale *= F
            acc = scale * acc
        w = acc
    return w


def test_long_periodic_runs_stay_within_the_f64_tolerance():
    u0 = inputs.uniform((12, 13, 14), -1.0, 1.0, 31)
    for T in (9, 50, 121):
        ref = oracle.run(OP.heat3d(u0.shape, T, "periodic"), [u0])[-1]
        got = _deferred_heat(u0, T)
        assert np.max(np.abs(got - ref)) <= 1e-12 * float(np.max(np.abs(u0))), T


def test_scaled_state_stays_finite_up_to_1e298():
    u0 = inputs.uniform((6, 7, 8), -1.0, 1.0, 32)
    u0[0, 0, 0] = 1e298
    got = _deferred_heat(u0, 18)
    assert np.isfinite(got).all()
    ref = oracle.run(OP.heat3d(u0.shape, 18, "periodic"), [u0])[-1]
    assert np.max(np.abs(got - ref)) <= 1e-12 * 1e298
