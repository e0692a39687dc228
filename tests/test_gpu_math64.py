"""Binary64 exp, sin and cos of the fused kernels against the oracle's libm,
in units in the last place, over the fast ranges (|x| < 704 for exp,
|x| < 2^17 for sin and cos), across their limits (where the kernels hand
the argument to CUDA's own functions) and at the special values.

The bound: the kernels' routines are within about 1.4 ulp of the exact value
on their fast paths, CUDA's functions within 2 ulp on the rest, and the
host's libm within 1 ulp, so two results differ by at most 3 ulp (4 where
the result is subnormal and the ulp is the fixed 2^-1074)."""
import math

import numpy as np
import pytest

import oracle
from paper_2107_00555_gb300 import Graph
from paper_2107_00555_gb300 import _capi as C

from gpu_util import to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _gpu_map(op, x):
    g = Graph()
    v = g.input("f64", x.shape)
    g.output(g.map(op, [v]))
    g.fuse(C.DCP_FUSE_ALL)
    (y,) = g.run([to_dev(x)])
    torch.cuda.synchronize()
    return to_host(y)


def _ulps(got, ref):
    ulp = np.array([math.ulp(float(r)) if np.isfinite(r) else 0.0 for r in ref])
    with np.errstate(invalid="ignore"):
        return np.abs(got - ref) / np.where(ulp > 0, ulp, 1.0)


def _args(op, rng):
    lim = 704.0 if op == "exp" else 2.0 ** 17
    edge = lim + np.arange(-64, 64) * math.ulp(lim)  # both sides of the fast path's limit
    parts = [
        rng.uniform(-lim, lim, 200_000),
        rng.normal(0.0, 1.0, 200_000),
        rng.normal(0.0, 10.0, 50_000),
        np.sign(rng.uniform(-1, 1, 20_000)) * 10.0 ** rng.uniform(-300, math.log10(lim), 20_000),
        edge,
        -edge,
    ]
    if op == "exp":
        parts.append(rng.uniform(-745.2, 709.78, 20_000))  # down to the subnormal results
    else:
        parts.append(np.arange(-3000, 3000) * (np.pi / 4))  # near the zeros and extrema
        parts.append(rng.uniform(-1e6, 1e6, 20_000))        # beyond the fast path
    return np.concatenate(parts)


@pytest.mark.parametrize("op", ["exp", "sin", "cos"])
def test_f64_transcendentals_within_3_ulp_of_libm(op):
    rng = np.random.default_rng({"exp": 61, "sin": 62, "cos": 63}[op])
    x = _args(op, rng)
    got = _gpu_map(op, x)
    ref = oracle.map_f(op, x)
    err = _ulps(got, ref)
    sub = np.abs(ref) < np.finfo(np.float64).tiny
    bound = np.where(sub, 4.0, 3.0)
    bad = ~(err <= bound)
    assert not bad.any(), (op, int(bad.sum()), x[bad][:5], got[bad][:5], ref[bad][:5])


@pytest.mark.parametrize("op", ["exp", "sin", "cos"])
def test_f64_transcendentals_special_values(op):
    x = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, 1e-300, -1e-300,
                  709.78, 709.79, -745.1, -746.0, 1e300, -1e300, 2.0 ** 17, -(2.0 ** 17)])
    got = _gpu_map(op, x)
    ref = oracle.map_f(op, x)
    for xi, gi, ri in zip(x, got, ref):
        if np.isnan(ri):
            assert np.isnan(gi), (op, xi, gi)
        elif np.isinf(ri) or ri == 0.0:
            assert gi == ri and np.signbit(gi) == np.signbit(ri), (op, xi, gi, ri)
        else:
            assert abs(gi - ri) <= 4 * math.ulp(ri), (op, xi, gi, ri)
