"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers; it contains none of the method's
arithmetic.  Tests feed the same arrays to the CUDA path and to the CPU
oracle; the benchmark uses the same recipes.  All draws come from
``numpy.random.default_rng(seed)`` (PCG64).  The paper's benchmark suite is
not available here, so these recipes stand in for its stencil / map /
reduction programs (jacobi_2d and heat3d forms, Sec. 3.4 and 4.3).

Recipes (seed 1000 + config number by default):
  cfg1  256 x 256 float64, U[0, 1)                       (2-D 5-point, 10 steps)
  cfg2  x, a, b of 2**26 elements, N(0, 1), float32 or float64
  cfg3  512**3 float64, U[-1, 1)                          (3-D 7-point, 50 steps)
  cfg4  4096 instances, side round(exp(U(ln 32, ln 512))) clamped to [32, 512],
        float32, U[0, 1)                                  (2-D 5-point, 20 steps)
  cfg5  256**3 float64, U[-1, 1)                          (tanh-stencil chain, 20 steps)
"""
from __future__ import annotations

import math

import numpy as np


def uniform(shape, lo, hi, seed, dtype=np.float64):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=shape).astype(dtype)


def normal(shape, seed, dtype=np.float64, count=1):
    """`count` independent N(0,1) arrays from one stream (drawn in float64, then cast)."""
    rng = np.random.default_rng(seed)
    out = [rng.standard_normal(size=shape).astype(dtype) for _ in range(count)]
    return out if count > 1 else out[0]


def cfg1(seed=1001, n=256):
    return uniform((n, n), 0.0, 1.0, seed)


def cfg2(dtype=np.float32, seed=1002, n=1 << 26):
    x, a, b = normal((n,), seed, dtype, count=3)
    return x, a, b


def cfg3(seed=1003, n=512):
    return uniform((n, n, n), -1.0, 1.0, seed)


def cfg4_sides(seed=1004, count=4096, lo=32, hi=512):
    rng = np.random.default_rng(seed)
    s = np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))
    return np.clip(np.rint(s), lo, hi).astype(np.int64)


def cfg4(seed=1004, count=4096, lo=32, hi=512, dtype=np.float32):
    sides = cfg4_sides(seed, count, lo, hi)
    rng = np.random.default_rng(seed + 7919)
    return [rng.uniform(0.0, 1.0, size=(int(s), int(s))).astype(dtype) for s in sides]


def cfg5(seed=1005, n=256):
    return uniform((n, n, n), -1.0, 1.0, seed)
