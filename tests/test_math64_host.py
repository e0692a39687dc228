"""The binary64 exp, sin and cos of k_math64.cuh, compiled for the host
(the CUDA rounding intrinsics mapped to their IEEE equivalents: __fma_rn to
fma, __dmul_rn / __dsub_rn to plain operations without contraction), against
120-bit values from mpmath: within 1.5 ulp on the fast paths, the special
values exact.  Catches a wrong constant, a dropped Taylor term or a wrong
quadrant without a GPU; the GPU tests check the same routines on the device
against libm."""
import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

KDIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2107_00555_gb300", "csrc", "kernels")

SHIM = r"""
#include <cmath>
#include <cstring>
#define __device__
#define __forceinline__ inline
static inline double __fma_rn(double a, double b, double c) { return std::fma(a, b, c); }
static inline double __dmul_rn(double a, double b) { return a * b; }
static inline double __dsub_rn(double a, double b) { return a - b; }
static inline long long __double_as_longlong(double x) { long long v; std::memcpy(&v, &x, 8); return v; }
static inline double __longlong_as_double(long long v) { double x; std::memcpy(&x, &v, 8); return x; }
static inline int __double2loint(double x) {
  return (int)(unsigned)(unsigned long long)__double_as_longlong(x);
}
static inline double __ldg(const double* p) { return *p; }
using std::exp; using std::sin; using std::cos;
#include "k_math64.cuh"
extern "C" void m64(int f, long n, const double* x, double* y) {
  for (long i = 0; i < n; ++i)
    y[i] = f == 0 ? dcp_exp64(x[i]) : (f == 1 ? dcp_sin64(x[i]) : dcp_cos64(x[i]));
}
"""


@pytest.fixture(scope="module")
def m64(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("m64")
    src = d / "m64.cpp"
    src.write_text(SHIM)
    lib = d / "libm64.so"
    subprocess.run([cxx, "-O2", "-ffp-contract=off", "-std=c++17", "-shared", "-fPIC",
                    "-I", KDIR, "-o", str(lib), str(src)], check=True)
    so = ctypes.CDLL(str(lib))

    def run(f, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty_like(x)
        so.m64(ctypes.c_int(f), ctypes.c_long(x.size), x.ctypes.data_as(ctypes.c_void_p),
               y.ctypes.data_as(ctypes.c_void_p))
        return y
    return run


def _max_ulp(fn, x, y):
    mpmath.mp.prec = 120
    worst = 0.0
    for xi, yi in zip(x.tolist(), y.tolist()):
        ref = fn(mpmath.mpf(xi))
        worst = max(worst, float(abs((mpmath.mpf(yi) - ref) / math.ulp(float(ref)))))
    return worst


@pytest.mark.parametrize("f,name", [(0, "exp"), (1, "sin"), (2, "cos")])
def test_fast_paths_within_1p5_ulp(m64, f, name):
    rng = np.random.default_rng(90 + f)
    lim = 703.9 if f == 0 else 131071.0
    x = np.concatenate([rng.uniform(-lim, lim, 3000), rng.normal(0.0, 1.0, 3000),
                        rng.uniform(-8.0, 8.0, 2000),
                        np.sign(rng.uniform(-1, 1, 1000)) * 10.0 ** rng.uniform(-20, 2, 1000)])
    if f:
        # near multiples of pi/4 and pi/2, where the reduction and quadrants meet
        k = np.arange(-400, 400)
        x = np.concatenate([x, k * (np.pi / 4), np.nextafter(k * (np.pi / 2), np.inf)])
    fn = {0: mpmath.exp, 1: mpmath.sin, 2: mpmath.cos}[f]
    assert _max_ulp(fn, x, m64(f, x)) <= 1.5


def test_special_values(m64):
    inf, nan = math.inf, math.nan
    assert m64(0, np.array([0.0, -0.0, inf, -inf, 800.0, -800.0])).tolist() == [1.0, 1.0, inf, 0.0, inf, 0.0]
    assert np.isnan(m64(0, np.array([nan]))).all()
    y = m64(1, np.array([0.0, -0.0, 5e-324, -5e-324]))
    assert y.tolist() == [0.0, 0.0, 5e-324, -5e-324] and np.signbit(y).tolist() == [False, True, False, True]
    assert m64(2, np.array([0.0, -0.0, 5e-324])).tolist() == [1.0, 1.0, 1.0]
    for f in (1, 2):
        assert np.isnan(m64(f, np.array([inf, -inf, nan]))).all()
    # the exponent scaling at both ends of the fast path stays normal
    y = m64(0, np.array([703.99, -703.99]))
    assert np.isfinite(y).all() and (y > np.finfo(np.float64).tiny).all()
