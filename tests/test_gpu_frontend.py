"""Traced NumPy-style programs on the GPU: the same bits as the equivalent
hand-built programs, and the oracle's values within the usual tolerances."""
import numpy as np
import pytest

import oracle
import paper_2107_00555_gb300 as dcp
from oracle import programs as OP
from paper_2107_00555_gb300 import _capi as C
from paper_2107_00555_gb300 import inputs, programs

from gpu_util import assert_close, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_traced_map_reduce_matches_builder_and_oracle(dtype):
    n = 100003
    npdt = np.float32 if dtype == "f32" else np.float64
    x, a, b = inputs.cfg2(npdt, seed=5, n=n)

    @dcp.program(x=(dtype, (n,)), a=(dtype, (n,)), b=(dtype, (n,)))
    def f(x, a, b):
        y = dcp.exp(a * x + b) * dcp.sin(x) - 0.5 * x * x
        return y.sum(), abs(y).max()

    dev = [to_dev(v) for v in (x, a, b)]
    s, m = (float(to_host(t)) for t in f(*dev))
    g = programs.map_reduce(n, dtype, fuse=C.DCP_FUSE_ALL)
    s0, m0 = (float(to_host(t)) for t in g.run(dev))
    assert m == m0  # (0.5*x)*x and 0.5*(x*x) round identically
    prog = OP.map_reduce(n)
    vals, extra = oracle.run(prog, [x, a, b], detail=True)
    sid, _ = prog.outputs
    tol = 1e-4 if dtype == "f32" else 1e-10
    assert abs(s - extra[sid]["fsum"]) <= tol * extra[sid]["abs"]


def test_traced_jacobi2d_paper_form_bitwise():
    n, T = 130, 4
    u0 = inputs.uniform((n, n), 0.0, 1.0, 15)

    @dcp.program(A=("f64", (n, n)), B=("f64", (n, n)))
    def jacobi_2d(A, B):
        for _ in range(T):
            B[1:-1, 1:-1] = 0.2 * (A[1:-1, 1:-1] + A[1:-1, :-2] + A[1:-1, 2:] + A[2:, 1:-1]
                                   + A[:-2, 1:-1])
            A[1:-1, 1:-1] = 0.2 * (B[1:-1, 1:-1] + B[1:-1, :-2] + B[1:-1, 2:] + B[2:, 1:-1]
                                   + B[:-2, 1:-1])
        return A

    got = to_host(jacobi_2d(to_dev(u0), to_dev(u0)))
    g = programs.jacobi2d((n, n), 2 * T, "fixed_ring", "f64", fuse=C.DCP_FUSE_ALL)
    ref_gpu = to_host(g.run([to_dev(u0)])[0])
    assert got.tobytes() == ref_gpu.tobytes()
    ref = oracle.run(OP.jacobi2d((n, n), 2 * T, "fixed_ring"), [u0])[-1]
    assert_close(got, ref, 1e-12, 1.0, "traced jacobi_2d")


def test_traced_row_reduction_and_1d_stencil():
    x = np.random.default_rng(3).normal(size=(300, 517)).astype(np.float32)

    @dcp.program(("f32", (300, 517)))
    def rows(v):
        return (v * v).sum(axis=1)

    got = to_host(rows(to_dev(x))).astype(np.float64)
    _, fs, ab = oracle.reduce_axis("sum", x.astype(np.float64) ** 2, 1)
    assert np.all(np.abs(got - fs) <= 1e-4 * ab)

    u = inputs.uniform((1000,), 0.0, 1.0, 16)

    @dcp.program(("f64", (1000,)))
    def jac1(A):
        for _ in range(6):
            A[1:-1] = 0.33333 * (A[:-2] + A[1:-1] + A[2:])
        return A

    got = to_host(jac1(to_dev(u)))
    p = oracle.Program()
    v = p.input("f64", (1000,))
    p.output(p.stencil(v, [(-1,), (0,), (1,)], [0.33333] * 3, "fixed_ring", 6))
    assert_close(got, oracle.run(p, [u])[-1], 1e-12, 1.0, "traced jacobi_1d")
