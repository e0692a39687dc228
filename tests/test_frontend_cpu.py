"""The NumPy-style tracer: what it records (plans only; no GPU needed)."""
import pytest

import paper_2107_00555_gb300 as dcp


def test_traced_map_reduce_is_one_kernel():
    n = 1 << 12

    @dcp.program(x=("f32", (n,)), a=("f32", (n,)), b=("f32", (n,)))
    def f(x, a, b):
        y = dcp.exp(a * x + b) * dcp.sin(x) - 0.5 * x * x
        return y.sum(), abs(y).max()

    (grp,) = f.plan()["groups"]
    assert grp["kind"] == "map" and grp["reductions"] == 2 and grp["stores"] == 0
    assert f.plan()["n_launches"] == 1


def test_traced_jacobi2d_paper_form_is_one_time_tiled_chain():
    n, T = 40, 3

    @dcp.program(A=("f64", (n, n)), B=("f64", (n, n)))
    def jacobi_2d(A, B):
        for _ in range(T):
            B[1:-1, 1:-1] = 0.2 * (A[1:-1, 1:-1] + A[1:-1, :-2] + A[1:-1, 2:] + A[2:, 1:-1]
                                   + A[:-2, 1:-1])
            A[1:-1, 1:-1] = 0.2 * (B[1:-1, 1:-1] + B[1:-1, :-2] + B[1:-1, 2:] + B[2:, 1:-1]
                                   + B[:-2, 1:-1])
        return A

    (grp,) = jacobi_2d.plan()["groups"]
    assert grp["kind"] == "stencil" and grp["steps"] == 2 * T
    assert grp["tile"] is not None


def test_traced_axis_reduction_and_stencil_1d():
    @dcp.program(("f32", (30, 40)))
    def rows(x):
        return (x * x).sum(axis=1)

    (grp,) = rows.plan()["groups"]
    assert grp["kind"] == "axis_reduce" and grp["members"] == 1

    @dcp.program(("f64", (100,)))
    def jac1(A):
        A[1:-1] = 0.33333 * (A[:-2] + A[1:-1] + A[2:])
        return A

    (grp,) = jac1.plan()["groups"]
    assert grp["kind"] == "stencil" and grp["steps"] == 1


def test_tracer_rejects_what_it_cannot_express():
    with pytest.raises(NotImplementedError):
        @dcp.program(("f32", (8,)))
        def div3(x):
            return x / 3.0
    with pytest.raises(NotImplementedError):
        @dcp.program(("f64", (10, 10)), ("f64", (10, 10)))
        def not_interior(A, B):
            B[1:-1, 2:] = 0.5 * (A[1:-1, 1:-1] + A[1:-1, 2:])  # region is not the interior
            return B
    with pytest.raises(ValueError):
        @dcp.program(("f64", (10, 10)), ("f64", (10, 10)))
        def extents(A, B):
            B[1:-1, 1:-1] = A[1:-1, 1:-1] + A[:-1, 1:-1]
            return B
    with pytest.raises(TypeError):
        @dcp.program(x=("f32", (8,)))
        def two(x, y):
            return x + y

    @dcp.program(("f32", (8,)))
    def half(x):
        return x / 2.0  # exact: multiplies by 0.5

    assert half.plan()["groups"][0]["kind"] == "map"
