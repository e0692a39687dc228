"""The workload programs, written against the dcp builder one NumPy-level
operation per call (the SSA form of Sec. 2.3).

* ``map_reduce``  y = exp(a*x + b) * sin(x) - 0.5*x*x; sum(y), max|y| (over
                  all elements, or along one axis)
* ``jacobi2d``    the 5-point averaging step of the paper's jacobi_2d
                  (Sec. 4.3), points in the order the paper sums them:
                  centre, west, east, south, north, all weighted 0.2
* ``heat3d``      3-D 7-point step, centre 0.4, six neighbours 0.1
* ``batch2d``     many independent jacobi2d instances of different sizes
* ``tanh_chain``  u_{t+1} = tanh(S u_t) with the 7-point S, loss = sum(u_T^2)
"""
from __future__ import annotations

from .graph import Graph

FIVE_POINT = [(0, 0), (0, -1), (0, 1), (1, 0), (-1, 0)]
FIVE_WEIGHTS = [0.2] * 5
SEVEN_POINT = [(0, 0, 0), (0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]
SEVEN_WEIGHTS = [0.4] + [0.1] * 6


def map_reduce(n, dtype="f32", fuse=None, axis=None):
    """``n`` is an element count (1-D arrays) or a shape; with ``axis`` the
    two reductions run along that axis (one result per remaining index)."""
    shape = (n,) if isinstance(n, int) else tuple(n)
    g = Graph()
    x = g.input(dtype, shape)
    a = g.input(dtype, shape)
    b = g.input(dtype, shape)
    t = g.map("mul", [a, x])
    t = g.map("add", [t, b])
    e = g.map("exp", [t])
    s = g.map("sin", [x])
    p = g.map("mul", [e, s])
    xx = g.map("mul", [x, x])
    h = g.map("mul_s", [xx], 0.5)
    y = g.map("sub", [p, h])
    g.output(g.reduce(y, "sum", axis=axis))
    g.output(g.reduce(y, "maxabs", axis=axis))
    if fuse is not None:
        g.fuse(fuse)
    return g


def jacobi2d(shape, steps, bc="zero", dtype="f64", fuse=None):
    g = Graph()
    u = g.input(dtype, shape)
    g.output(g.stencil(u, FIVE_POINT, FIVE_WEIGHTS, bc, steps))
    if fuse is not None:
        g.fuse(fuse)
    return g


def heat3d(shape, steps, bc="periodic", dtype="f64", fuse=None):
    g = Graph()
    u = g.input(dtype, shape)
    g.output(g.stencil(u, SEVEN_POINT, SEVEN_WEIGHTS, bc, steps))
    if fuse is not None:
        g.fuse(fuse)
    return g


def batch2d(sides, steps, bc="zero", dtype="f32", fuse=None):
    g = Graph()
    for s in sides:
        u = g.input(dtype, (int(s), int(s)))
        g.output(g.stencil(u, FIVE_POINT, FIVE_WEIGHTS, bc, steps))
    if fuse is not None:
        g.fuse(fuse)
    return g


def tanh_chain(shape, steps, bc="periodic", dtype="f64", fuse=None):
    g = Graph()
    u = g.input(dtype, shape)
    for _ in range(steps):
        u = g.map("tanh", [g.stencil(u, SEVEN_POINT, SEVEN_WEIGHTS, bc, 1)])
    g.output(g.reduce(g.map("square", [u]), "sum"))
    if fuse is not None:
        g.fuse(fuse)
    return g
