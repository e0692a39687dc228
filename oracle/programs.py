"""The workload programs in the oracle's own vocabulary (test infrastructure).

Written independently of the product's builders: each is the unfused SSA
program of the paper's form, one oracle op per NumPy-level statement.
"""
from . import Program

FIVE = [(0, 0), (0, -1), (0, 1), (1, 0), (-1, 0)]   # centre, west, east, south, north
SEVEN = [(0, 0, 0), (0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]
W5 = [0.2] * 5
W7 = [0.4] + [0.1] * 6


def map_reduce(n, dtype="f64", axis=None):
    """y = exp(a*x + b) * sin(x) - 0.5*x*x, then sum(y) and max|y| (``n`` an
    element count or a shape; with ``axis``, along that axis).
    Handles: x, a, b, ax, t, e, s, p, xx, h, y, sum, maxabs."""
    shape = (n,) if isinstance(n, int) else tuple(n)
    p = Program()
    x = p.input(dtype, shape)
    a = p.input(dtype, shape)
    b = p.input(dtype, shape)
    ax = p.map("mul", [a, x])
    t = p.map("add", [ax, b])
    e = p.map("exp", [t])
    s = p.map("sin", [x])
    pr = p.map("mul", [e, s])
    xx = p.map("mul", [x, x])
    h = p.map("mul_s", [xx], 0.5)
    y = p.map("sub", [pr, h])
    p.output(p.reduce(y, "sum", axis=axis))
    p.output(p.reduce(y, "maxabs", axis=axis))
    p.handles = dict(x=x, a=a, b=b, p=pr, h=h, y=y)
    return p


def jacobi2d(shape, steps, bc="zero", dtype="f64"):
    p = Program()
    u = p.input(dtype, shape)
    p.output(p.stencil(u, FIVE, W5, bc, steps))
    return p


def heat3d(shape, steps, bc="periodic", dtype="f64"):
    p = Program()
    u = p.input(dtype, shape)
    p.output(p.stencil(u, SEVEN, W7, bc, steps))
    return p


def tanh_chain(shape, steps, bc="periodic", dtype="f64"):
    p = Program()
    u = p.input(dtype, shape)
    for _ in range(steps):
        u = p.map("tanh", [p.stencil(u, SEVEN, W7, bc, 1)])
    p.output(p.reduce(p.map("square", [u]), "sum"))
    return p
