"""GPU axis reductions (x.sum(axis=a), max, min, max|x| along one axis)
against the oracle.  Sums: |gpu - exact| <= tol * sum|y| per output (the
backward-stable bound of any summation order); max / min / maxabs of the
inputs themselves: exact; integer reductions: bit-exact.  Shapes cover every
thread layout (contiguous and strided reduced axis, tiny and long axes, the
split of a long axis over several blocks) and the degenerate cases."""
import numpy as np
import pytest

import oracle
from oracle import Program
from paper_2107_00555_gb300 import Graph
from paper_2107_00555_gb300 import _capi as C

from gpu_util import red_tol_for, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NP = {"f32": np.float32, "f64": np.float64, "i32": np.int32, "i64": np.int64}
SHAPES_AXES = [((1,), 0), ((5,), 0), ((37, 45), 0), ((37, 45), 1), ((3, 5, 7), 0),
               ((3, 5, 7), 1), ((3, 5, 7), 2), ((1000, 3), 0), ((1000, 3), 1),
               ((3, 100003), 1), ((100003, 3), 0), ((64, 4096), 1), ((4096, 64), 0),
               ((2, 1, 5), 1), ((7, 300, 9), 1), ((1, 1 << 20), 1), ((1 << 20, 1), 0),
               # extents divisible by the vector width: 16-byte loads along the
               # contiguous axis (inner, or the reduced axis for contiguous rows)
               ((36, 44), 0), ((36, 44), 1), ((8, 5, 12), 0), ((8, 5, 12), 1), ((8, 5, 12), 2),
               ((4, 100000), 0), ((100000, 4), 1), ((3, 100004), 1), ((100004, 8), 0),
               ((64, 8), 1), ((5, 4096), 1)]


def _data(shape, dtype, seed):
    rng = np.random.default_rng(seed)
    if dtype.startswith("i"):
        return rng.integers(-1000, 1000, size=shape).astype(NP[dtype])
    return rng.normal(size=shape).astype(NP[dtype])


def _graph(shape, dtype, axis, reds, pre=None):
    g = Graph()
    x = g.input(dtype, shape)
    y = x if pre is None else pre(g, x)
    for r in reds:
        g.output(g.reduce(y, r, axis=axis))
    return g


@pytest.mark.parametrize("shape,axis", SHAPES_AXES)
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_float_axis_reductions(shape, axis, dtype):
    x = _data(shape, dtype, 50 + len(shape))
    reds = ["sum", "max", "min", "maxabs"]
    g = _graph(shape, dtype, axis, reds)
    assert g.fuse(C.DCP_FUSE_ALL) == 1
    outs = [to_host(o) for o in g.run([to_dev(x)])]
    s, fs, ab = oracle.reduce_axis("sum", x, axis)
    assert outs[0].shape == s.shape
    assert np.all(np.abs(outs[0].astype(np.float64) - fs) <= red_tol_for(dtype) * ab + 1e-300)
    for got, r in zip(outs[1:], reds[1:]):
        ref = oracle.reduce_axis(r, x, axis)
        assert np.array_equal(got.astype(np.float64), ref), r


@pytest.mark.parametrize("shape,axis", [((37, 45), 0), ((3, 5, 7), 2), ((3, 100003), 1),
                                        ((100003, 3), 0)])
@pytest.mark.parametrize("dtype", ["i32", "i64"])
def test_integer_axis_reductions_bit_exact(shape, axis, dtype):
    x = _data(shape, dtype, 60)
    if dtype == "i32":
        x = (x.astype(np.int64) * (1 << 20)).astype(np.int32)  # sums wrap
    reds = ["sum", "max", "min", "maxabs"]
    g = _graph(shape, dtype, axis, reds)
    g.fuse(C.DCP_FUSE_ALL)
    outs = [to_host(o) for o in g.run([to_dev(x)])]
    bits = 32 if dtype == "i32" else 64
    for got, r in zip(outs, reds):
        ref = oracle.reduce_axis_i(r, bits, x, axis)
        assert np.array_equal(got.astype(np.int64), ref), r


@pytest.mark.parametrize("shape,axis", [((256, 1000), 1), ((1000, 256), 0), ((5, 200003), 1)])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_fused_prologue_row_and_column_reductions(shape, axis, dtype):
    """y = exp(a*x + b) * sin(x) - 0.5*x*x reduced along an axis: the map
    chain is the prologue of the one reduction kernel."""
    rng = np.random.default_rng(7)
    x, a, b = (rng.normal(size=shape).astype(NP[dtype]) for _ in range(3))
    p = Program()
    px, pa, pb = (p.input(dtype, shape) for _ in range(3))
    e = p.map("exp", [p.map("add", [p.map("mul", [pa, px]), pb])])
    es = p.map("mul", [e, p.map("sin", [px])])
    hh = p.map("mul_s", [p.map("mul", [px, px])], 0.5)
    y = p.map("sub", [es, hh])
    hs, hm = p.output(p.reduce(y, "sum", axis=axis)), p.output(p.reduce(y, "maxabs", axis=axis))
    vals, extra = oracle.run(p, [x, a, b], detail=True)
    g = Graph()
    gx, ga, gb = (g.input(dtype, shape) for _ in range(3))
    ge = g.map("exp", [g.map("add", [g.map("mul", [ga, gx]), gb])])
    gy = g.map("sub", [g.map("mul", [ge, g.map("sin", [gx])]),
                       g.map("mul_s", [g.map("mul", [gx, gx])], 0.5)])
    g.output(g.reduce(gy, "sum", axis=axis))
    g.output(g.reduce(gy, "maxabs", axis=axis))
    assert g.fuse(C.DCP_FUSE_ALL) == 1
    (grp,) = g.plan()["groups"]
    assert grp["kind"] == "axis_reduce" and grp["members"] == 8 and grp["stores"] == 0
    s, m = (to_host(o).astype(np.float64) for o in g.run([to_dev(x), to_dev(a), to_dev(b)]))
    tol = red_tol_for(dtype)
    assert np.all(np.abs(s - extra[hs]["fsum"]) <= tol * extra[hs]["abs"])
    # maxabs of a computed value: the map's rounding, bounded by the map tolerance
    mt = 1e-5 if dtype == "f32" else 1e-12
    ym = vals[hm]
    scale = oracle.reduce_axis("maxabs", np.abs(vals[es]) + np.abs(vals[hh]), axis)
    assert np.all(np.abs(m - ym) <= mt * np.maximum(ym, scale))


def test_determinism_and_repeated_runs():
    x = _data((3, 300007), "f32", 9)
    g = _graph((3, 300007), "f32", 1, ["sum"])
    g.fuse(C.DCP_FUSE_ALL)
    d = to_dev(x)
    runs = [to_host(g.run([d])[0]).tobytes() for _ in range(4)]
    assert all(r == runs[0] for r in runs)
    g.set_option(C.DCP_OPT_USE_GRAPH, 1)
    runs2 = [to_host(g.run([d])[0]).tobytes() for _ in range(3)]
    assert all(r == runs[0] for r in runs2)


def test_empty_and_unit_axes():
    g = _graph((0, 5), "f32", 0, ["sum"])
    g.fuse(C.DCP_FUSE_ALL)
    out = to_host(g.run([torch.empty((0, 5), dtype=torch.float32, device="cuda")])[0])
    assert out.shape == (5,) and np.all(out == 0)
    g = _graph((5, 0), "f64", 0, ["sum"])
    g.fuse(C.DCP_FUSE_ALL)
    out = g.run([torch.empty((5, 0), dtype=torch.float64, device="cuda")])[0]
    assert tuple(out.shape) == (0,)
    x = _data((4, 1, 6), "f64", 11)
    g = _graph((4, 1, 6), "f64", 1, ["sum", "max"])
    g.fuse(C.DCP_FUSE_ALL)
    s, m = (to_host(o) for o in g.run([to_dev(x)]))
    assert np.array_equal(s, x[:, 0, :]) and np.array_equal(m, x[:, 0, :])


def test_axis_reduction_op_by_op_and_errors():
    x = _data((50, 70), "f64", 12)
    g = Graph()
    v = g.input("f64", (50, 70))
    g.output(g.reduce(g.map("abs", [v]), "sum", axis=0))
    g.fuse(0)
    assert len(g.plan()["groups"]) == 2
    s, fs, ab = oracle.reduce_axis("sum", np.abs(x), 0)
    got = to_host(g.run([to_dev(x)])[0])
    assert np.all(np.abs(got - fs) <= 1e-10 * ab)
    g = Graph()
    v = g.input("f64", (3, 4))
    r = g.reduce(v, "sum", axis=1)
    g.output(r)
    g.fuse(C.DCP_FUSE_ALL)
    with pytest.raises(C.DcpError) as e:
        g.adjoint([to_dev(np.ones((3, 4)))], [to_dev(np.ones(3))])
    assert e.value.status == C.DCP_E_UNSUPPORTED


@pytest.mark.parametrize("offset", [1, 2, 3])
@pytest.mark.parametrize("shape,axis", [((64, 400), 0), ((64, 400), 1)])
def test_unaligned_buffers_take_the_scalar_variant(offset, shape, axis):
    """Inputs that start off a 16-byte boundary use the element-wise loads."""
    n = int(np.prod(shape))
    x = _data((n + offset,), "f32", 13)
    d = to_dev(x)[offset:].view(shape)
    g = _graph(shape, "f32", axis, ["sum", "max"])
    g.fuse(C.DCP_FUSE_ALL)
    s, m = (to_host(o) for o in g.run([d]))
    xs = x[offset:].reshape(shape)
    _, fs, ab = oracle.reduce_axis("sum", xs, axis)
    assert np.all(np.abs(s.astype(np.float64) - fs) <= 1e-4 * ab)
    assert np.array_equal(m.astype(np.float64), oracle.reduce_axis("max", xs, axis))
