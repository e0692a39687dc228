"""Arrays beyond 2^31 elements (64-bit indexing in every kernel family).

Inputs are all ones and the stencil weights are powers of two, so every
value is exact: sums of ones are integers, interior stencil cells stay 1,
and the cells near a border equal those of a small array with the same
nearby border (the far borders lie outside the dependence cone), which the
oracle computes."""
import numpy as np
import pytest

import oracle
from paper_2107_00555_gb300 import Graph
from paper_2107_00555_gb300 import _capi as C

from gpu_util import to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BIG = (1 << 31) + 5


def _free():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def test_map_and_reductions_over_2p31_elements():
    x = torch.ones(BIG, dtype=torch.float64, device="cuda")
    g = Graph()
    v = g.input("f64", (BIG,))
    y = g.map("add_s", [v], 1.0)
    g.output(y)
    g.output(g.reduce(v, "sum"))
    g.output(g.reduce(y, "max"))
    g.fuse(C.DCP_FUSE_ALL)
    out_y, s, m = g.run([x])
    assert float(to_host(s)) == float(BIG) and float(to_host(m)) == 2.0
    assert bool((out_y[-1000:] == 2.0).all()) and bool((out_y[(1 << 31) - 3:(1 << 31) + 3] == 2.0).all())
    assert int((out_y == 2.0).sum()) == BIG
    del x, out_y
    _free()
    xi = torch.ones(BIG, dtype=torch.int32, device="cuda")
    g = Graph()
    v = g.input("i32", (BIG,))
    g.output(g.reduce(v, "sum"))
    g.fuse(C.DCP_FUSE_ALL)
    (si,) = g.run([xi])
    assert int(to_host(si)) == np.int64(BIG - (1 << 32))  # wraps modulo 2^32
    del xi
    _free()


def test_axis_reductions_over_2p31_elements():
    R = (1 << 29) + 3
    x = torch.ones((4, R), dtype=torch.float64, device="cuda")  # 2^31 + 12 elements
    g = Graph()
    v = g.input("f64", (4, R))
    g.output(g.reduce(v, "sum", axis=1))
    g.output(g.reduce(v, "sum", axis=0))
    g.fuse(C.DCP_FUSE_ALL)
    rows, cols = g.run([x])
    assert np.array_equal(to_host(rows), np.full(4, float(R)))
    assert int((cols == 4.0).sum()) == R
    del x, rows, cols
    _free()


def _corner_ref(shape_small, steps, offs, w):
    p = oracle.Program()
    u = p.input("f64", shape_small)
    p.output(p.stencil(u, offs, w, "zero", steps))
    return oracle.run(p, [np.ones(shape_small)])[-1]


@pytest.mark.parametrize("kernel", [0, 1])
def test_2d_stencil_over_2p31_cells(kernel):
    n = 46341  # n * n > 2^31
    offs = [(0, 0), (0, -1), (0, 1), (1, 0), (-1, 0)]
    w = [0.5, 0.125, 0.125, 0.125, 0.125]
    T = 3
    x = torch.ones((n, n), dtype=torch.float32, device="cuda")
    g = Graph()
    v = g.input("f32", (n, n))
    g.output(g.stencil(v, offs, w, "zero", T))
    g.set_option(C.DCP_OPT_STENCIL_KERNEL, kernel)
    g.set_option(C.DCP_OPT_TIME_TILE_DEPTH, T)
    g.fuse(C.DCP_FUSE_ALL)
    (out,) = g.run([x])
    ref = _corner_ref((32, 32), T, offs, w)
    assert np.array_equal(to_host(out[:8, :8]).astype(np.float64), ref[:8, :8])
    assert np.array_equal(to_host(out[-8:, -8:]).astype(np.float64), ref[-8:, -8:])
    assert np.array_equal(to_host(out[-8:, :8]).astype(np.float64), ref[-8:, :8])
    assert bool((out[T:-T, T:-T] == 1.0).all())
    del x, out
    _free()


def test_3d_stencil_over_2p31_cells():
    n = 1291  # n^3 > 2^31
    offs = [(0, 0, 0), (0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]
    w = [0.25] + [0.125] * 6
    x = torch.ones((n, n, n), dtype=torch.float32, device="cuda")
    g = Graph()
    v = g.input("f32", (n, n, n))
    g.output(g.stencil(v, offs, w, "zero", 2))
    g.fuse(C.DCP_FUSE_ALL)
    (out,) = g.run([x])
    ref = _corner_ref((16, 16, 16), 2, offs, w)
    assert np.array_equal(to_host(out[:4, :4, :4]).astype(np.float64), ref[:4, :4, :4])
    assert np.array_equal(to_host(out[-4:, -4:, -4:]).astype(np.float64), ref[-4:, -4:, -4:])
    assert bool((out[2:-2, 2:-2, 2:-2] == 1.0).all())
    del x, out
    _free()
