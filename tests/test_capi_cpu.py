"""C ABI checks that need no GPU: the library loads and exports every symbol
include/dcp.h declares, the builder rejects malformed programs with the
documented status codes, and the planner fuses programs into the expected
kernels (plan structure), compiling every generated kernel for sm_103a."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2107_00555_gb300 import DcpError, Graph, programs
from paper_2107_00555_gb300 import _capi as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    text = open(os.path.join(ROOT, "include", "dcp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dcp_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(C.lib_path())
    names = _header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(C.EXPORTED), set(names) - set(C.EXPORTED)


def _err(fn, *args):
    with pytest.raises(DcpError) as e:
        fn(*args)
    return e.value.status


def test_builder_validation():
    g = Graph()
    x = g.input("f32", (10,))
    y = g.input("f64", (10,))
    z = g.input("f32", (11,))
    i = g.input("i32", (10,))
    s = g.input("f32", ())
    assert _err(g.map, "add", [x, y]) == C.DCP_E_DTYPE
    assert _err(g.map, "add", [x, z]) == C.DCP_E_SHAPE
    assert _err(g.map, "exp", [i]) == C.DCP_E_DTYPE
    assert _err(g.map, "div", [i, i]) == C.DCP_E_DTYPE
    assert _err(g.map, 99, [x]) == C.DCP_E_INVALID_ARG
    assert _err(g.map, "add", [x]) == C.DCP_E_INVALID_ARG
    assert _err(g.map, "add_s", [i], 0.5) == C.DCP_E_INVALID_ARG
    assert _err(g.map, "neg", [12345]) == C.DCP_E_INVALID_ARG
    assert _err(g.stencil, i, [(0,)], [1.0]) == C.DCP_E_DTYPE
    assert _err(g.stencil, x, [(5,)], [1.0]) == C.DCP_E_INVALID_ARG
    assert _err(g.stencil, s, [(0,)], [1.0]) == C.DCP_E_SHAPE
    assert _err(g.stencil, x, [(0,)], [1.0], 7) == C.DCP_E_INVALID_ARG
    e = g.input("f64", (0,))
    assert _err(g.reduce, e, "max") == C.DCP_E_SHAPE
    g.reduce(e, "sum")  # sum of empty is 0
    assert _err(g.output, x) == C.DCP_E_INVALID_ARG  # inputs cannot be outputs
    v = g.map("add", [x, s])  # 0-axis operand broadcasts
    assert g.shape[v] == (10,)
    assert _err(g.fuse, 0) == C.DCP_E_STATE  # no outputs yet
    g.output(v)
    assert _err(g.output, v) == C.DCP_E_INVALID_ARG
    assert g.fuse(C.DCP_FUSE_ALL) == 1
    assert _err(g.map, "neg", [x]) == C.DCP_E_STATE
    assert _err(g.fuse, 0) == C.DCP_E_STATE
    assert _err(C.dcp_fuse, g._h, 1 << 20) == C.DCP_E_STATE


def test_unknown_fuse_flag_and_options():
    g = Graph()
    x = g.input("f32", (4,))
    g.output(g.map("neg", [x]))
    assert _err(C.dcp_fuse, g._h, 1 << 20) == C.DCP_E_INVALID_ARG
    assert _err(g.set_option, 999, 1) == C.DCP_E_INVALID_ARG
    assert _err(g.set_option, C.DCP_OPT_TIME_TILE_DEPTH, 0) == C.DCP_E_INVALID_ARG
    assert _err(g.set_option, C.DCP_OPT_TILE_X, 12) == C.DCP_E_INVALID_ARG
    assert _err(g.set_option, C.DCP_OPT_TILE_Z, 0) == C.DCP_E_INVALID_ARG
    assert _err(g.set_option, C.DCP_OPT_TILE_Z, 1025) == C.DCP_E_INVALID_ARG
    g.set_option(C.DCP_OPT_TILE_Z, 16)
    assert _err(g.set_option, C.DCP_OPT_CELLS_PER_THREAD, 3) == C.DCP_E_INVALID_ARG
    assert _err(g.set_option, C.DCP_OPT_MAP_UNROLL, 9) == C.DCP_E_INVALID_ARG
    g.set_option(C.DCP_OPT_MAP_UNROLL, 3)
    g.set_option(C.DCP_OPT_CELLS_PER_THREAD, 2)
    g.set_option(C.DCP_OPT_TIME_TILE_DEPTH, 3)
    g.fuse(0)
    assert _err(g.set_option, C.DCP_OPT_TIME_TILE_DEPTH, 2) == C.DCP_E_STATE


def test_null_handles():
    lib = C.load()
    assert lib.dcp_add_input(None, 1, 1, None, None) == C.DCP_E_INVALID_ARG
    assert "NULL" in C.dcp_last_error()
    assert lib.dcp_graph_destroy(None) == C.DCP_OK
    assert lib.dcp_run(None, None, None, None) == C.DCP_E_INVALID_ARG


def test_plan_map_reduce():
    g = programs.map_reduce(1 << 20, "f32", fuse=C.DCP_FUSE_ALL)
    p = g.plan()
    assert p["n_launches"] == 1 and len(p["groups"]) == 1
    grp = p["groups"][0]
    assert grp["members"] == 8 and grp["reductions"] == 2 and grp["stores"] == 0
    assert grp["loads"] == 3 and p["transient_bytes"] == 0
    g0 = programs.map_reduce(1 << 20, "f32", fuse=0)
    p0 = g0.plan()
    assert p0["n_launches"] == 10
    # every one of the 8 map temporaries is materialised op by op
    assert p0["transient_bytes"] == 8 * (1 << 20) * 4


def test_plan_maps_only_keeps_reductions_separate():
    g = programs.map_reduce(1000, "f64", fuse=C.DCP_FUSE_MAPS)
    p = g.plan()
    # one fused map kernel storing y, then one kernel per reduction
    assert p["n_launches"] == 3
    assert p["transient_bytes"] == 1000 * 8


def test_plan_tanh_chain_epilogues_and_loss():
    g = programs.tanh_chain((16, 16, 16), 5, fuse=C.DCP_FUSE_ALL)
    p = g.plan()
    assert len(p["groups"]) == 1
    grp = p["groups"][0]
    # 5 tanh epilogues, and the loss's square folds into the last step's epilogue
    assert grp["kind"] == "stencil" and grp["steps"] == 5 and grp["epilogue_ops"] == 6
    assert grp["post"] == 0 and grp["reductions"] == 1 and grp["stores"] == 0
    assert p["n_launches"] == 5 and p["transient_bytes"] == 0


def test_plan_prologue_fusion():
    g = Graph()
    u = g.input("f64", (64, 64))
    w = g.input("f64", (64, 64))
    v = g.map("mul", [g.map("exp", [u]), w])
    g.output(g.stencil(v, programs.FIVE_POINT, programs.FIVE_WEIGHTS, "periodic", 3))
    g.fuse(C.DCP_FUSE_ALL)
    p = g.plan()
    assert len(p["groups"]) == 1
    assert p["groups"][0]["members"] == 2 and p["groups"][0]["loads"] == 2


def test_plan_time_tile_depth():
    g = programs.jacobi2d((300, 300), 10, "zero", "f32")
    g.set_option(C.DCP_OPT_TIME_TILE_DEPTH, 4)
    assert g.fuse(C.DCP_FUSE_ALL) == 3
    g = programs.jacobi2d((300, 300), 10, "zero", "f32", fuse=C.DCP_FUSE_SUBGRAPH)
    assert g.n_kernels == 10  # no time tiling without the flag


def test_plan_batch():
    g = programs.batch2d([33, 64, 100, 512], 20, fuse=C.DCP_FUSE_ALL | C.DCP_BATCH)
    p = g.plan()
    assert len(p["groups"]) == 1 and p["groups"][0]["kind"] == "batch"
    assert p["groups"][0]["instances"] == 4


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32", "i64"])
def test_every_op_compiles(dtype):
    g = Graph()
    a = g.input(dtype, (33,))
    b = g.input(dtype, (33,))
    s = g.input(dtype, ())
    v = a
    ops = ["neg", "abs", "square", "add", "sub", "mul", "max", "min", "add_s", "mul_s", "sub_s",
           "rsub_s"]
    if dtype.startswith("f"):
        ops += ["exp", "sin", "cos", "tanh", "sqrt", "div"]
    for op in ops:
        if op in ("add", "sub", "mul", "max", "min", "div"):
            v = g.map(op, [v, b])
        elif op.endswith("_s"):
            v = g.map(op, [v], 3.0)
        else:
            v = g.map(op, [v])
    v = g.map("add", [v, s])
    g.output(v)
    for red in ("sum", "max", "min", "maxabs"):
        g.output(g.reduce(v, red))
    assert g.fuse(C.DCP_FUSE_ALL) == 1


@pytest.mark.parametrize("bc", ["zero", "periodic", "fixed_ring"])
@pytest.mark.parametrize("shape", [(50,), (20, 30), (9, 10, 11)])
def test_stencil_kernels_compile(bc, shape):
    nd = len(shape)
    offs = [tuple([0] * nd), tuple([1] + [0] * (nd - 1)), tuple([0] * (nd - 1) + [-2])]
    for dtype in ("f32", "f64"):
        g = Graph()
        u = g.input(dtype, shape)
        v = g.map("sin", [u])
        st = g.stencil(v, offs, [0.5, 0.25, 0.25], bc, 3)
        t = g.map("tanh", [st])
        g.output(g.reduce(g.map("square", [t]), "sum"))
        g.output(t)
        g.fuse(C.DCP_FUSE_ALL)


def test_plan_3d_tile_options():
    g = programs.heat3d((40, 24, 64), 2, "periodic", "f64")
    g.set_option(C.DCP_OPT_TILE_Z, 16)
    g.set_option(C.DCP_OPT_TILE_Y, 4)
    g.set_option(C.DCP_OPT_TILE_X, 64)
    g.fuse(C.DCP_FUSE_ALL)
    (grp,) = [x for x in g.plan()["groups"] if x["kind"] == "stencil"]
    assert grp["tile"] == [16, 4, 64]


def test_axis_reduce_shapes_and_errors():
    g = Graph()
    x = g.input("f32", (3, 4, 5))
    assert g.shape[g.reduce(x, "sum", axis=1)] == (3, 5)
    assert g.shape[g.reduce(x, "max", axis=-1)] == (3, 4)
    with pytest.raises(DcpError) as e:
        g.reduce(x, "sum", axis=3)
    assert e.value.status == C.DCP_E_INVALID_ARG
    s = g.reduce(x, "sum")
    with pytest.raises(DcpError) as e:
        g.reduce(s, "sum", axis=0)
    assert e.value.status == C.DCP_E_SHAPE
    z = g.input("f32", (0, 4))
    with pytest.raises(DcpError) as e:
        g.reduce(z, "max", axis=0)
    assert e.value.status == C.DCP_E_SHAPE
    g.reduce(z, "sum", axis=0)


def test_plan_axis_reduce_fusion():
    g = Graph()
    x = g.input("f64", (8, 9))
    y = g.map("square", [x])
    g.output(g.reduce(y, "sum", axis=0))
    g.output(g.reduce(y, "max", axis=0))
    g.output(g.reduce(x, "min", axis=1))
    assert g.fuse(C.DCP_FUSE_ALL) == 2
    k = [(gr["kind"], gr["axis"], gr["members"], gr["reductions"]) for gr in g.plan()["groups"]]
    assert k == [("axis_reduce", 0, 1, 2), ("axis_reduce", 1, 0, 1)]
    # a value also needed elsewhere stays a map group of its own
    g = Graph()
    x = g.input("f64", (8, 9))
    y = g.map("square", [x])
    g.output(y)
    g.output(g.reduce(y, "sum", axis=1))
    assert g.fuse(C.DCP_FUSE_ALL) == 2
    assert [gr["kind"] for gr in g.plan()["groups"]] == ["map", "axis_reduce"]


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32", "i64"])
def test_every_kernel_family_compiles(dtype):
    """dcp_fuse generates and NVRTC-compiles (for sm_103a, no GPU needed)
    every kernel family the dtype supports: fused maps with full and axis
    reductions, and for floating types 1-D / 2-D / 3-D stencils under every
    boundary rule and kernel form, batches and the reverse-pass maps."""
    g = Graph()
    x = g.input(dtype, (6, 7, 8))
    y = g.map("add", [g.map("mul", [x, x]), x])
    g.output(g.reduce(y, "sum"))
    g.output(g.reduce(y, "max", axis=0))
    g.output(g.reduce(y, "min", axis=1))
    g.output(g.reduce(y, "maxabs", axis=2))
    g.output(g.reduce(x, "sum", axis=-1))
    g.fuse(C.DCP_FUSE_ALL)
    g0 = Graph()
    x0 = g0.input(dtype, (6, 7))
    g0.output(g0.reduce(g0.map("neg", [x0]), "sum", axis=1))
    g0.fuse(0)
    if dtype.startswith("i"):
        return
    for bc in ("zero", "periodic", "fixed_ring"):
        for kernel in (0, 1):
            for shape, offs in (((40,), [(-1,), (0,), (1,)]),
                                ((20, 30), [(0, 0), (0, -1), (0, 1), (1, 0), (-1, 0)]),
                                ((20, 30), [(0, 0), (0, -2), (0, 2), (2, 0), (-2, 0)])):
                g = Graph()
                v = g.input(dtype, shape)
                s = g.map("tanh", [g.stencil(g.map("abs", [v]), offs, [0.2] * len(offs), bc, 3)])
                g.output(g.reduce(g.stencil(s, offs, [0.2] * len(offs), bc, 2), "sum"))
                g.set_option(C.DCP_OPT_STENCIL_KERNEL, kernel)
                g.fuse(C.DCP_FUSE_ALL)
        programs.heat3d((9, 10, 11), 2, bc, dtype, fuse=C.DCP_FUSE_ALL)
        g = programs.heat3d((9, 10, 11), 2, bc, dtype)
        g.set_option(C.DCP_OPT_CELLS_PER_THREAD, 2)
        g.fuse(C.DCP_FUSE_ALL)
    programs.batch2d([5, 40, 70], 6, "zero", dtype, fuse=C.DCP_FUSE_ALL | C.DCP_BATCH)
    programs.tanh_chain((8, 9, 10), 2, "periodic", dtype, fuse=C.DCP_FUSE_ALL)


def test_math64_constants_are_the_generated_roundings():
    """k_math64.cuh holds exactly what its generator computes in 200-bit
    arithmetic (2^(j/64), the split ln2/64 and pi/2, 1/n!), and the values
    are the ones the mathematics fixes: the table's entries double from j to
    j + 64, the splits sum to the constants, the Taylor coefficients
    alternate in sign as 1/n! does."""
    mpmath = pytest.importorskip("mpmath")
    import importlib.util
    import math
    from fractions import Fraction
    kdir = os.path.join(os.path.dirname(C.__file__), "csrc", "kernels")
    spec = importlib.util.spec_from_file_location("gen_math64_constants",
                                                  os.path.join(kdir, "gen_math64_constants.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    text = open(os.path.join(kdir, "k_math64.cuh")).read()
    a = text.index("// BEGIN generated")
    b = text.index("// END generated")
    assert text[a:b] + "// END generated by gen_math64_constants.py\n" == gen.block()
    c = gen.constants()
    tab = c["DCP_M64_EXP_TAB"]
    assert tab[0] == 1.0 and tab[32] == float.fromhex("0x1.6a09e667f3bcdp+0")  # sqrt(2)
    assert all(abs(tab[j] * tab[64 - j] - 2.0) <= 4 * math.ulp(2.0) for j in range(1, 64))
    assert all(1.0 <= t < 2.0 for t in tab) and tab == sorted(tab)
    mpmath.mp.prec = 200
    hi, lo = c["DCP_M64_L"]
    assert abs(Fraction(hi) + Fraction(lo) - gen.to_fraction(mpmath.log(2) / 64)) < Fraction(1, 2 ** 110)
    p1, p2, p3 = c["DCP_M64_PIO2"]
    assert p1 == math.pi / 2
    assert abs(Fraction(p1) + Fraction(p2) + Fraction(p3) - gen.to_fraction(mpmath.pi / 2)) < Fraction(1, 2 ** 160)
    assert c["DCP_M64_SIN_TAYLOR"][0] == -1 / 6 and c["DCP_M64_COS_TAYLOR"][0] == -0.5
    for k, v in enumerate(c["DCP_M64_SIN_TAYLOR"], start=1):
        assert v == float(Fraction((-1) ** k, math.factorial(2 * k + 1)))
    for k, v in enumerate(c["DCP_M64_COS_TAYLOR"], start=1):
        assert v == float(Fraction((-1) ** k, math.factorial(2 * k)))


def test_plan_deferred_common_weight():
    """Linear runs of f64 steps with weights f * r_k (r_k exact) run on the
    ratios and apply f^m at the end of every chunk of m <= D steps,
    (sum |r_k|)^D <= 2^32: D = 9 for the 7-point heat stencil (0.4 = 4 * 0.1,
    sum of ratios 10), 13 for the 5-point average.  Fixed rings, single
    steps, f32 and weights without exact ratios keep the plain weighted sum
    (no "deferred_scales" in the launch)."""
    def scales(g):
        out = []
        for l in g.plan()["launches"]:
            out += l.get("deferred_scales", [None] * (l["steps"][1] - l["steps"][0]))
        return out

    sc = scales(programs.heat3d((8, 9, 10), 23, "periodic", "f64", fuse=C.DCP_FUSE_ALL))
    chunk_ends = {8: 1e-9, 17: 1e-9, 22: 1e-5}
    assert len(sc) == 23
    for i, s in enumerate(sc):
        assert s == pytest.approx(chunk_ends.get(i, 1.0), rel=1e-15), (i, s)
    assert scales(programs.heat3d((8, 9, 10), 18, "zero", "f64", fuse=C.DCP_FUSE_ALL))[-1] == \
        pytest.approx(1e-9, rel=1e-15)
    # 2-D, every kernel form and time-tile depth: the same per-step plan
    for kernel in (0, 1):
        for depth in (1, 3, 10):
            g = programs.jacobi2d((40, 50), 30, "zero", "f64")
            g.set_option(C.DCP_OPT_STENCIL_KERNEL, kernel)
            g.set_option(C.DCP_OPT_TIME_TILE_DEPTH, depth)
            g.fuse(C.DCP_FUSE_ALL)
            sc = scales(g)
            assert len(sc) == 30
            for i, s in enumerate(sc):
                want = 0.2 ** 13 if i in (12, 25) else (0.2 ** 4 if i == 29 else 1.0)
                assert s == pytest.approx(want, rel=1e-14), (kernel, depth, i, s)
    for g in (programs.heat3d((8, 9, 10), 5, "fixed_ring", "f64", fuse=C.DCP_FUSE_ALL),
              programs.heat3d((8, 9, 10), 1, "periodic", "f64", fuse=C.DCP_FUSE_ALL),
              programs.heat3d((8, 9, 10), 5, "periodic", "f32", fuse=C.DCP_FUSE_ALL),
              programs.jacobi2d((40, 50), 10, "zero", "f32", fuse=C.DCP_FUSE_ALL),
              programs.jacobi2d((40, 50), 10, "fixed_ring", "f64", fuse=C.DCP_FUSE_ALL),
              programs.tanh_chain((8, 9, 10), 3, fuse=C.DCP_FUSE_ALL)):
        assert all(s is None for s in scales(g))
    g = Graph()
    x = g.input("f64", (8, 9, 10))
    g.output(g.stencil(x, programs.SEVEN_POINT, [0.3] + [0.7 / 6] * 6, "zero", 4))
    g.fuse(C.DCP_FUSE_ALL)
    assert all(s is None for s in scales(g))
    # negative weights: f = -0.125 (the most frequent), ratios -4 and 1
    g = Graph()
    x = g.input("f64", (30, 40))
    g.output(g.stencil(x, programs.FIVE_POINT, [0.5, -0.125, -0.125, -0.125, -0.125], "periodic", 5))
    g.fuse(C.DCP_FUSE_ALL)
    assert scales(g) == [1.0] * 4 + [pytest.approx((-0.125) ** 5, rel=1e-15)]
    # one point: the steps are copies and the factor w^T comes once; a factor
    # that would underflow keeps the plain sum
    for T, deferred in ((10, True), (2000, False)):
        g = Graph()
        x = g.input("f64", (30, 40))
        g.output(g.stencil(x, [(0, 0)], [0.5], "zero", T))
        g.fuse(C.DCP_FUSE_ALL)
        sc = scales(g)
        assert (sc[-1] == pytest.approx(0.5 ** T, rel=1e-15)) if deferred else all(v is None for v in sc)
    # a fused chain of equal one-step nodes is one run, like one five-step node
    g = Graph()
    v = g.input("f64", (8, 9, 10))
    for _ in range(5):
        v = g.stencil(v, programs.SEVEN_POINT, programs.SEVEN_WEIGHTS, "periodic", 1)
    g.output(v)
    g.fuse(C.DCP_FUSE_ALL)
    assert scales(g)[:4] == [1.0] * 4 and scales(g)[4] == pytest.approx(1e-5, rel=1e-15)


def test_deferred_weight_option_and_run_start():
    """DCP_OPT_DEFERRED_WEIGHT = 0 (before dcp_fuse) keeps the plain weighted
    sum everywhere; the option takes 0 or 1 only and is frozen by dcp_fuse.
    A run of equal steps after a step of other weights is deferred too (its
    chunk ends count from the run's own first step)."""
    def scales(g):
        out = []
        for l in g.plan()["launches"]:
            out += l.get("deferred_scales", [None] * (l["steps"][1] - l["steps"][0]))
        return out

    g = programs.heat3d((8, 9, 10), 12, "periodic", "f64")
    g.set_option(C.DCP_OPT_DEFERRED_WEIGHT, 0)
    g.fuse(C.DCP_FUSE_ALL)
    assert all(s is None for s in scales(g))
    with pytest.raises(C.DcpError) as e:
        g.set_option(C.DCP_OPT_DEFERRED_WEIGHT, 1)
    assert e.value.status == C.DCP_E_STATE
    g = programs.heat3d((8, 9, 10), 12, "periodic", "f64")
    with pytest.raises(C.DcpError):
        g.set_option(C.DCP_OPT_DEFERRED_WEIGHT, 2)
    g = Graph()
    v = g.input("f64", (8, 9, 10))
    v = g.stencil(v, programs.SEVEN_POINT, [0.3] + [0.7 / 6] * 6, "periodic", 1)
    for _ in range(4):
        v = g.stencil(v, programs.SEVEN_POINT, programs.SEVEN_WEIGHTS, "periodic", 1)
    g.output(v)
    g.fuse(C.DCP_FUSE_ALL)
    assert scales(g)[0] is None and scales(g)[1:4] == [1.0] * 3
    assert scales(g)[4] == pytest.approx(1e-4, rel=1e-15)


def _chain2d(shape, steps, bc, dtype, epi=("tanh",), depth=None, radius2=False):
    offs = programs.FIVE_POINT if not radius2 else [(0, 0), (0, -2), (0, 2), (2, 0), (-2, 0)]
    g = Graph()
    u = g.input(dtype, shape)
    for _ in range(steps):
        u = g.stencil(u, offs, programs.FIVE_WEIGHTS, bc, 1)
        for e in epi:
            u = g.map(e, [u])
    g.output(g.reduce(g.map("square", [u]), "sum"))
    if depth is not None:
        g.set_option(C.DCP_OPT_ADJOINT_DEPTH, depth)
    g.fuse(C.DCP_FUSE_ALL)
    return g


def _adj_kernels(plan, prefix):
    return [l for l in plan["adjoint"]["launches"] if l["kernel"].startswith(prefix)]


def test_plan_time_tiled_reverse():
    """dcp_prepare_adjoint plans and compiles the reverse pass without a GPU.
    A float32 2-D tanh chain of 10 steps with DCP_OPT_ADJOINT_DEPTH = 4 runs
    its reverse in chunks of 4: the forward pass stores only u_4 and u_8 and
    stops there (the last chunk's states are recomputed in its tile), the
    reverse is one broadcast of the loss cotangent and 3 chunk launches
    (2 + 4 + 4 steps).  The default (0) is one launch per step and the full
    tape."""
    state = 64 * 80 * 4
    p = _chain2d((64, 80), 10, "periodic", "f32", depth=4).prepare_adjoint()
    a = p["adjoint"]
    assert a["tape_bytes"] == 2 * state and not a["checkpointed"]
    assert len(_adj_kernels(p, "dcp_adj_")) == 3
    assert [l["phase"] for l in a["launches"]] == ["forward"] * 2 + ["reverse"] * 4
    assert len(set(l["kernel"] for l in _adj_kernels(p, "dcp_adj_"))) == 2  # 2-step and 4-step
    p0 = _chain2d((64, 80), 10, "periodic", "f32").prepare_adjoint()
    assert p0["adjoint"]["tape_bytes"] == 10 * state
    assert not _adj_kernels(p0, "dcp_adj_") and len(p0["adjoint"]["launches"]) == 20


def test_plan_time_tiled_reverse_rules():
    """3-D chains and chains linear up to their last step never take the
    tiled form; every 1-D / 2-D form compiles for both boundaries, radius 2
    and epilogues whose reverse needs the pre-epilogue value."""
    p = _chain2d((30, 40), 6, "zero", "f64", depth=3).prepare_adjoint()
    assert len(_adj_kernels(p, "dcp_adj_")) == 2
    lin = _chain2d((30, 40), 6, "zero", "f32", epi=(), depth=3).prepare_adjoint()
    assert not _adj_kernels(lin, "dcp_adj_")
    g3 = programs.tanh_chain((8, 9, 10), 4, "periodic", "f32")
    g3.set_option(C.DCP_OPT_ADJOINT_DEPTH, 2)
    g3.fuse(C.DCP_FUSE_ALL)
    assert not _adj_kernels(g3.prepare_adjoint(), "dcp_adj_")
    for dt, bc, epi in (("f32", "zero", ("tanh",)), ("f32", "periodic", ("sin", "square")),
                        ("f64", "zero", ("exp", "sqrt")), ("f64", "periodic", ("abs", "cos"))):
        for shape in ((50,), (20, 30)):
            p = _chain2d(shape, 5, bc, dt, epi, depth=2,
                         radius2=len(shape) == 2 and epi[0] == "sin").prepare_adjoint()
            assert len(_adj_kernels(p, "dcp_adj_")) == 3
    g = _chain2d((20, 30), 4, "zero", "f32")
    with pytest.raises(DcpError) as e:
        g.set_option(C.DCP_OPT_ADJOINT_DEPTH, 1)  # after dcp_fuse
    assert e.value.status == C.DCP_E_STATE
    g = Graph()
    with pytest.raises(DcpError) as e:
        g.set_option(C.DCP_OPT_ADJOINT_DEPTH, 65)
    assert e.value.status == C.DCP_E_INVALID_ARG
    with pytest.raises(DcpError) as e:
        C.dcp_prepare_adjoint(g._h, 1 << 20)  # before dcp_fuse
    assert e.value.status == C.DCP_E_STATE


def test_plan_cooperative_form():
    """DCP_OPT_STENCIL_KERNEL = 2 plans every step of a 1-D / 2-D group as one
    cooperative launch (one thread per tile cell) and compiles it for every
    boundary; groups it cannot run are rejected on the host."""
    for bc in ("zero", "periodic", "fixed_ring"):
        for shape, tile in (((256, 256), (14, 32)), ((1000,), (1, 32))):
            g = programs.jacobi2d(shape, 10, bc, "f64") if len(shape) == 2 else Graph()
            if len(shape) == 1:
                v = g.input("f32", shape)
                g.output(g.reduce(g.stencil(g.map("tanh", [v]), [(-1,), (0,), (1,)],
                                            [0.25, 0.5, 0.25], bc, 7), "sum"))
            g.set_option(C.DCP_OPT_STENCIL_KERNEL, 2)
            g.set_option(C.DCP_OPT_TILE_Y, tile[0])
            g.set_option(C.DCP_OPT_TILE_X, tile[1])
            g.fuse(C.DCP_FUSE_ALL)
            p = g.plan()
            (grp,) = [x for x in p["groups"] if x["kind"] == "stencil"]
            assert grp["kernel_form"] == "coop" and grp["depth"] == grp["steps"]
            assert grp["threads"] == (448 if len(shape) == 2 else 64)
            assert len(p["launches"]) == 1 and p["launches"][0]["kernel"].startswith("dcp_coop_")
    g = programs.jacobi2d((64, 64), 64, "zero", "f64")  # more than 63 steps
    g.set_option(C.DCP_OPT_STENCIL_KERNEL, 2)
    assert _err(g.fuse, C.DCP_FUSE_ALL) == C.DCP_E_UNSUPPORTED
    g2 = Graph()  # an edge tile 1 row tall under a radius of 2
    v = g2.input("f64", (65, 64))
    g2.output(g2.stencil(v, [(0, 0), (2, 0), (-2, 0)], [0.5, 0.25, 0.25], "zero", 3))
    g2.set_option(C.DCP_OPT_STENCIL_KERNEL, 2)
    g2.set_option(C.DCP_OPT_TILE_Y, 16)
    assert _err(g2.fuse, C.DCP_FUSE_ALL) == C.DCP_E_UNSUPPORTED
    assert _err(Graph().set_option, C.DCP_OPT_STENCIL_KERNEL, 3) == C.DCP_E_INVALID_ARG


def test_plan_time_tiled_reverse_chain_rules():
    """Which parts of a program the tiled reverse takes (plans only): a chain
    is cut where an intermediate state is also a program output; steps may
    change weights (same offsets); a float64 chain with a step that has no
    epilogue keeps one launch per step; under a small tape budget the
    checkpointed segments run their own tiled chunks."""
    F, W = programs.FIVE_POINT, programs.FIVE_WEIGHTS

    def chain(dt, steps, out_at=None, epi_skip=None, weights=None):
        g = Graph()
        u = g.input(dt, (30, 40))
        for i in range(steps):
            u = g.stencil(u, F, (weights(i) if weights else W), "zero", 1)
            if epi_skip is None or i != epi_skip:
                u = g.map("tanh", [u])
            if out_at is not None and i == out_at:
                g.output(u)
        g.output(g.reduce(g.map("square", [u]), "sum"))
        g.set_option(C.DCP_OPT_ADJOINT_DEPTH, 3)
        g.fuse(C.DCP_FUSE_ALL)
        return g

    # an intermediate output after step 4 cuts the 9-step chain into 5 + 4
    # steps: chunks (3 + 2) and (3 + 1)
    p = chain("f32", 9, out_at=4).prepare_adjoint()
    assert len(_adj_kernels(p, "dcp_adj_")) == 4
    # per-step weights may differ
    p = chain("f32", 6, weights=lambda i: [0.2 + 0.01 * i, 0.2, 0.2, 0.2, 0.2 - 0.01 * i]).prepare_adjoint()
    assert len(_adj_kernels(p, "dcp_adj_")) == 2
    # float64: a step without an epilogue could run on a deferred common
    # weight in the forward pass, so the chain keeps the per-step reverse
    p = chain("f64", 6, epi_skip=2).prepare_adjoint()
    assert not _adj_kernels(p, "dcp_adj_")
    p = chain("f32", 6, epi_skip=2).prepare_adjoint()
    assert len(_adj_kernels(p, "dcp_adj_")) == 2
    # checkpointed: 16 steps, chunks of 3, a budget below the 5-state tape
    g = chain("f32", 16)
    state = 30 * 40 * 4
    full = g.prepare_adjoint()["adjoint"]
    assert full["tape_bytes"] == 5 * state and not full["checkpointed"]
    ck = g.prepare_adjoint(4 * state)["adjoint"]
    assert ck["checkpointed"] and ck["tape_bytes"] <= 4 * state
    assert any(l["kernel"].startswith("dcp_adj_") for l in ck["launches"] if l["phase"] == "reverse")


def test_prepare_adjoint_budget_errors():
    """dcp_prepare_adjoint reports, without a GPU, a tape budget that even
    sqrt(T) checkpointing cannot meet (DCP_E_OOM), and plans a fitting one."""
    g = programs.tanh_chain((16, 16, 16), 9, fuse=C.DCP_FUSE_ALL)
    state = 16 * 16 * 16 * 8
    with pytest.raises(DcpError) as e:
        g.prepare_adjoint(state)
    assert e.value.status == C.DCP_E_OOM
    a = g.prepare_adjoint(5 * state)["adjoint"]
    assert a["checkpointed"] and a["tape_bytes"] <= 5 * state
