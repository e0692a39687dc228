"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Floating tolerances are the mixed bounds |gpu - ref| <= tol * max(|ref|, s):
1e-12 (f64) / 1e-5 (f32) for maps and stencils, with s the magnitude scale of
the computation (for the fused map: |exp(ax+b) sin x| + |0.5 x^2|; for the
averaging stencils, whose weights are non-negative and sum to 1:
||u0||_inf); reductions use 1e-10 / 1e-4 times sum|y_i| (the backward-stable
bound of any summation order).  Integer work is compared bit-exactly.
"""
import numpy as np
import pytest

import oracle
from oracle import programs as OP
from paper_2107_00555_gb300 import Graph, inputs, programs
from paper_2107_00555_gb300 import _capi as C

from gpu_util import assert_close, red_tol_for, tol_for, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NP = {"f32": np.float32, "f64": np.float64}
FUSED = C.DCP_FUSE_ALL
OPBYOP = 0


def _map_reduce_check(dtype, n, flags, seed):
    x, a, b = inputs.cfg2(NP[dtype], seed=seed, n=n)
    prog = OP.map_reduce(n)
    vals, extra = oracle.run(prog, [x, a, b], detail=True)
    H = prog.handles
    y = vals[H["y"]]
    scale = np.abs(vals[H["p"]]) + np.abs(vals[H["h"]])
    s_id, m_id = prog.outputs
    g = programs.map_reduce(n, dtype, fuse=flags)
    out = g.run([to_dev(x), to_dev(a), to_dev(b)])
    torch.cuda.synchronize()
    s_gpu, m_gpu = float(to_host(out[0])), float(to_host(out[1]))
    tol, rtol = tol_for(dtype), red_tol_for(dtype)
    fs, sa = extra[s_id]["fsum"], extra[s_id]["abs"]
    assert abs(s_gpu - fs) <= rtol * max(sa, 1e-300), (s_gpu, fs, sa)
    m_ref = float(vals[m_id])
    assert abs(m_gpu - m_ref) <= tol * max(float(scale.max()) if n else 0.0, m_ref), (m_gpu, m_ref)
    return y, scale


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("n", [1, 3, 8, 1000, 4099, (1 << 20) + 5])
@pytest.mark.parametrize("flags", [FUSED, OPBYOP])
def test_map_reduce_small(dtype, n, flags):
    _map_reduce_check(dtype, n, flags, seed=1 + n % 3)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_map_reduce_materialised_y(dtype):
    """Same program with y also an output: elementwise check of the fused map."""
    n = 70001
    x, a, b = inputs.cfg2(NP[dtype], seed=2, n=n)
    prog = OP.map_reduce(n)
    vals = oracle.run(prog, [x, a, b])
    H = prog.handles
    scale = np.abs(vals[H["p"]]) + np.abs(vals[H["h"]])
    g = Graph()
    xv, av, bv = (g.input(dtype, (n,)) for _ in range(3))
    t = g.map("add", [g.map("mul", [av, xv]), bv])
    y = g.map("sub", [g.map("mul", [g.map("exp", [t]), g.map("sin", [xv])]),
                      g.map("mul_s", [g.map("mul", [xv, xv])], 0.5)])
    g.output(y)
    g.output(g.reduce(y, "sum"))
    assert g.fuse(FUSED) == 1
    out = g.run([to_dev(x), to_dev(a), to_dev(b)])
    assert_close(to_host(out[0]), vals[H["y"]], tol_for(dtype), scale, "y")


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_map_reduce_full_size(dtype):
    """The benchmark workload: 2**26 elements, every element against the oracle."""
    n = 1 << 26
    x, a, b = inputs.cfg2(NP[dtype], n=n)
    prog = OP.map_reduce(n)
    vals, extra = oracle.run(prog, [x, a, b], detail=True)
    H = prog.handles
    s_id, m_id = prog.outputs
    g = programs.map_reduce(n, dtype, fuse=FUSED)
    out = g.run([to_dev(x), to_dev(a), to_dev(b)])
    torch.cuda.synchronize()
    fs, sa = extra[s_id]["fsum"], extra[s_id]["abs"]
    assert abs(float(to_host(out[0])) - fs) <= red_tol_for(dtype) * sa
    scale = np.abs(vals[H["p"]]) + np.abs(vals[H["h"]])
    assert abs(float(to_host(out[1])) - float(vals[m_id])) <= tol_for(dtype) * max(
        float(scale.max()), float(vals[m_id]))


def test_reductions_deterministic():
    n = (1 << 22) + 17
    x, a, b = inputs.cfg2(np.float32, seed=3, n=n)
    g = programs.map_reduce(n, "f32", fuse=FUSED)
    d = [to_dev(x), to_dev(a), to_dev(b)]
    r1 = [to_host(t).copy() for t in g.run(d)]
    r2 = [to_host(t).copy() for t in g.run(d)]
    assert r1[0].tobytes() == r2[0].tobytes() and r1[1].tobytes() == r2[1].tobytes()


# ---------------------------------------------------------------------------
# stencils
# ---------------------------------------------------------------------------

def _stencil_check(build_dev, build_orc, shape, steps, bc, dtype, flags, seed, depth=None):
    u0 = inputs.uniform(shape, -1.0, 1.0, seed, NP[dtype])
    ref = oracle.run(build_orc(shape, steps, bc), [u0])[-1]
    g = build_dev(shape, steps, bc, dtype)
    if depth is not None:
        g.set_option(C.DCP_OPT_TIME_TILE_DEPTH, depth)
    g.fuse(flags)
    out = g.run([to_dev(u0)])
    s = float(np.max(np.abs(u0))) if u0.size else 0.0
    assert_close(to_host(out[0]), ref, tol_for(dtype), s, "stencil %s %s %s" % (shape, bc, dtype))
    return to_host(out[0])


@pytest.mark.parametrize("bc", ["zero", "periodic", "fixed_ring"])
@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (5, 7), (37, 45), (64, 200), (256, 256)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_jacobi2d(bc, shape, dtype):
    for flags, depth in ((FUSED, None), (FUSED, 3), (OPBYOP, None)):
        _stencil_check(programs.jacobi2d, OP.jacobi2d, shape, 7, bc, dtype, flags, seed=11,
                       depth=depth)


@pytest.mark.parametrize("bc", ["zero", "periodic", "fixed_ring"])
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 4, 5), (17, 19, 40), (40, 33, 70)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_heat3d(bc, shape, dtype):
    for flags in (FUSED, OPBYOP):
        _stencil_check(programs.heat3d, OP.heat3d, shape, 3, bc, dtype, flags, seed=12)


def test_jacobi2d_config1_full():
    """256 x 256 float64, zero boundary, 10 steps, U[0,1) (the small configuration),
    fused, op by op, and in the benchmark's launch configuration (autotuned,
    CUDA-graph replay, prepared call)."""
    u0 = inputs.cfg1()
    ref = oracle.run(OP.jacobi2d((256, 256), 10, "zero"), [u0])[-1]
    for flags in (FUSED, OPBYOP):
        g = programs.jacobi2d((256, 256), 10, "zero", "f64", fuse=flags)
        out = g.run([to_dev(u0)])
        assert_close(to_host(out[0]), ref, 1e-12, float(u0.max()), "cfg1")
    g = programs.jacobi2d((256, 256), 10, "zero", "f64")
    g.set_option(C.DCP_OPT_USE_GRAPH, 1)
    g.fuse(FUSED | C.DCP_AUTOTUNE)
    call = g.prepare([to_dev(u0)])
    for _ in range(3):  # tuning run, eager run, graph replay
        out = call()
        assert_close(to_host(out[0]), ref, 1e-12, float(u0.max()), "cfg1 bench form")


def test_map_reduce_rows_full_size_sampled_rows():
    """8192 x 8192 float32, the row-reduced program as the benchmark runs it;
    sampled rows against the oracle run on just those rows (each row's
    results depend on that row only)."""
    shape = (8192, 8192)
    x, a, b = (v.reshape(shape) for v in inputs.cfg2(np.float32, n=shape[0] * shape[1]))
    g = programs.map_reduce(shape, "f32", fuse=FUSED, axis=1)
    dev = [to_dev(v) for v in (x, a, b)]
    s, m = (to_host(o).astype(np.float64) for o in g.prepare(dev)())
    rows = [0, 1, 4095, 8191] + list(range(17, 8192, 1021))
    sub = [v[rows] for v in (x, a, b)]
    prog = OP.map_reduce((len(rows), shape[1]), axis=1)
    vals, extra = oracle.run(prog, sub, detail=True)
    sid, mid = prog.outputs
    assert np.all(np.abs(s[rows] - extra[sid]["fsum"]) <= 1e-4 * extra[sid]["abs"])
    H = prog.handles
    scale = oracle.reduce_axis("maxabs", np.abs(vals[H["p"]]) + np.abs(vals[H["h"]]), 1)
    assert np.all(np.abs(m[rows] - vals[mid]) <= 1e-5 * np.maximum(vals[mid], scale))


def test_time_tiling_is_bit_exact():
    """k steps per launch give bit-identical results to one step per launch."""
    u0 = inputs.uniform((300, 257), 0.0, 1.0, 5)
    res = []
    for depth in (1, 2, 5):
        g = programs.jacobi2d((300, 257), 10, "zero", "f64")
        g.set_option(C.DCP_OPT_TIME_TILE_DEPTH, depth)
        g.fuse(FUSED)
        res.append(to_host(g.run([to_dev(u0)])[0]).copy())
    assert res[0].tobytes() == res[1].tobytes() == res[2].tobytes()


def test_jacobi1d_paper_form():
    u0 = inputs.uniform((1000,), 0.0, 1.0, 9)
    offs, w = [(-1,), (0,), (1,)], [0.33333] * 3
    p = oracle.Program()
    v = p.input("f64", (1000,))
    p.output(p.stencil(v, offs, w, "fixed_ring", 12))
    ref = oracle.run(p, [u0])[-1]
    g = Graph()
    v = g.input("f64", (1000,))
    g.output(g.stencil(v, offs, w, "fixed_ring", 12))
    g.fuse(FUSED)
    assert_close(to_host(g.run([to_dev(u0)])[0]), ref, 1e-12, 1.0, "jacobi1d")


@pytest.mark.parametrize("shape", [(70, 20, 28), (100, 9, 33), (33, 40, 65)])
@pytest.mark.parametrize("tz", [None, 16])
def test_stencil3d_fused_loss_over_many_z_chunks(shape, tz):
    """A 3-D stencil chain with a fused reduction whose grid spans several
    z-chunks: the cross-block pass must number blocks over the whole grid.
    Repeated runs must agree bitwise (the ticket is reset for the next run)."""
    T = 3
    u0 = inputs.uniform(shape, -1.0, 1.0, 31)
    prog = OP.tanh_chain(shape, T)
    vals, extra = oracle.run(prog, [u0], detail=True)
    (lid,) = prog.outputs
    g = programs.tanh_chain(shape, T)
    if tz is not None:
        g.set_option(C.DCP_OPT_TILE_Z, tz)
        g.set_option(C.DCP_OPT_TILE_Y, 4)
        g.set_option(C.DCP_OPT_TILE_X, 64)
    g.fuse(FUSED)
    plan = g.plan()
    assert len(plan["launches"]) == T
    d = to_dev(u0)
    got = [float(to_host(g.run([d])[0])) for _ in range(3)]
    assert got[0] == got[1] == got[2]
    fs, sa = extra[lid]["fsum"], extra[lid]["abs"]
    assert abs(got[0] - fs) <= 1e-10 * sa, (got[0], fs, sa)


@pytest.mark.parametrize("shape", [(1, 1000), (1000, 1), (5, 7), (37, 45), (300, 257), (130, 1030)])
@pytest.mark.parametrize("bc", ["zero", "fixed_ring"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_stream_kernel_options_bitwise(shape, bc, dtype):
    """The warp-stream kernel under several depths, prefetch depths, CTA sizes
    and rows per work item reproduces the one-step tile kernel bit for bit,
    and the oracle within tolerance."""
    T = 10
    u0 = inputs.uniform(shape, 0.0, 1.0, 33, NP[dtype])
    build = programs.jacobi2d
    ref = oracle.run(OP.jacobi2d(shape, T, bc), [u0])[-1]
    g0 = build(shape, T, bc, dtype)
    g0.set_option(C.DCP_OPT_STENCIL_KERNEL, 0)
    g0.set_option(C.DCP_OPT_TIME_TILE_DEPTH, 1)
    g0.fuse(FUSED)
    base = to_host(g0.run([to_dev(u0)])[0])
    assert_close(base, ref, tol_for(dtype), float(np.max(u0)), "tile kernel")
    for depth, pf, th, rows in ((3, 1, 128, None), (5, 2, 64, 17), (10, 2, 32, 1), (4, 4, 256, 300)):
        g = build(shape, T, bc, dtype)
        g.set_option(C.DCP_OPT_STENCIL_KERNEL, 1)
        g.set_option(C.DCP_OPT_TIME_TILE_DEPTH, depth)
        g.set_option(C.DCP_OPT_STREAM_PREFETCH, pf)
        g.set_option(C.DCP_OPT_STREAM_THREADS, th)
        if rows is not None:
            g.set_option(C.DCP_OPT_STREAM_ROWS, rows)
        g.fuse(FUSED)
        (grp,) = g.plan()["groups"]
        if grp["kernel_form"] != "stream":
            continue  # too narrow a strip for this depth: tile kernel chosen
        got = to_host(g.run([to_dev(u0)])[0])
        assert got.tobytes() == base.tobytes(), (depth, pf, th, rows)


@pytest.mark.parametrize("bc", ["zero", "periodic", "fixed_ring"])
@pytest.mark.parametrize("shape", [(17, 19, 40), (40, 33, 71), (5, 9, 2)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_heat3d_paired_cells_bitwise(bc, shape, dtype):
    """Two cells per thread along x give the bits of one cell per thread."""
    u0 = inputs.uniform(shape, -1.0, 1.0, 17, NP[dtype])
    res = []
    for cx, tile in ((1, None), (2, None), (2, (4, 16, 32)), (2, (8, 4, 64))):
        g = programs.heat3d(shape, 3, bc, dtype)
        g.set_option(C.DCP_OPT_CELLS_PER_THREAD, cx)
        if tile is not None:
            g.set_option(C.DCP_OPT_TILE_Z, tile[0])
            g.set_option(C.DCP_OPT_TILE_Y, tile[1])
            g.set_option(C.DCP_OPT_TILE_X, tile[2])
        g.fuse(FUSED)
        assert g.plan()["groups"][0]["cells_per_thread"] == cx
        res.append(to_host(g.run([to_dev(u0)])[0]).tobytes())
    assert all(r == res[0] for r in res)


@pytest.mark.parametrize("bc", ["zero", "periodic"])
def test_heat3d_deferred_weight_chunks_magnitudes_nan(bc):
    """23 steps run as chunks of 9, 9 and 5 on the ratios 4 and 1 of the
    heat weights, the factor 0.1^m applied at each chunk's end: values near
    1e280 stay finite and within the f64 tolerance of the oracle's plain
    weighted sum, a NaN spreads over the same dependence cone, and every tile
    shape gives the same bits."""
    shape, T = (9, 10, 11), 23
    u0 = inputs.uniform(shape, -1.0, 1.0, 19) * 1e280
    ref = oracle.run(OP.heat3d(shape, T, bc), [u0])[-1]
    g = programs.heat3d(shape, T, bc, "f64", fuse=FUSED)
    assert ["deferred_scales" in l for l in g.plan()["launches"]] == [True] * T
    got = to_host(g.run([to_dev(u0)])[0])
    assert np.isfinite(got).all()
    assert_close(got, ref, 1e-12, float(np.max(np.abs(u0))), "deferred weight, 1e280 %s" % bc)
    shape = (9, 10, 60)  # long enough in x for cells outside the NaN's cone
    u1 = inputs.uniform(shape, -1.0, 1.0, 20)
    u1[4, 5, 2] = np.nan
    ref = oracle.run(OP.heat3d(shape, T, bc), [u1])[-1]
    assert 0 < np.isnan(ref).sum() < ref.size
    res = []
    for cx, tile in ((1, None), (2, None), (2, (4, 16, 32)), (1, (8, 4, 64))):
        g = programs.heat3d(shape, T, bc, "f64")
        g.set_option(C.DCP_OPT_CELLS_PER_THREAD, cx)
        if tile is not None:
            g.set_option(C.DCP_OPT_TILE_Z, tile[0])
            g.set_option(C.DCP_OPT_TILE_Y, tile[1])
            g.set_option(C.DCP_OPT_TILE_X, tile[2])
        g.fuse(FUSED)
        got = to_host(g.run([to_dev(u1)])[0])
        res.append(got.tobytes())
    assert all(r == res[0] for r in res)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    ok = ~np.isnan(ref)
    assert_close(got[ok], ref[ok], 1e-12, 1.0, "deferred weight with NaN %s" % bc)


@pytest.mark.parametrize("bc", ["zero", "periodic"])
def test_jacobi2d_deferred_weight_forms_magnitudes_nan(bc):
    """30 steps of the 5-point average run as chunks of 13, 13 and 4 on ratio
    1 (4 adds per cell), 0.2^m applied at each chunk's end, in every kernel
    form and time-tile depth: the same bits in all of them, within the f64
    tolerance of the oracle on inputs near 1e290, and NaN over the same
    dependence cone."""
    T = 30
    shape = (37, 150)
    u0 = inputs.uniform(shape, -1.0, 1.0, 21) * 1e290
    u0[5, 70] = np.nan
    ref = oracle.run(OP.jacobi2d(shape, T, bc), [u0])[-1]
    assert 0 < np.isnan(ref).sum() < ref.size
    res = []
    for kernel, depth in ((0, 1), (0, 4), (1, 1), (1, 5), (1, 13)):
        g = programs.jacobi2d(shape, T, bc, "f64")
        g.set_option(C.DCP_OPT_STENCIL_KERNEL, kernel)
        g.set_option(C.DCP_OPT_TIME_TILE_DEPTH, depth)
        g.fuse(FUSED)
        got = to_host(g.run([to_dev(u0)])[0])
        res.append(got.tobytes())
    assert all(r == res[0] for r in res)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    ok = ~np.isnan(ref)
    assert np.isfinite(got[ok]).all()
    assert_close(got[ok], ref[ok], 1e-12, 1e290, "deferred weight 2-D %s" % bc)


@pytest.mark.parametrize("prog", ["heat3d", "jacobi2d_tile", "jacobi2d_stream"])
def test_deferred_weight_guard_reports_large_inputs(prog):
    """An input above the magnitude the deferred common weight keeps finite
    (about 1.8e299 for the heat step, 1.5e299 for the 5-point average) is
    reported when the caller synchronises (DCP_E_UNSUPPORTED, naming the
    option); with DCP_OPT_DEFERRED_WEIGHT = 0 the same program runs the plain
    weighted sum and matches the oracle.  Inputs below the bound, and NaN /
    inf inputs, are not reported."""
    T = 12
    if prog == "heat3d":
        shape = (10, 12, 14)
        build = lambda: programs.heat3d(shape, T, "periodic", "f64")
        ref_prog = OP.heat3d(shape, T, "periodic")
    else:
        shape = (40, 70)
        kernel = 0 if prog == "jacobi2d_tile" else 1

        def build():
            g = programs.jacobi2d(shape, T, "zero", "f64")
            g.set_option(C.DCP_OPT_STENCIL_KERNEL, kernel)
            return g
        ref_prog = OP.jacobi2d(shape, T, "zero")
    u0 = inputs.uniform(shape, -1.0, 1.0, 27)
    u0.flat[u0.size // 3] = 1e300
    g = build()
    g.fuse(FUSED)
    g.run([to_dev(u0)])
    with pytest.raises(C.DcpError) as e:
        g.sync()
    assert e.value.status == C.DCP_E_UNSUPPORTED and "DCP_OPT_DEFERRED_WEIGHT" in str(e.value)
    g.sync()  # reported once
    g0 = build()
    g0.set_option(C.DCP_OPT_DEFERRED_WEIGHT, 0)
    g0.fuse(FUSED)
    assert all("deferred_scales" not in l for l in g0.plan()["launches"])
    got = to_host(g0.run([to_dev(u0)])[0])
    g0.sync()
    ref = oracle.run(ref_prog, [u0])[-1]
    assert_close(got, ref, 1e-12, 1e300, "plain sum on 1e300 inputs, %s" % prog)
    # below the bound, and with NaN / inf: nothing to report
    u1 = inputs.uniform(shape, -1.0, 1.0, 28) * 1e298
    u1.flat[7] = np.nan
    u1.flat[11] = np.inf
    g.run([to_dev(u1)])
    g.sync()


def test_deferred_weight_guard_host_runs():
    """The host-buffer entry point waits for its stream and so reports the
    magnitude guard itself (pageable and page-locked buffers alike)."""
    shape, T = (10, 12, 14), 12
    u0 = inputs.uniform(shape, -1.0, 1.0, 29)
    u0[2, 3, 4] = -1e300
    g = programs.heat3d(shape, T, "periodic", "f64", fuse=FUSED)
    with pytest.raises(C.DcpError) as e:
        g.run_host([u0])
    assert e.value.status == C.DCP_E_UNSUPPORTED
    u1 = inputs.uniform(shape, -1.0, 1.0, 30)
    out = g.run_host([u1])[0]
    ref = oracle.run(OP.heat3d(shape, T, "periodic"), [u1])[-1]
    assert_close(out, ref, 1e-12, 1.0, "host run below the bound")


def test_radius2_3d_stencil_paired_cells():
    shape = (12, 14, 37)
    offs = [(0, 0, 0), (0, 0, -2), (0, 0, 2), (0, -2, 0), (0, 2, 0), (-2, 0, 0), (2, 0, 0),
            (0, 0, -1), (0, 1, 1)]
    w = [0.3, 0.1, 0.1, 0.1, 0.1, 0.1, 0.1, 0.05, 0.05]
    u0 = inputs.uniform(shape, -1.0, 1.0, 18)
    p = oracle.Program()
    v = p.input("f64", shape)
    p.output(p.stencil(v, offs, w, "zero", 2))
    ref = oracle.run(p, [u0])[-1]
    for cx in (1, 2):
        g = Graph()
        x = g.input("f64", shape)
        g.output(g.stencil(x, offs, w, "zero", 2))
        g.set_option(C.DCP_OPT_CELLS_PER_THREAD, cx)
        g.fuse(FUSED)
        assert_close(to_host(g.run([to_dev(u0)])[0]), ref, 1e-12, 1.0, "radius-2 3-D cx=%d" % cx)


def test_tanh_chain_paired_cells_loss():
    shape, T = (33, 20, 50), 3
    u0 = inputs.uniform(shape, -1.0, 1.0, 19)
    out = []
    for cx in (1, 2):
        g = programs.tanh_chain(shape, T)
        g.set_option(C.DCP_OPT_CELLS_PER_THREAD, cx)
        g.fuse(FUSED)
        out.append(float(to_host(g.run([to_dev(u0)])[0])))
    prog = OP.tanh_chain(shape, T)
    vals, extra = oracle.run(prog, [u0], detail=True)
    (lid,) = prog.outputs
    for v in out:
        assert abs(v - extra[lid]["fsum"]) <= 1e-10 * extra[lid]["abs"]


def _heat3d_full(u0_host, flags=FUSED | C.DCP_AUTOTUNE):
    """The 512^3, 50-step periodic 3-D workload as the benchmark launches it
    (autotuned kernel form and tiles)."""
    n = u0_host.shape[0]
    g = programs.heat3d((n, n, n), 50, "periodic", "f64", fuse=flags)
    d = to_dev(u0_host)
    out = g.run([d])[0]
    torch.cuda.synchronize()
    return g, d, out


def test_config3_full_size_fourier_mode():
    """A periodic Fourier mode is an eigenvector of the 7-point step:
    S cos(2 pi k.p / n) = lam cos(...), lam = 0.4 + 0.2 (cos tx + cos ty + cos tz),
    so after 50 steps every one of the 512^3 cells equals lam^50 u0."""
    n, T = 512, 50
    k = (1, 2, 3)
    ax = [np.cos(2 * np.pi * k[d] * np.arange(n) / n) for d in range(3)]
    th = [2 * np.pi * k[d] / n for d in range(3)]
    # separable product of per-axis modes (a product of cosines is also an eigenvector)
    u0 = (ax[0][:, None, None] * ax[1][None, :, None] * ax[2][None, None, :]).astype(np.float64)
    lam = 0.4 + 0.2 * (np.cos(th[0]) + np.cos(th[1]) + np.cos(th[2]))
    _, d, out = _heat3d_full(u0)
    want = torch.from_numpy(u0).cuda() * (lam ** T)
    err = float((out - want).abs().max())
    assert err <= 1e-12 * 1.0, err
    del d, out, want
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def test_config3_full_size_sampled_points():
    """Sampled cells of the 512^3, 50-step run against the oracle's
    dependence-cone evaluation of the same cells."""
    u0 = inputs.cfg3()
    _, d, out = _heat3d_full(u0)
    offs = programs.SEVEN_POINT
    w = programs.SEVEN_WEIGHTS
    rng = np.random.default_rng(77)
    pts = [(0, 0, 0), (511, 511, 511), (5, 300, 511)] + [tuple(int(v) for v in rng.integers(0, 512, 3))
                                                         for _ in range(2)]
    for p in pts:
        ref = oracle.stencil_point(u0, offs, w, "periodic", 50, p)
        got = float(out[p].item())
        assert abs(got - ref) <= 1e-12 * max(abs(ref), 1.0), (p, got, ref)
    del d, out
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("epi", [[("square", 0.0), ("rsub_s", 0.25)], [("mul_s", 0.5), ("add_s", 0.1)],
                                 [("tanh", 0.0)]])
@pytest.mark.parametrize("radius2", [False, True])
def test_step_epilogues_same_bits_in_every_form(dtype, epi, radius2):
    """Six steps, each followed by epilogue maps -- including ones the
    compiler could contract into a fused multiply-add (0.25 - v*v, 0.5 v +
    0.1) -- give the same bits in the tile and warp-stream kernels at
    depths 1 and 3 (zero boundary, radius 1 and 2)."""
    offs = ([(0, 0), (0, -2), (0, -1), (0, 1), (0, 2), (-2, 0), (-1, 0), (1, 0), (2, 0)]
            if radius2 else programs.FIVE_POINT)
    w = [0.36, 0.05, 0.12, 0.14, -0.03, 0.06, 0.11, 0.13, 0.06] if radius2 else programs.FIVE_WEIGHTS
    shape = (40, 41)
    x = inputs.uniform(shape, -1.0, 1.0, 3, NP[dtype])
    res = {}
    for kernel in (0, 1):
        for depth in (1, 3):
            g = Graph()
            u = g.input(dtype, shape)
            for _ in range(6):
                u = g.stencil(u, offs, w, "zero", 1)
                for op, imm in epi:
                    u = g.map(op, [u], imm)
            g.output(u)
            g.set_option(C.DCP_OPT_STENCIL_KERNEL, kernel)
            g.set_option(C.DCP_OPT_TIME_TILE_DEPTH, depth)
            g.fuse(FUSED)
            res[(g.plan()["groups"][0]["kernel_form"], depth)] = to_host(g.run([to_dev(x)])[0]).tobytes()
    assert {f for f, _ in res} == {"tile", "stream"}
    assert len(set(res.values())) == 1
