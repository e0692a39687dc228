"""Cooperative stencil form (DCP_OPT_STENCIL_KERNEL = 2): every step of a
1-D / 2-D stencil group in one launch, one tile per resident CTA, border
rings exchanged between neighbouring tiles through device memory with
bounded flag waits.

Checked bit for bit against the shared-memory tile form (the same per-step
arithmetic), against the oracle within the dtype's tolerance, across
repeated runs and CUDA-graph replays (the per-launch epochs), with fused
prologues, epilogues and reductions; the bounded wait's error path runs by
host-side injection (DCP_FAULT=coop_wait: every wait gives up after 1000
polls, no flag is ever set late, nothing hangs)."""
import numpy as np
import pytest

import oracle
from oracle import programs as OP
from paper_2107_00555_gb300 import Graph, inputs, programs
from paper_2107_00555_gb300 import _capi as C

from gpu_util import assert_close, red_tol_for, to_dev, to_host, tol_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIVE = programs.FIVE_POINT
NINE_R2 = [(0, 0), (0, -2), (0, 2), (2, 0), (-2, 0), (1, 1), (-1, -1), (0, -1), (0, 1)]
W_R2 = [0.2, 0.1, 0.1, 0.1, 0.1, 0.1, 0.1, 0.1, 0.1]
LINE = [(0,), (-1,), (1,), (-2,)]
W_LINE = [0.4, 0.25, 0.25, 0.1]


def _build(b, shape, offs, w, bc, dtype, steps):
    """|x| -> (steps // 2) steps with a tanh epilogue each -> the rest plain;
    outputs: the final state and its sum."""
    x = b.input(dtype, shape)
    u = b.map("abs", [x])
    k = steps // 2
    for _ in range(k):
        u = b.map("tanh", [b.stencil(u, offs, w, bc, 1)])
    u = b.stencil(u, offs, w, bc, steps - k)
    b.output(u)
    b.output(b.reduce(u, "sum"))
    return b


def _run(shape, offs, w, bc, dtype, steps, form, tile=None, graph=False, runs=1, seed=41):
    g = Graph()
    _build(g, shape, offs, w, bc, dtype, steps)
    g.set_option(C.DCP_OPT_STENCIL_KERNEL, form)
    if tile is not None:
        g.set_option(C.DCP_OPT_TILE_Y, tile[0])
        g.set_option(C.DCP_OPT_TILE_X, tile[1])
    if graph:
        g.set_option(C.DCP_OPT_USE_GRAPH, 1)
    g.fuse(C.DCP_FUSE_ALL)
    plan = g.plan()
    np_dt = np.float32 if dtype == "f32" else np.float64
    x = inputs.uniform(shape, -1.0, 1.0, seed).astype(np_dt)
    outs = []
    dx = to_dev(x)
    for _ in range(runs):
        outs.append([to_host(t) for t in g.run([dx])])
    g.sync()
    return x, outs, plan


CASES = [
    # shape, offsets, weights, bc, dtype, steps, tile
    ((256, 256), FIVE, programs.FIVE_WEIGHTS, "zero", "f64", 10, (14, 32)),
    ((256, 256), FIVE, programs.FIVE_WEIGHTS, "periodic", "f64", 9, (16, 32)),
    ((100, 130), FIVE, programs.FIVE_WEIGHTS, "fixed_ring", "f64", 7, (13, 16)),
    ((70, 90), NINE_R2, W_R2, "zero", "f32", 8, (16, 32)),
    ((70, 90), NINE_R2, W_R2, "periodic", "f64", 6, (9, 16)),
    ((37, 41), FIVE, programs.FIVE_WEIGHTS, "periodic", "f32", 12, (8, 8)),
    ((5, 7), FIVE, programs.FIVE_WEIGHTS, "periodic", "f64", 5, (3, 8)),   # one tile column wraps onto itself
    ((3000,), LINE, W_LINE, "zero", "f64", 11, (1, 32)),
    ((999,), LINE, W_LINE, "periodic", "f32", 6, (1, 16)),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-%s-%s-T%d" % (c[0], c[3], c[4], c[5]))
def test_coop_matches_tile_form_and_oracle(case):
    shape, offs, w, bc, dt, steps, tile = case
    x, (got,), plan = _run(shape, offs, w, bc, dt, steps, 2, tile)
    grp = [gr for gr in plan["groups"] if gr["kind"] == "stencil"]
    assert len(grp) == 1 and grp[0]["kernel_form"] == "coop" and grp[0]["depth"] == steps
    assert sum(1 for l in plan["launches"] if l["kernel"].startswith("dcp_coop_")) == 1
    _, (ref,), _ = _run(shape, offs, w, bc, dt, steps, 0)
    assert got[0].tobytes() == ref[0].tobytes()
    p = oracle.Program()
    _build(p, shape, offs, w, bc, "f64", steps)
    vals, extra = oracle.run(p, [x.astype(np.float64)], detail=True)
    s_id = p.outputs[1]
    u_ref = vals[p.outputs[0]]
    assert_close(got[0], u_ref, tol_for(dt), float(np.max(np.abs(x))), "cooperative stencil")
    assert abs(float(got[1]) - extra[s_id]["fsum"]) <= red_tol_for(dt) * extra[s_id]["abs"]


def test_coop_config1_bitwise():
    """The 256^2 f64 ten-step average (zero boundary) on 152 tiles of 14 x 32:
    the same bits as the tile form, and the oracle's values within 1e-12."""
    g = programs.jacobi2d((256, 256), 10, "zero", "f64")
    g.set_option(C.DCP_OPT_STENCIL_KERNEL, 2)
    g.set_option(C.DCP_OPT_TILE_Y, 14)
    g.set_option(C.DCP_OPT_TILE_X, 32)
    g.fuse(C.DCP_FUSE_ALL)
    u0 = inputs.cfg1(seed=1001, n=256)
    ref = oracle.run(OP.jacobi2d((256, 256), 10, "zero"), [u0])[-1]
    g0 = programs.jacobi2d((256, 256), 10, "zero", "f64", fuse=C.DCP_FUSE_ALL)
    base = to_host(g0.run([to_dev(u0)])[0])
    got = to_host(g.run([to_dev(u0)])[0])
    assert got.tobytes() == base.tobytes()
    assert_close(got, ref, 1e-12, 1.0, "config 1, cooperative")


def test_coop_repeated_runs_and_graph_replay():
    """Ten runs in a row and ten CUDA-graph replays (each launch reads the
    epoch the previous one advanced) give identical bits."""
    args = ((120, 150), FIVE, programs.FIVE_WEIGHTS, "periodic", "f64", 9)
    _, outs, _ = _run(*args, 2, (16, 32), runs=10)
    _, gouts, _ = _run(*args, 2, (16, 32), graph=True, runs=10)
    for o in outs + gouts:
        assert o[0].tobytes() == outs[0][0].tobytes()
        assert o[1].tobytes() == outs[0][1].tobytes()


def test_coop_autotuner_keeps_the_tile_form():
    """Under DCP_AUTOTUNE the option's cooperative form is kept (the autotuner
    tunes the other forms only) and still computes the tile form's bits."""
    g = programs.jacobi2d((256, 256), 10, "zero", "f64")
    g.set_option(C.DCP_OPT_STENCIL_KERNEL, 2)
    g.set_option(C.DCP_OPT_TILE_Y, 14)
    g.set_option(C.DCP_OPT_TILE_X, 32)
    g.fuse(C.DCP_FUSE_ALL | C.DCP_AUTOTUNE)
    u0 = inputs.cfg1(seed=1001, n=256)
    got = to_host(g.run([to_dev(u0)])[0])
    again = to_host(g.run([to_dev(u0)])[0])
    g0 = programs.jacobi2d((256, 256), 10, "zero", "f64", fuse=C.DCP_FUSE_ALL)
    base = to_host(g0.run([to_dev(u0)])[0])
    assert got.tobytes() == base.tobytes() == again.tobytes()


def test_coop_bounded_wait_reports_timeout(monkeypatch):
    """DCP_FAULT=coop_wait compiles the waits with an unreachable target and a
    1000-poll limit: every wait gives up, the launch ends, and dcp_sync
    reports DCP_E_TIMEOUT once; the graph and the GPU stay usable."""
    monkeypatch.setenv("DCP_FAULT", "coop_wait")
    g = programs.jacobi2d((64, 64), 4, "zero", "f64")
    g.set_option(C.DCP_OPT_STENCIL_KERNEL, 2)
    g.set_option(C.DCP_OPT_TILE_Y, 16)
    g.set_option(C.DCP_OPT_TILE_X, 16)
    g.fuse(C.DCP_FUSE_ALL)
    monkeypatch.delenv("DCP_FAULT")
    u0 = inputs.cfg1(seed=3, n=64)
    g.run([to_dev(u0)])
    with pytest.raises(C.DcpError) as e:
        g.sync()
    assert e.value.status == C.DCP_E_TIMEOUT
    g.sync()  # reported once
    g2 = programs.jacobi2d((64, 64), 4, "zero", "f64")
    g2.set_option(C.DCP_OPT_STENCIL_KERNEL, 2)
    g2.set_option(C.DCP_OPT_TILE_Y, 16)
    g2.set_option(C.DCP_OPT_TILE_X, 16)
    g2.fuse(C.DCP_FUSE_ALL)
    ref = oracle.run(OP.jacobi2d((64, 64), 4, "zero"), [u0])[-1]
    got = to_host(g2.run([to_dev(u0)])[0])
    g2.sync()
    assert_close(got, ref, 1e-12, 1.0, "after the injected timeout")
