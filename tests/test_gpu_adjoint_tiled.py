"""Time-tiled reverse pass of 1-D / 2-D stencil chains: each launch reads a
checkpoint u_t and the cotangent of u_{t+k}, recomputes the k forward states
inside its tile and runs the k reverse steps (DCP_OPT_ADJOINT_DEPTH = k).

Checked against the oracle's op-by-op reverse pass (fp64, full tape) within
the stencil tolerance of the dtype, and bit for bit against the library's
own one-launch-per-step reverse pass (DCP_OPT_ADJOINT_DEPTH = 0): every
recomputed forward level and reverse step does the same arithmetic in the
same order as the per-step kernels."""
import numpy as np
import pytest

import oracle
from paper_2107_00555_gb300 import Graph, inputs, programs
from paper_2107_00555_gb300 import _capi as C

from gpu_util import assert_close, to_dev, to_host, tol_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIVE, W5 = programs.FIVE_POINT, programs.FIVE_WEIGHTS
# radius-2 cross with unequal, partly negative weights (its transpose differs
# from itself only through the point order)
CROSS2 = [(0, 0), (0, -2), (0, -1), (0, 1), (0, 2), (-2, 0), (-1, 0), (1, 0), (2, 0)]
WCROSS2 = [0.36, 0.05, 0.12, 0.14, -0.03, 0.06, 0.11, 0.13, 0.06]
LINE3 = [(0,), (-1,), (1,)]
WLINE3 = [0.5, 0.3, 0.2]


def _build(builder, shape, steps, offsets, weights, bc, dtype, epi, prologue=False):
    """u_{t+1} = epi(S u_t) for `steps` steps, loss = sum(u_T^2) (+ sum(x*u_T)
    when `prologue`: the chain then starts from x*x and x is read twice)."""
    p = builder
    x = p.input(dtype, shape)
    u = p.map("mul", [x, x]) if prologue else x
    for _ in range(steps):
        u = p.stencil(u, offsets, weights, bc, 1)
        for op, imm in epi:
            u = p.map(op, [u], imm)
    loss = p.reduce(p.map("square", [u]), "sum")
    p.output(loss)
    if prologue:
        p.output(p.reduce(p.map("mul", [x, u]), "sum"))
    return p


def _grads(shape, steps, offsets, weights, bc, dtype, epi, depth, prologue=False, budget=1 << 62,
           tile=None, seed=31):
    g = Graph()
    _build(g, shape, steps, offsets, weights, bc, dtype, epi, prologue)
    g.set_option(C.DCP_OPT_ADJOINT_DEPTH, depth)
    if tile is not None:
        g.set_option(C.DCP_OPT_TILE_Y, tile[0])
        g.set_option(C.DCP_OPT_TILE_X, tile[1])
    g.fuse(C.DCP_FUSE_ALL)
    np_dt = np.float32 if dtype == "f32" else np.float64
    u0 = inputs.uniform(shape, -1.0, 1.0, seed).astype(np_dt)
    outs = [np.array(1.0, dtype=np_dt)] + ([np.array(0.5, dtype=np_dt)] if prologue else [])
    (got,) = [to_host(t) for t in g.adjoint([to_dev(u0)], [to_dev(o) for o in outs],
                                            tape_budget_bytes=budget)]
    plan = g.plan()
    return u0, outs, got, plan


def _oracle(u0, outs, shape, steps, offsets, weights, bc, epi, prologue=False):
    p = oracle.Program()
    _build(p, shape, steps, offsets, weights, bc, "f64", epi, prologue)
    (ref,) = oracle.adjoint(p, [u0.astype(np.float64)], [float(o) for o in outs])
    return ref


def _reverse_kernels(plan):
    return [l for l in plan["adjoint"]["launches"]
            if l["phase"] == "reverse" and l["kernel"].startswith("dcp_adj_")]


CASES = [
    # shape, steps, offsets, weights, bc, dtype, epilogue, depth
    ((64, 80), 10, FIVE, W5, "periodic", "f32", [("tanh", 0.0)], 4),
    ((37, 53), 7, FIVE, W5, "zero", "f32", [("tanh", 0.0)], 3),
    ((45, 70), 6, FIVE, W5, "zero", "f64", [("tanh", 0.0)], 2),
    ((33, 41), 5, FIVE, W5, "periodic", "f64", [("sin", 0.0), ("mul_s", 0.9)], 5),
    ((50, 29), 9, CROSS2, WCROSS2, "zero", "f32", [("neg", 0.0), ("exp", 0.0), ("mul_s", 0.5)], 4),
    ((40, 40), 6, CROSS2, WCROSS2, "periodic", "f64", [("square", 0.0), ("rsub_s", 0.25)], 3),
    ((40, 41), 6, CROSS2, WCROSS2, "zero", "f32", [("square", 0.0), ("rsub_s", 0.25)], 3),
    ((1000,), 8, LINE3, WLINE3, "zero", "f64", [("cos", 0.0)], 3),
    ((777,), 5, LINE3, WLINE3, "periodic", "f32", [("tanh", 0.0), ("add_s", 0.1)], 8),
    ((6, 5), 7, FIVE, W5, "periodic", "f64", [("tanh", 0.0)], 4),   # halo wider than the array
    ((3, 70), 4, FIVE, W5, "zero", "f32", [("abs", 0.0), ("neg", 0.0)], 2),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-%s-%s-k%d" % (c[0], c[4], c[5], c[7]))
def test_tiled_reverse_vs_oracle_and_per_step(case):
    shape, steps, offs, w, bc, dt, epi, k = case
    u0, outs, got, plan = _grads(shape, steps, offs, w, bc, dt, epi, k)
    assert len(_reverse_kernels(plan)) == (steps + k - 1) // k
    ref = _oracle(u0, outs, shape, steps, offs, w, bc, epi)
    assert_close(got, ref, tol_for(dt), float(np.max(np.abs(ref))), "tiled reverse")
    _, _, base, plan0 = _grads(shape, steps, offs, w, bc, dt, epi, 0)
    assert not _reverse_kernels(plan0)
    assert got.tobytes() == base.tobytes()


def test_tiled_reverse_prologue_and_shared_input():
    """The chain starts from x*x and x is also read by a second output: the
    chain's cotangent is accumulated with the other contribution."""
    args = ((48, 36), 6, FIVE, W5, "periodic", "f32", [("tanh", 0.0)])
    u0, outs, got, plan = _grads(*args, 4, prologue=True)
    assert len(_reverse_kernels(plan)) == 2
    ref = _oracle(u0, outs, *args[:5], args[6], prologue=True)
    assert_close(got, ref, 1e-5, float(np.max(np.abs(ref))), "tiled reverse with prologue")
    _, _, base, _ = _grads(*args, 0, prologue=True)
    assert got.tobytes() == base.tobytes()


@pytest.mark.parametrize("tile", [(8, 16), (16, 64), (32, 8)])
def test_tiled_reverse_tile_shapes_bitwise(tile):
    args = ((70, 90), 8, FIVE, W5, "zero", "f64", [("tanh", 0.0)])
    _, _, got, _ = _grads(*args, 4, tile=tile)
    _, _, ref, _ = _grads(*args, 4)
    assert got.tobytes() == ref.tobytes()


def test_tiled_reverse_checkpointed_equals_full_tape():
    """sqrt(T) checkpoints with tiled reverse chunks give the full tape's bits.
    With chunks of 2 steps the tape keeps every 2nd state (7 of 16; the
    per-step reverse keeps all 16); a budget of 5 states cuts the chain into
    4 segments (3 checkpoints + one segment's tape)."""
    shape, steps = (40, 56), 16
    args = (shape, steps, FIVE, W5, "periodic", "f32", [("tanh", 0.0)])
    _, _, full, plan = _grads(*args, 2)
    _, _, _, plan0 = _grads(*args, 0)
    state = shape[0] * shape[1] * 4
    assert plan["adjoint"]["tape_bytes"] == 7 * state
    assert plan0["adjoint"]["tape_bytes"] == steps * state
    _, _, ck, plan_ck = _grads(*args, 2, budget=5 * state)
    assert plan_ck["adjoint"]["checkpointed"]
    assert plan_ck["adjoint"]["tape_bytes"] == 4 * state
    assert ck.tobytes() == full.tobytes()


def test_tiled_reverse_central_differences():
    """f64 2-D tanh chain: the tiled reverse pass against central differences
    of the forward program along a random direction."""
    shape, T = (40, 44), 6
    g = Graph()
    _build(g, shape, T, FIVE, W5, "zero", "f64", [("tanh", 0.0)])
    g.set_option(C.DCP_OPT_ADJOINT_DEPTH, 3)
    g.fuse(C.DCP_FUSE_ALL)
    u0 = inputs.uniform(shape, -1.0, 1.0, 33)
    (grad,) = [to_host(t) for t in g.adjoint([to_dev(u0)], [to_dev(np.array(1.0))])]
    d = np.random.default_rng(34).normal(size=shape)
    eps = 1e-6
    lp = float(to_host(g.run([to_dev(u0 + eps * d)])[0]))
    lm = float(to_host(g.run([to_dev(u0 - eps * d)])[0]))
    fd = (lp - lm) / (2 * eps)
    assert abs(fd - float(np.sum(grad * d))) <= 1e-7 * max(1.0, abs(fd))


def test_tanh_adjoint_2d_full_size_sampled():
    """The benchmark's configuration (4096^2 f32, periodic, 20 steps, 3 reverse
    steps per launch): bit for bit the per-step reverse everywhere, and the
    oracle's gradient at sampled cells.  d loss / d u0[p] depends only on u0
    within 2T cells of p (T steps forward, T back), so the oracle runs the
    same program on the 81 x 81 window around p (wrapped): its boundary's
    errors move one cell per step and never reach the centre."""
    n, T = 4096, 20
    shape = (n, n)
    g = Graph()
    _build(g, shape, T, FIVE, W5, "periodic", "f32", [("tanh", 0.0)])
    g.set_option(C.DCP_OPT_ADJOINT_DEPTH, 3)
    g.fuse(C.DCP_FUSE_ALL)
    u0 = inputs.uniform(shape, -1.0, 1.0, 1006).astype(np.float32)
    du = to_dev(u0)
    one = to_dev(np.array(1.0, dtype=np.float32))
    (got,) = [to_host(t) for t in g.adjoint([du], [one])]
    g0 = Graph()
    _build(g0, shape, T, FIVE, W5, "periodic", "f32", [("tanh", 0.0)])
    g0.fuse(C.DCP_FUSE_ALL)
    (base,) = [to_host(t) for t in g0.adjoint([du], [one])]
    assert got.tobytes() == base.tobytes()
    R = 2 * T
    rng = np.random.default_rng(35)
    pts = [(0, 0), (n - 1, n - 1), (0, n - 1), (17, 4000)] + [tuple(rng.integers(0, n, 2)) for _ in range(8)]
    p = oracle.Program()
    _build(p, (2 * R + 1, 2 * R + 1), T, FIVE, W5, "zero", "f64", [("tanh", 0.0)])
    refs, vals = [], []
    for (y, x) in pts:
        rows = np.arange(y - R, y + R + 1) % n
        cols = np.arange(x - R, x + R + 1) % n
        win = u0[np.ix_(rows, cols)].astype(np.float64)
        (gw,) = oracle.adjoint(p, [win], [1.0])
        refs.append(gw[R, R])
        vals.append(float(got[y, x]))
    refs, vals = np.array(refs), np.array(vals)
    assert_close(vals, refs, 1e-5, float(np.max(np.abs(refs))), "sampled full-size gradient")
