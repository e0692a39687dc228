"""GPU reverse pass (dcp_run_adjoint) against the oracle's reverse pass,
central finite differences of the GPU forward program, and the
full-tape / sqrt(T)-checkpoint equivalence."""
import numpy as np
import pytest

import oracle
from oracle import programs as OP
from paper_2107_00555_gb300 import Graph, inputs, programs
from paper_2107_00555_gb300 import _capi as C

from gpu_util import assert_close, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _adjoint(g, ins, out_grads, budget=1 << 62):
    return [to_host(t) for t in g.adjoint([to_dev(a) for a in ins],
                                          [to_dev(np.asarray(o)) for o in out_grads],
                                          tape_budget_bytes=budget)]


@pytest.mark.parametrize("shape,T", [((16, 16, 16), 3), ((9, 13, 20), 5)])
def test_tanh_chain_adjoint_vs_oracle(shape, T):
    u0 = inputs.uniform(shape, -1.0, 1.0, 21)
    (ref,) = oracle.adjoint(OP.tanh_chain(shape, T), [u0], [1.0])
    g = programs.tanh_chain(shape, T, fuse=C.DCP_FUSE_ALL)
    (got,) = _adjoint(g, [u0], [np.array(1.0)])
    assert_close(got, ref, 1e-12, float(np.max(np.abs(ref))), "tanh chain adjoint")


def test_linear_heat_chain_adjoint_vs_oracle():
    """loss = sum(u_T^2) for u_T = S^T u0 (12 periodic heat steps, one linear
    run): the reverse pass's transposed chain also runs on the deferred
    common weight (chunks of 9 and 3) and matches the oracle's reverse pass."""
    shape, T = (10, 12, 14), 12
    u0 = inputs.uniform(shape, -1.0, 1.0, 24)
    p = oracle.Program()
    pv = p.input("f64", shape)
    p.output(p.reduce(p.map("square", [p.stencil(pv, OP.SEVEN, OP.W7, "periodic", T)]), "sum"))
    (ref,) = oracle.adjoint(p, [u0], [1.0])
    g = Graph()
    gv = g.input("f64", shape)
    g.output(g.reduce(g.map("square", [g.stencil(gv, programs.SEVEN_POINT, programs.SEVEN_WEIGHTS,
                                                  "periodic", T)]), "sum"))
    g.fuse(C.DCP_FUSE_ALL)
    (got,) = _adjoint(g, [u0], [np.array(1.0)])
    assert_close(got, ref, 1e-12, float(np.max(np.abs(ref))), "linear heat chain adjoint")


def test_checkpointed_equals_full_tape_bitwise():
    shape, T = (20, 24, 28), 9
    u0 = inputs.uniform(shape, -1.0, 1.0, 22)
    g = programs.tanh_chain(shape, T, fuse=C.DCP_FUSE_ALL)
    (full,) = _adjoint(g, [u0], [np.array(1.0)])
    state_bytes = u0.nbytes
    (ck,) = _adjoint(g, [u0], [np.array(1.0)], budget=5 * state_bytes)
    assert full.tobytes() == ck.tobytes()
    with pytest.raises(C.DcpError) as e:
        _adjoint(g, [u0], [np.array(1.0)], budget=state_bytes)
    assert e.value.status == C.DCP_E_OOM


def test_tanh_chain_central_differences():
    shape, T = (16, 16, 16), 3
    u0 = inputs.uniform(shape, -1.0, 1.0, 23)
    g = programs.tanh_chain(shape, T, fuse=C.DCP_FUSE_ALL)
    (grad,) = _adjoint(g, [u0], [np.array(1.0)])
    rng = np.random.default_rng(5)
    d = rng.normal(size=shape)
    eps = 1e-6
    lp = float(to_host(g.run([to_dev(u0 + eps * d)])[0]))
    lm = float(to_host(g.run([to_dev(u0 - eps * d)])[0]))
    fd = (lp - lm) / (2 * eps)
    assert abs(fd - float(np.sum(grad * d))) <= 1e-7 * max(1.0, abs(fd))


@pytest.mark.parametrize("bc", ["zero", "periodic"])
def test_jacobi2d_adjoint(bc):
    shape, T = (70, 90), 6
    u0 = inputs.uniform(shape, 0.0, 1.0, 24)
    gout = inputs.uniform(shape, -1.0, 1.0, 25)
    (ref,) = oracle.adjoint(OP.jacobi2d(shape, T, bc), [u0], [gout])
    for flags in (C.DCP_FUSE_ALL, 0):
        g = programs.jacobi2d(shape, T, bc, "f64", fuse=flags)
        (got,) = _adjoint(g, [u0], [gout])
        assert_close(got, ref, 1e-12, float(np.max(np.abs(ref))), "jacobi2d adjoint")


def test_map_program_adjoint_vs_oracle():
    n = 5003
    rng = np.random.default_rng(26)
    x, a = rng.normal(size=n), rng.normal(size=n)
    ops = ["mul", "sin", "cos", "exp", "div", "max", "min", "sqrt", "tanh", "abs", "neg", "square"]
    p = oracle.Program()
    g = Graph()
    px, pa = p.input("f64", (n,)), p.input("f64", (n,))
    gx, ga = g.input("f64", (n,)), g.input("f64", (n,))

    def both(op, args, imm=0.0):
        return (p.map(op, [h[0] for h in args], imm), g.map(op, [h[1] for h in args], imm))

    X, A = (px, gx), (pa, ga)
    v = both("mul", [A, X])
    v = both("add", [v, both("sin", [X])])
    v = both("sub", [v, both("cos", [A])])
    v = both("div", [v, both("add_s", [both("exp", [X])], 1.0)])
    v = both("max", [v, both("neg", [A])])
    v = both("min", [v, both("mul_s", [X], 3.0)])
    v = both("sqrt", [both("add_s", [both("square", [v])], 0.5)])
    v = both("tanh", [both("rsub_s", [both("sub_s", [v], 0.25)], 2.0)])
    v = both("abs", [both("add", [v, both("neg", [X])])])
    s = (p.reduce(v[0], "sum"), g.reduce(v[1], "sum"))
    p.output(s[0]); g.output(s[1])
    p.output(v[0]); g.output(v[1])
    gy = rng.normal(size=n)
    ref = oracle.adjoint(p, [x, a], [0.7, gy])
    g.fuse(C.DCP_FUSE_ALL)
    got = _adjoint(g, [x, a], [np.array(0.7), gy])
    for r, gg in zip(ref, got):
        assert_close(gg, r, 1e-12, float(np.max(np.abs(r))), "map adjoint")


def test_max_min_adjoint_ties_route_to_the_selected_operand():
    """Inputs drawn from a few integers and signed zeros tie often; at a tie
    the forward pass returns b and the adjoint goes to b, on both sides.
    Each adjoint is one cotangent or a sum of two, so the match is exact."""
    n = 4099
    rng = np.random.default_rng(27)
    vals = np.array([-1.0, -0.0, 0.0, 1.0, 2.0])
    x, a = rng.choice(vals, n), rng.choice(vals, n)
    p, g = oracle.Program(), Graph()
    px, pa = p.input("f64", (n,)), p.input("f64", (n,))
    gx, ga = g.input("f64", (n,)), g.input("f64", (n,))
    for op in ("max", "min"):
        p.output(p.map(op, [px, pa]))
        g.output(g.map(op, [gx, ga]))
    gy, gz = rng.normal(size=n), rng.normal(size=n)
    ref = oracle.adjoint(p, [x, a], [gy, gz])
    g.fuse(C.DCP_FUSE_ALL)
    got = _adjoint(g, [x, a], [gy, gz])
    for r, gg in zip(ref, got):
        assert np.array_equal(gg, r)


def test_config5_adjoint_full_size():
    """256^3 float64, 20 steps of tanh(S u), loss = sum(u_T^2): GPU reverse pass
    against the oracle's reverse pass, full tape and checkpointed."""
    shape, T = (256, 256, 256), 20
    u0 = inputs.cfg5()
    (ref,) = oracle.adjoint(OP.tanh_chain(shape, T), [u0], [1.0])
    g = programs.tanh_chain(shape, T, fuse=C.DCP_FUSE_ALL)
    (got,) = _adjoint(g, [u0], [np.array(1.0)])
    assert_close(got, ref, 1e-12, float(np.max(np.abs(ref))), "cfg5 adjoint")
    (ck,) = _adjoint(g, [u0], [np.array(1.0)], budget=2 * 10 ** 9)
    assert ck.tobytes() == got.tobytes()


def test_autograd_function_gradcheck():
    from paper_2107_00555_gb300.autograd import apply
    shape, T = (6, 7, 8), 2
    g = programs.tanh_chain(shape, T, fuse=C.DCP_FUSE_ALL)
    u = torch.tensor(inputs.uniform(shape, -1.0, 1.0, 27), device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda t: apply(g, t), (u,), eps=1e-6, atol=1e-7, rtol=1e-6)
    loss = apply(g, u)
    loss.backward()
    (ref,) = oracle.adjoint(OP.tanh_chain(shape, T), [u.detach().cpu().numpy()], [1.0])
    assert_close(u.grad.cpu().numpy(), ref, 1e-12, float(np.max(np.abs(ref))), "autograd")


def test_plan_lists_the_reverse_pass_kernels():
    shape, T = (12, 10, 14), 9
    u0 = inputs.uniform(shape, -1.0, 1.0, 24)
    g = programs.tanh_chain(shape, T, fuse=C.DCP_FUSE_ALL)
    _adjoint(g, [u0], [np.array(1.0)])
    adj = g.plan()["adjoint"]
    phases = [l["phase"] for l in adj["launches"]]
    assert phases[0] == "forward" and "reverse" in phases and not adj["checkpointed"]
    assert adj["tape_bytes"] > 0
    _adjoint(g, [u0], [np.array(1.0)], budget=5 * u0.nbytes)
    adj = g.plan()["adjoint"]
    assert adj["checkpointed"] and "recompute" in [l["phase"] for l in adj["launches"]]


def _paired_tanh_chain(shape, T):
    """u_{t+1} = tanh(S(S(u_t))), loss = sum(u_T^2): every pair of separate
    one-step heat nodes is one deferred common-weight run of two steps."""
    p = oracle.Program()
    pv = p.input("f64", shape)
    g = Graph()
    gv = g.input("f64", shape)
    for _ in range(T):
        for _ in range(2):
            pv = p.stencil(pv, OP.SEVEN, OP.W7, "periodic", 1)
            gv = g.stencil(gv, programs.SEVEN_POINT, programs.SEVEN_WEIGHTS, "periodic", 1)
        pv = p.map("tanh", [pv])
        gv = g.map("tanh", [gv])
    p.output(p.reduce(p.map("square", [pv]), "sum"))
    g.output(g.reduce(g.map("square", [gv]), "sum"))
    g.fuse(C.DCP_FUSE_ALL)
    return p, g


def test_checkpoint_cuts_do_not_split_a_deferred_run():
    """Eight stencil nodes in four deferred runs of two: sqrt(8) checkpointing
    would cut after the third node, inside a run, where the full-tape forward
    applies no factor; the planner moves the cut to the run's end, so the
    checkpointed gradient is bitwise the full tape's, and both match the
    oracle's reverse pass."""
    shape = (12, 14, 16)
    u0 = inputs.uniform(shape, -1.0, 1.0, 25)
    p, g = _paired_tanh_chain(shape, 4)
    (ref,) = oracle.adjoint(p, [u0], [1.0])
    (full,) = _adjoint(g, [u0], [np.array(1.0)])
    (ck,) = _adjoint(g, [u0], [np.array(1.0)], budget=3 * u0.nbytes)
    assert g.plan()["adjoint"]["checkpointed"] is True
    assert full.tobytes() == ck.tobytes()
    assert_close(full, ref, 1e-12, float(np.max(np.abs(ref))), "paired tanh chain adjoint")
