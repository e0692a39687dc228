"""Seeded random differentiable programs (maps including broadcast 0-axis
operands, zero / periodic stencils, sum reductions; array and scalar
outputs with random cotangents): dcp_run_adjoint against the oracle's
reverse pass of the unfused program, and a checkpointed tape against the
full tape bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2107_00555_gb300 import _capi as C

from gpu_util import to_dev, to_host
from test_gpu_random_programs import STAR, Twin

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _random_diff_program(seed):
    rng = np.random.default_rng(1000 + seed)
    nd = int(rng.integers(1, 4))
    shape = tuple(int(rng.integers(2, 24 if nd < 3 else 10)) for _ in range(nd))
    t = Twin("f64")
    full = [t.input(shape) for _ in range(int(rng.integers(1, 3)))]
    scal = [t.input(()) for _ in range(int(rng.integers(0, 2)))]
    outs = []
    n_stencils = 0
    for _ in range(int(rng.integers(3, 10))):
        k = rng.random()
        a = full[int(rng.integers(len(full)))]
        if k < 0.3:
            op = ["neg", "sin", "cos", "tanh", "square"][int(rng.integers(5))]
            v = t.map(op, [a])
            if op == "square":
                v = t.map("tanh", [v])
        elif k < 0.4:
            v = t.map("exp", [t.map("tanh", [a])])
        elif k < 0.45:
            v = t.map("sqrt", [t.map("add_s", [t.map("square", [a])], 1.0)])
        elif k < 0.65:
            b = (scal + full)[int(rng.integers(len(scal) + len(full)))]
            op = ["add", "sub", "mul", "max", "min"][int(rng.integers(5))]
            v = t.map(op, [a, b] if rng.random() < 0.5 else [b, a])
            if op == "mul":
                v = t.map("tanh", [v])
        elif k < 0.7:
            d = t.map("add_s", [t.map("square", [full[int(rng.integers(len(full)))]])], 1.0)
            v = t.map("div", [a, d])
        elif k < 0.75:
            op = ["add_s", "mul_s", "sub_s", "rsub_s"][int(rng.integers(4))]
            v = t.map("tanh", [t.map(op, [a], float(rng.uniform(-2, 2)))])
        else:
            offs = STAR[nd][int(rng.integers(2))]
            w = rng.uniform(0.1, 1.0, len(offs))
            v = t.stencil(a, offs, list(w / w.sum()), ["zero", "periodic"][int(rng.integers(2))],
                          int(rng.integers(1, 4)))
            n_stencils += 1
        full.append(v)
        if rng.random() < 0.2:
            outs.append(v)
    outs.append(full[-1])
    outs.append(t.reduce(full[int(rng.integers(len(full)))], "sum"))
    outs = [i for i in dict.fromkeys(outs) if t.vals[i][0] not in t.p.inputs]
    for i in outs:
        t.output(i)
    return t, outs, rng, n_stencils


@pytest.mark.parametrize("seed", range(40))
def test_random_program_adjoint(seed):
    t, outs, rng, n_stencils = _random_diff_program(seed)
    ins = [rng.uniform(-1.5, 1.5, size=t.p.nodes[h].shape) for h in t.p.inputs]
    cots = [rng.uniform(-1.0, 1.0, size=t.vals[i][2]) for i in outs]
    ref = oracle.adjoint(t.p, ins, cots)
    t.g.fuse(C.DCP_FUSE_ALL)
    dev_in = [to_dev(np.asarray(a)) for a in ins]
    dev_cot = [to_dev(np.asarray(c)) for c in cots]
    got = [to_host(x) for x in t.g.adjoint(dev_in, dev_cot)]
    for r, g_ in zip(ref, got):
        r = np.asarray(r)
        assert g_.shape == r.shape
        scale = max(float(np.max(np.abs(r))) if r.size else 0.0, 1.0)
        assert np.all(np.abs(g_ - r) <= 1e-9 * scale), (seed, float(np.max(np.abs(g_ - r))))
    if n_stencils >= 2:
        # the smallest tape budget the planner accepts reproduces the full tape's bits
        state = int(np.prod(t.vals[0][2])) * 8
        for mult in (3, 4, 6, 10):
            try:
                ck = [to_host(x) for x in t.g.adjoint(dev_in, dev_cot,
                                                       tape_budget_bytes=mult * state)]
            except C.DcpError as e:
                assert e.status == C.DCP_E_OOM
                continue
            for a, b in zip(got, ck):
                assert a.tobytes() == b.tobytes(), (seed, mult)
            break
