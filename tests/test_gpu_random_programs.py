"""Seeded random programs (maps, scalar broadcasts, stencils of every
boundary rule, whole-array and axis reductions, intermediate outputs) built
identically in the oracle and in the library, run fused and op by op, and
compared output by output.  Values are kept bounded (tanh before exp, |x|+1
under sqrt and as divisor), so mixed tolerances scaled by the output's
magnitude apply; sums use the backward-stable bound sum|y_i|."""
import numpy as np
import pytest

import oracle
from paper_2107_00555_gb300 import Graph
from paper_2107_00555_gb300 import _capi as C

from gpu_util import to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STAR = {1: [[(0,), (-1,), (1,)], [(0,), (-2,), (2,), (-1,), (1,)]],
        2: [[(0, 0), (0, -1), (0, 1), (1, 0), (-1, 0)],
            [(0, 0), (1, 1), (-1, -1), (0, 2), (-2, 0)]],
        3: [[(0, 0, 0), (0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)],
            [(0, 0, 0), (0, 0, 2), (0, -1, 1), (1, 0, 0)]]}


class Twin:
    """Records every operation in both the oracle program and the graph."""

    def __init__(self, dtype):
        self.p, self.g, self.dt = oracle.Program(), Graph(), dtype
        self.vals = []      # (oracle handle, graph handle, shape)

    def input(self, shape):
        self.vals.append((self.p.input(self.dt, shape), self.g.input(self.dt, shape), shape))
        return len(self.vals) - 1

    def map(self, op, ins, imm=0.0):
        ph = self.p.map(op, [self.vals[i][0] for i in ins], imm)
        gh = self.g.map(op, [self.vals[i][1] for i in ins], imm)
        shape = max((self.vals[i][2] for i in ins), key=len)
        self.vals.append((ph, gh, shape))
        return len(self.vals) - 1

    def stencil(self, i, offs, w, bc, steps):
        ph = self.p.stencil(self.vals[i][0], offs, w, bc, steps)
        gh = self.g.stencil(self.vals[i][1], offs, w, bc, steps)
        self.vals.append((ph, gh, self.vals[i][2]))
        return len(self.vals) - 1

    def reduce(self, i, red, axis=None):
        ph = self.p.reduce(self.vals[i][0], red, axis=axis)
        gh = self.g.reduce(self.vals[i][1], red, axis=axis)
        shape = () if axis is None else tuple(s for d, s in enumerate(self.vals[i][2]) if d != axis)
        self.vals.append((ph, gh, shape))
        return len(self.vals) - 1

    def output(self, i):
        self.p.output(self.vals[i][0])
        self.g.output(self.vals[i][1])


def _random_program(seed):
    rng = np.random.default_rng(seed)
    dtype = "f64" if rng.random() < 0.5 else "f32"
    nd = int(rng.integers(1, 4))
    shape = tuple(int(rng.integers(1, 40 if nd < 3 else 14)) for _ in range(nd))
    t = Twin(dtype)
    full = [t.input(shape) for _ in range(int(rng.integers(1, 4)))]
    scal = [t.input(()) for _ in range(int(rng.integers(0, 2)))]
    reductions, outs = [], []
    for _ in range(int(rng.integers(3, 12))):
        k = rng.random()
        a = full[int(rng.integers(len(full)))]
        if k < 0.35:
            op = ["neg", "abs", "sin", "cos", "tanh", "square"][int(rng.integers(6))]
            v = t.map(op, [a])
            if op == "square":
                v = t.map("tanh", [v])
        elif k < 0.45:
            v = t.map("exp", [t.map("tanh", [a])])
        elif k < 0.5:
            v = t.map("sqrt", [t.map("add_s", [t.map("abs", [a])], 1.0)])
        elif k < 0.7:
            b = (scal + full)[int(rng.integers(len(scal) + len(full)))]
            op = ["add", "sub", "mul", "max", "min"][int(rng.integers(5))]
            ins = [a, b] if rng.random() < 0.5 else [b, a]
            v = t.map(op, ins)
            if op == "mul":
                v = t.map("tanh", [v])
        elif k < 0.75:
            d = t.map("add_s", [t.map("abs", [full[int(rng.integers(len(full)))]])], 1.0)
            v = t.map("div", [a, d])
        elif k < 0.8:
            op = ["add_s", "mul_s", "sub_s", "rsub_s"][int(rng.integers(4))]
            v = t.map(op, [a], float(rng.uniform(-2, 2)))
            v = t.map("tanh", [v])
        else:
            offs = STAR[nd][int(rng.integers(2))]
            w = rng.uniform(0.1, 1.0, len(offs))
            w = list(w / w.sum())
            bc = ["zero", "periodic", "fixed_ring"][int(rng.integers(3))]
            v = t.stencil(a, offs, w, bc, int(rng.integers(1, 4)))
        full.append(v)
        if rng.random() < 0.25:
            outs.append(v)
    last = full[-1]
    outs.append(last)
    for _ in range(int(rng.integers(1, 3))):
        red = ["sum", "max", "min", "maxabs"][int(rng.integers(4))]
        src = full[int(rng.integers(len(full)))]
        axis = None if rng.random() < 0.5 else int(rng.integers(nd))
        reductions.append(t.reduce(src, red, axis))
    for i in dict.fromkeys(outs + reductions):
        if t.vals[i][0] not in t.p.inputs:
            t.output(i)
    return t, dtype, shape, rng


@pytest.mark.parametrize("seed", range(100))
def test_random_program_fused_and_op_by_op(seed):
    t, dtype, shape, rng = _random_program(seed)
    npdt = np.float32 if dtype == "f32" else np.float64
    ins = []
    for h in t.p.inputs:
        shp = t.p.nodes[h].shape
        ins.append(rng.uniform(-1.5, 1.5, size=shp).astype(npdt))
    vals, extra = oracle.run(t.p, ins, detail=True)
    tol = 2e-4 if dtype == "f32" else 1e-9
    for flags in (C.DCP_FUSE_ALL, 0):
        g = t.g
        if flags == 0:
            # the same program, rebuilt op by op
            t2, _, _, _ = _random_program(seed)
            g = t2.g
        g.fuse(flags)
        outs = [to_host(o).astype(np.float64) for o in g.run([to_dev(a) for a in ins])]
        for h, got in zip(t.p.outputs, outs):
            ref = np.asarray(vals[h], dtype=np.float64)
            assert got.shape == ref.shape, (seed, h)
            if h in extra:  # sums: backward-stable bound
                assert np.all(np.abs(got - extra[h]["fsum"]) <= tol * (extra[h]["abs"] + 1.0)), \
                    (seed, flags, h)
            else:
                scale = float(np.max(np.abs(ref))) if ref.size else 0.0
                assert np.all(np.abs(got - ref) <= tol * max(scale, 1.0)), \
                    (seed, flags, h, float(np.max(np.abs(got - ref))) if ref.size else 0.0)
