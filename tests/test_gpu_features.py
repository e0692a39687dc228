"""GPU parity of the remaining features through the C ABI: integer maps
(bit-exact), 0-axis broadcast operands, unaligned buffers (element-wise
path), empty arrays, every fusion pattern around stencils (map prologue,
step epilogues, post maps, fused reductions), host-buffer runs and CUDA-graph
replay."""
import numpy as np
import pytest

import oracle
from oracle import programs as OP
from paper_2107_00555_gb300 import Graph, inputs, programs
from paper_2107_00555_gb300 import _capi as C

from gpu_util import assert_close, red_tol_for, tol_for, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIVE = [(0, 0), (0, -1), (0, 1), (1, 0), (-1, 0)]
SEVEN = [(0, 0, 0), (0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]


class Twin:
    """Builds the same program in the oracle and in dcp, op by op."""

    def __init__(self):
        self.p = oracle.Program()
        self.g = Graph()

    def input(self, dtype, shape):
        return (self.p.input(dtype, shape), self.g.input(dtype, shape))

    def map(self, op, ins, imm=0.0):
        return (self.p.map(op, [i[0] for i in ins], imm), self.g.map(op, [i[1] for i in ins], imm))

    def stencil(self, v, offs, w, bc, steps):
        return (self.p.stencil(v[0], offs, w, bc, steps), self.g.stencil(v[1], offs, w, bc, steps))

    def reduce(self, v, red):
        return (self.p.reduce(v[0], red), self.g.reduce(v[1], red))

    def output(self, v):
        self.p.output(v[0])
        self.g.output(v[1])


@pytest.mark.parametrize("dtype", ["i32", "i64"])
@pytest.mark.parametrize("flags", [C.DCP_FUSE_ALL, 0])
def test_integer_program_bit_exact(dtype, flags):
    n = 100003
    bits = 32 if dtype == "i32" else 64
    rng = np.random.default_rng(31)
    npd = np.int32 if dtype == "i32" else np.int64
    lo, hi = np.iinfo(npd).min, np.iinfo(npd).max
    a = rng.integers(lo, hi, n, dtype=npd, endpoint=True)
    b = rng.integers(lo, hi, n, dtype=npd, endpoint=True)
    t = Twin()
    x, y = t.input(dtype, (n,)), t.input(dtype, (n,))
    v = t.map("mul", [x, y])
    v = t.map("add", [v, t.map("square", [x])])
    v = t.map("sub", [v, t.map("abs", [y])])
    v = t.map("max", [v, t.map("neg", [x])])
    v = t.map("min", [v, t.map("mul_s", [y], 12345)])
    v = t.map("rsub_s", [t.map("add_s", [v], -7)], 99)
    t.output(v)
    for red in ("sum", "max", "min", "maxabs"):
        t.output(t.reduce(v, red))
    vals = oracle.run(t.p, [a, b])
    t.g.fuse(flags)
    outs = t.g.run([to_dev(a), to_dev(b)])
    for h, o in zip(t.p.outputs, outs):
        ref = np.asarray(vals[h]).astype(np.int64)
        got = to_host(o).astype(np.int64)
        wrapped = ((ref + (1 << (bits - 1))) % (1 << bits)) - (1 << (bits - 1)) if bits == 32 else ref
        assert np.array_equal(got, wrapped)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_scalar_broadcast_operands(dtype):
    """x - mean(x), scaled by 1/max|x|: reductions feeding later maps as 0-axis operands."""
    n = 50001
    x0 = inputs.normal((n,), 32, {"f32": np.float32, "f64": np.float64}[dtype])
    t = Twin()
    x = t.input(dtype, (n,))
    s = t.reduce(x, "sum")
    mean = t.map("mul_s", [s], 1.0 / n)
    m = t.reduce(x, "maxabs")
    c = t.map("sub", [x, mean])
    y = t.map("div", [c, m])
    t.output(y)
    t.output(t.reduce(t.map("square", [y]), "sum"))
    vals = oracle.run(t.p, [x0])
    t.g.fuse(C.DCP_FUSE_ALL)
    outs = t.g.run([to_dev(x0)])
    yref = vals[t.p.outputs[0]]
    assert_close(to_host(outs[0]), yref, 4 * tol_for(dtype), 1.0, "broadcast")
    sq = float(np.sum(yref * yref))
    assert abs(float(to_host(outs[1])) - sq) <= red_tol_for(dtype) * sq * 10


@pytest.mark.parametrize("offset", [1, 2, 3])
def test_unaligned_buffers_take_elementwise_path(offset):
    n = 10007
    x0 = inputs.normal((n + 4,), 33, np.float32)
    t = Twin()
    x = t.input("f32", (n,))
    t.output(t.map("exp", [t.map("sin", [x])]))
    t.output(t.reduce(x, "sum"))
    t.g.fuse(C.DCP_FUSE_ALL)
    d = to_dev(x0)[offset:offset + n]   # 4-byte aligned, not 16-byte aligned
    outs = t.g.run([d])
    vals = oracle.run(t.p, [x0[offset:offset + n]])
    assert_close(to_host(outs[0]), vals[t.p.outputs[0]], 1e-5, 1.0, "unaligned map")
    ref = vals[t.p.outputs[1]]
    assert abs(float(to_host(outs[1])) - float(ref)) <= 1e-4 * float(np.sum(np.abs(x0)))


def test_empty_arrays():
    g = Graph()
    x = g.input("f32", (0,))
    g.output(g.map("neg", [x]))
    g.output(g.reduce(x, "sum"))
    g.fuse(C.DCP_FUSE_ALL)
    outs = g.run([torch.empty(0, device="cuda")])
    torch.cuda.synchronize()
    assert outs[0].numel() == 0 and float(outs[1]) == 0.0


@pytest.mark.parametrize("bc", ["zero", "periodic", "fixed_ring"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_stencil_fusion_patterns(bc, dtype):
    """prologue maps -> 2-step stencil with epilogues -> 3-step stencil -> post maps,
    stored values and reductions, fused against op-by-op and the oracle."""
    shape = (61, 75)
    npd = {"f32": np.float32, "f64": np.float64}[dtype]
    a0 = inputs.uniform(shape, -1.0, 1.0, 34, npd)
    b0 = inputs.uniform(shape, 0.5, 1.5, 35, npd)
    t = Twin()
    a, b = t.input(dtype, shape), t.input(dtype, shape)
    v = t.map("mul", [t.map("sin", [a]), b])          # prologue
    v = t.stencil(v, FIVE, [0.2] * 5, bc, 2)
    v = t.map("tanh", [t.map("mul_s", [v], 1.5)])      # step epilogue
    v = t.stencil(v, FIVE, [0.3, 0.2, 0.2, 0.15, 0.15], bc, 3)
    w = t.map("add", [t.map("square", [v]), b])        # post
    t.output(v)
    t.output(w)
    t.output(t.reduce(w, "sum"))
    t.output(t.reduce(v, "maxabs"))
    vals = oracle.run(t.p, [a0, b0])
    for flags in (C.DCP_FUSE_ALL, 0):
        t2 = Twin()
        a2, b2 = t2.input(dtype, shape), t2.input(dtype, shape)
        v2 = t2.map("mul", [t2.map("sin", [a2]), b2])
        v2 = t2.stencil(v2, FIVE, [0.2] * 5, bc, 2)
        v2 = t2.map("tanh", [t2.map("mul_s", [v2], 1.5)])
        v2 = t2.stencil(v2, FIVE, [0.3, 0.2, 0.2, 0.15, 0.15], bc, 3)
        w2 = t2.map("add", [t2.map("square", [v2]), b2])
        t2.output(v2)
        t2.output(w2)
        t2.output(t2.reduce(w2, "sum"))
        t2.output(t2.reduce(v2, "maxabs"))
        t2.g.fuse(flags)
        if flags:
            assert t2.g.n_kernels <= 3
        outs = t2.g.run([to_dev(a0), to_dev(b0)])
        tol = tol_for(dtype) * 4
        assert_close(to_host(outs[0]), vals[t.p.outputs[0]], tol, 1.0, "v")
        assert_close(to_host(outs[1]), vals[t.p.outputs[1]], tol, 2.0, "w")
        sw = float(np.sum(np.abs(vals[t.p.outputs[1]])))
        assert abs(float(to_host(outs[2])) - float(vals[t.p.outputs[2]])) <= red_tol_for(dtype) * sw
        assert abs(float(to_host(outs[3])) - float(vals[t.p.outputs[3]])) <= tol


def test_3d_prologue_and_reduction():
    shape = (20, 33, 47)
    a0 = inputs.uniform(shape, -1.0, 1.0, 36)
    t = Twin()
    a = t.input("f64", shape)
    v = t.stencil(t.map("exp", [a]), SEVEN, [0.4] + [0.1] * 6, "zero", 2)
    t.output(v)
    t.output(t.reduce(t.map("mul", [v, a]), "sum"))
    vals = oracle.run(t.p, [a0])
    t.g.fuse(C.DCP_FUSE_ALL)
    outs = t.g.run([to_dev(a0)])
    assert_close(to_host(outs[0]), vals[t.p.outputs[0]], 1e-12, 3.0, "3d")
    ref = float(vals[t.p.outputs[1]])
    assert abs(float(to_host(outs[1])) - ref) <= 1e-10 * float(np.sum(np.abs(vals[t.p.outputs[0]] * a0)))


def test_run_host_buffers():
    n = 300001
    x0 = inputs.normal((n,), 37, np.float32)
    t = Twin()
    x = t.input("f32", (n,))
    t.output(t.map("mul", [x, x]))
    t.output(t.reduce(x, "maxabs"))
    t.g.fuse(C.DCP_FUSE_ALL)
    outs = t.g.run_host([x0])
    vals = oracle.run(t.p, [x0])
    assert_close(outs[0], vals[t.p.outputs[0]], 1e-6, 0.0, "host map")
    assert float(outs[1]) == float(vals[t.p.outputs[1]])


def test_graph_replay_for_a_stencil_program():
    u0 = inputs.uniform((128, 130), 0.0, 1.0, 38)
    t = Twin()
    u = t.input("f64", (128, 130))
    t.output(t.stencil(u, FIVE, [0.2] * 5, "zero", 10))
    t.g.set_option(C.DCP_OPT_USE_GRAPH, 1)
    t.g.fuse(C.DCP_FUSE_ALL)
    d = to_dev(u0)
    o = t.g.run([d])
    o = t.g.run([d], o)
    o = t.g.run([d], o)
    ref = oracle.run(t.p, [u0])[-1]
    assert_close(to_host(o[0]), ref, 1e-12, 1.0, "graph replay")


def test_determinism_of_fused_stencil_reductions():
    u0 = inputs.uniform((40, 64, 64), -1.0, 1.0, 39)
    g = Graph()
    u = g.input("f64", (40, 64, 64))
    v = g.stencil(u, SEVEN, [0.4] + [0.1] * 6, "periodic", 3)
    g.output(g.reduce(g.map("square", [v]), "sum"))
    g.fuse(C.DCP_FUSE_ALL)
    d = to_dev(u0)
    r = [to_host(g.run([d])[0]).tobytes() for _ in range(3)]
    assert r[0] == r[1] == r[2]


def test_autotune_picks_a_config_and_keeps_results():
    u0 = inputs.uniform((300, 270), 0.0, 1.0, 41).astype(np.float32)
    t = Twin()
    u = t.input("f32", (300, 270))
    t.output(t.stencil(u, FIVE, [0.2] * 5, "zero", 12))
    t.g.fuse(C.DCP_FUSE_ALL | C.DCP_AUTOTUNE)
    ref = oracle.run(t.p, [u0])[-1]
    d = to_dev(u0)
    o1 = to_host(t.g.run([d])[0]).copy()      # tuning run
    o2 = to_host(t.g.run([d])[0]).copy()      # tuned run
    assert_close(o1, ref, 1e-5, 1.0, "tuning run")
    assert o1.tobytes() == o2.tobytes()
    plan = t.g.plan()
    grp = plan["groups"][0]
    assert 1 <= grp["depth"] <= 12
    assert plan["n_launches"] == -(-12 // grp["depth"])


def test_autotune_small_f64_grid_keeps_bits():
    """The 256^2 binary64 five-point program (10 steps): the autotuner also
    tries tile shapes balanced over the SMs with 256, 512 and 1024 threads;
    whatever it keeps computes the same bits as the untuned plan, within the
    f64 tolerance of the oracle."""
    u0 = inputs.cfg1(seed=43, n=256)
    ref = oracle.run(OP.jacobi2d((256, 256), 10, "zero"), [u0])[-1]
    g0 = programs.jacobi2d((256, 256), 10, "zero", "f64", fuse=C.DCP_FUSE_ALL)
    want = to_host(g0.run([to_dev(u0)])[0]).copy()
    g = programs.jacobi2d((256, 256), 10, "zero", "f64")
    g.set_option(C.DCP_OPT_USE_GRAPH, 1)
    g.fuse(C.DCP_FUSE_ALL | C.DCP_AUTOTUNE)
    d = to_dev(u0)
    o1 = to_host(g.run([d])[0]).copy()   # tuning run
    o2 = to_host(g.run([d])[0]).copy()   # tuned run (graph replay)
    assert o1.tobytes() == want.tobytes() == o2.tobytes()
    assert_close(o2, ref, 1e-12, 1.0, "tuned 256^2 f64")


@pytest.mark.parametrize("direct", [1, 0])
def test_run_host_pinned_buffers(direct):
    """Page-locked host buffers: the kernels access them directly (or, with
    the option off, through staging copies); both give the oracle's result."""
    n = 1 << 20
    x0 = inputs.normal((n,), 42, np.float32)
    t = Twin()
    x = t.input("f32", (n,))
    t.output(t.map("mul_s", [t.map("sin", [x])], 3.0))
    t.output(t.reduce(x, "sum"))
    t.g.set_option(C.DCP_OPT_HOST_ACCESS, direct)
    t.g.fuse(C.DCP_FUSE_ALL)
    xin = torch.empty(n, dtype=torch.float32, pin_memory=True)
    xin.copy_(torch.from_numpy(x0))
    out0 = torch.empty(n, dtype=torch.float32, pin_memory=True)
    out1 = torch.empty((), dtype=torch.float32, pin_memory=True)
    for _ in range(2):
        t.g.run_host([xin.numpy()], [out0.numpy(), out1.numpy()])
        vals = oracle.run(t.p, [x0])
        assert_close(out0.numpy(), vals[t.p.outputs[0]], 1e-5, 3.0, "pinned map")
        assert abs(float(out1) - float(vals[t.p.outputs[1]])) <= 1e-4 * float(np.sum(np.abs(x0)))


def test_prepared_call_matches_run():
    sides = [33, 70]
    us = [inputs.uniform((s, s), 0.0, 1.0, 43 + s).astype(np.float32) for s in sides]
    g = Graph()
    vs = [g.input("f32", u.shape) for u in us]
    for v in vs:
        g.output(g.stencil(v, FIVE, [0.2] * 5, "zero", 6))
    g.fuse(C.DCP_FUSE_ALL | C.DCP_BATCH)
    d = [to_dev(u) for u in us]
    call = g.prepare(d)
    a = [to_host(o).copy() for o in call()]
    b = [to_host(o) for o in g.run(d)]
    for x, y in zip(a, b):
        assert x.tobytes() == y.tobytes()


@pytest.mark.parametrize("pinned", [True, False])
def test_prepared_host_call_matches_run(pinned):
    """Batched instances in host memory (page-locked: read and written in
    place by the kernels; pageable: staged) give the device run's bits."""
    sides = [33, 70, 5]
    us = [inputs.uniform((s, s), 0.0, 1.0, 47 + s).astype(np.float32) for s in sides]
    g = Graph()
    vs = [g.input("f32", u.shape) for u in us]
    for v in vs:
        g.output(g.stencil(v, FIVE, [0.2] * 5, "zero", 6))
    g.fuse(C.DCP_FUSE_ALL | C.DCP_BATCH)
    ref = [to_host(o) for o in g.run([to_dev(u) for u in us])]
    if pinned:
        hin = [torch.from_numpy(u).pin_memory().numpy() for u in us]
        hout = [torch.empty(u.shape, dtype=torch.float32, pin_memory=True).numpy() for u in us]
    else:
        hin = [u.copy() for u in us]
        hout = [np.empty_like(u) for u in us]
    call = g.prepare_host(hin, hout)
    for _ in range(2):
        got = call()
        torch.cuda.synchronize()
        for x, y in zip(got, ref):
            assert x.tobytes() == y.tobytes()


@pytest.mark.parametrize("graph_replay", [0, 1])
def test_injected_faults_leave_the_graph_usable(monkeypatch, graph_replay):
    """DCP_FAULT makes the next device allocation or launch fail on the host
    with the status a real failure returns; the graph stays usable and the
    following run is correct (the CUDA-graph capture path included)."""
    shape, T = (40, 50), 6
    u0 = inputs.uniform(shape, 0.0, 1.0, 61)
    ref = oracle.run(OP.jacobi2d(shape, T, "zero"), [u0])[-1]
    g = programs.jacobi2d(shape, T, "zero", "f64")
    g.set_option(C.DCP_OPT_TIME_TILE_DEPTH, 2)  # three launches, state buffers
    g.set_option(C.DCP_OPT_USE_GRAPH, graph_replay)
    g.fuse(C.DCP_FUSE_ALL)
    d = to_dev(u0)
    for fault, status in (("alloc", C.DCP_E_OOM), ("launch", C.DCP_E_CUDA)):
        monkeypatch.setenv("DCP_FAULT", fault)
        with pytest.raises(C.DcpError) as e:
            g.run([d])
        torch.cuda.synchronize()
        assert e.value.status == status and "injected" in str(e.value)
        monkeypatch.delenv("DCP_FAULT")
        out = to_host(g.run([d])[0])
        assert np.max(np.abs(out - ref)) <= 1e-12


def test_graphs_on_concurrent_host_threads():
    """Different graphs run from several host threads at once, each on its
    own stream (first runs compile and tune concurrently), give the bits of
    serial runs."""
    import threading

    def make(k):
        if k % 3 == 0:
            return programs.jacobi2d((70 + k, 90), 6, "zero", "f64", fuse=C.DCP_FUSE_ALL | C.DCP_AUTOTUNE)
        if k % 3 == 1:
            return programs.map_reduce(50000 + 1000 * k, "f32", fuse=C.DCP_FUSE_ALL)
        return programs.heat3d((20, 18, 40 + k), 2, "periodic", "f64", fuse=C.DCP_FUSE_ALL)

    def inputs_for(k, g):
        rng = np.random.default_rng(100 + k)
        return [to_dev(rng.uniform(-1, 1, size=g.shape[v]).astype(
            np.float32 if g.dtype[v] == C.DCP_F32 else np.float64)) for v in g.inputs]

    serial = []
    for k in range(6):
        g = make(k)
        serial.append([to_host(o).tobytes() for o in g.run(inputs_for(k, g))])
    torch.cuda.synchronize()
    results = [None] * 6
    errors = []

    def worker(k):
        try:
            torch.cuda.set_device(0)
            s = torch.cuda.Stream()
            g = make(k)
            ins = inputs_for(k, g)
            with torch.cuda.stream(s):
                for _ in range(3):
                    outs = g.run(ins, stream=s)
            s.synchronize()
            results[k] = [to_host(o).tobytes() for o in outs]
        except Exception as e:  # reported below
            errors.append((k, repr(e)))

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(6)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    for k in range(6):
        assert results[k] == serial[k], k


@pytest.mark.gpu
def test_fp64_probe_reports_a_plausible_rate():
    """dcp_probe_fp64 (the FP64 roofline denominator): fused multiply-add, add
    and multiply each give a positive lane rate, at most the FP32 rate of a
    GB300 (152 SMs x 128 lanes x 2.07 GHz), and arguments are validated."""
    torch.cuda.init()
    s = torch.cuda.current_stream().cuda_stream
    cap = 152 * 128 * 2.1
    for op in (0, 1, 2, 3, 4):
        g, ms = C.dcp_probe_fp64(op, 1024, s)
        assert 0 < g < cap and ms > 0, (op, g, ms)
    with pytest.raises(C.DcpError):
        C.dcp_probe_fp64(5, 1024, s)
    with pytest.raises(C.DcpError):
        C.dcp_probe_fp64(0, 0, s)
