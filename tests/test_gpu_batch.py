"""Batched persistent stencil launches (many independent instances of uneven
size in one launch) against the oracle, against one-at-a-time runs of the
same instances, and against the closed-form decay of zero-boundary sine
modes at the full 4096-instance size."""
import math

import numpy as np
import pytest

import oracle
from oracle import programs as OP
from paper_2107_00555_gb300 import inputs, programs
from paper_2107_00555_gb300 import _capi as C

from gpu_util import assert_close, tol_for, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NP = {"f32": np.float32, "f64": np.float64}
BATCH = C.DCP_FUSE_ALL | C.DCP_BATCH


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("bc", ["zero", "periodic", "fixed_ring"])
def test_small_batch_vs_oracle(dtype, bc):
    sides = [1, 2, 5, 33, 64, 100, 130, 7, 65]
    T = 20
    us = [inputs.uniform((s, s), 0.0, 1.0, 40 + i, NP[dtype]) for i, s in enumerate(sides)]
    g = programs.batch2d(sides, T, bc, dtype, fuse=BATCH)
    plan = g.plan()
    assert len(plan["groups"]) == 1 and plan["groups"][0]["kind"] == "batch"
    outs = g.run([to_dev(u) for u in us])
    for u, o in zip(us, outs):
        ref = oracle.run(OP.jacobi2d(u.shape, T, bc), [u])[-1]
        assert_close(to_host(o), ref, tol_for(dtype), float(np.max(u)), "batch %s" % (u.shape,))


def test_batched_equals_one_at_a_time_bitwise():
    sides = [40, 97, 128, 200]
    T = 20
    us = [inputs.uniform((s, s), 0.0, 1.0, 60 + s) for s in sides]
    us = [u.astype(np.float32) for u in us]
    gb = programs.batch2d(sides, T, "zero", "f32", fuse=BATCH)
    ob = [to_host(o) for o in gb.run([to_dev(u) for u in us])]
    for u, o in zip(us, ob):
        g1 = programs.jacobi2d(u.shape, T, "zero", "f32", fuse=C.DCP_FUSE_ALL)
        assert to_host(g1.run([to_dev(u)])[0]).tobytes() == o.tobytes()


def _bench_batch(sides):
    """The batched program in the launch configuration the benchmark times:
    autotuned kernel form, depth and work items, CUDA-graph replay."""
    g = programs.batch2d(sides, 20, "zero", "f32")
    g.set_option(C.DCP_OPT_USE_GRAPH, 1)
    g.fuse(BATCH | C.DCP_AUTOTUNE)
    return g


def test_config4_full_batch_sine_modes():
    """All 4096 instances (sides log-uniform in [32, 512]) start from a
    zero-boundary sine mode, which the 5-point average scales by
    lam = 0.2 (1 + 2 cos(pi p/(N+1)) + 2 cos(pi q/(N+1))) per step."""
    sides = inputs.cfg4_sides()
    T = 20
    us, refs = [], []
    for k, n in enumerate(sides):
        n = int(n)
        p, q = 1 + k % 3, 1 + (k // 3) % 2
        i = np.arange(n)
        mode = np.outer(np.sin(np.pi * p * (i + 1) / (n + 1)), np.sin(np.pi * q * (i + 1) / (n + 1)))
        lam = 0.2 * (1 + 2 * math.cos(math.pi * p / (n + 1)) + 2 * math.cos(math.pi * q / (n + 1)))
        us.append(mode.astype(np.float32))
        refs.append(lam ** T * mode)
    g = _bench_batch(sides)
    dev = [to_dev(u) for u in us]
    call = g.prepare(dev)
    call()             # first run: autotuned, eager
    outs = call()      # replayed CUDA graph, the timed form
    torch.cuda.synchronize()
    for k in range(len(sides)):
        # fp32 input rounding is propagated exactly by the linear map; stay within fp32 tolerance
        assert_close(to_host(outs[k]), refs[k], 1e-5, 1.0, "instance %d" % k)


def test_config4_sample_vs_oracle():
    """The benchmark's inputs: a sample of instances (smallest, largest and
    every 97th) against the oracle."""
    us = inputs.cfg4()
    sides = [u.shape[0] for u in us]
    g = _bench_batch(sides)
    call = g.prepare([to_dev(u) for u in us])
    call()
    outs = call()
    torch.cuda.synchronize()
    idx = sorted(set([int(np.argmin(sides)), int(np.argmax(sides))] + list(range(0, len(us), 97))))
    for k in idx:
        ref = oracle.run(OP.jacobi2d(us[k].shape, 20, "zero", "f32"), [us[k]])[-1]
        assert_close(to_host(outs[k]), ref, 1e-5, 1.0, "instance %d" % k)


def test_graph_replay_and_rebinding():
    sides = [50, 80, 120]
    us = [inputs.uniform((s, s), 0.0, 1.0, 70 + s).astype(np.float32) for s in sides]
    g = programs.batch2d(sides, 8, "zero", "f32")
    g.set_option(C.DCP_OPT_USE_GRAPH, 1)
    g.fuse(BATCH)
    d = [to_dev(u) for u in us]
    o1 = g.run(d)        # eager run + capture
    o2 = g.run(d, o1)    # replay into the same buffers
    r = [to_host(o).copy() for o in o2]
    d2 = [to_dev(u * 2) for u in us]
    o3 = g.run(d2)       # new pointers: re-capture
    for a, b, u in zip(r, o3, us):
        ref = oracle.run(OP.jacobi2d(u.shape, 8, "zero", "f32"), [u])[-1]
        assert_close(a, ref, 1e-5, 1.0, "replay")
        assert_close(to_host(b), 2 * ref, 1e-5, 2.0, "rebound")


@pytest.mark.parametrize("kernel,depth,prefetch,threads,rows", [
    (0, 4, 1, 128, 64), (1, 1, 1, 128, 64), (1, 4, 1, 128, 32), (1, 5, 2, 64, 128),
    (1, 8, 2, 128, 64), (1, 6, 1, 32, 1)])
def test_batch_kernel_forms_bitwise(kernel, depth, prefetch, threads, rows):
    """Every kernel form, depth, prefetch depth, CTA size and work-item size
    of the batched launch gives the bits of one-at-a-time one-step runs."""
    sides = [1, 3, 40, 97, 128, 200, 33]
    T = 20
    us = [inputs.uniform((s, s), 0.0, 1.0, 70 + i, np.float32) for i, s in enumerate(sides)]
    g = programs.batch2d(sides, T, "zero", "f32")
    g.set_option(C.DCP_OPT_STENCIL_KERNEL, kernel)
    g.set_option(C.DCP_OPT_TIME_TILE_DEPTH, depth)
    g.set_option(C.DCP_OPT_STREAM_PREFETCH, prefetch)
    g.set_option(C.DCP_OPT_STREAM_THREADS, threads)
    g.set_option(C.DCP_OPT_STREAM_ROWS, rows)
    g.fuse(BATCH)
    (grp,) = g.plan()["groups"]
    assert grp["kernel_form"] == ("stream" if kernel == 1 else "tile")
    outs = [to_host(o) for o in g.run([to_dev(u) for u in us])]
    for u, o in zip(us, outs):
        g1 = programs.jacobi2d(u.shape, T, "zero", "f32")
        g1.set_option(C.DCP_OPT_STENCIL_KERNEL, 0)
        g1.set_option(C.DCP_OPT_TIME_TILE_DEPTH, 1)
        g1.fuse(C.DCP_FUSE_ALL)
        assert to_host(g1.run([to_dev(u)])[0]).tobytes() == o.tobytes(), u.shape
