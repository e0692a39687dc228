"""Sharded execution with the library's kernels (Sec. 4.1 block split, Sec. 4.3
slab split with halo exchange), two ranks as two processes on the one GPU of
the box.  The halos travel over gloo through host copies (NCCL does not run
two ranks on one device); no kernel of one rank waits on the other rank, so
the two processes never depend on each other's kernels.  Each rank's owned
planes are compared with the whole-domain oracle, the map+reduce result with
the whole-array oracle.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

SEVEN = [(0, 0, 0), (0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]
W7 = [0.4] + [0.1] * 6


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _spawn(target, world, *args):
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=target, args=(r, world, port, out) + args) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
    for p in procs:
        if p.is_alive():
            p.kill()
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    return dict(out)


def _init(rank, world, port):
    import torch.distributed as dist
    from datetime import timedelta
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=120))
    return dist


def _stencil_rank(rank, world, port, out, shape, bc, steps, depth, seed):
    import oracle
    from paper_2107_00555_gb300 import _capi as C
    from paper_2107_00555_gb300 import inputs, programs, shard
    dist = _init(rank, world, port)
    torch.cuda.set_device(0)
    u0 = inputs.uniform(shape, -1.0, 1.0, seed)
    plan = shard.SlabPlan(shape, 1, bc, steps, world, rank, depth)
    bufs = [torch.zeros(plan.local_shape, dtype=torch.float64, device="cuda") for _ in range(2)]
    graphs, calls = {}, {}
    for c in plan.chunks:
        if c.steps not in graphs:
            graphs[c.steps] = programs.heat3d(plan.local_shape, c.steps, bc, "f64",
                                              fuse=C.DCP_FUSE_ALL)
            for i in range(2):
                calls[(c.steps, i)] = graphs[c.steps].prepare([bufs[i]], [bufs[1 - i]])
    which = {id(bufs[0]): 0, id(bufs[1]): 1}
    it = iter(bufs)
    ss = shard.ShardedStencil(plan, lambda src, k, dst: calls[(k, which[id(src)])](),
                              lambda: next(it), dist)
    ss.load(torch.from_numpy(plan.slab_of(u0).copy()).cuda())
    got = ss.run().cpu().numpy()
    ref = oracle.stencil(u0, SEVEN, W7, bc, steps)[plan.z0:plan.z1]
    scale = float(np.max(np.abs(u0)))
    err = float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), scale)))
    out[rank] = (err, plan.h, len(plan.chunks))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("bc,steps,depth", [("periodic", 7, 2), ("zero", 6, 3),
                                            ("fixed_ring", 5, 2)])
def test_two_rank_slab_split_heat_step_matches_oracle(bc, steps, depth):
    res = _spawn(_stencil_rank, 2, (34, 20, 28), bc, steps, depth, 31)
    for r in range(2):
        err, h, nchunks = res[r]
        assert err <= 1e-12, (r, err)
        assert h == depth and nchunks == -(-steps // depth)


def _map_reduce_rank(rank, world, port, out, n, seed):
    import oracle
    from oracle import programs as OP
    from paper_2107_00555_gb300 import _capi as C
    from paper_2107_00555_gb300 import Graph, inputs, programs, shard
    dist = _init(rank, world, port)
    torch.cuda.set_device(0)
    x, a, b = inputs.cfg2(np.float64, seed=seed, n=n)
    lo, hi = shard.block_range(n, world, rank)
    dev = [torch.from_numpy(v[lo:hi].copy()).cuda() for v in (x, a, b)]
    g = programs.map_reduce(hi - lo, "f64", fuse=C.DCP_FUSE_ALL)
    combs = []
    for red in ("sum", "maxabs"):
        cg = Graph()
        t = cg.input("f64", (world,))
        cg.output(cg.reduce(t, red))
        cg.fuse(C.DCP_FUSE_ALL)
        combs.append(cg)

    def local_run(lo_, hi_):
        # gloo moves host tensors: the partials go through host memory
        return [t.cpu() for t in g.run(dev)]

    def combine(j, table):
        return float(combs[j].run([table.cuda()])[0].cpu())

    s, m = shard.ShardedMapReduce(n, world, rank, local_run, combine, dist).run()
    prog = OP.map_reduce(n)
    vals, extra = oracle.run(prog, [x, a, b], detail=True)
    sid, mid = prog.outputs
    out[rank] = (s, m, extra[sid]["fsum"], extra[sid]["abs"], float(vals[mid]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_block_split_map_reduce_matches_oracle():
    res = _spawn(_map_reduce_rank, 2, 200003, 41)
    s0, m0 = res[0][:2]
    for r in range(2):
        s, m, exact, mag, mx = res[r]
        assert (s, m) == (s0, m0)
        assert abs(s - exact) <= 1e-10 * mag
        assert abs(m - mx) <= 1e-12 * mx
