"""Sharded execution over several ranks on CPU (gloo): the partition, the halo
schedule and the exchange of partial results (Sec. 4.1 block distribution of
element-wise operations; Sec. 4.3 local views with halo exchange).

Each rank advances its own slab plus halos with the oracle -- the compute a
GPU rank does with the library's kernels -- and the owned planes must equal
the whole-domain oracle's bit for bit: every cell is the same weighted sum of
the same neighbour values.  The block-split map+reduce combines per-rank
partials from an all-gather in rank order and must meet the reduction
tolerance against the whole-array oracle.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from oracle import programs as OP
from paper_2107_00555_gb300 import inputs, shard

FIVE = [(0, 0), (0, -1), (0, 1), (1, 0), (-1, 0)]
W5 = [0.2] * 5
SEVEN = [(0, 0, 0), (0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]
W7 = [0.4] + [0.1] * 6
# radius 2 along the split axis, unequal weights, one negative
WIDE = [(0, 0, 0), (-2, 0, 0), (2, 0, 0), (0, 1, 0), (0, 0, -1), (-1, 0, 1)]
WW = [0.5, 0.125, 0.25, -0.0625, 0.0625, 0.125]


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
        p.join(120)
    for p in procs:
        if p.is_alive():
            p.kill()
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    return dict(out)


def _init(rank, world, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from datetime import timedelta
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=60))


def _stencil_rank(rank, world, port, out, shape, offs, w, bc, steps, depth, seed):
    _init(rank, world, port)
    u0 = inputs.uniform(shape, -1.0, 1.0, seed)
    plan = shard.SlabPlan(shape, shard.stencil_radius(offs), bc, steps, world, rank, depth)

    def advance(src, k, dst):
        dst[...] = torch.from_numpy(oracle.stencil(src.numpy(), offs, w, bc, k))

    ss = shard.ShardedStencil(plan, advance,
                              lambda: torch.full(plan.local_shape, float("nan"), dtype=torch.float64),
                              dist)
    ss.load(torch.from_numpy(plan.slab_of(u0).copy()))
    got = ss.run().numpy().copy()
    ref = oracle.stencil(u0, offs, w, bc, steps)[plan.z0:plan.z1]
    out[rank] = (bool(np.array_equal(got, ref)), plan.k, plan.h, len(plan.chunks),
                 float(np.max(np.abs(got - ref))))
    dist.barrier()
    dist.destroy_process_group()


CASES = [
    # shape, offsets, weights, bc, steps, depth, world
    ((13, 6, 7), SEVEN, W7, "periodic", 5, 2, 2),
    ((13, 6, 7), SEVEN, W7, "zero", 5, 2, 3),
    ((13, 6, 7), SEVEN, W7, "fixed_ring", 7, 3, 3),
    ((11, 9), FIVE, W5, "zero", 6, 4, 2),
    ((11, 9), FIVE, W5, "periodic", 4, 1, 3),
    ((12, 5, 6), WIDE, WW, "periodic", 5, 2, 2),
    ((12, 5, 6), WIDE, WW, "zero", 4, 8, 3),   # depth clamped to the slab / radius
]


@pytest.mark.parametrize("shape,offs,w,bc,steps,depth,world", CASES)
def test_sharded_stencil_equals_whole_domain_oracle(shape, offs, w, bc, steps, depth, world):
    res = _spawn(_stencil_rank, world, shape, offs, w, bc, steps, depth, 11)
    for r in range(world):
        ok, k, h, nchunks, err = res[r]
        assert ok, (r, err)
        assert h == k * shard.stencil_radius(offs)
        assert nchunks == -(-steps // k)


def test_slab_plan_partition_and_schedule():
    for n0, world, R, bc in [(13, 3, 1, "zero"), (12, 2, 2, "periodic"), (9, 4, 1, "fixed_ring")]:
        plans = [shard.SlabPlan((n0, 4), R, bc, 10, world, r, depth=2) for r in range(world)]
        # slabs tile the axis in rank order, sizes differ by at most one
        assert plans[0].z0 == 0 and plans[-1].z1 == n0
        assert all(a.z1 == b.z0 for a, b in zip(plans, plans[1:]))
        assert max(p.n for p in plans) - min(p.n for p in plans) <= 1
        # halo depth never exceeds a neighbour's slab
        assert all(p.h <= min(q.n for q in plans) for p in plans)
        # every send is matched by exactly one receive with the same tag
        sends = [(p.rank, peer, tag) for p in plans for kind, peer, tag, _ in shard.halo_schedule(p)
                 if kind == "send"]
        recvs = [(peer, p.rank, tag) for p in plans for kind, peer, tag, _ in shard.halo_schedule(p)
                 if kind == "recv"]
        assert sorted(sends) == sorted(recvs)
        if bc != "periodic":
            assert plans[0].hl == 0 and plans[-1].hh == 0
    with pytest.raises(ValueError):
        shard.SlabPlan((3, 4), 2, "zero", 5, 3, 0)  # slabs thinner than the radius


def test_two_rank_periodic_messages_match_in_posting_order():
    # NCCL matches the messages between one pair of ranks in posting order;
    # with two periodic ranks both neighbours are the same peer
    p0, p1 = (shard.SlabPlan((10, 3), 1, "periodic", 4, 2, r) for r in range(2))
    s0 = [tag for kind, peer, tag, _ in shard.halo_schedule(p0) if kind == "send"]
    r1 = [tag for kind, peer, tag, _ in shard.halo_schedule(p1) if kind == "recv"]
    assert s0 == r1 == [1, 2]


def test_block_range_covers_once():
    for n in (0, 1, 7, 100, 2 ** 20 + 3):
        for world in (1, 2, 3, 8):
            ranges = [shard.block_range(n, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [hi - lo for lo, hi in ranges]
            assert max(sizes) - min(sizes) <= 1


def _map_reduce_rank(rank, world, port, out, n, seed):
    _init(rank, world, port)
    x, a, b = inputs.cfg2(np.float64, seed=seed, n=n)
    prog = OP.map_reduce(n)

    def local_run(lo, hi):
        vals, extra = oracle.run(OP.map_reduce(hi - lo), [x[lo:hi], a[lo:hi], b[lo:hi]], detail=True)
        sid, mid = OP.map_reduce(hi - lo).outputs
        return [torch.tensor(float(vals[sid]), dtype=torch.float64),
                torch.tensor(float(vals[mid]), dtype=torch.float64)]

    def combine(j, table):
        t = table.numpy()
        return float(oracle.sum_seq(t)) if j == 0 else float(oracle.reduce_ext("max", t)[0])

    sm = shard.ShardedMapReduce(n, world, rank, local_run, combine, dist)
    s, m = sm.run()
    vals, extra = oracle.run(prog, [x, a, b], detail=True)
    sid, mid = prog.outputs
    out[rank] = (s, m, extra[sid]["fsum"], extra[sid]["abs"], float(vals[mid]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_map_reduce_matches_whole_array_oracle(world):
    n = 100003
    res = _spawn(_map_reduce_rank, world, n, 21)
    first = res[0]
    for r in range(world):
        s, m, exact, mag, mx = res[r]
        assert (s, m) == first[:2]              # every rank holds the same result
        assert abs(s - exact) <= 1e-10 * mag    # backward-stable bound of any order
        assert m == mx                          # max is order-free
