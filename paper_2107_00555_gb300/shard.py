"""One program split over several GPUs, one process per GPU.

Two partitionings, after the paper's distributed Python (Sec. 4):

* **Block split of maps with reductions** (Sec. 4.1: element-wise operations
  on contiguous arrays are distributed as a 1-D block distribution, each rank
  computes its block with no further communication, and reduced outputs are
  combined).  Rank r owns elements [lo_r, hi_r) (sizes differ by at most
  one); it runs the fused map+reduce program on its block, producing one
  partial per reduction; one exchange (an all-gather of the partials) and a
  combination in a fixed order give every rank the same results,
  deterministic for a given number of ranks.

* **Slab split of iterated stencils with halo exchange** (Sec. 4.3: local
  views of a block distribution, advanced in time with explicit Isend /
  Irecv halo exchanges).  The first axis (z of a 3-D grid, rows of a 2-D
  grid) is split into slabs; rank r owns slab [z0_r, z1_r).  Every chunk of
  k steps, each rank receives h = k * R planes (R the stencil's radius along
  the axis) from each neighbour into the halo planes of its own buffer,
  advances its slab with halos by k steps with the library's (time-tiled)
  kernels under the global boundary rule, and keeps its own planes.  The
  planes next to a local end are wrong after the chunk (they read zeros, a
  local wrap-around or a fixed ring), but that error moves at most R planes
  per step, so after k steps it has reached the halo planes only.  At a
  global edge of a zero or fixed-ring boundary there is no halo: the local
  boundary rule is then the global one.

Compute and transport are injected: ``advance(buf, steps, out)`` advances a
local buffer by ``steps`` stencil steps (the GPU path builds it from the
library; tests may pass the oracle), and the exchange uses
``torch.distributed`` point-to-point operations -- NCCL on device buffers
(grouped, so the two directions of a pair cannot deadlock), or any other
backend through host copies.  Received halos land in the rank's own buffer
before the chunk is computed; no rank reads another rank's memory.
"""
from __future__ import annotations

from dataclasses import dataclass


def block_range(n, world, rank):
    """Elements [lo, hi) of rank `rank` in a 1-D block split of n elements over
    `world` ranks: the first n % world ranks get one element more."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad block split: n=%r world=%r rank=%r" % (n, world, rank))
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def stencil_radius(offsets, axis=0):
    """Largest |offset| of the stencil along `axis` (R)."""
    return max(abs(int(o[axis])) for o in offsets)


@dataclass
class Chunk:
    steps: int   # stencil steps in this chunk (k, or fewer for the last one)


class SlabPlan:
    """Partition and halo schedule of a slab-split iterated stencil.

    shape     global array shape (the first axis is split)
    radius    R, the stencil's largest |offset| along the first axis
    bc        "zero" | "periodic" | "fixed_ring" (the global boundary rule)
    steps     T, total stencil steps
    depth     k, steps per chunk (halo exchanges happen every k steps)
    """

    def __init__(self, shape, radius, bc, steps, world, rank, depth=2):
        self.shape = tuple(int(s) for s in shape)
        self.R = int(radius)
        self.bc = bc
        self.T = int(steps)
        self.world = int(world)
        self.rank = int(rank)
        if bc not in ("zero", "periodic", "fixed_ring"):
            raise ValueError("unknown boundary rule %r" % bc)
        n0 = self.shape[0]
        self.z0, self.z1 = block_range(n0, self.world, self.rank)
        self.n = self.z1 - self.z0
        smallest = n0 // self.world
        k = max(1, min(int(depth), self.T if self.T > 0 else 1))
        if self.R > 0:
            # a halo may not reach past the neighbour's slab
            k = max(1, min(k, smallest // self.R))
            if self.world > 1 and smallest < self.R:
                raise ValueError("slabs of %d planes are thinner than the stencil radius %d: "
                                 "use fewer ranks" % (smallest, self.R))
        self.k = k
        self.h = self.k * self.R
        periodic = bc == "periodic"
        many = self.world > 1
        self.has_lo = many and (periodic or self.rank > 0) and self.h > 0
        self.has_hi = many and (periodic or self.rank < self.world - 1) and self.h > 0
        self.hl = self.h if self.has_lo else 0
        self.hh = self.h if self.has_hi else 0
        self.left = (self.rank - 1) % self.world
        self.right = (self.rank + 1) % self.world
        self.local_shape = (self.hl + self.n + self.hh,) + self.shape[1:]

    @property
    def chunks(self):
        out, t = [], 0
        while t < self.T:
            s = min(self.k, self.T - t)
            out.append(Chunk(s))
            t += s
        return out

    def owned(self, buf):
        """The rank's own planes inside a local buffer (a view)."""
        return buf[self.hl:self.hl + self.n]

    def slab_of(self, global_array):
        """The rank's own planes of a global array (a view)."""
        return global_array[self.z0:self.z1]

    def send_lo(self, buf):
        """First h owned planes: the left neighbour's high halo."""
        return buf[self.hl:self.hl + self.h]

    def send_hi(self, buf):
        """Last h owned planes: the right neighbour's low halo."""
        return buf[self.hl + self.n - self.h:self.hl + self.n]

    def recv_lo(self, buf):
        return buf[:self.hl]

    def recv_hi(self, buf):
        return buf[self.hl + self.n:]

    def describe(self):
        return ("z-slabs of the first axis over %d GPUs, halo of %d plane(s) exchanged every %d "
                "step(s)" % (self.world, self.h, self.k))


def halo_schedule(plan):
    """Point-to-point operations of one halo exchange as (kind, peer, tag,
    region), in a canonical order: sends to the left then to the right,
    receives from the right then from the left.  Tag 1 carries a rank's
    first planes (its left neighbour's high halo), tag 2 its last planes
    (its right neighbour's low halo).  Between two ranks that are each
    other's left and right neighbour (two ranks, periodic) the messages then
    also match in posting order, which NCCL requires (it ignores tags)."""
    ops = []
    if plan.world > 1 and plan.h > 0:
        left_has_hi = plan.bc == "periodic" or plan.rank > 0
        right_has_lo = plan.bc == "periodic" or plan.rank < plan.world - 1
        if left_has_hi:
            ops.append(("send", plan.left, 1, "send_lo"))
        if right_has_lo:
            ops.append(("send", plan.right, 2, "send_hi"))
        if plan.has_hi:
            ops.append(("recv", plan.right, 1, "recv_hi"))
        if plan.has_lo:
            ops.append(("recv", plan.left, 2, "recv_lo"))
    return ops


def exchange_halos(dist, plan, buf, backend=None):
    """Fills the halo planes of `buf` from the neighbours' owned planes.
    NCCL: device views are sent and received in place, as one group.  Other
    backends (gloo): through host copies, matched by tag."""
    sched = halo_schedule(plan)
    if not sched:
        return
    backend = backend or dist.get_backend()
    if backend == "nccl":
        ops = []
        for kind, peer, tag, region in sched:
            view = getattr(plan, region)(buf)
            op = dist.isend if kind == "send" else dist.irecv
            ops.append(dist.P2POp(op, view, peer, tag=tag))
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        return
    reqs, landing = [], []
    for kind, peer, tag, region in sched:
        view = getattr(plan, region)(buf)
        host = view.detach().to("cpu", copy=True).contiguous()
        if kind == "send":
            reqs.append(dist.isend(host, peer, tag=tag))
        else:
            reqs.append(dist.irecv(host, peer, tag=tag))
            landing.append((view, host))
    for req in reqs:
        req.wait()
    for view, host in landing:
        view.copy_(host)


class ShardedStencil:
    """Runs `steps` applications of a stencil on a slab-split array.

    advance(src, steps, dst) writes into `dst` the local buffer `src` advanced
    by `steps` stencil steps under the global boundary rule (both buffers of
    plan.local_shape).  `new_buffer()` returns an empty local buffer.
    """

    def __init__(self, plan, advance, new_buffer, dist=None, backend=None):
        self.plan = plan
        self.advance = advance
        self.dist = dist
        self.backend = backend
        self.a = new_buffer()
        self.b = new_buffer()

    def load(self, owned):
        """Copies the rank's own planes into the working buffer."""
        self.plan.owned(self.a)[...] = owned

    def run(self):
        """Advances the loaded slab by all steps; returns a view of the
        rank's own planes of the result."""
        for chunk in self.plan.chunks:
            if self.dist is not None:
                exchange_halos(self.dist, self.plan, self.a, self.backend)
            self.advance(self.a, chunk.steps, self.b)
            self.a, self.b = self.b, self.a
        return self.plan.owned(self.a)


def gather_partials(dist, partial, world):
    """All-gather of one partial result per rank (a 0-D or 1-element tensor);
    returns a (world,) tensor in rank order."""
    import torch
    part = partial.reshape(1)
    out = [torch.empty_like(part) for _ in range(world)]
    dist.all_gather(out, part)
    return torch.cat(out)


class ShardedMapReduce:
    """Block split of a fused map+reduce program over `world` ranks.

    local_run(lo, hi) runs the program on the rank's block [lo, hi) and
    returns one partial per reduction (0-D tensors); combine(j, table)
    combines reduction j's (world,) table of partials, laid out in rank
    order, into the final value.  With the library, both steps are its
    kernels (the fused program on the block, then a reduction of the
    gathered table); the combination order is fixed by the rank layout, so
    results are deterministic for a given number of ranks.
    """

    def __init__(self, n, world, rank, local_run, combine, dist=None):
        self.n, self.world, self.rank = int(n), int(world), int(rank)
        self.lo, self.hi = block_range(self.n, self.world, self.rank)
        self.local_run = local_run
        self.combine = combine
        self.dist = dist

    def run(self):
        parts = self.local_run(self.lo, self.hi)
        if self.dist is None or self.world == 1:
            tables = [p.reshape(1) for p in parts]
        else:
            tables = [gather_partials(self.dist, p, self.world) for p in parts]
        return [self.combine(j, t) for j, t in enumerate(tables)]

    def describe(self):
        return ("1-D blocks of %d elements over %d GPUs; one all-gather of the partial results, "
                "combined in rank order" % (self.hi - self.lo, self.world))
