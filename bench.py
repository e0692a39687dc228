#!/usr/bin/env python3
"""Benchmark of the fused executor on one batch of synthetic input per step.

Default workload (the largest configuration that fits one GPU, at the
paper's binary64 arithmetic): the 3-D 7-point heat step (centre 0.4, six
neighbours 0.1) on a 512^3 float64 grid with periodic boundaries, 50 steps,
input U[-1, 1) from seed 1003 -- the heat3d form of the paper's stencil
benchmarks.  One step = one dcp_run of the fused program (50 stencil
launches).  The grid (1.07 GB) exceeds the 129 MB L2, so no flush is needed
between steps.

Metric: effective HBM GB/s = algorithmic bytes per step / device time per
step; for iterated stencils the per-step convention (every stencil step
reads and writes the grid once: 2 * steps * cells * 8 bytes).  The roofline
of the dominant kernel is reported against the bound that holds on GB300:
the FP64 pipes for binary64 programs (the 13 flops of the 7-point step as
defined, over the FP64 rate measured in the same run by dcp_probe_fp64),
with the FP64 issue fraction and the HBM fraction alongside; device memory
for float32 programs.  Also reported: the same program op-by-op (one kernel
per NumPy statement) and as torch eager ops (the CuPy analogue of the
paper's GPU comparison), the oracle on the host cores (cpu_baseline: one
thread, and the OpenMP build on every core), the end-to-end rate through
dcp_run_host (host buffers, copies inside the timed region), and the SM
clocks sampled during the timed region.

Other workloads (--workload): map_reduce_f32 / map_reduce_f64 (2^26
elements), map_reduce_rows_f32, jacobi2d (256^2 f64, 10 steps), batch2d
(4096 instances f32, 20 steps), tanh_adjoint (256^3 f64, 20 steps, steps/s
of the reverse pass), tanh_adjoint_2d (4096^2 f32, 20 steps, the time-tiled
reverse pass that recomputes each chunk's forward states in its tiles).

--impl reference times the oracle (the plain CPU interpreter the kernels are
checked against) on the same workload and config, with the same bounded
sample as the main line's cpu_baseline.

Multi-GPU (torchrun, one rank per GPU): heat3d and map_reduce_* split ONE
problem over the ranks (z-slabs with halo exchange; 1-D blocks with one
exchange of partial results; strong scaling); the other workloads run one
independent instance per rank (weak scaling, no data-path collective).  The
time is the max over ranks and `value` is the whole job's rate.
"""
from __future__ import annotations

import argparse
import glob
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GB = 1e9


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        time.sleep(0.25)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        for line in self.lines:
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

class Workload:
    name = ""
    dtype = ""
    metric = "Effective HBM GB/s"
    unit = "GB/s"
    higher_is_better = True

    def setup(self, torch, dev):
        raise NotImplementedError

    def step(self):
        raise NotImplementedError

    def value(self, t_step):
        """Metric value for one step taking t_step seconds."""
        return self.bytes / t_step / GB

    # -- the oracle on the host cores (cpu_baseline and the reference arm) --
    # cpu_run() times one bounded sample of the workload through the oracle
    # and returns its seconds; cpu_value(t) turns a sample time into the
    # metric; cpu_scale is (one whole workload step) / (one sample), used to
    # state the reference arm's ms_per_step; cpu_desc says what a sample is.
    cpu_scale = 1.0

    def cpu_value(self, t):
        return self.value(t)


def _np_dtype(d):
    import numpy as np
    return {"f32": np.float32, "f64": np.float64}[d]


class MapReduce(Workload):
    def __init__(self, dtype, n=1 << 26):
        self.dtype = dtype
        self.n = n
        self.name = "map_reduce_%s" % dtype
        self.bytes = 3 * n * (4 if dtype == "f32" else 8)

    def roof(self):
        # f32: device memory bound (3 arrays read once).  f64: bound by the
        # FP64 pipes; exp and sin in binary64 have no algorithmic flop
        # count, so the f64 line reports how busy the FP64 pipe is (the FP64
        # instructions per element that ncu counted on this exact kernel,
        # recorded in profiles/, over the probe's rate) and the HBM fraction
        # (a sharded rank's map kernel reads its own block)
        n = getattr(self, "roof_elements", self.n)
        nbytes = 3 * n * (4 if self.dtype == "f32" else 8)
        if self.dtype == "f64":
            return {"bound": "alu_issue", "hbm_bytes": nbytes, "elements": n}
        return {"bound": "hbm", "bytes": nbytes}

    def describe(self):
        return {"workload": "fused map+reduce: y = exp(a*x+b)*sin(x) - 0.5*x*x; sum(y), max|y|",
                "elements": self.n, "dtype": self.dtype, "inputs": "x, a, b ~ N(0,1), seed 1002",
                "l2": "inputs %.0f MB > 129 MB L2: no flush between steps" % (self.bytes / 1e6),
                "algorithmic_bytes_per_step": self.bytes}

    def host_setup(self):
        from paper_2107_00555_gb300 import inputs
        self.host = inputs.cfg2(_np_dtype(self.dtype), n=self.n)

    def setup(self, torch, dev):
        from paper_2107_00555_gb300 import _capi as C
        from paper_2107_00555_gb300 import programs
        self.host_setup()
        self.dev = [torch.from_numpy(a).to(dev) for a in self.host]
        self.g = programs.map_reduce(self.n, self.dtype, fuse=C.DCP_FUSE_ALL)
        self.g0 = programs.map_reduce(self.n, self.dtype, fuse=0)
        self.out = self.g.empty_outputs(dev)
        self.out0 = self.g0.empty_outputs(dev)
        # buffers marshalled once: a step is one C call
        self.call = self.g.prepare(self.dev, self.out)
        self.call0 = self.g0.prepare(self.dev, self.out0)
        plan = self.g.plan()
        self.kernels = [l["kernel"] for l in plan["launches"]]
        self.n_launch = len(self.kernels)
        self.n_launch0 = self.g0.n_kernels

    def step(self):
        self.call()

    def step_opbyop(self):
        self.call0()

    def legs(self):
        return [("op_by_op", self.step_opbyop, self.n_launch0), ("torch_eager", self.step_torch, None)]

    def step_torch(self):
        import torch
        x, a, b = self.dev
        y = torch.exp(a * x + b) * torch.sin(x) - 0.5 * x * x
        return y.sum(), y.abs().max()

    # end-to-end through the C ABI with host buffers (pinned)
    def setup_e2e(self, torch):
        import numpy as np
        self.pinned = []
        for a in self.host:
            t = torch.empty(a.shape, dtype=torch.from_numpy(a).dtype, pin_memory=True)
            t.copy_(torch.from_numpy(a))
            self.pinned.append(t.numpy())
        # page-locked outputs too: the kernels then access host memory directly
        tdt = torch.float32 if self.dtype == "f32" else torch.float64
        self.host_out = [torch.empty((), dtype=tdt, pin_memory=True).numpy() for _ in range(2)]
        self.h2d = sum(a.nbytes for a in self.pinned)
        self.d2h = sum(o.nbytes for o in self.host_out)
        # the same call forced through device staging copies, for comparison
        from paper_2107_00555_gb300 import _capi as C
        from paper_2107_00555_gb300 import programs
        self.g_staged = programs.map_reduce(self.n, self.dtype)
        self.g_staged.set_option(C.DCP_OPT_HOST_ACCESS, 0)
        self.g_staged.fuse(C.DCP_FUSE_ALL)
        self.call_host = self.g.prepare_host(self.pinned, self.host_out)
        self.call_staged = self.g_staged.prepare_host(self.pinned, self.host_out)

    def step_e2e(self):
        # page-locked host buffers: the fused kernel reads them directly
        self.call_host()

    # -- one problem split over several GPUs (torchrun): 1-D blocks
    shardable = True

    def shard_desc(self, world):
        from paper_2107_00555_gb300 import shard
        return shard.ShardedMapReduce(self.n, world, 0, None, None).describe()

    def setup_sharded(self, torch, dev, dist, rank, world):
        from paper_2107_00555_gb300 import _capi as C
        from paper_2107_00555_gb300 import Graph, programs, shard
        self.host_setup()
        lo, hi = shard.block_range(self.n, world, rank)
        self.dev = [torch.from_numpy(a[lo:hi].copy()).to(dev) for a in self.host]
        self.g = programs.map_reduce(hi - lo, self.dtype, fuse=C.DCP_FUSE_ALL)
        self.out = self.g.empty_outputs(dev)
        call = self.g.prepare(self.dev, self.out)
        combs = []
        for red in ("sum", "maxabs"):
            g = Graph()
            t = g.input(self.dtype, (world,))
            g.output(g.reduce(t, red))
            g.fuse(C.DCP_FUSE_ALL)
            combs.append(g)
        self.combine_graphs = combs

        def local_run(lo_, hi_):
            return call()

        def combine(j, table):
            return combs[j].run([table.contiguous()])[0]

        self.sm = shard.ShardedMapReduce(self.n, world, rank, local_run, combine, dist)
        self.kernels = [l["kernel"] for l in self.g.plan()["launches"]]
        self.n_launch = len(self.kernels) + 2
        # roofline of the block's map kernel: the step is that launch plus two
        # one-CTA combines and an all-gather of a few bytes
        self.roof_elements = hi - lo
        self.roof_launches = 1
        self.legs = lambda: []
        self.step = self.sm.run
        self.setup_e2e = self._setup_e2e_sharded
        self.step_e2e = self._step_e2e_sharded

    def _setup_e2e_sharded(self, torch):
        # this rank's blocks from page-locked host memory, the results back
        self.pin_in = []
        for t in self.dev:
            p = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
            p.copy_(t)
            self.pin_in.append(p)
        self.pin_out = [torch.empty((), dtype=self.dev[0].dtype, pin_memory=True) for _ in range(2)]
        self.h2d = sum(p.numel() * p.element_size() for p in self.pin_in)
        self.d2h = sum(p.element_size() for p in self.pin_out)

    def _step_e2e_sharded(self):
        for d, p in zip(self.dev, self.pin_in):
            d.copy_(p, non_blocking=True)
        res = self.sm.run()
        for p, r in zip(self.pin_out, res):
            p.copy_(r, non_blocking=True)

    def step_e2e_staged(self):
        self.call_staged()

    cpu_desc = "the full workload step: one oracle pass over all 2^26 elements"

    def cpu_run(self):
        import oracle
        from oracle import programs as OP
        prog = OP.map_reduce(self.n)
        t0 = time.perf_counter()
        oracle.run(prog, list(self.host))
        return time.perf_counter() - t0


class MapReduceRows(Workload):
    """The map+reduce program reduced along rows: 8192 x 8192 f32 inputs,
    sum and max|y| of every row (a fused axis reduction, one kernel)."""

    def __init__(self, name="map_reduce_rows_f32", n=None):
        self.name = name
        self.dtype = "f32"
        side = n or 8192
        self.shape = (side, side)
        self.n = side * side
        self.bytes = 3 * self.n * 4 + 2 * side * 4

    def roof(self):
        return {"bound": "hbm", "bytes": self.bytes}

    def describe(self):
        return {"workload": "fused map + axis reduction: y = exp(a*x+b)*sin(x) - 0.5*x*x on "
                            "%dx%d; sum(y) and max|y| of every row" % self.shape,
                "dtype": "f32", "inputs": "x, a, b ~ N(0,1), seed 1002",
                "l2": "inputs %.0f MB > 129 MB L2: no flush between steps" % (3 * self.n * 4 / 1e6),
                "algorithmic_bytes_per_step": self.bytes}

    def host_setup(self):
        import numpy as np
        from paper_2107_00555_gb300 import inputs
        self.host = [a.reshape(self.shape) for a in inputs.cfg2(np.float32, n=self.n)]

    def setup(self, torch, dev):
        from paper_2107_00555_gb300 import _capi as C
        from paper_2107_00555_gb300 import programs
        self.host_setup()
        self.dev = [torch.from_numpy(a).to(dev) for a in self.host]
        self.g = programs.map_reduce(self.shape, "f32", fuse=C.DCP_FUSE_ALL, axis=1)
        self.g0 = programs.map_reduce(self.shape, "f32", fuse=0, axis=1)
        self.out = self.g.empty_outputs(dev)
        self.out0 = self.g0.empty_outputs(dev)
        self.call = self.g.prepare(self.dev, self.out)
        self.call0 = self.g0.prepare(self.dev, self.out0)
        self.kernels = [l["kernel"] for l in self.g.plan()["launches"]]
        self.n_launch = len(self.kernels)
        self.n_launch0 = self.g0.n_kernels

    def step(self):
        self.call()

    def legs(self):
        return [("op_by_op", self.call0, self.n_launch0),
                ("torch_eager", self.step_torch, None)]

    def step_torch(self):
        import torch
        x, a, b = self.dev
        y = torch.exp(a * x + b) * torch.sin(x) - 0.5 * x * x
        return y.sum(dim=1), y.abs().amax(dim=1)

    def setup_e2e(self, torch):
        import numpy as np
        self.pinned = []
        for a in self.host:
            t = torch.empty(a.shape, dtype=torch.float32, pin_memory=True)
            t.copy_(torch.from_numpy(a))
            self.pinned.append(t.numpy())
        self.host_out = [torch.empty((self.shape[0],), dtype=torch.float32, pin_memory=True).numpy()
                         for _ in range(2)]
        self.h2d = sum(a.nbytes for a in self.pinned)
        self.d2h = sum(o.nbytes for o in self.host_out)
        self.call_host = self.g.prepare_host(self.pinned, self.host_out)

    def step_e2e(self):
        self.call_host()

    @property
    def cpu_rows(self):
        return min(512, self.shape[0])

    @property
    def cpu_desc(self):
        return "the first %d of the %d rows, scaled per byte" % (self.cpu_rows, self.shape[0])

    @property
    def cpu_scale(self):
        return self.shape[0] / self.cpu_rows

    def cpu_value(self, t):
        return 3 * self.cpu_rows * self.shape[1] * 4 / t / GB

    def cpu_run(self):
        import oracle
        from oracle import programs as OP
        sub = [a[:self.cpu_rows] for a in self.host]
        prog = OP.map_reduce((self.cpu_rows, self.shape[1]), axis=1)
        t0 = time.perf_counter()
        oracle.run(prog, sub)
        return time.perf_counter() - t0


class Stencil(Workload):
    """Iterated stencil workloads; bytes follow the per-step convention
    (every step reads and writes the whole grid once: 2 * T * cells * size)."""

    def __init__(self, name, n=None):
        self.name = name
        import numpy as np
        if name == "jacobi2d":
            self.shape, self.T, self.bc, self.dtype = (256, 256), 10, "zero", "f64"
        elif name == "heat3d":
            self.shape, self.T, self.bc, self.dtype = (512, 512, 512), 50, "periodic", "f64"
        else:
            raise SystemExit("unknown workload %s" % name)
        if n:  # smaller grid of the same program (profiling)
            self.shape = (n,) * len(self.shape)
        self.cells = int(np.prod(self.shape))
        self.size = 8
        self.bytes = 2 * self.T * self.cells * self.size

    @property
    def npts(self):
        return 5 if self.name == "jacobi2d" else 7

    def roof(self):
        # FP64 ALU bound.  Algorithmic work: the step as defined, p weighted
        # terms per cell (a multiply and an add each, except the first add:
        # 2p - 1 flops; 13 for the 7-point step).  Alongside: the FP64
        # instructions the kernels execute per useful cell and step (p - 1
        # on a deferred common weight, plus one multiply at chunk ends; p for
        # the plain weighted sum), and the compulsory device-memory traffic
        # of one launch (the grid read once and written once).
        # (a sharded rank's launches process its slab with halos)
        cells = getattr(self, "roof_cells", self.cells)
        steps_per_launch = self.T / max(1, self.n_launch)
        return {"bound": "alu",
                "flops": (2 * self.npts - 1) * cells * steps_per_launch,
                "fp64_inst": self.fp64_inst_per_cell_step * cells * steps_per_launch,
                "fp64_inst_per_cell_step": self.fp64_inst_per_cell_step,
                "hbm_bytes": 2 * cells * self.size}

    def plan_model(self, plan):
        """FP64 instructions per useful cell and step, averaged over the run,
        from the plan's per-step deferral factors."""
        total, steps = 0.0, 0
        for l in plan["launches"]:
            lo, hi = l["steps"]
            scales = l.get("deferred_scales")
            for k in range(hi - lo):
                if scales is None:
                    total += self.npts          # one multiply + p - 1 FMAs
                else:
                    f = scales[k] if k < len(scales) else 1
                    total += (self.npts - 1) + (0 if f == 1 else 1)
                steps += 1
        self.fp64_inst_per_cell_step = total / max(1, steps)

    def describe(self):
        form = ("2-D 5-point 0.2*(c+w+e+s+n)" if self.name == "jacobi2d"
                else "3-D 7-point 0.4*c + 0.1*(6 neighbours) (heat3d form)")
        grid_mb = self.cells * self.size / 1e6
        return {"workload": "%s, %s, %s boundary, %d steps" % (form, "x".join(map(str, self.shape)),
                                                           self.bc, self.T),
                "dtype": self.dtype,
                "inputs": ("U[0,1), seed 1001" if self.name == "jacobi2d" else "U[-1,1), seed 1003"),
                "algorithmic_bytes_per_step": self.bytes,
                "bytes_convention": "2 * steps * cells * 8 (each step reads and writes the grid)",
                "l2": ("working set %.1f MB: L2-resident, launch-latency bound" % (2 * grid_mb)
                       if grid_mb * 2 < 129 else
                       "grid %.0f MB > 129 MB L2: no flush between steps" % grid_mb)}

    def host_setup(self):
        from paper_2107_00555_gb300 import inputs
        if self.name == "jacobi2d":
            self.host = [inputs.cfg1(n=self.shape[0])]
        else:
            self.host = [inputs.cfg3(n=self.shape[0])]

    def setup(self, torch, dev):
        from paper_2107_00555_gb300 import _capi as C
        from paper_2107_00555_gb300 import programs
        self.host_setup()
        self.dev = [torch.from_numpy(a).to(dev) for a in self.host]
        build = programs.jacobi2d if self.name == "jacobi2d" else programs.heat3d
        self.g = build(self.shape, self.T, self.bc, self.dtype)
        if self.name == "jacobi2d":
            # the small grid: tile shape, depth, kernel form and CTA size picked
            # by the autotuner on the first (warm-up) run; CUDA-graph replay
            self.g.set_option(C.DCP_OPT_USE_GRAPH, 1)
            self.g.fuse(C.DCP_FUSE_ALL | C.DCP_AUTOTUNE)
        else:
            # 512^3: the planner's tiles (candidate tiles change the step by
            # under 1 %), so the kernels, and the names its ncu counters are
            # recorded under, are the same on every run
            self.g.fuse(C.DCP_FUSE_ALL)
        self.g0 = build(self.shape, self.T, self.bc, self.dtype, fuse=0)
        self.out = self.g.empty_outputs(dev)
        self.out0 = self.g0.empty_outputs(dev)
        self.call_coop = None
        if self.name == "jacobi2d":
            # the cooperative form: all 10 steps in one launch on 152 tiles of
            # 14 x 32, neighbour flags between steps (graph replay as well)
            self.gc = build(self.shape, self.T, self.bc, self.dtype)
            self.gc.set_option(C.DCP_OPT_STENCIL_KERNEL, 2)
            self.gc.set_option(C.DCP_OPT_TILE_Y, 14)
            self.gc.set_option(C.DCP_OPT_TILE_X, 32)
            self.gc.set_option(C.DCP_OPT_USE_GRAPH, 1)
            self.gc.fuse(C.DCP_FUSE_ALL)
            self.outc = self.gc.empty_outputs(dev)
            self.call_coop = self.gc.prepare(self.dev, self.outc)
        # buffers marshalled once: a step is one C call (the 256^2 run is
        # shorter than the Python-side checks of an unprepared call)
        self.call = self.g.prepare(self.dev, self.out)
        self.call0 = self.g0.prepare(self.dev, self.out0)
        plan = self.g.plan()
        self.kernels = [l["kernel"] for l in plan["launches"]]
        self.n_launch = len(self.kernels)
        self.n_launch0 = self.g0.n_kernels
        self.plan_model(plan)

    def step(self):
        self.call()

    def step_opbyop(self):
        self.call0()

    def legs(self):
        legs = [("op_by_op", self.step_opbyop, self.n_launch0), ("torch_eager", self.step_torch, None)]
        if self.call_coop is not None:
            legs.append(("cooperative_one_launch", self.call_coop, 1))
        return legs

    def step_torch(self):
        """The paper's NumPy form as torch eager ops (slices into temporaries)."""
        import torch
        A = self.dev[0]
        if self.name == "jacobi2d":
            P = torch.zeros((A.shape[0] + 2, A.shape[1] + 2), dtype=A.dtype, device=A.device)
            P[1:-1, 1:-1] = A
            for _ in range(self.T):
                B = 0.2 * (P[1:-1, 1:-1] + P[1:-1, :-2] + P[1:-1, 2:] + P[2:, 1:-1] + P[:-2, 1:-1])
                P[1:-1, 1:-1] = B
            return P
        U = A
        for _ in range(self.T):
            U = 0.4 * U + 0.1 * (torch.roll(U, 1, 2) + torch.roll(U, -1, 2) + torch.roll(U, 1, 1)
                                 + torch.roll(U, -1, 1) + torch.roll(U, 1, 0) + torch.roll(U, -1, 0))
        return U

    def setup_e2e(self, torch):
        import numpy as np
        t = torch.empty(self.shape, dtype=torch.float64, pin_memory=True)
        t.copy_(torch.from_numpy(self.host[0]))
        self.pinned = [t.numpy()]
        self.host_out = [torch.empty(self.shape, dtype=torch.float64, pin_memory=True).numpy()]
        self.h2d = self.pinned[0].nbytes
        self.d2h = self.host_out[0].nbytes
        self.call_host = self.g.prepare_host(self.pinned, self.host_out)

    def step_e2e(self):
        self.call_host()

    # -- one problem split over several GPUs (torchrun): z-slabs, halo exchange
    @property
    def shardable(self):
        return self.name == "heat3d"

    def shard_desc(self, world):
        from paper_2107_00555_gb300 import shard
        plan = shard.SlabPlan(self.shape, 1, self.bc, self.T, world, 0, self.shard_depth)
        return plan.describe()

    shard_depth = int(os.environ.get("DCP_SHARD_DEPTH", "2"))

    def setup_sharded(self, torch, dev, dist, rank, world):
        from paper_2107_00555_gb300 import _capi as C
        from paper_2107_00555_gb300 import programs, shard
        self.host_setup()
        offs = programs.SEVEN_POINT
        plan = shard.SlabPlan(self.shape, shard.stencil_radius(offs), self.bc, self.T, world, rank,
                              self.shard_depth)
        self.plan_sh = plan
        self.slab_host = plan.slab_of(self.host[0])
        self.slab_dev = torch.from_numpy(self.slab_host.copy()).to(dev)
        bufs = [torch.zeros(plan.local_shape, dtype=torch.float64, device=dev) for _ in range(2)]
        self.local_graphs, calls = {}, {}
        for c in plan.chunks:
            if c.steps in self.local_graphs:
                continue
            g = programs.heat3d(plan.local_shape, c.steps, self.bc, self.dtype)
            g.fuse(C.DCP_FUSE_ALL)
            self.local_graphs[c.steps] = g
            for i in range(2):
                calls[(c.steps, i)] = g.prepare([bufs[i]], [bufs[1 - i]])
        handle = {id(bufs[0]): 0, id(bufs[1]): 1}

        def advance(src, k, dst):
            calls[(k, handle[id(src)])]()

        it = iter(bufs)
        self.ss = shard.ShardedStencil(plan, advance, lambda: next(it), dist,
                                       backend=dist.get_backend())
        g0 = self.local_graphs[plan.chunks[0].steps]
        plan0 = g0.plan()
        self.kernels = [l["kernel"] for l in plan0["launches"]]
        self.n_launch = sum(len(self.local_graphs[c.steps].plan()["launches"]) for c in plan.chunks)
        self.plan_model({"launches": [l for c in plan.chunks
                                      for l in self.local_graphs[c.steps].plan()["launches"]]})
        self.roof_cells = 1
        for d in plan.local_shape:
            self.roof_cells *= d
        self.legs = lambda: []
        self.step = self._step_sharded
        self.setup_e2e = self._setup_e2e_sharded
        self.step_e2e = self._step_e2e_sharded

    def _step_sharded(self):
        self.ss.load(self.slab_dev)
        return self.ss.run()

    def _setup_e2e_sharded(self, torch):
        # this rank's slab from page-locked host memory, its result back to it
        self.pin_in = torch.empty(self.slab_dev.shape, dtype=torch.float64, pin_memory=True)
        self.pin_in.copy_(torch.from_numpy(self.slab_host))
        self.pin_out = torch.empty_like(self.pin_in, pin_memory=True)
        self.h2d = self.pin_in.numel() * 8
        self.d2h = self.pin_out.numel() * 8

    def _step_e2e_sharded(self):
        self.slab_dev.copy_(self.pin_in, non_blocking=True)
        res = self._step_sharded()
        self.pin_out.copy_(res, non_blocking=True)

    # the oracle: the whole 2-D workload; for 3-D one of the steps on a slab
    # of at most 64 planes with the full x-y extent (the same work per cell;
    # periodic in the slab), scaled per cell
    @property
    def cpu_planes(self):
        return self.shape[0] if len(self.shape) == 2 else min(64, self.shape[0])

    @property
    def cpu_desc(self):
        if len(self.shape) == 2:
            return "the full workload step (%s, %d steps)" % ("x".join(map(str, self.shape)), self.T)
        return ("one of the %d steps on a %dx%dx%d slab (the full x-y extent; the same work per "
                "cell), scaled per cell" % (self.T, self.cpu_planes, self.shape[1], self.shape[2]))

    @property
    def cpu_scale(self):
        if len(self.shape) == 2:
            return 1.0
        return self.T * self.shape[0] / self.cpu_planes

    def cpu_value(self, t):
        return self.bytes / (t * self.cpu_scale) / GB

    def cpu_run(self):
        import oracle
        from oracle import programs as OP
        if len(self.shape) == 2:
            prog = OP.jacobi2d(self.shape, self.T, self.bc)
            u = self.host[0]
        else:
            u = self.host[0][:self.cpu_planes]
            prog = OP.heat3d(u.shape, 1, self.bc)
        t0 = time.perf_counter()
        oracle.run(prog, [u])
        return time.perf_counter() - t0


class Batch(Workload):
    """4096 independent 2-D 5-point instances, float32, 20 steps, one launch."""

    def __init__(self, name="batch2d"):
        self.name = name
        self.dtype = "f32"
        self.T = 20

    def roof(self):
        # compulsory device-memory traffic of one launch: every instance read
        # and written once (the launch advances all instances `depth` steps)
        return {"bound": "hbm", "bytes": 2 * self.cells * 4}

    def describe(self):
        return {"workload": "4096 independent 2-D 5-point instances (0.2 weights, zero boundary), "
                            "side log-uniform in [32, 512], 20 steps each, one batched launch",
                "instances": len(self.sides), "cells": int(self.cells), "dtype": "f32",
                "algorithmic_bytes_per_step": self.bytes,
                "bytes_convention": "2 * steps * cells * 4 (each step reads and writes every grid)"}

    def host_setup(self):
        from paper_2107_00555_gb300 import inputs
        self.host = inputs.cfg4()
        self.sides = [a.shape[0] for a in self.host]
        self.cells = sum(a.size for a in self.host)
        self.bytes = 2 * self.T * self.cells * 4

    def setup(self, torch, dev):
        from paper_2107_00555_gb300 import _capi as C
        from paper_2107_00555_gb300 import programs
        self.host_setup()
        self.dev = [torch.from_numpy(a).to(dev) for a in self.host]
        self.g = programs.batch2d(self.sides, self.T, "zero", "f32")
        self.g.set_option(C.DCP_OPT_USE_GRAPH, 1)
        # autotuned kernel form, depth and work-item size (first warm-up run)
        self.g.fuse(C.DCP_FUSE_ALL | C.DCP_BATCH | C.DCP_AUTOTUNE)
        self.out = self.g.empty_outputs(dev)
        self.kernels = [l["kernel"] for l in self.g.plan()["launches"]]
        self.n_launch = len(self.kernels)
        # 8192 buffers: marshal them once so a step is one C call
        self.call = self.g.prepare(self.dev, self.out)
        # comparison forms: every instance as its own fused program, and op by op
        self.g1 = programs.batch2d(self.sides, self.T, "zero", "f32", fuse=C.DCP_FUSE_ALL)
        self.g0 = programs.batch2d(self.sides, self.T, "zero", "f32", fuse=0)
        self.call1 = self.g1.prepare(self.dev)
        self.call0 = self.g0.prepare(self.dev)

    def step(self):
        self.call()

    def legs(self):
        return [("unbatched_fused", self.call1, self.g1.n_kernels),
                ("op_by_op", self.call0, self.g0.n_kernels)]

    def setup_e2e(self, torch):
        # every instance in page-locked host memory, read and written there
        # directly by the batched launches through dcp_run_host
        self.pinned = []
        for a in self.host:
            t = torch.empty(a.shape, dtype=torch.float32, pin_memory=True)
            t.copy_(torch.from_numpy(a))
            self.pinned.append(t.numpy())
        self.host_out = [torch.empty(a.shape, dtype=torch.float32, pin_memory=True).numpy()
                         for a in self.host]
        self.h2d = sum(a.nbytes for a in self.pinned)
        self.d2h = sum(o.nbytes for o in self.host_out)
        self.call_host = self.g.prepare_host(self.pinned, self.host_out)

    def step_e2e(self):
        self.call_host()

    cpu_desc = "the first 64 of the 4096 instances, all 20 steps, scaled per cell"

    @property
    def cpu_cells(self):
        return sum(a.size for a in self.host[:64])

    @property
    def cpu_scale(self):
        return self.cells / self.cpu_cells

    def cpu_value(self, t):
        return 2 * self.T * self.cpu_cells * 4 / t / GB

    def cpu_run(self):
        import oracle
        from oracle import programs as OP
        t0 = time.perf_counter()
        for a in self.host[:64]:
            oracle.run(OP.jacobi2d(a.shape, self.T, "zero"), [a])
        return time.perf_counter() - t0


class Adjoint(Workload):
    """Reverse pass of u_{t+1} = tanh(S u_t), loss = sum(u_T^2), 256^3 f64, T = 20."""

    metric = "adjoint steps/s"
    unit = "steps/s"

    def __init__(self, name="tanh_adjoint", n=None):
        self.name = name
        self.dtype = "f64"
        self.shape, self.T = ((n or 256),) * 3, 20
        self.bytes = None

    def value(self, t_step):
        return self.T / t_step

    def roof(self):
        # FP64 ALU bound; count the stencil arithmetic only (13 flops per cell per
        # forward step and per reverse step), tanh and its derivative excluded
        cells = self.shape[0] ** 3
        return {"bound": "alu", "flops": 13 * cells * 2 * self.T / max(1, self.n_launch)}

    def describe(self):
        return {"workload": "reverse pass of u_{t+1} = tanh(S7 u_t), loss = sum(u_T^2); 256^3 f64, "
                            "20 steps, periodic; forward tape + 20 reverse steps per call",
                "dtype": "f64", "tape": "full (20 states, 2.7 GB)"}

    def host_setup(self):
        from paper_2107_00555_gb300 import inputs
        self.host = [inputs.cfg5(n=self.shape[0])]

    def setup(self, torch, dev):
        from paper_2107_00555_gb300 import _capi as C
        from paper_2107_00555_gb300 import programs
        self.host_setup()
        self.dev = [torch.from_numpy(a).to(dev) for a in self.host]
        self.prog = programs.tanh_chain(self.shape, self.T, fuse=C.DCP_FUSE_ALL)
        self.ones = [torch.ones((), dtype=torch.float64, device=dev)]
        self.grad = [torch.empty_like(self.dev[0])]
        self.kernels = []
        self.n_launch = 2 * self.T
        self.g0 = programs.tanh_chain(self.shape, self.T, fuse=0)
        self.grad0 = [torch.empty_like(self.dev[0])]

    def step(self):
        self.prog.adjoint(self.dev, self.ones, self.grad)

    def legs(self):
        # the same call under a tape budget of 8 states (1.07 GB < the 2.7 GB
        # full tape): sqrt(T) checkpoints, segments recomputed in the reverse pass
        budget = 8 * self.dev[0].numel() * 8
        return [("op_by_op", lambda: self.g0.adjoint(self.dev, self.ones, self.grad0), None),
                ("checkpointed_8_states", lambda: self.prog.adjoint(self.dev, self.ones, self.grad,
                                                                    tape_budget_bytes=budget), None)]

    def setup_e2e(self, torch):
        # u0 from page-locked host memory, the gradient back to it
        self.torch = torch
        self.u_host = torch.empty(self.shape, dtype=torch.float64, pin_memory=True)
        self.u_host.copy_(torch.from_numpy(self.host[0]))
        self.g_host = torch.empty(self.shape, dtype=torch.float64, pin_memory=True)
        self.h2d = self.u_host.numel() * 8
        self.d2h = self.g_host.numel() * 8

    def step_e2e(self):
        self.dev[0].copy_(self.u_host, non_blocking=True)
        self.prog.adjoint(self.dev, self.ones, self.grad)
        self.g_host.copy_(self.grad[0], non_blocking=True)

    cpu_desc = "a 64^3 sub-grid, all 20 steps forward and reverse, scaled per cell"

    @property
    def cpu_scale(self):
        return self.shape[0] ** 3 / 64 ** 3

    def cpu_value(self, t):
        return self.T / (t * self.cpu_scale)

    def cpu_run(self):
        import oracle
        from oracle import programs as OP
        prog = OP.tanh_chain((64, 64, 64), self.T)
        u = self.host[0][:64, :64, :64].copy()
        t0 = time.perf_counter()
        oracle.adjoint(prog, [u], [1.0])
        return time.perf_counter() - t0


class Adjoint2D(Adjoint):
    """Reverse pass of u_{t+1} = tanh(S5 u_t), loss = sum(u_T^2), 4096^2 f32,
    periodic, T = 20, with the time-tiled reverse: every launch recomputes
    the forward states of a chunk of 3 steps inside its tiles from the
    checkpoint the forward pass stored (DCP_OPT_ADJOINT_DEPTH = 3)."""

    DEPTH = 3

    def __init__(self, name="tanh_adjoint_2d", n=None):
        self.name = name
        self.dtype = "f32"
        self.shape, self.T = ((n or 4096),) * 2, 20
        self.bytes = None

    def _graph(self, depth, fuse):
        from paper_2107_00555_gb300 import Graph, programs
        from paper_2107_00555_gb300 import _capi as C
        g = Graph()
        u = g.input("f32", self.shape)
        for _ in range(self.T):
            u = g.map("tanh", [g.stencil(u, programs.FIVE_POINT, programs.FIVE_WEIGHTS, "periodic", 1)])
        g.output(g.reduce(g.map("square", [u]), "sum"))
        g.set_option(C.DCP_OPT_ADJOINT_DEPTH, depth)
        g.fuse(C.DCP_FUSE_ALL if fuse else 0)
        return g

    def roof(self):
        # compulsory device-memory traffic of the tiled schedule: each forward
        # launch reads one state and writes one, each reverse chunk reads u_t
        # and g_{t+k} and writes g_t, the loss cotangent is written once
        k, T = self.DEPTH, self.T
        chunks = (T + k - 1) // k
        states = 2 * (chunks - 1) + 3 * chunks + 1
        nbytes = states * self.shape[0] * self.shape[1] * 4
        return {"bound": "hbm", "bytes": nbytes / max(1, self.n_launch)}

    def describe(self):
        return {"workload": "reverse pass of u_{t+1} = tanh(S5 u_t), loss = sum(u_T^2); 4096^2 "
                            "f32, 20 steps, periodic; time-tiled reverse, 3 steps per launch",
                "dtype": "f32", "tape": "every 3rd state (6 states, 403 MB)",
                "l2": "states of 67 MB; the tape and cotangents together exceed L2"}

    def host_setup(self):
        from paper_2107_00555_gb300 import inputs
        import numpy as np
        self.host = [inputs.uniform(self.shape, -1.0, 1.0, 1006).astype(np.float32)]

    def setup(self, torch, dev):
        self.host_setup()
        self.dev = [torch.from_numpy(a).to(dev) for a in self.host]
        self.prog = self._graph(self.DEPTH, True)
        self.g_step = self._graph(0, True)
        self.g0 = self._graph(0, False)
        self.ones = [torch.ones((), dtype=torch.float32, device=dev)]
        self.grad = [torch.empty_like(self.dev[0])]
        self.grad0 = [torch.empty_like(self.dev[0])]
        self.kernels = []
        self.n_launch = 2 * self.T

    def legs(self):
        return [("per_step_reverse", lambda: self.g_step.adjoint(self.dev, self.ones, self.grad0), None),
                ("op_by_op", lambda: self.g0.adjoint(self.dev, self.ones, self.grad0), None)]

    def setup_e2e(self, torch):
        self.torch = torch
        self.u_host = torch.empty(self.shape, dtype=torch.float32, pin_memory=True)
        self.u_host.copy_(torch.from_numpy(self.host[0]))
        self.g_host = torch.empty(self.shape, dtype=torch.float32, pin_memory=True)
        self.h2d = self.u_host.numel() * 4
        self.d2h = self.g_host.numel() * 4

    cpu_desc = "a 256^2 sub-grid, all 20 steps forward and reverse, scaled per cell"

    @property
    def cpu_scale(self):
        return self.shape[0] * self.shape[1] / 256 ** 2

    def cpu_run(self):
        import oracle
        prog = oracle.Program()
        u = prog.input("f64", (256, 256))
        for _ in range(self.T):
            u = prog.map("tanh", [prog.stencil(u, [(0, 0), (0, -1), (0, 1), (1, 0), (-1, 0)],
                                               [0.2] * 5, "periodic", 1)])
        prog.output(prog.reduce(prog.map("square", [u]), "sum"))
        x = self.host[0][:256, :256].astype("float64")
        t0 = time.perf_counter()
        oracle.adjoint(prog, [x], [1.0])
        return time.perf_counter() - t0


def make_workload(name, n=None):
    if name in ("map_reduce_f32", "map_reduce_f64"):
        return MapReduce(name[-3:], n or (1 << 26))
    if name == "map_reduce_rows_f32":
        return MapReduceRows(n=n)
    if name in ("jacobi2d", "heat3d"):
        return Stencil(name, n)
    if name == "batch2d":
        return Batch()
    if name == "tanh_adjoint":
        return Adjoint(n=n)
    if name == "tanh_adjoint_2d":
        return Adjoint2D(n=n)
    raise SystemExit("unknown workload %s" % name)


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def _time_device(torch, fn, steps, stream):
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(steps):
        fn()
    end.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(end) / 1e3


def _step_times(torch, fn, steps, stream):
    """Device duration of each of `steps` single steps (events around each), s."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    torch.cuda.synchronize()
    for a, b in evs:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) / 1e3 for a, b in evs]


def median_ci95(xs):
    """Median and a distribution-free 95 % confidence interval of the median
    (order statistics of the binomial(n, 1/2) law, as the paper reports its
    timings): returns (median, low, high)."""
    from math import comb
    v = sorted(xs)
    n = len(v)
    med = statistics.median(v)
    # largest k with P(Binomial(n, 1/2) < k) <= 2.5 %: [v[k-1], v[n-k]] covers >= 95 %
    k, cum = 0, 0.0
    while k < n:
        p = comb(n, k) / 2.0 ** n
        if cum + p > 0.025:
            break
        cum += p
        k += 1
    if k == 0:
        return med, v[0], v[-1]
    return med, v[k - 1], v[n - k]


FP64_NOMINAL_GFLOPS = 1250.0  # nominal GB300 FP64 rate (a DFMA counted as 2 flops)
HBM_NOMINAL_GBS = 8000.0      # nominal GB300 HBM3e bandwidth


def reduce_max(value, dist=None, device=None):
    """Largest `value` over all ranks (timing only)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(per_rank_work, world, t_max):
    """Whole-job throughput: the work of all ranks over the slowest rank's time."""
    return world * per_rank_work / t_max


def _profile_value(key, kernel_name):
    """A per-kernel figure recorded from an ncu capture of exactly this kernel
    (profiles/*.md lines '<key>: <kernel> <number>'); None otherwise, e.g.
    once the kernel's source (and so its name) has changed."""
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for line in open(path):
            m = re.match(r"\s*%s:\s+(\S+)\s+([0-9.eE+]+)" % re.escape(key), line)
            if m and m.group(1) == kernel_name:
                return float(m.group(2))
    return None


def _ncu_traffic(kernel_name):
    v = _profile_value("ncu-traffic", kernel_name)
    return int(v) if v is not None else None


def measure_fp64_peak(stream):
    """FP64 rate of this GPU, measured now by the library's probe (every SM
    running independent DFMA chains; best of three launches)."""
    from paper_2107_00555_gb300 import _capi as C
    best = 0.0
    for _ in range(3):
        g, _ms = C.dcp_probe_fp64(0, 8192, stream.cuda_stream)
        best = max(best, g)
    return {"dfma_ginst_s": round(best, 2), "gflops": round(2 * best, 2),
            "how": "dcp_probe_fp64: full-occupancy CTAs on every SM, 8 independent DFMA "
                   "chains per thread, CUDA events; a DFMA = 2 flops; best of 3"}


def _roofline(wl, per_launch_s, fp64):
    """Roofline of the dominant kernel from its algorithmic work per launch."""
    r = wl.roof()
    kernel = wl.kernels[0] if wl.kernels else None
    hbm_peak, src = _peaks()
    if r["bound"] == "hbm":
        achieved = r["bytes"] / per_launch_s / GB
        return {"bound": "hbm", "achieved": round(achieved, 2), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 4), "traffic": _ncu_traffic(kernel),
                "kernel": kernel, "peak_source": src,
                "frac_of_nominal": round(achieved / HBM_NOMINAL_GBS, 4)}
    out = {}
    if r["bound"] == "alu":
        achieved = r["flops"] / per_launch_s / 1e9
        out = {"bound": "alu", "achieved": round(achieved, 2), "peak": fp64["gflops"],
               "unit": "GFLOP/s", "frac": round(achieved / fp64["gflops"], 4),
               "traffic": _ncu_traffic(kernel), "kernel": kernel,
               "peak_source": "measured in this run (dcp_probe_fp64, DFMA rate x 2)",
               "frac_of_nominal": round(achieved / FP64_NOMINAL_GFLOPS, 4),
               "work": "algorithmic flops of the step as defined (2p - 1 per cell and step)"}
        if "fp64_inst" in r:
            ach_i = r["fp64_inst"] / per_launch_s / 1e9
            out["fp64_issue"] = {
                "inst_per_cell_step": round(r["fp64_inst_per_cell_step"], 4),
                "achieved_ginst_s": round(ach_i, 2), "peak_ginst_s": fp64["dfma_ginst_s"],
                "frac": round(ach_i / fp64["dfma_ginst_s"], 4),
                "note": "FP64 instructions per useful cell and step executed by the kernels"}
    else:  # FP64-bound without an algorithmic flop count (binary64 exp, sin)
        per_el = _profile_value("ncu-fp64-inst-per-element", kernel)
        out = {"bound": "alu", "unit": "G FP64 inst/s", "kernel": kernel,
               "traffic": _ncu_traffic(kernel), "peak": fp64["dfma_ginst_s"],
               "peak_source": "measured in this run (dcp_probe_fp64, DFMA lane rate)",
               "work": "FP64 instructions per element counted by ncu on this kernel "
                       "(issue fraction of the FP64 pipe; exp and sin have no flop count)"}
        if per_el is not None:
            ach_i = per_el * r["elements"] / per_launch_s / 1e9
            out.update(achieved=round(ach_i, 2), frac=round(ach_i / fp64["dfma_ginst_s"], 4),
                       fp64_inst_per_element=per_el)
        else:
            out.update(achieved=None, frac=None, fp64_inst_per_element=None)
    if "hbm_bytes" in r:
        ach_b = r["hbm_bytes"] / per_launch_s / GB
        out["hbm"] = {"bytes_per_launch": r["hbm_bytes"], "achieved_gbs": round(ach_b, 2),
                      "peak_gbs": hbm_peak, "frac": round(ach_b / hbm_peak, 4),
                      "peak_source": src}
    return out


def _parallelism(wl, world):
    if world <= 1:
        return "single GPU"
    if getattr(wl, "shardable", False):
        return wl.shard_desc(world)
    return "replicas: one independent workload per GPU"


def _config(wl, world):
    return dict(wl.describe(), parallelism=_parallelism(wl, world))


def cpu_baseline(wl, runs=3, all_cores=False):
    """The oracle, as it stands, on the host cores: the median of `runs`
    bounded samples (wl.cpu_run), in the workload's metric."""
    import oracle
    if all_cores:
        with oracle.all_cores() as ac:
            if not ac.available:
                return None
            wl.cpu_run()  # first call loads the OpenMP build
            t = statistics.median(wl.cpu_run() for _ in range(runs))
            cores = ac.threads
        kind = "oracle, OpenMP build (maps and stencil steps on every core; reductions and " \
               "the transposed stencil sequential)"
    else:
        t = statistics.median(wl.cpu_run() for _ in range(runs))
        cores, kind = 1, "oracle"
    return {"value": round(wl.cpu_value(t), 6), "unit": wl.unit, "cores": cores, "kind": kind,
            "sample": "%s; median of %d samples" % (wl.cpu_desc, runs)}


def run_dcp(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # one rank per GPU; more ranks than GPUs share them (gloo only: NCCL
    # takes one rank per device)
    local = local % max(1, torch.cuda.device_count())
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        if args.dist_backend == "nccl":
            dist.init_process_group("nccl", device_id=dev)
        else:
            dist.init_process_group(args.dist_backend)
    wl = make_workload(args.workload, args.n)
    sharded = world > 1 and getattr(wl, "shardable", False)
    if sharded:
        wl.setup_sharded(torch, dev, dist, rank, world)
    else:
        wl.setup(torch, dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(t):
        return reduce_max(t, dist, dev)

    for _ in range(args.warmup):
        wl.step()
    barrier()
    if hasattr(wl, "g") and not sharded:
        # the autotuner may have changed the plan during the warm-up runs; the
        # dominant (most frequent) kernel first
        plan = wl.g.plan()
        names = [l["kernel"] for l in plan["launches"]]
        if names:
            wl.kernels = sorted(set(names), key=lambda k: (-names.count(k), names.index(k)))
        wl.n_launch = len(plan["launches"]) or wl.n_launch
        if hasattr(wl, "plan_model"):
            wl.plan_model(plan)
    if hasattr(wl, "prog"):
        # reverse pass: its kernels, the most frequent first
        names = [l["kernel"] for l in wl.prog.plan().get("adjoint", {}).get("launches", [])]
        if names:
            # ties go to the time-tiled reverse kernels
            wl.kernels = sorted(set(names), key=lambda k: (-names.count(k), not k.startswith("dcp_adj")))
            wl.n_launch = len(names)
    fp64 = measure_fp64_peak(stream)
    barrier()
    with ClockSampler(local) as clk:
        t = _time_device(torch, wl.step, args.steps, stream)
        barrier()
    t = max_over_ranks(t)
    t_step = t / args.steps
    if sharded:
        value = wl.value(t_step)          # the whole problem's rate (strong scaling)
    else:
        value = weak_scaling_value(wl.value(t_step) * t_step, world, t_step)

    # per-step device times: the dominant kernel's average launch duration
    # inside a step, and the median with its 95 % interval
    times = _step_times(torch, wl.step, max(10, min(args.steps, 30)), stream)
    per_launch = statistics.mean(times) / max(1, getattr(wl, "roof_launches", wl.n_launch))
    med, lo, hi = median_ci95(times)
    if args.quick:
        if rank == 0:
            groups = wl.g.plan().get("groups") if hasattr(wl, "g") else None
            print(json.dumps({"quick": True, "workload": wl.name, "ms_per_step": t_step * 1e3,
                              "value": value, "per_launch_ms": per_launch * 1e3,
                              "median_ms": med * 1e3, "kernels": wl.kernels,
                              "fp64_peak": fp64, "groups": groups}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    extra = {}
    for name, fn, nk in wl.legs():
        k = max(3, min(args.steps // 2, 10))
        fn()
        t_leg = max_over_ranks(_time_device(torch, fn, k, stream) / k)
        extra[name] = {"value": round(wl.value(t_leg) if sharded else world * wl.value(t_leg), 3),
                       "unit": wl.unit, "kernels_per_step": nk,
                       "speedup_fused": round(t_leg / t_step, 3)}
    e2e = None
    wl.setup_e2e(torch) if hasattr(wl, "setup_e2e") else None
    if getattr(wl, "h2d", None):
        wl.step_e2e()
        k_e2e = max(3, min(args.steps, 10))
        barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            wl.step_e2e()
        torch.cuda.synchronize()
        t_e2e = max_over_ranks((time.perf_counter() - t0) / k_e2e)
        e2e = {"value": round(wl.value(t_e2e) if sharded else world * wl.value(t_e2e), 2),
               "unit": wl.unit, "h2d_bytes_per_step": wl.h2d * (world if sharded else 1),
               "d2h_bytes_per_step": wl.d2h * (world if sharded else 1)}
        if hasattr(wl, "step_e2e_staged"):
            wl.step_e2e_staged()
            barrier()
            t0 = time.perf_counter()
            for _ in range(k_e2e):
                wl.step_e2e_staged()
            torch.cuda.synchronize()
            t_st = max_over_ranks((time.perf_counter() - t0) / k_e2e)
            extra["e2e_staged_copies"] = {"value": round(world * wl.value(t_st), 2),
                                          "unit": wl.unit}

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    if not hasattr(wl, "host") or wl.host is None:
        wl.host_setup()
    line = {
        "metric": wl.metric,
        "value": round(value, 3),
        "unit": wl.unit,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(t_step * 1e3, 5),
        "higher_is_better": True,
        "scaling": "strong" if sharded else "weak",
        "vs_baseline": None,
        "dtype": wl.dtype,
        "data": "synthetic",
        "config": _config(wl, world),
        "roofline": _roofline(wl, per_launch, fp64),
        "cpu_baseline": cpu_baseline(wl),
        "cpu_baseline_all_cores": cpu_baseline(wl, all_cores=True),
        "e2e": e2e,
        "gpu_launches": wl.n_launch * args.steps,
        "clocks": clk.summary(),
        "fp64_peak_probe": fp64,
        "step_time_ms": {"median": round(med * 1e3, 5), "ci95": [round(lo * 1e3, 5), round(hi * 1e3, 5)],
                         "runs": len(times), "timed_separately": True},
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_reference(args):
    """The reference arm: the oracle (the plain CPU interpreter the kernels are
    checked against), as it stands, single-threaded on the host cores, on the
    same workload and config as the main line; every step is the workload's
    bounded sample (the one its cpu_baseline times)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    wl = make_workload(args.workload, args.n)
    wl.host_setup()
    for _ in range(args.warmup):
        wl.cpu_run()
    total = sum(wl.cpu_run() for _ in range(args.steps))
    t = total / args.steps
    value = wl.cpu_value(t)
    line = {
        "impl": "reference",
        "metric": wl.metric,
        "value": round(value, 6),
        "unit": wl.unit,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(t * wl.cpu_scale * 1e3, 3),
        "higher_is_better": True,
        "scaling": "strong" if world > 1 and getattr(wl, "shardable", False) else "weak",
        "vs_baseline": None,
        "dtype": wl.dtype,
        "data": "synthetic",
        "config": _config(wl, world),
        "cpu_baseline": {"value": round(value, 6), "unit": wl.unit, "cores": 1, "kind": "oracle",
                         "sample": "%s; one sample per timed step" % wl.cpu_desc},
        "e2e": {"value": round(value, 6), "unit": wl.unit, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_probe(args):
    """The FP64 rate of this GPU for each binary64 operation (the roofline
    denominator of the f64 workloads; an add is also timed as a fused
    multiply-add by a run-time 1.0), with the SM clocks sampled meanwhile."""
    import torch
    from paper_2107_00555_gb300 import _capi as C
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    C.dcp_probe_fp64(0, 8192, stream.cuda_stream)  # load the module, wake the clocks
    res = {}
    with ClockSampler(0) as clk:
        for op, name in ((0, "dfma"), (1, "dadd"), (2, "dmul"), (3, "dadd_as_dfma"),
                         (4, "dadd_as_dfma_own_one")):
            runs = [C.dcp_probe_fp64(op, 65536, stream.cuda_stream) for _ in range(5)]
            res[name] = {"ginst_s": round(max(g for g, _ in runs), 2),
                         "median_ginst_s": round(statistics.median(g for g, _ in runs), 2),
                         "ms": round(statistics.median(m for _, m in runs), 3)}
    props = torch.cuda.get_device_properties(0)
    print(json.dumps({"probe": "fp64", "device": props.name, "sms": props.multi_processor_count,
                      "ops": res, "gflops_dfma": round(2 * res["dfma"]["ginst_s"], 2),
                      "clocks": clk.summary()}), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="dcp", choices=["dcp", "reference"])
    ap.add_argument("--workload", default="heat3d")
    ap.add_argument("--n", "--size", dest="n", type=int, default=None,
                    help="element count or grid side override (profiling; --size under torchrun, "
                         "whose own options --n abbreviates)")
    ap.add_argument("--quick", action="store_true",
                    help="time the fused program only (no comparison legs); for profiling")
    ap.add_argument("--probe", action="store_true",
                    help="measure the FP64 rate (fma, add, mul) with clocks sampled, and exit")
    ap.add_argument("--dist-backend", default="nccl", choices=["nccl", "gloo"],
                    help="process group under torchrun (gloo moves halos and partials through "
                         "host memory; it lets several ranks share one GPU)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.probe:
        run_probe(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_dcp(args)


if __name__ == "__main__":
    main()
