#!/usr/bin/env python3
"""Benchmark of the fused executor on one batch of synthetic input per step.

Default workload (the configuration the headline metric is quoted on): the
fused map+reduce program y = exp(a*x + b) * sin(x) - 0.5*x*x with sum(y) and
max|y| over x, a, b of 2**26 float32 elements drawn N(0, 1).  One step = one
dcp_run of the fused program (one kernel).  Inputs (805 MB) exceed the 129 MB
L2, so no flush is needed between steps.

Metric: effective HBM GB/s = algorithmic bytes per step / device time per
step (algorithmic bytes = every input read once, every output written once).
Also reported: the same program op-by-op (one kernel per NumPy statement,
every temporary in device memory) and as torch eager ops (the CuPy analogue
of the paper's GPU comparison), the oracle on the host cores (cpu_baseline),
the end-to-end rate through dcp_run_host (host buffers, copies inside the
timed region), the roofline of the dominant kernel and the SM clocks sampled
during the timed region.

Other workloads (--workload): map_reduce_f64, jacobi2d (256^2 f64, 10
steps), heat3d (512^3 f64, 50 steps), batch2d (4096 instances f32, 20
steps), tanh_adjoint (256^3 f64, 20 steps, steps/s of the reverse pass).

Multi-GPU (torchrun, one rank per GPU): each rank runs its own instance of
the workload (weak scaling, no data-path collective); the time is the max
over ranks and `value` aggregates all ranks.
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


def _ncu_traffic(kernel_name):
    """DRAM bytes per launch recorded by an ncu capture of exactly this kernel
    (profiles/*.md lines 'ncu-traffic: <kernel> <bytes>'); None otherwise."""
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for line in open(path):
            m = re.match(r"\s*ncu-traffic:\s+(\S+)\s+(\d+)", line)
            if m and m.group(1) == kernel_name:
                return int(m.group(2))
    return None


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


def _np_dtype(d):
    import numpy as np
    return {"f32": np.float32, "f64": np.float64}[d]


class MapReduce(Workload):
    def __init__(self, dtype, n=1 << 26):
        self.dtype = dtype
        self.n = n
        self.name = "map_reduce_%s" % dtype
        self.bytes = 3 * n * (4 if dtype == "f32" else 8)

    # FP64 operations per element of the f64 program as executed: exp and sin
    # in binary64 have no fixed operation count, so the FP64 work is the one
    # counted by ncu on the fused kernel (22 DFMA, 4 DADD, 5 DMUL per element
    # with the kernels' own exp and sin, a DFMA counted as 2 flops)
    F64_FLOPS_PER_ELEMENT = 53

    def roof(self):
        # f32: device memory bound (3 arrays read once); f64: the FP64 pipes
        if self.dtype == "f64":
            return "alu", self.F64_FLOPS_PER_ELEMENT * self.n, "flop"
        return "hbm", self.bytes, "bytes"

    def describe(self):
        return {"workload": "fused map+reduce: y = exp(a*x+b)*sin(x) - 0.5*x*x; sum(y), max|y|",
                "elements": self.n, "dtype": self.dtype, "inputs": "x, a, b ~ N(0,1), seed 1002",
                "l2": "inputs %.0f MB > 129 MB L2: no flush between steps" % (self.bytes / 1e6),
                "algorithmic_bytes_per_step": self.bytes}

    def setup(self, torch, dev):
        from paper_2107_00555_gb300 import _capi as C
        from paper_2107_00555_gb300 import inputs, programs
        self.host = inputs.cfg2(_np_dtype(self.dtype), n=self.n)
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

    def step_e2e_staged(self):
        self.call_staged()

    def cpu_sample(self):
        """Oracle on the full workload (2**26 elements), single thread."""
        import oracle
        from oracle import programs as OP
        prog = OP.map_reduce(self.n)
        t0 = time.perf_counter()
        oracle.run(prog, list(self.host))
        dt = time.perf_counter() - t0
        return self.bytes / dt / GB, "full workload: 2^26 elements, one oracle pass", 1


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
        return "hbm", self.bytes, "bytes"

    def describe(self):
        return {"workload": "fused map + axis reduction: y = exp(a*x+b)*sin(x) - 0.5*x*x on "
                            "%dx%d; sum(y) and max|y| of every row" % self.shape,
                "dtype": "f32", "inputs": "x, a, b ~ N(0,1), seed 1002",
                "l2": "inputs %.0f MB > 129 MB L2: no flush between steps" % (3 * self.n * 4 / 1e6),
                "algorithmic_bytes_per_step": self.bytes}

    def setup(self, torch, dev):
        import numpy as np
        from paper_2107_00555_gb300 import _capi as C
        from paper_2107_00555_gb300 import inputs, programs
        self.host = [a.reshape(self.shape) for a in inputs.cfg2(np.float32, n=self.n)]
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

    def cpu_sample(self):
        """Oracle on the first 512 rows (1/16 of the workload), scaled per byte."""
        import oracle
        from oracle import programs as OP
        rows = min(512, self.shape[0])
        sub = [a[:rows] for a in self.host]
        prog = OP.map_reduce((rows, self.shape[1]), axis=1)
        t0 = time.perf_counter()
        oracle.run(prog, sub)
        dt = time.perf_counter() - t0
        return 3 * rows * self.shape[1] * 4 / dt / GB, "first %d of %d rows" % (rows, self.shape[0]), 1


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

    def roof(self):
        # FP64 ALU bound: 5 (2-D) / 7 (3-D) weighted terms per cell and step,
        # each a multiply and an add except the first (2k - 1 flops) -- the
        # step as defined; with the deferred common weight the kernels
        # execute k - 1 FP64 operations per cell and step
        npts = 5 if self.name == "jacobi2d" else 7
        steps_per_launch = self.T / max(1, self.n_launch)
        return "alu", (2 * npts - 1) * self.cells * steps_per_launch, "flop"

    def describe(self):
        form = ("2-D 5-point 0.2*(c+w+e+s+n)" if self.name == "jacobi2d"
                else "3-D 7-point 0.4*c + 0.1*(6 neighbours)")
        return {"workload": "%s, %s, %s boundary, %d steps" % (form, "x".join(map(str, self.shape)),
                                                           self.bc, self.T),
                "dtype": self.dtype, "algorithmic_bytes_per_step": self.bytes,
                "bytes_convention": "2 * steps * cells * 8 (each step reads and writes the grid)",
                "l2": ("working set 1 MiB: L2-resident, launch-latency bound"
                       if self.name == "jacobi2d" else "grid 1.07 GB > L2")}

    def setup(self, torch, dev):
        from paper_2107_00555_gb300 import _capi as C
        from paper_2107_00555_gb300 import inputs, programs
        if self.name == "jacobi2d":
            self.host = [inputs.cfg1(n=self.shape[0])]
        else:
            self.host = [inputs.cfg3(n=self.shape[0])]
        self.dev = [torch.from_numpy(a).to(dev) for a in self.host]
        build = programs.jacobi2d if self.name == "jacobi2d" else programs.heat3d
        self.g = build(self.shape, self.T, self.bc, self.dtype)
        if self.name == "jacobi2d":
            self.g.set_option(C.DCP_OPT_USE_GRAPH, 1)
        # tile shape, depth and kernel form picked by the autotuner on the first
        # (warm-up) run
        self.g.fuse(C.DCP_FUSE_ALL | C.DCP_AUTOTUNE)
        self.g0 = build(self.shape, self.T, self.bc, self.dtype, fuse=0)
        self.out = self.g.empty_outputs(dev)
        self.out0 = self.g0.empty_outputs(dev)
        # buffers marshalled once: a step is one C call (the 256^2 run is
        # shorter than the Python-side checks of an unprepared call)
        self.call = self.g.prepare(self.dev, self.out)
        self.call0 = self.g0.prepare(self.dev, self.out0)
        self.kernels = [l["kernel"] for l in self.g.plan()["launches"]]
        self.n_launch = len(self.kernels)
        self.n_launch0 = self.g0.n_kernels

    def step(self):
        self.call()

    def step_opbyop(self):
        self.call0()

    def legs(self):
        return [("op_by_op", self.step_opbyop, self.n_launch0), ("torch_eager", self.step_torch, None)]

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

    def cpu_sample(self):
        import oracle
        from oracle import programs as OP
        if self.name == "jacobi2d":
            prog = OP.jacobi2d(self.shape, self.T, self.bc)
            t0 = time.perf_counter()
            oracle.run(prog, self.host)
            dt = time.perf_counter() - t0
            return self.bytes / dt / GB, "full workload (256^2, 10 steps)", 1
        # 3-D: 2 of the 50 steps on the full 512^3 grid, scaled per step
        prog = OP.heat3d(self.shape, 2, self.bc)
        t0 = time.perf_counter()
        oracle.run(prog, self.host)
        dt = time.perf_counter() - t0
        return 2 * 2 * self.cells * 8 / dt / GB, "2 of 50 steps on the full 512^3 grid", 1


class Batch(Workload):
    """4096 independent 2-D 5-point instances, float32, 20 steps, one launch."""

    def __init__(self, name="batch2d"):
        self.name = name
        self.dtype = "f32"
        self.T = 20

    def roof(self):
        # compulsory device-memory traffic of one launch: every instance read
        # and written once (the launch advances all instances `depth` steps)
        return "hbm", 2 * self.cells * 4, "bytes"

    def describe(self):
        return {"workload": "4096 independent 2-D 5-point instances (0.2 weights, zero boundary), "
                            "side log-uniform in [32, 512], 20 steps each, one batched launch",
                "instances": len(self.sides), "cells": int(self.cells), "dtype": "f32",
                "algorithmic_bytes_per_step": self.bytes,
                "bytes_convention": "2 * steps * cells * 4 (each step reads and writes every grid)"}

    def setup(self, torch, dev):
        from paper_2107_00555_gb300 import _capi as C
        from paper_2107_00555_gb300 import inputs, programs
        self.host = inputs.cfg4()
        self.sides = [a.shape[0] for a in self.host]
        self.cells = sum(a.size for a in self.host)
        self.bytes = 2 * self.T * self.cells * 4
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

    def cpu_sample(self):
        import oracle
        from oracle import programs as OP
        sample = self.host[:64]
        cells = sum(a.size for a in sample)
        t0 = time.perf_counter()
        for a in sample:
            oracle.run(OP.jacobi2d(a.shape, self.T, "zero"), [a])
        dt = time.perf_counter() - t0
        return 2 * self.T * cells * 4 / dt / GB, "first 64 of 4096 instances, all 20 steps", 1


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
        return "alu", 13 * cells * 2 * self.T / max(1, self.n_launch), "flop"

    def describe(self):
        return {"workload": "reverse pass of u_{t+1} = tanh(S7 u_t), loss = sum(u_T^2); 256^3 f64, "
                            "20 steps, periodic; forward tape + 20 reverse steps per call",
                "dtype": "f64", "tape": "full (20 states, 2.7 GB)"}

    def setup(self, torch, dev):
        from paper_2107_00555_gb300 import _capi as C
        from paper_2107_00555_gb300 import inputs, programs
        self.host = [inputs.cfg5(n=self.shape[0])]
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

    def cpu_sample(self):
        import oracle
        from oracle import programs as OP
        shape = (64, 64, 64)
        prog = OP.tanh_chain(shape, self.T)
        u = self.host[0][:64, :64, :64].copy()
        t0 = time.perf_counter()
        oracle.adjoint(prog, [u], [1.0])
        dt = time.perf_counter() - t0
        scale = 64 ** 3 / 256 ** 3
        return self.T / dt * scale, "64^3 sub-grid, 20 steps, scaled by cells to 256^3", 1


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


FP64_PEAK_GFLOPS = 1250.0  # nominal GB300 FP64 rate (DFMA counted as 2 flops)
HBM_NOMINAL_GBS = 8000.0   # nominal GB300 HBM3e bandwidth


def reduce_max(value, dist=None, device=None):
    """Largest `value` over all ranks.  Used for timing only: the workload
    itself has no collective (every rank runs an independent instance)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(per_rank_work, world, t_max):
    """Whole-job throughput: the work of all ranks over the slowest rank's time."""
    return world * per_rank_work / t_max


def _roofline(wl, per_launch_s):
    """Roofline of the dominant kernel from its algorithmic work per launch."""
    bound, work, unit = wl.roof()
    if bound == "hbm":
        peak, src = _peaks()
        achieved = work / per_launch_s / GB
        return {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": _ncu_traffic(wl.kernels[0]),
                "kernel": wl.kernels[0], "peak_source": src,
                "frac_of_nominal": round(achieved / HBM_NOMINAL_GBS, 4)}
    achieved = work / per_launch_s / 1e9
    return {"bound": "alu", "achieved": round(achieved, 2), "peak": FP64_PEAK_GFLOPS,
            "unit": "GFLOP/s", "frac": round(achieved / FP64_PEAK_GFLOPS, 4),
            "traffic": _ncu_traffic(wl.kernels[0]) if wl.kernels else None,
            "kernel": wl.kernels[0] if wl.kernels else None,
            "peak_source": "nominal FP64 1.25 TFLOP/s (probe measured 1.20)"}


def run_dcp(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wl = make_workload(args.workload, args.n)
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
    if hasattr(wl, "g"):
        # the autotuner may have changed the plan during the warm-up runs
        plan = wl.g.plan()
        wl.kernels = [l["kernel"] for l in plan["launches"]] or wl.kernels
        wl.n_launch = len(plan["launches"]) or wl.n_launch
    if hasattr(wl, "prog"):
        # reverse pass: its kernels, the most frequent first
        names = [l["kernel"] for l in wl.prog.plan().get("adjoint", {}).get("launches", [])]
        if names:
            wl.kernels = sorted(set(names), key=lambda k: -names.count(k))
            wl.n_launch = len(names)
    with ClockSampler(local) as clk:
        t = _time_device(torch, wl.step, args.steps, stream)
        barrier()
    t = max_over_ranks(t)
    t_step = t / args.steps
    value = weak_scaling_value(wl.value(t_step) * t_step, world, t_step)

    # per-step device times: the dominant kernel's average launch duration
    # inside a step, and the median with its 95 % interval
    times = _step_times(torch, wl.step, max(10, min(args.steps, 30)), stream)
    per_launch = statistics.mean(times) / max(1, wl.n_launch)
    med, lo, hi = median_ci95(times)
    if args.quick:
        if rank == 0:
            print(json.dumps({"quick": True, "workload": wl.name, "ms_per_step": t_step * 1e3,
                              "value": value, "per_launch_ms": per_launch * 1e3,
                              "median_ms": med * 1e3, "kernels": wl.kernels}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    extra = {}
    for name, fn, nk in wl.legs():
        k = max(3, min(args.steps // 2, 10))
        fn()
        t_leg = _time_device(torch, fn, k, stream) / k
        extra[name] = {"value": round(wl.value(t_leg), 3), "unit": wl.unit,
                       "kernels_per_step": nk, "speedup_fused": round(t_leg / t_step, 3)}
    e2e = None
    wl.setup_e2e(torch) if hasattr(wl, "setup_e2e") else None
    if getattr(wl, "h2d", None):
        wl.step_e2e()
        k_e2e = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            wl.step_e2e()
        torch.cuda.synchronize()
        t_e2e = max_over_ranks((time.perf_counter() - t0) / k_e2e)
        e2e = {"value": round(world * wl.value(t_e2e), 2), "unit": wl.unit,
               "h2d_bytes_per_step": wl.h2d, "d2h_bytes_per_step": wl.d2h}
        if hasattr(wl, "step_e2e_staged"):
            wl.step_e2e_staged()
            torch.cuda.synchronize()
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
    cpu_value, cpu_sample, cores = wl.cpu_sample()
    line = {
        "metric": wl.metric,
        "value": round(value, 3),
        "unit": wl.unit,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(t_step * 1e3, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": wl.dtype,
        "data": "synthetic",
        "config": dict(wl.describe(), parallelism="replicas: one independent workload per GPU"
                       if world > 1 else "single GPU"),
        "roofline": _roofline(wl, per_launch),
        "cpu_baseline": {"value": round(cpu_value, 6), "unit": wl.unit, "cores": cores,
                         "kind": "oracle", "sample": cpu_sample},
        "e2e": e2e,
        "gpu_launches": wl.n_launch * args.steps,
        "clocks": clk.summary(),
        "step_time_ms": {"median": round(med * 1e3, 5), "ci95": [round(lo * 1e3, 5), round(hi * 1e3, 5)],
                         "runs": len(times), "timed_separately": True},
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_reference(args):
    """The oracle (plain CPU interpreter) as the reference arm, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import oracle
    from oracle import programs as OP
    from paper_2107_00555_gb300 import inputs
    dtype = "f32" if args.workload.endswith("f32") else "f64"
    n = 1 << 22  # bounded sample per step
    host = inputs.cfg2(_np_dtype(dtype), n=n)
    prog = OP.map_reduce(n)
    for _ in range(args.warmup):
        oracle.run(prog, list(host))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(prog, list(host))
    t = (time.perf_counter() - t0) / args.steps
    bytes_ = 3 * n * (4 if dtype == "f32" else 8)
    value = bytes_ / t / GB
    sample = "2^22 of the 2^26 elements per step, single thread"
    line = {
        "impl": "reference",
        "metric": "Effective HBM GB/s",
        "value": round(value, 4),
        "unit": "GB/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(t * 1e3, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": dtype,
        "data": "synthetic",
        "config": MapReduce(dtype).describe(),
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="dcp", choices=["dcp", "reference"])
    ap.add_argument("--workload", default="map_reduce_f32")
    ap.add_argument("--n", type=int, default=None, help="element count override (profiling)")
    ap.add_argument("--quick", action="store_true",
                    help="time the fused program only (no comparison legs); for profiling")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_dcp(args)


if __name__ == "__main__":
    main()
