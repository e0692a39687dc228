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
                 "--format=csv,noheader,nounits", "-lms", "100"],
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


def _np_dtype(d):
    import numpy as np
    return {"f32": np.float32, "f64": np.float64}[d]


class MapReduce(Workload):
    def __init__(self, dtype, n=1 << 26):
        self.dtype = dtype
        self.n = n
        self.name = "map_reduce_%s" % dtype
        self.bytes = 3 * n * (4 if dtype == "f32" else 8)

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
        plan = self.g.plan()
        self.kernels = [l["kernel"] for l in plan["launches"]]
        self.n_launch = len(self.kernels)
        self.n_launch0 = self.g0.n_kernels

    def step(self):
        self.g.run(self.dev, self.out)

    def step_opbyop(self):
        self.g0.run(self.dev, self.out0)

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
        self.host_out = [np.empty((), dtype=_np_dtype(self.dtype)) for _ in range(2)]
        self.h2d = sum(a.nbytes for a in self.pinned)
        self.d2h = sum(o.nbytes for o in self.host_out)

    def step_e2e(self):
        self.g.run_host(self.pinned, self.host_out)

    def cpu_sample(self):
        """Oracle on the full workload (2**26 elements), single thread."""
        import oracle
        from oracle import programs as OP
        prog = OP.map_reduce(self.n)
        t0 = time.perf_counter()
        oracle.run(prog, list(self.host))
        dt = time.perf_counter() - t0
        return self.bytes / dt / GB, "full workload: 2^26 elements, one oracle pass", 1


def make_workload(name, n=None):
    if name in ("map_reduce_f32", "map_reduce_f64"):
        return MapReduce(name[-3:], n or (1 << 26))
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


def _per_launch(torch, fn, steps, stream):
    """Average device duration of single launches (events around each)."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    torch.cuda.synchronize()
    for a, b in evs:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in evs) / 1e3


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

    for _ in range(args.warmup):
        wl.step()
    barrier()
    with ClockSampler(local) as clk:
        t = _time_device(torch, wl.step, args.steps, stream)
        barrier()
    if dist is not None:
        tt = torch.tensor([t], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    value = world * wl.bytes * args.steps / t / GB

    # comparison forms and roofline (rank-local)
    per_launch = _per_launch(torch, wl.step, max(5, args.steps), stream)
    if args.quick:
        if rank == 0:
            print(json.dumps({"quick": True, "workload": wl.name, "elements": wl.n,
                              "ms_per_step": t / args.steps * 1e3,
                              "value": world * wl.bytes * args.steps / t / GB,
                              "per_launch_ms": per_launch * 1e3,
                              "kernels": wl.kernels}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    for _ in range(2):
        wl.step_opbyop()
    t_op = _time_device(torch, wl.step_opbyop, max(3, args.steps // 2), stream) / max(3, args.steps // 2)
    for _ in range(2):
        wl.step_torch()
    t_torch = _time_device(torch, wl.step_torch, max(3, args.steps // 2), stream) / max(3, args.steps // 2)

    # end to end through the C ABI with host buffers
    wl.setup_e2e(torch)
    for _ in range(2):
        wl.step_e2e()
    k_e2e = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        wl.step_e2e()
    torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / k_e2e
    if dist is not None:
        tt = torch.tensor([t_e2e], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_e2e = float(tt.item())

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    peak, peak_kind = _peaks()
    achieved = wl.bytes / per_launch / GB
    kname = wl.kernels[0] if wl.kernels else None
    cpu_value, cpu_sample, cores = wl.cpu_sample()
    line = {
        "metric": wl.metric,
        "value": round(value, 2),
        "unit": wl.unit,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(t / args.steps * 1e3, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": wl.dtype,
        "data": "synthetic",
        "config": dict(wl.describe(), parallelism="replicas: one independent workload per GPU"
                       if world > 1 else "single GPU"),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": _ncu_traffic(kname),
                     "kernel": kname, "peak_source": peak_kind},
        "cpu_baseline": {"value": round(cpu_value, 4), "unit": "GB/s", "cores": cores,
                         "kind": "oracle", "sample": cpu_sample},
        "e2e": {"value": round(wl.bytes / t_e2e / GB * world, 2), "unit": "GB/s",
                "h2d_bytes_per_step": wl.h2d, "d2h_bytes_per_step": wl.d2h},
        "gpu_launches": wl.n_launch * args.steps,
        "clocks": clk.summary(),
        "op_by_op": {"value": round(wl.bytes / t_op / GB, 2), "unit": "GB/s",
                     "kernels_per_step": wl.n_launch0, "speedup_fused": round(t_op / (t / args.steps), 3)},
        "torch_eager": {"value": round(wl.bytes / t_torch / GB, 2), "unit": "GB/s",
                        "speedup_fused": round(t_torch / (t / args.steps), 3)},
    }
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
