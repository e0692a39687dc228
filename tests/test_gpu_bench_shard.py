"""The benchmark's multi-GPU path (one problem split over the ranks), run the
way a multi-GPU launch runs it -- torchrun, one process per rank -- with two
ranks sharing the one GPU of the box.  NCCL takes one rank per device, so
the ranks use gloo, which moves the halos and partial results through host
memory; no kernel of one rank waits on the other.  The splits themselves are
checked against the oracle in test_gpu_shard.py; this checks that the
benchmark's sharded workloads run end to end and report a strong-scaling
line."""
import json
import os
import socket
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _torchrun(args):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py")] + args + ["--dist-backend", "gloo"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-3000:]
    return json.loads(lines[0])


def test_bench_heat3d_slabs_on_two_ranks():
    line = _torchrun(["--workload", "heat3d", "--size", "64", "--steps", "2", "--warmup", "3"])
    assert line["n_gpus"] == 2 and line["scaling"] == "strong"
    assert "z-slabs" in line["config"]["parallelism"]
    assert line["value"] > 0 and line["gpu_launches"] > 0
    assert line["roofline"]["bound"] == "alu" and line["e2e"]["value"] > 0


def test_bench_map_reduce_blocks_on_two_ranks():
    line = _torchrun(["--workload", "map_reduce_f32", "--size", str(1 << 22), "--steps", "3",
                      "--warmup", "3", "--quick"])
    assert line["quick"] and line["value"] > 0
