"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): each rank
runs an independent instance of the workload; the only collective is the
timing reduction, and the reported value aggregates all ranks' work over the
slowest rank's time (weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_time = [0.25, 0.40][rank]
    t = bench.reduce_max(local_time, dist, "cpu")
    out[rank] = t
    dist.barrier()
    dist.destroy_process_group()


def test_timing_is_max_over_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert out[0] == out[1] == 0.40


def test_weak_scaling_value():
    # 2 ranks each moving 1e9 bytes; slowest rank took 0.5 s -> 4e9 B/s whole-job
    assert bench.weak_scaling_value(1e9, 2, 0.5) == 4e9
    assert bench.reduce_max(3.0) == 3.0


def test_median_confidence_interval_order_statistics():
    """The distribution-free 95 % interval of the median uses the order
    statistics of Binomial(n, 1/2): ranks (2, 9) for n = 10 and (10, 21)
    for n = 30 (1-based), the textbook values."""
    import bench
    v10 = list(range(1, 11))
    assert bench.median_ci95(v10) == (5.5, 2, 9)
    v30 = list(range(1, 31))
    med, lo, hi = bench.median_ci95(v30[::-1])
    assert (med, lo, hi) == (15.5, 10, 21)
    assert bench.median_ci95([7.0]) == (7.0, 7.0, 7.0)
