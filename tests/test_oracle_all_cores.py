"""The oracle's OpenMP build (used only to time the oracle on every host core
for the benchmark's all-core CPU baseline) computes the same bits as the
single-threaded checker build: its parallel loops write disjoint outputs,
each the same expression in the same order."""
import numpy as np
import pytest

import oracle
from oracle import programs as OP
from paper_2107_00555_gb300 import inputs


def _both(prog, ins):
    ref = oracle.run(prog, ins)
    with oracle.all_cores() as ac:
        if not ac.available:
            pytest.skip("host compiler has no OpenMP")
        got = oracle.run(prog, ins)
    return ref, got


@pytest.mark.parametrize("bc", ["zero", "periodic", "fixed_ring"])
def test_all_cores_stencil_bitwise(bc):
    u = inputs.uniform((12, 17, 23), -1.0, 1.0, 5)
    ref, got = _both(OP.heat3d(u.shape, 4, bc), [u])
    assert np.array_equal(ref[-1], got[-1])
    u2 = inputs.cfg1(seed=6, n=40)
    ref, got = _both(OP.jacobi2d(u2.shape, 5, bc), [u2])
    assert np.array_equal(ref[-1], got[-1])


def test_all_cores_maps_bitwise():
    x, a, b = inputs.cfg2(np.float64, seed=7, n=30011)
    ref, got = _both(OP.map_reduce(30011), [x, a, b])
    for r, g in zip(ref, got):
        assert np.array_equal(np.asarray(r), np.asarray(g))
