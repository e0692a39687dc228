"""The no-allocation reduction entry point against the graph reduction.

dcp_reduce_noalloc serves callers that cannot allocate device memory (their
own pool allocator owns the GPU, or they are recovering from an
out-of-memory error); it keeps its scratch in a fixed array inside the
library.  It must agree with the ordinary graph path (input -> reduce ->
output) within the reduction tolerance used everywhere else, on two calls
in a row (the second call reuses the scratch the first one left behind).
It is also checked against the oracle (the exactly rounded sum with the
backward-stable bound, exact max / min, wrapped integer sums), and a
warmed-up call must leave the device's free memory unchanged.
This file is collected last on purpose.
"""
import gc

import numpy as np
import pytest

import oracle
from paper_2107_00555_gb300 import Graph, inputs
from paper_2107_00555_gb300 import _capi as C

from gpu_util import red_tol_for, tol_for, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CODES = {"f32": C.DCP_F32, "f64": C.DCP_F64, "i32": C.DCP_I32, "i64": C.DCP_I64}
REDS = {"sum": C.DCP_SUM, "max": C.DCP_MAX_R, "min": C.DCP_MIN_R, "maxabs": C.DCP_MAXABS}


def _data(dtype, n):
    if dtype.startswith("f"):
        return inputs.normal((n,), 77, {"f32": np.float32, "f64": np.float64}[dtype])
    rng = np.random.default_rng(78)
    return rng.integers(-1000, 1000, n).astype({"i32": np.int32, "i64": np.int64}[dtype])


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32", "i64"])
@pytest.mark.parametrize("red", ["sum", "max", "min", "maxabs"])
@pytest.mark.parametrize("n", [1, 1000, 3_000_001])
def test_noalloc_matches_graph_reduction(dtype, red, n):
    x = _data(dtype, n)
    xd = to_dev(x)
    g = Graph()
    v = g.input(dtype, (n,))
    g.output(g.reduce(v, red))
    g.fuse(C.DCP_FUSE_ALL)
    ref = float(to_host(g.run([xd])[0]))
    stream = torch.cuda.current_stream()
    for _ in range(2):  # two calls in a row share the scratch
        out = torch.full((), 12345, dtype=xd.dtype, device=xd.device)
        C.dcp_reduce_noalloc(xd.data_ptr(), n, CODES[dtype], REDS[red], out.data_ptr(),
                             stream.cuda_stream)
        torch.cuda.synchronize()
        got = float(to_host(out))
        if dtype.startswith("i") or red != "sum":
            assert got == ref, (got, ref)  # integer work and max/min are exact
        else:
            scale = float(np.sum(np.abs(x.astype(np.float64))))
            assert abs(got - ref) <= red_tol_for(dtype) * scale, (got, ref)


def test_noalloc_rejects_sizes_beyond_the_maximum():
    x = torch.zeros(4, device="cuda")
    out = torch.zeros((), device="cuda")
    with pytest.raises(C.DcpError) as e:
        C.dcp_reduce_noalloc(x.data_ptr(), (1 << 31) + 1, C.DCP_F32, C.DCP_SUM, out.data_ptr(), 0)
    assert e.value.status == C.DCP_E_INVALID_ARG and "maximum" in str(e.value)
    with pytest.raises(C.DcpError) as e:
        C.dcp_reduce_noalloc(x.data_ptr(), 0, C.DCP_F32, C.DCP_MAX_R, out.data_ptr(), 0)
    assert e.value.status == C.DCP_E_SHAPE
    C.dcp_reduce_noalloc(x.data_ptr(), 0, C.DCP_F32, C.DCP_SUM, out.data_ptr(), 0)
    torch.cuda.synchronize()
    assert float(out) == 0.0


def _oracle_reduce(red, dtype, x):
    if dtype.startswith("i"):
        bits = 32 if dtype == "i32" else 64
        return oracle.reduce_i(red, bits, x.astype(np.int64)), None
    x64 = x.astype(np.float64)
    if red == "sum":
        return oracle.fsum(x64), oracle.sum_abs(x64)
    return oracle.reduce_ext(red, x64)[0], None


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32", "i64"])
@pytest.mark.parametrize("red", ["sum", "max", "min", "maxabs"])
def test_noalloc_matches_oracle_and_allocates_nothing(dtype, red):
    n = 2_500_003
    x = _data(dtype, n)
    if dtype.startswith("i"):
        # sums that wrap: large magnitudes
        x = (x.astype(np.int64) * (1 << (20 if dtype == "i32" else 52))).astype(x.dtype)
    xd = to_dev(x)
    out = torch.zeros((), dtype=xd.dtype, device=xd.device)
    s = torch.cuda.current_stream().cuda_stream
    ref, mag = _oracle_reduce(red, dtype, x)
    # warm-up: the first call on a device looks up the scratch and loads the kernel
    C.dcp_reduce_noalloc(xd.data_ptr(), n, CODES[dtype], REDS[red], out.data_ptr(), s)
    torch.cuda.synchronize()
    gc.collect()  # tensors of earlier tests freed now, not inside the measured calls
    free0, _ = torch.cuda.mem_get_info()
    torch_bytes0 = torch.cuda.memory_allocated()
    for _ in range(2):
        out.fill_(7)
        C.dcp_reduce_noalloc(xd.data_ptr(), n, CODES[dtype], REDS[red], out.data_ptr(), s)
        torch.cuda.synchronize()
        got = to_host(out).item()
        if dtype.startswith("i"):
            assert int(got) == int(ref), (got, ref)
        elif red == "sum":
            assert abs(float(got) - ref) <= red_tol_for(dtype) * mag, (got, ref)
        else:
            want = ref if dtype == "f64" else float(np.float32(ref))
            assert float(got) == want, (got, want)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_allocated() <= torch_bytes0  # nothing through torch's allocator
