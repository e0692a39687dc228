"""ctypes binding of the dcp C ABI (``include/dcp.h``): argument marshalling only.

Every function here has the name of the C entry point it calls and raises
``DcpError`` (carrying the status code and ``dcp_last_error()``) when the call
returns a non-zero status.  No computation happens in Python.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

# status codes (include/dcp.h)
DCP_OK = 0
DCP_E_INVALID_ARG = -1
DCP_E_SHAPE = -2
DCP_E_DTYPE = -3
DCP_E_UNSUPPORTED = -4
DCP_E_OOM = -5
DCP_E_CUDA = -6
DCP_E_COMPILE = -7
DCP_E_TIMEOUT = -8
DCP_E_STATE = -9

DCP_F32, DCP_F64, DCP_I32, DCP_I64 = 1, 2, 3, 4

(DCP_NEG, DCP_ABS, DCP_EXP, DCP_SIN, DCP_COS, DCP_TANH, DCP_SQRT, DCP_SQUARE,
 DCP_ADD, DCP_SUB, DCP_MUL, DCP_DIV, DCP_MAX, DCP_MIN,
 DCP_ADD_S, DCP_MUL_S, DCP_SUB_S, DCP_RSUB_S) = range(18)

DCP_BC_ZERO, DCP_BC_PERIODIC, DCP_BC_FIXED_RING = 0, 1, 2
DCP_SUM, DCP_MAX_R, DCP_MIN_R, DCP_MAXABS = 0, 1, 2, 3

DCP_FUSE_MAPS = 1 << 0
DCP_FUSE_SUBGRAPH = 1 << 1
DCP_TIME_TILE = 1 << 2
DCP_BATCH = 1 << 3
DCP_AUTOTUNE = 1 << 4
DCP_FUSE_ALL = DCP_FUSE_MAPS | DCP_FUSE_SUBGRAPH | DCP_TIME_TILE

DCP_OPT_TIME_TILE_DEPTH = 1
DCP_OPT_TILE_X = 2
DCP_OPT_TILE_Y = 3
DCP_OPT_MAP_BLOCKS_PER_SM = 4
DCP_OPT_USE_GRAPH = 5
DCP_OPT_STENCIL_KERNEL = 7
DCP_OPT_HOST_ACCESS = 8
DCP_OPT_STREAM_ROWS = 9
DCP_OPT_TILE_Z = 10
DCP_OPT_STREAM_PREFETCH = 11
DCP_OPT_STREAM_THREADS = 12
DCP_OPT_CELLS_PER_THREAD = 13
DCP_OPT_MAP_UNROLL = 14
DCP_OPT_DEFERRED_WEIGHT = 15
DCP_OPT_STREAM_MIN_CTAS = 16
DCP_OPT_ADJOINT_DEPTH = 17

_STATUS_NAMES = {v: k for k, v in globals().items() if k.startswith("DCP_E_") or k == "DCP_OK"}


class DcpError(RuntimeError):
    """A dcp entry point returned a non-zero status."""

    def __init__(self, status, func, message):
        self.status = status
        self.func = func
        super().__init__("%s failed with %s (%d): %s"
                         % (func, _STATUS_NAMES.get(status, "?"), status, message))


_lib = None

# (name, restype, argtypes)
_P = ctypes.c_void_p
_SIG = [
    ("dcp_graph_create", ctypes.c_int32, [ctypes.POINTER(_P)]),
    ("dcp_graph_destroy", ctypes.c_int32, [_P]),
    ("dcp_add_input", ctypes.c_int32, [_P, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]),
    ("dcp_add_map", ctypes.c_int32, [_P, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.POINTER(ctypes.c_int32), ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_int32)]),
    ("dcp_add_stencil", ctypes.c_int32, [_P, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                         ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    ("dcp_add_reduce", ctypes.c_int32, [_P, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_int32)]),
    ("dcp_add_reduce_axis", ctypes.c_int32, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_int32)]),
    ("dcp_mark_output", ctypes.c_int32, [_P, ctypes.c_int32]),
    ("dcp_fuse", ctypes.c_int32, [_P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int32)]),
    ("dcp_run", ctypes.c_int32, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _P]),
    ("dcp_run_host", ctypes.c_int32, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _P]),
    ("dcp_run_adjoint", ctypes.c_int32, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                         ctypes.POINTER(_P), ctypes.c_size_t, _P]),
    ("dcp_prepare_adjoint", ctypes.c_int32, [_P, ctypes.c_size_t]),
    ("dcp_sync", ctypes.c_int32, [_P, _P]),
    ("dcp_set_option", ctypes.c_int32, [_P, ctypes.c_int32, ctypes.c_int64]),
    ("dcp_plan_info", ctypes.c_int32, [_P, ctypes.c_char_p, ctypes.c_size_t,
                                       ctypes.POINTER(ctypes.c_size_t)]),
    ("dcp_reduce_noalloc", ctypes.c_int32, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                            _P, _P]),
    ("dcp_probe_fp64", ctypes.c_int32, [ctypes.c_int32, ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double), _P]),
    ("dcp_last_error", ctypes.c_char_p, []),
    ("dcp_version", ctypes.c_char_p, []),
]

EXPORTED = [name for name, _, _ in _SIG]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libdcp.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise OSError("libdcp.so not built: %s" % path)
        lib = ctypes.CDLL(path)
        for name, res, args in _SIG:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(name, status):
    if status != DCP_OK:
        raise DcpError(status, name, load().dcp_last_error().decode(errors="replace"))


def _ptrs(seq):
    arr = (_P * max(1, len(seq)))()
    for i, p in enumerate(seq):
        arr[i] = p
    return arr


def dcp_graph_create():
    h = _P()
    _check("dcp_graph_create", load().dcp_graph_create(ctypes.byref(h)))
    return h


def dcp_graph_destroy(g):
    _check("dcp_graph_destroy", load().dcp_graph_destroy(g))


def dcp_add_input(g, dtype, shape):
    shape = [int(s) for s in shape]
    arr = (ctypes.c_int64 * max(1, len(shape)))(*shape)
    out = ctypes.c_int32()
    _check("dcp_add_input", load().dcp_add_input(g, dtype, len(shape), arr, ctypes.byref(out)))
    return out.value


def dcp_add_map(g, op, ins, imm=0.0):
    arr = (ctypes.c_int32 * max(1, len(ins)))(*ins)
    out = ctypes.c_int32()
    _check("dcp_add_map", load().dcp_add_map(g, op, len(ins), arr, float(imm), ctypes.byref(out)))
    return out.value


def dcp_add_stencil(g, v, offsets, weights, bc, steps):
    flat = [int(o) for pt in offsets for o in pt]
    offs = (ctypes.c_int32 * max(1, len(flat)))(*flat)
    w = (ctypes.c_double * max(1, len(weights)))(*[float(x) for x in weights])
    out = ctypes.c_int32()
    _check("dcp_add_stencil", load().dcp_add_stencil(g, v, len(weights), offs, w, bc, int(steps),
                                                     ctypes.byref(out)))
    return out.value


def dcp_add_reduce(g, v, red):
    out = ctypes.c_int32()
    _check("dcp_add_reduce", load().dcp_add_reduce(g, v, red, ctypes.byref(out)))
    return out.value


def dcp_add_reduce_axis(g, v, red, axis):
    out = ctypes.c_int32()
    _check("dcp_add_reduce_axis", load().dcp_add_reduce_axis(g, v, red, axis, ctypes.byref(out)))
    return out.value


def dcp_mark_output(g, v):
    _check("dcp_mark_output", load().dcp_mark_output(g, v))


def dcp_fuse(g, flags):
    n = ctypes.c_int32()
    _check("dcp_fuse", load().dcp_fuse(g, flags, ctypes.byref(n)))
    return n.value


def dcp_run(g, inputs, outputs, stream=0):
    _check("dcp_run", load().dcp_run(g, _ptrs(inputs), _ptrs(outputs), stream))


def dcp_run_host(g, inputs, outputs, stream=0):
    _check("dcp_run_host", load().dcp_run_host(g, _ptrs(inputs), _ptrs(outputs), stream))


def dcp_run_adjoint(g, inputs, out_grads, in_grads, tape_budget_bytes, stream=0):
    _check("dcp_run_adjoint", load().dcp_run_adjoint(g, _ptrs(inputs), _ptrs(out_grads),
                                                     _ptrs(in_grads), int(tape_budget_bytes),
                                                     stream))


def dcp_prepare_adjoint(g, tape_budget_bytes):
    _check("dcp_prepare_adjoint", load().dcp_prepare_adjoint(g, int(tape_budget_bytes)))


def dcp_sync(g, stream=0):
    _check("dcp_sync", load().dcp_sync(g, stream))


def dcp_set_option(g, key, value):
    _check("dcp_set_option", load().dcp_set_option(g, key, int(value)))


def dcp_plan_info(g):
    need = ctypes.c_size_t()
    _check("dcp_plan_info", load().dcp_plan_info(g, None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value)
    _check("dcp_plan_info", load().dcp_plan_info(g, buf, need.value, None))
    return buf.value.decode()


def dcp_reduce_noalloc(in_ptr, n, dtype, red, out_ptr, stream=0):
    _check("dcp_reduce_noalloc", load().dcp_reduce_noalloc(in_ptr, int(n), dtype, red, out_ptr,
                                                           stream))


def dcp_probe_fp64(op=0, iters=8192, stream=0):
    """Returns (10^9 FP64 lane operations per second, milliseconds) of the probe."""
    g, ms = ctypes.c_double(), ctypes.c_double()
    _check("dcp_probe_fp64", load().dcp_probe_fp64(int(op), int(iters), ctypes.byref(g),
                                                   ctypes.byref(ms), stream))
    return g.value, ms.value


def dcp_last_error():
    return load().dcp_last_error().decode(errors="replace")


def dcp_version():
    return load().dcp_version().decode()
