"""dcp oracle: the plain CPU interpreter that the GPU executor is checked against.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library (``paper_2107_00555_gb300``) never imports it and
shares no code with it; the two meet only in the test harness, which feeds
both the same seeded input arrays.

The oracle runs a program the way the paper's frontend first translates it
(Sec. 2.3): one NumPy-level operation per SSA statement, each materialising its
whole output array, evaluated in IEEE binary64 with host libm.  The per-op
loops live in ``dcp_oracle.c`` (plain C, no FMA contraction, no
reassociation); this module only walks the program in order and keeps every
intermediate value (a full tape).

Program vocabulary (the oracle's own names):

* ``input(dtype, shape)`` -- a data container (Sec. 2: arrays with a NumPy
  dtype).  ``dtype`` in {"f32", "f64", "i32", "i64"}.  Floating programs are
  evaluated in binary64 whatever the container type (an f32 input is widened
  exactly; intermediates are not rounded back to f32); integer programs wrap
  modulo 2**bits after every op, like NumPy.
* ``map(op, ins, imm)`` -- elementwise op (Table 1: an element-wise assignment
  is a map scope with one tasklet per element).
* ``stencil(v, offsets, weights, bc, steps)`` -- ``steps`` out-of-place
  applications of ``out[p] = sum_k w_k * in[p + o_k]`` (the jacobi programs of
  Sec. 2.2 and Sec. 4.3), boundary rule ``bc`` in {"zero", "periodic",
  "fixed_ring"}.
* ``reduce(v, red, axis=None)`` -- write-conflict resolution of all elements
  into one scalar (Sec. 2.3, ``alpha += C[i, j]``), or along one axis with one
  result per remaining index (``x.sum(axis=a)``), ``red`` in {"sum", "max",
  "min", "maxabs"}.

``run`` returns every value; ``adjoint`` runs the reverse pass of the unfused
program (each op's vector-Jacobian product in reverse order, full tape);
``jvp`` runs the forward tangent pass.  Reductions report, besides the
sequential flat-order sum, the exactly rounded sum (Shewchuk) and the sum of
magnitudes.

Parity status of each function is stated in the test files that pin it; all
functions here are pinned (closed forms, brute force, library special cases,
finite differences), none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dcp_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libdcp_oracle.so")
_lock = threading.Lock()
_lib = None

UNARY = ["neg", "abs", "exp", "sin", "cos", "tanh", "sqrt", "square"]
BINARY = ["add", "sub", "mul", "div", "max", "min"]
SCALAR = ["add_s", "mul_s", "sub_s", "rsub_s"]
OPS = UNARY + BINARY + SCALAR
_OPCODE = {name: i for i, name in enumerate(OPS)}
_INT_OK = {"neg", "abs", "square", "add", "sub", "mul", "max", "min",
           "add_s", "mul_s", "sub_s", "rsub_s"}
BCS = {"zero": 0, "periodic": 1, "fixed_ring": 2}
REDS = {"sum": 0, "max": 1, "min": 2, "maxabs": 3}
DTYPES = ("f32", "f64", "i32", "i64")


_LIB_OMP = os.path.join(_HERE, "_build", "libdcp_oracle_omp.so")
_lib_omp = None
_use_omp = False


def _compile(out, extra):
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + ".tmp%d" % os.getpid()
    subprocess.check_call([
        "gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
        "-shared", _SRC, "-o", tmp] + extra + ["-lm"])
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile the oracle's C loops with the host compiler (binary64 kept literal)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            _compile(_LIB, [])
    return _LIB


def build_all_cores(force: bool = False):
    """The same C loops built with OpenMP, for timing the oracle on every host
    core (maps and stencil steps run in parallel; each output element is the
    same expression in the same order, so results are bitwise those of the
    checker build).  Returns the library path, or None if the host compiler
    has no OpenMP."""
    with _lock:
        if force or not os.path.exists(_LIB_OMP) or \
                os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC):
            try:
                _compile(_LIB_OMP, ["-fopenmp"])
            except (subprocess.CalledProcessError, OSError):
                return None
    return _LIB_OMP


class all_cores:
    """Context manager: oracle calls inside it use the OpenMP build (timing only).
    ``threads`` is the number of threads it uses (``OMP_NUM_THREADS`` if set,
    else every core this process may run on)."""

    def __init__(self):
        self.threads = int(os.environ.get("OMP_NUM_THREADS", "0")) or len(os.sched_getaffinity(0))
        self.available = False

    def __enter__(self):
        global _lib_omp, _use_omp
        if _lib_omp is None:
            path = build_all_cores()
            if path is None:
                return self
            os.environ.setdefault("OMP_NUM_THREADS", str(self.threads))
            _lib_omp = _declare(ctypes.CDLL(path))
        _use_omp = True
        self.available = True
        return self

    def __exit__(self, *exc):
        global _use_omp
        _use_omp = False


def _load():
    global _lib
    if _use_omp and _lib_omp is not None:
        return _lib_omp
    if _lib is None:
        build()
        _lib = _declare(ctypes.CDLL(_LIB))
    return _lib


def _declare(lib):
    """Argument and result types of the C entry points."""
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    I = ctypes.c_int
    D = ctypes.c_double
    lib.orc_map_f.argtypes = [I, I64, P, P, D, P]
    lib.orc_map_i.argtypes = [I, I, I64, P, P, I64, P]
    lib.orc_stencil_f.argtypes = [I, P, P, P, I, P, P, I, I]
    lib.orc_stencil_vjp_f.argtypes = [I, P, P, P, I, P, P, I, I]
    lib.orc_stencil_point_f.argtypes = [I, P, P, I, P, P, I, I, P, P]
    lib.orc_stencil_point_f.restype = D
    lib.orc_sum_seq.argtypes = [I64, P]
    lib.orc_sum_seq.restype = D
    lib.orc_sum_abs.argtypes = [I64, P]
    lib.orc_sum_abs.restype = D
    lib.orc_fsum.argtypes = [I64, P, P]
    lib.orc_fsum.restype = D
    lib.orc_reduce_ext_f.argtypes = [I, I64, P, P, P]
    lib.orc_reduce_i.argtypes = [I, I, I64, P, P]
    lib.orc_reduce_axis_f.argtypes = [I, I64, I64, I64, P, P, P, P]
    lib.orc_reduce_axis_i.argtypes = [I, I, I64, I64, I64, P, P]
    lib.orc_map_vjp_f.argtypes = [I, I64, P, P, D, P, P, P, P]
    lib.orc_map_jvp_f.argtypes = [I, I64, P, P, D, P, P, P, P]
    for f in (lib.orc_map_f, lib.orc_map_i, lib.orc_stencil_f, lib.orc_stencil_vjp_f,
              lib.orc_reduce_ext_f, lib.orc_reduce_i, lib.orc_map_vjp_f, lib.orc_map_jvp_f,
              lib.orc_reduce_axis_f, lib.orc_reduce_axis_i):
        f.restype = I
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s failed with status %d" % (what, rc))


# --------------------------------------------------------------------------
# Single operations (thin wrappers over the C loops)
# --------------------------------------------------------------------------

def map_f(op, a, b=None, imm=0.0):
    """One floating elementwise op in binary64 (Sec. 2.3, Table 1)."""
    lib = _load()
    a = _f64(a)
    b = _f64(b) if b is not None else None
    if op in BINARY and (b is None or b.shape != a.shape):
        raise ValueError("binary op %s needs two operands of one shape" % op)
    y = np.empty_like(a)
    _check(lib.orc_map_f(_OPCODE[op], a.size, _p(a), _p(b), float(imm), _p(y)), op)
    return y


def map_i(op, bits, a, b=None, imm=0):
    """One integer elementwise op, wrapped modulo 2**bits (NumPy semantics)."""
    if op not in _INT_OK:
        raise ValueError("op %s is not defined on integers" % op)
    lib = _load()
    a = _i64(a)
    b = _i64(b) if b is not None else None
    y = np.empty_like(a)
    _check(lib.orc_map_i(_OPCODE[op], bits, a.size, _p(a), _p(b), int(imm), _p(y)), op)
    return y


def _stencil_args(shape, offsets, weights):
    shape = np.ascontiguousarray(shape, dtype=np.int64)
    offs = np.ascontiguousarray(offsets, dtype=np.int32).reshape(-1)
    w = _f64(weights).reshape(-1)
    ndim = shape.size
    if offs.size != w.size * ndim:
        raise ValueError("offsets must be npoints x ndim")
    return shape, offs, w, ndim


def stencil(u0, offsets, weights, bc, steps):
    """``steps`` Jacobi applications of the weighted-offset stencil (Sec. 2.2, 4.3)."""
    lib = _load()
    u0 = _f64(u0)
    shape, offs, w, ndim = _stencil_args(u0.shape, offsets, weights)
    out = np.empty_like(u0)
    _check(lib.orc_stencil_f(ndim, _p(shape), _p(u0), _p(out), w.size, _p(offs), _p(w),
                             BCS[bc], int(steps)), "stencil")
    return out


def stencil_vjp(g_out, offsets, weights, bc, steps):
    """Adjoint of ``stencil``: (S^T)^steps g_out, by scattering (the transpose)."""
    lib = _load()
    g_out = _f64(g_out)
    shape, offs, w, ndim = _stencil_args(g_out.shape, offsets, weights)
    g_in = np.empty_like(g_out)
    _check(lib.orc_stencil_vjp_f(ndim, _p(shape), _p(g_out), _p(g_in), w.size, _p(offs), _p(w),
                                 BCS[bc], int(steps)), "stencil_vjp")
    return g_in


def stencil_point(u0, offsets, weights, bc, steps, point):
    """Value of ``stencil(u0, ...)`` at one cell, from its dependence cone only."""
    lib = _load()
    u0 = _f64(u0)
    shape, offs, w, ndim = _stencil_args(u0.shape, offsets, weights)
    p3 = np.zeros(3, dtype=np.int64)
    p3[3 - ndim:] = np.asarray(point, dtype=np.int64)
    st = ctypes.c_int(0)
    v = lib.orc_stencil_point_f(ndim, _p(shape), _p(u0), w.size, _p(offs), _p(w), BCS[bc],
                                int(steps), _p(p3), ctypes.byref(st))
    _check(st.value, "stencil_point")
    return v


def sum_seq(y):
    """Sequential sum in flat index order."""
    y = _f64(y)
    return _load().orc_sum_seq(y.size, _p(y))


def sum_abs(y):
    """Sequential sum of |y_i| (scale of the backward-stable error bound)."""
    y = _f64(y)
    return _load().orc_sum_abs(y.size, _p(y))


def fsum(y):
    """Exactly rounded sum (Shewchuk 1997 expansion arithmetic)."""
    y = _f64(y)
    st = ctypes.c_int(0)
    v = _load().orc_fsum(y.size, _p(y), ctypes.byref(st))
    _check(st.value, "fsum")
    return v


def reduce_ext(red, y):
    """max / min / maxabs with NaN propagation; returns (value, first arg index)."""
    y = _f64(y)
    out = ctypes.c_double(0.0)
    arg = ctypes.c_int64(0)
    _check(_load().orc_reduce_ext_f(REDS[red], y.size, _p(y), ctypes.byref(out),
                                    ctypes.byref(arg)), red)
    return out.value, arg.value


def reduce_i(red, bits, y):
    """Integer reduction (sum wraps modulo 2**bits)."""
    y = _i64(y)
    out = ctypes.c_int64(0)
    _check(_load().orc_reduce_i(REDS[red], bits, y.size, _p(y), ctypes.byref(out)), red)
    return out.value


def _axis_view(shape, axis):
    nd = len(shape)
    if not -nd <= axis < nd:
        raise ValueError("axis %d out of range for %d axes" % (axis, nd))
    axis %= nd
    outer = int(np.prod(shape[:axis], dtype=np.int64))
    inner = int(np.prod(shape[axis + 1:], dtype=np.int64))
    return axis, outer, int(shape[axis]), inner, tuple(s for d, s in enumerate(shape) if d != axis)


def reduce_axis(red, y, axis):
    """Floating reduction along one axis; for "sum" returns (sequential sum,
    exactly rounded sum, magnitude sum) per output, else the reduced array."""
    y = _f64(y)
    axis, outer, R, inner, oshape = _axis_view(y.shape, axis)
    out = np.empty(outer * inner)
    fs = np.empty(outer * inner) if red == "sum" else None
    ab = np.empty(outer * inner) if red == "sum" else None
    _check(_load().orc_reduce_axis_f(REDS[red], outer, R, inner, _p(y), _p(out), _p(fs), _p(ab)),
           red + " along an axis")
    if red == "sum":
        return out.reshape(oshape), fs.reshape(oshape), ab.reshape(oshape)
    return out.reshape(oshape)


def reduce_axis_i(red, bits, y, axis):
    """Integer reduction along one axis (sum wraps modulo 2**bits)."""
    y = _i64(y)
    axis, outer, R, inner, oshape = _axis_view(y.shape, axis)
    out = np.empty(outer * inner, dtype=np.int64)
    _check(_load().orc_reduce_axis_i(REDS[red], bits, outer, R, inner, _p(y), _p(out)),
           red + " along an axis")
    return out.reshape(oshape)


def map_vjp(op, a, b, imm, y, g):
    """Adjoints (ga, gb) of one floating map op given its forward output y."""
    lib = _load()
    a = _f64(a)
    b = _f64(b) if b is not None else None
    ga = np.zeros_like(a)
    gb = np.zeros_like(a) if b is not None else None
    _check(lib.orc_map_vjp_f(_OPCODE[op], a.size, _p(a), _p(b), float(imm), _p(_f64(y)),
                             _p(_f64(g)), _p(ga), _p(gb)), op + " vjp")
    return ga, gb


def map_jvp(op, a, b, imm, y, da, db):
    """Tangent dy of one floating map op."""
    lib = _load()
    a = _f64(a)
    b = _f64(b) if b is not None else None
    dy = np.empty_like(a)
    _check(lib.orc_map_jvp_f(_OPCODE[op], a.size, _p(a), _p(b), float(imm), _p(_f64(y)),
                             _p(_f64(da)), _p(_f64(db) if db is not None else None), _p(dy)),
           op + " jvp")
    return dy


# --------------------------------------------------------------------------
# Programs: SSA op lists interpreted one op at a time
# --------------------------------------------------------------------------

@dataclass
class _Node:
    kind: str                 # "input" | "map" | "stencil" | "reduce"
    dtype: str
    shape: tuple
    op: str = ""
    ins: tuple = ()
    imm: float = 0.0
    offsets: object = None
    weights: object = None
    bc: str = "zero"
    steps: int = 1
    axis: object = None       # reduce: None = all axes, else the reduced axis


@dataclass
class Program:
    """An SSA program: values are integer handles in creation order."""
    nodes: list = field(default_factory=list)
    inputs: list = field(default_factory=list)
    outputs: list = field(default_factory=list)

    def input(self, dtype, shape):
        if dtype not in DTYPES:
            raise ValueError(dtype)
        self.nodes.append(_Node("input", dtype, tuple(int(s) for s in shape)))
        self.inputs.append(len(self.nodes) - 1)
        return len(self.nodes) - 1

    def map(self, op, ins, imm=0.0):
        ins = tuple(ins)
        if op not in OPS:
            raise ValueError(op)
        n0 = self.nodes[ins[0]]
        need = 2 if op in BINARY else 1
        if len(ins) != need:
            raise ValueError("%s takes %d operands" % (op, need))
        shape = n0.shape
        for v in ins:
            if self.nodes[v].dtype != n0.dtype:
                raise ValueError("operands of one op share a dtype")
            s = self.nodes[v].shape
            if s != shape:
                # NumPy broadcasting of a 0-axis (scalar) container
                if s == ():
                    continue
                if shape == ():
                    shape = s
                    continue
                raise ValueError("operand shapes differ (only 0-axis operands broadcast)")
        if n0.dtype.startswith("i") and op not in _INT_OK:
            raise ValueError("%s is not defined on integers" % op)
        self.nodes.append(_Node("map", n0.dtype, shape, op=op, ins=ins, imm=imm))
        return len(self.nodes) - 1

    def stencil(self, v, offsets, weights, bc, steps):
        n0 = self.nodes[v]
        if n0.dtype.startswith("i"):
            raise ValueError("stencils are floating point")
        self.nodes.append(_Node("stencil", n0.dtype, n0.shape, ins=(v,),
                                offsets=np.asarray(offsets, dtype=np.int32),
                                weights=np.asarray(weights, dtype=np.float64), bc=bc,
                                steps=int(steps)))
        return len(self.nodes) - 1

    def reduce(self, v, red, axis=None):
        n0 = self.nodes[v]
        if axis is None:
            self.nodes.append(_Node("reduce", n0.dtype, (), op=red, ins=(v,)))
        else:
            axis, _, _, _, oshape = _axis_view(n0.shape, int(axis))
            self.nodes.append(_Node("reduce", n0.dtype, oshape, op=red, ins=(v,), axis=axis))
        return len(self.nodes) - 1

    def output(self, v):
        self.outputs.append(v)
        return v


def _is_int(dtype):
    return dtype in ("i32", "i64")


def _bits(dtype):
    return 32 if dtype == "i32" else 64


def _operands(vals, nd):
    """Operand arrays of a map node, a 0-axis operand broadcast to the node's shape."""
    ops = [vals[v] for v in nd.ins]
    ops = [np.array(np.broadcast_to(o, nd.shape)) if o.shape != nd.shape else o for o in ops]
    return ops[0], (ops[1] if len(ops) > 1 else None)


def run(prog: Program, inputs, detail=False):
    """Evaluate every value of ``prog`` in program order.

    ``inputs`` are arrays in ``prog.inputs`` order.  Float values come back as
    float64 arrays, integer values as int64 arrays, reductions as 0-d arrays.
    With ``detail=True`` also returns, for every sum reduction, a dict with
    the exactly rounded sum ``fsum`` and the magnitude sum ``abs``.
    """
    vals = [None] * len(prog.nodes)
    extra = {}
    for h, arr in zip(prog.inputs, inputs):
        nd = prog.nodes[h]
        arr = np.asarray(arr)
        if arr.shape != nd.shape:
            raise ValueError("input %d has shape %s, expected %s" % (h, arr.shape, nd.shape))
        vals[h] = _i64(arr) if _is_int(nd.dtype) else _f64(arr)
    for h, nd in enumerate(prog.nodes):
        if nd.kind == "input":
            continue
        if nd.kind == "map":
            a, b = _operands(vals, nd)
            if _is_int(nd.dtype):
                vals[h] = map_i(nd.op, _bits(nd.dtype), a, b, int(nd.imm)).reshape(nd.shape)
            else:
                vals[h] = map_f(nd.op, a, b, nd.imm).reshape(nd.shape)
        elif nd.kind == "stencil":
            vals[h] = stencil(vals[nd.ins[0]], nd.offsets, nd.weights, nd.bc, nd.steps)
        elif nd.kind == "reduce" and nd.axis is not None:
            y = vals[nd.ins[0]]
            if _is_int(nd.dtype):
                vals[h] = reduce_axis_i(nd.op, _bits(nd.dtype), y, nd.axis)
            elif nd.op == "sum":
                vals[h], fs, ab = reduce_axis("sum", y, nd.axis)
                if detail:
                    extra[h] = {"fsum": fs, "abs": ab}
            else:
                vals[h] = reduce_axis(nd.op, y, nd.axis)
        elif nd.kind == "reduce":
            y = vals[nd.ins[0]]
            if _is_int(nd.dtype):
                vals[h] = np.array(reduce_i(nd.op, _bits(nd.dtype), y), dtype=np.int64)
            elif nd.op == "sum":
                vals[h] = np.array(sum_seq(y))
                if detail:
                    extra[h] = {"fsum": fsum(y), "abs": sum_abs(y)}
            else:
                if y.size == 0:
                    raise ValueError("%s of an empty array is undefined" % nd.op)
                vals[h] = np.array(reduce_ext(nd.op, y)[0])
    if detail:
        return vals, extra
    return vals


def adjoint(prog: Program, inputs, out_grads):
    """Reverse pass of the unfused program (floating programs only).

    ``out_grads`` holds one cotangent per entry of ``prog.outputs`` (scalars
    for reductions).  Returns the cotangent of every input, in input order.
    Each op's vector-Jacobian product is applied in reverse program order on a
    full tape of forward values; cotangents of values used twice add up.
    """
    if any(nd.kind == "reduce" and nd.axis is not None for nd in prog.nodes):
        raise ValueError("the adjoint of axis reductions is not implemented")
    vals = run(prog, inputs)
    grads = [None] * len(prog.nodes)

    def acc(h, g):
        grads[h] = g if grads[h] is None else grads[h] + g

    for h, g in zip(prog.outputs, out_grads):
        acc(h, np.array(np.broadcast_to(np.asarray(g, dtype=np.float64), prog.nodes[h].shape)))
    for h in range(len(prog.nodes) - 1, -1, -1):
        nd = prog.nodes[h]
        g = grads[h]
        if g is None or nd.kind == "input":
            continue
        if _is_int(nd.dtype):
            raise ValueError("integer programs have no adjoint")
        if nd.kind == "map":
            a, b = _operands(vals, nd)
            ga, gb = map_vjp(nd.op, a, b, nd.imm, vals[h], g)
            # a broadcast 0-axis operand receives the sum of its cotangents
            for v, gv in zip(nd.ins, (ga, gb)):
                if gv is None:
                    continue
                if prog.nodes[v].shape != nd.shape:
                    gv = np.array(fsum(gv))
                acc(v, gv.reshape(prog.nodes[v].shape))
        elif nd.kind == "stencil":
            acc(nd.ins[0], stencil_vjp(g, nd.offsets, nd.weights, nd.bc, nd.steps))
        elif nd.kind == "reduce":
            y = vals[nd.ins[0]]
            gs = float(g)
            if nd.op == "sum":
                acc(nd.ins[0], np.full(y.shape, gs))
            else:
                _, arg = reduce_ext(nd.op, y)
                gy = np.zeros(y.size)
                gy[arg] = gs if nd.op != "maxabs" else gs * float(np.sign(y.reshape(-1)[arg]))
                acc(nd.ins[0], gy.reshape(y.shape))
    return [grads[h] if grads[h] is not None else np.zeros(prog.nodes[h].shape)
            for h in prog.inputs]


def jvp(prog: Program, inputs, tangents):
    """Forward tangent pass: the directional derivative of every output."""
    if any(nd.kind == "reduce" and nd.axis is not None for nd in prog.nodes):
        raise ValueError("the tangent of axis reductions is not implemented")
    vals = run(prog, inputs)
    tans = [None] * len(prog.nodes)
    for h, t in zip(prog.inputs, tangents):
        tans[h] = _f64(t)
    for h, nd in enumerate(prog.nodes):
        if nd.kind == "input":
            continue
        if nd.kind == "map":
            a, b = _operands(vals, nd)
            ta = np.array(np.broadcast_to(tans[nd.ins[0]], nd.shape))
            tb = (np.array(np.broadcast_to(tans[nd.ins[1]], nd.shape))
                  if len(nd.ins) > 1 else None)
            tans[h] = map_jvp(nd.op, a, b, nd.imm, vals[h], ta, tb).reshape(nd.shape)
        elif nd.kind == "stencil":
            # the step is linear in its input, so its tangent map is the step itself
            tans[h] = stencil(tans[nd.ins[0]], nd.offsets, nd.weights, nd.bc, nd.steps)
        elif nd.kind == "reduce":
            y = vals[nd.ins[0]]
            if nd.op == "sum":
                tans[h] = np.array(fsum(tans[nd.ins[0]]))
            else:
                _, arg = reduce_ext(nd.op, y)
                t = tans[nd.ins[0]].reshape(-1)[arg]
                if nd.op == "maxabs":
                    t = t * np.sign(y.reshape(-1)[arg])
                tans[h] = np.array(t)
    return [tans[h] for h in prog.outputs]
