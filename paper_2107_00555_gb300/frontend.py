"""NumPy-style front end: trace a Python function over array proxies into a
dcp program, one builder call per array operation (the SSA form of Sec. 2.3).

    import paper_2107_00555_gb300 as dcp

    @dcp.program(x=("f32", (n,)), a=("f32", (n,)), b=("f32", (n,)))
    def f(x, a, b):
        y = dcp.exp(a * x + b) * dcp.sin(x) - 0.5 * x * x
        return y.sum(), abs(y).max()

    s, m = f(x_t, a_t, b_t)          # torch CUDA tensors in, tensors out

The function runs once, at decoration time, on ``Array`` proxies: every
operator, ufunc-like call and reduction records the matching ``dcp_add_*``
call, and the returned proxies become the program outputs.  Python control
flow runs during tracing, so a ``for t in range(T)`` time loop unrolls into
T stencil statements that the planner chains and time-tiles (the paper's
frontend turns such loops into state machines instead; the resulting
dataflow is the same).

Stencils are written the paper's way, as a weighted sum of shifted slices of
one array assigned to the interior of another (Sec. 2.2, jacobi_1d; Sec. 4.3,
jacobi_2d):

    B[1:-1, 1:-1] = 0.2 * (A[1:-1, 1:-1] + A[1:-1, :-2] + A[1:-1, 2:]
                           + A[2:, 1:-1] + A[:-2, 1:-1])

This records one fixed-ring stencil step of A whose offsets are the slices'
shifts relative to the assigned region, in the order the terms are written,
and rebinds B to it.  Scalar factors are distributed over the terms (the
weighted sum is formed term by term).  The assigned region must be the
interior left by the largest shift on each axis, and the ring (border) cells
of the result are A's, as in the paper's programs, where both arrays start
from the same values.
"""
from __future__ import annotations

import builtins
import inspect
import math
import numbers

from . import _capi as C
from .graph import Graph

__all__ = ["Array", "program", "exp", "sin", "cos", "tanh", "sqrt", "square", "maximum",
           "minimum"]


class _Tracer:
    def __init__(self):
        self.g = Graph()


class Array:
    """A traced array value: a handle into the program being built."""

    __array_priority__ = 1000  # numpy scalars defer to Array's operators

    def __init__(self, tr, handle):
        self._tr = tr
        self._h = handle

    # -- metadata ------------------------------------------------------------
    @property
    def shape(self):
        return self._tr.g.shape[self._h]

    @property
    def ndim(self):
        return len(self.shape)

    @property
    def dtype(self):
        return {C.DCP_F32: "f32", C.DCP_F64: "f64", C.DCP_I32: "i32",
                C.DCP_I64: "i64"}[self._tr.g.dtype[self._h]]

    def _new(self, h):
        return Array(self._tr, h)

    # -- elementwise maps ------------------------------------------------------
    def _binary(self, other, op, op_s=None, rop_s=None, reflected=False):
        g = self._tr.g
        if isinstance(other, Array):
            if other._tr is not self._tr:
                raise ValueError("operands belong to different programs")
            ins = [other._h, self._h] if reflected else [self._h, other._h]
            return self._new(g.map(op, ins))
        if isinstance(other, numbers.Real):
            name = rop_s if reflected else op_s
            if name is None:
                raise NotImplementedError("%s with a Python scalar on this side" % op)
            return self._new(g.map(name, [self._h], float(other)))
        if isinstance(other, _Linear):
            return NotImplemented
        return NotImplemented

    def __add__(self, o):
        return self._binary(o, "add", "add_s", "add_s")

    def __radd__(self, o):
        return self._binary(o, "add", "add_s", "add_s", reflected=True)

    def __sub__(self, o):
        return self._binary(o, "sub", "sub_s", "rsub_s")

    def __rsub__(self, o):
        return self._binary(o, "sub", "sub_s", "rsub_s", reflected=True)

    def __mul__(self, o):
        return self._binary(o, "mul", "mul_s", "mul_s")

    def __rmul__(self, o):
        return self._binary(o, "mul", "mul_s", "mul_s", reflected=True)

    def __truediv__(self, o):
        if isinstance(o, numbers.Real):
            # x / s equals x * (1/s) exactly only when 1/s is a power of two
            inv = 1.0 / float(o)
            m, _ = math.frexp(inv)
            if inv != 0.0 and builtins.abs(m) == 0.5:
                return self._new(self._tr.g.map("mul_s", [self._h], inv))
            raise NotImplementedError("division by a scalar that is not a power of two")
        return self._binary(o, "div")

    def __rtruediv__(self, o):
        if isinstance(o, Array):
            return o._binary(self, "div")
        raise NotImplementedError("a scalar divided by an array")

    def __neg__(self):
        return self._new(self._tr.g.map("neg", [self._h]))

    def __pos__(self):
        return self

    def __abs__(self):
        return self._new(self._tr.g.map("abs", [self._h]))

    def __pow__(self, e):
        if e == 2:
            return self._new(self._tr.g.map("square", [self._h]))
        if e == 1:
            return self
        raise NotImplementedError("only x**2 is supported")

    # -- reductions --------------------------------------------------------------
    def _reduce(self, red, axis):
        return self._new(self._tr.g.reduce(self._h, red, axis=axis))

    def sum(self, axis=None):
        return self._reduce("sum", axis)

    def max(self, axis=None):
        return self._reduce("max", axis)

    def min(self, axis=None):
        return self._reduce("min", axis)

    # -- shifted views and stencil assignment --------------------------------------
    def __getitem__(self, key):
        return _View(self, _region(key, self.shape))

    def __setitem__(self, key, value):
        dest = _region(key, self.shape)
        if isinstance(value, _View):
            value = _Linear([(1.0, value)])
        if not isinstance(value, _Linear):
            raise NotImplementedError("only weighted sums of shifted slices can be assigned "
                                      "to a region")
        self._h = value._emit_stencil(dest, self.shape)


def _region(key, shape):
    """Per-axis (start, stop) of a basic slice with step 1."""
    if not isinstance(key, tuple):
        key = (key,)
    if len(key) != len(shape):
        raise NotImplementedError("index every axis with a slice")
    out = []
    for k, n in zip(key, shape):
        if not isinstance(k, slice) or k.step not in (None, 1):
            raise NotImplementedError("only step-1 slices form stencil views")
        start, stop, _ = k.indices(n)
        if stop <= start:
            raise ValueError("empty slice")
        out.append((start, stop))
    return tuple(out)


class _View:
    """A shifted window of an array, the operand of a stencil term."""

    def __init__(self, base, region):
        self.base = base
        self.h = base._h  # the value the slice reads, fixed when the slice is taken
        self.region = region

    def _lin(self):
        return _Linear([(1.0, self)])

    def __add__(self, o):
        return self._lin() + o

    def __radd__(self, o):
        return self._lin() + o

    def __sub__(self, o):
        return self._lin() - o

    def __mul__(self, s):
        return self._lin() * s

    def __rmul__(self, s):
        return self._lin() * s

    def __neg__(self):
        return self._lin() * -1.0


class _Linear:
    """sum_k w_k * view_k, in the order the terms were written."""

    def __init__(self, terms):
        self.terms = terms

    def __add__(self, o):
        if isinstance(o, _View):
            o = o._lin()
        if not isinstance(o, _Linear):
            return NotImplemented
        return _Linear(self.terms + o.terms)

    __radd__ = __add__

    def __sub__(self, o):
        if isinstance(o, _View):
            o = o._lin()
        if not isinstance(o, _Linear):
            return NotImplemented
        return _Linear(self.terms + [(-w, v) for w, v in o.terms])

    def __mul__(self, s):
        if not isinstance(s, numbers.Real):
            return NotImplemented
        return _Linear([(float(s) * w, v) for w, v in self.terms])

    __rmul__ = __mul__

    def __truediv__(self, s):
        if not isinstance(s, numbers.Real):
            return NotImplemented
        return _Linear([(w / float(s), v) for w, v in self.terms])

    def _emit_stencil(self, dest, shape):
        handles = {v.h for _, v in self.terms}
        if len(handles) != 1:
            raise NotImplementedError("a stencil reads one array")
        src = self.terms[0][1].base
        h = self.terms[0][1].h
        if src._tr.g.shape[h] != tuple(shape):
            raise ValueError("source and destination shapes differ")
        ext = tuple(b - a for a, b in dest)
        offsets = []
        for _, v in self.terms:
            if tuple(b - a for a, b in v.region) != ext:
                raise ValueError("every slice must have the extent of the assigned region")
            offsets.append(tuple(va - da for (va, _), (da, _) in zip(v.region, dest)))
        ring = [builtins.max(builtins.abs(o[d]) for o in offsets) for d in range(len(shape))]
        want = tuple((r, n - r) for r, n in zip(ring, shape))
        if tuple(dest) != want:
            raise NotImplementedError("the assigned region must be the interior left by the "
                                      "largest shift on each axis (fixed-ring stencil)")
        g = src._tr.g
        return g.stencil(h, offsets, [w for w, _ in self.terms], "fixed_ring", 1)


def _unary(name):
    def f(x):
        if not isinstance(x, Array):
            raise TypeError("%s expects a traced array" % name)
        return x._new(x._tr.g.map(name, [x._h]))
    f.__name__ = name
    f.__doc__ = "Elementwise %s of a traced array." % name
    return f


exp = _unary("exp")
sin = _unary("sin")
cos = _unary("cos")
tanh = _unary("tanh")
sqrt = _unary("sqrt")
square = _unary("square")


def maximum(a, b):
    """Elementwise larger value (NaN-propagating, like np.maximum)."""
    return a._binary(b, "max")


def minimum(a, b):
    """Elementwise smaller value (NaN-propagating, like np.minimum)."""
    return a._binary(b, "min")


class Program:
    """A traced, fused program; call it with device tensors."""

    def __init__(self, fn, args, flags):
        self.__name__ = getattr(fn, "__name__", "program")
        tr = _Tracer()
        self.graph = tr.g
        proxies = [Array(tr, tr.g.input(dt, shape)) for dt, shape in args]
        out = fn(*proxies)
        self._single = isinstance(out, Array)
        outs = [out] if self._single else list(out)
        if not outs or not all(isinstance(o, Array) for o in outs):
            raise TypeError("a program returns traced arrays")
        for o in outs:
            h = o._h
            if h in tr.g.inputs:
                h = tr.g.map("add_s", [h], 0.0)  # an input returned unchanged: a copy
            tr.g.output(h)
        self.graph.fuse(flags)

    def plan(self):
        return self.graph.plan()

    def __call__(self, *tensors, outputs=None, stream=None):
        res = self.graph.run(list(tensors), outputs, stream)
        return res[0] if self._single else tuple(res)


def program(*arg_specs, flags=C.DCP_FUSE_ALL, **kw_specs):
    """Decorator: ``@program(x=("f32", shape), ...)`` (or positional specs in
    parameter order) traces the function once and returns a ``Program``."""
    def wrap(fn):
        params = list(inspect.signature(fn).parameters)
        if arg_specs and kw_specs:
            raise TypeError("give the argument specs positionally or by name, not both")
        if kw_specs:
            missing = [p for p in params if p not in kw_specs]
            if missing:
                raise TypeError("no dtype/shape given for %s" % ", ".join(missing))
            specs = [kw_specs[p] for p in params]
        else:
            specs = list(arg_specs)
        if len(specs) != len(params):
            raise TypeError("%d argument specs for %d parameters" % (len(specs), len(params)))
        return Program(fn, [(dt, tuple(int(s) for s in shape)) for dt, shape in specs], flags)
    return wrap
