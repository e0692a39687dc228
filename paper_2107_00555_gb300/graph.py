"""Pythonic wrapper over the dcp C ABI: build a program one NumPy-level
operation per call (Sec. 2.3 SSA form), fuse it (Sec. 3.1), run it on torch
device tensors.  PyTorch only supplies device memory and the current stream;
every operation of the program runs in the library's kernels.
"""
from __future__ import annotations

import json

from . import _capi as C

OPS = {"neg": C.DCP_NEG, "abs": C.DCP_ABS, "exp": C.DCP_EXP, "sin": C.DCP_SIN,
       "cos": C.DCP_COS, "tanh": C.DCP_TANH, "sqrt": C.DCP_SQRT, "square": C.DCP_SQUARE,
       "add": C.DCP_ADD, "sub": C.DCP_SUB, "mul": C.DCP_MUL, "div": C.DCP_DIV,
       "max": C.DCP_MAX, "min": C.DCP_MIN, "add_s": C.DCP_ADD_S, "mul_s": C.DCP_MUL_S,
       "sub_s": C.DCP_SUB_S, "rsub_s": C.DCP_RSUB_S}
BCS = {"zero": C.DCP_BC_ZERO, "periodic": C.DCP_BC_PERIODIC, "fixed_ring": C.DCP_BC_FIXED_RING}
REDS = {"sum": C.DCP_SUM, "max": C.DCP_MAX_R, "min": C.DCP_MIN_R, "maxabs": C.DCP_MAXABS}
DTYPES = {"f32": C.DCP_F32, "f64": C.DCP_F64, "i32": C.DCP_I32, "i64": C.DCP_I64}
FLAGS = {"maps": C.DCP_FUSE_MAPS, "subgraph": C.DCP_FUSE_SUBGRAPH, "time_tile": C.DCP_TIME_TILE,
         "batch": C.DCP_BATCH, "autotune": C.DCP_AUTOTUNE}


def _torch_dtype(code):
    import torch
    return {C.DCP_F32: torch.float32, C.DCP_F64: torch.float64,
            C.DCP_I32: torch.int32, C.DCP_I64: torch.int64}[code]


def _numpy_dtype(code):
    import numpy as np
    return {C.DCP_F32: np.float32, C.DCP_F64: np.float64,
            C.DCP_I32: np.int32, C.DCP_I64: np.int64}[code]


class Graph:
    """A dcp program.  Values are integer handles returned by the builder calls."""

    def __init__(self):
        self._h = C.dcp_graph_create()
        self.inputs = []
        self.outputs = []
        self.shape = {}
        self.dtype = {}
        self.fused = False
        self.n_kernels = None

    # -- construction --------------------------------------------------------
    def input(self, dtype, shape):
        code = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        v = C.dcp_add_input(self._h, code, shape)
        self.inputs.append(v)
        self.shape[v] = tuple(int(s) for s in shape)
        self.dtype[v] = code
        return v

    def map(self, op, ins, imm=0.0):
        code = OPS[op] if isinstance(op, str) else int(op)
        ins = list(ins)
        v = C.dcp_add_map(self._h, code, ins, imm)
        shapes = [self.shape[i] for i in ins]
        self.shape[v] = max(shapes, key=len)
        self.dtype[v] = self.dtype[ins[0]]
        return v

    def stencil(self, v, offsets, weights, bc="zero", steps=1):
        code = BCS[bc] if isinstance(bc, str) else int(bc)
        out = C.dcp_add_stencil(self._h, v, offsets, weights, code, steps)
        self.shape[out] = self.shape[v]
        self.dtype[out] = self.dtype[v]
        return out

    def reduce(self, v, red="sum", axis=None):
        """Reduction of all elements (axis=None) or along one axis (NumPy's
        ``x.sum(axis=axis)``; negative axes count from the end)."""
        code = REDS[red] if isinstance(red, str) else int(red)
        if axis is None:
            out = C.dcp_add_reduce(self._h, v, code)
            self.shape[out] = ()
        else:
            out = C.dcp_add_reduce_axis(self._h, v, code, int(axis))
            shp = self.shape[v]
            ax = int(axis) + len(shp) if int(axis) < 0 else int(axis)
            self.shape[out] = tuple(s for d, s in enumerate(shp) if d != ax)
        self.dtype[out] = self.dtype[v]
        return out

    def output(self, v):
        C.dcp_mark_output(self._h, v)
        self.outputs.append(v)
        return v

    def set_option(self, key, value):
        C.dcp_set_option(self._h, key, value)

    # -- optimisation --------------------------------------------------------
    def fuse(self, flags=C.DCP_FUSE_ALL):
        if isinstance(flags, (list, tuple, set)):
            flags = sum(FLAGS[f] for f in flags)
        self.n_kernels = C.dcp_fuse(self._h, int(flags))
        self.fused = True
        return self.n_kernels

    def plan(self):
        return json.loads(C.dcp_plan_info(self._h))

    # -- execution -------------------------------------------------------------
    def _check_tensor(self, t, v, what):
        import torch
        if not isinstance(t, torch.Tensor):
            raise TypeError("%s must be a torch tensor" % what)
        if t.device.type != "cuda":
            raise ValueError("%s must be a CUDA tensor" % what)
        if tuple(t.shape) != self.shape[v]:
            raise ValueError("%s has shape %s, expected %s" % (what, tuple(t.shape), self.shape[v]))
        if t.dtype != _torch_dtype(self.dtype[v]):
            raise ValueError("%s has dtype %s, expected %s" % (what, t.dtype, _torch_dtype(self.dtype[v])))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % what)

    def empty_outputs(self, device=None):
        import torch
        return [torch.empty(self.shape[v], dtype=_torch_dtype(self.dtype[v]),
                            device=device or "cuda") for v in self.outputs]

    def run(self, inputs, outputs=None, stream=None):
        """Run on CUDA tensors (asynchronous on ``stream``, default: torch's current)."""
        import torch
        if len(inputs) != len(self.inputs):
            raise ValueError("expected %d inputs" % len(self.inputs))
        for i, (t, v) in enumerate(zip(inputs, self.inputs)):
            self._check_tensor(t, v, "input %d" % i)
        if outputs is None:
            outputs = self.empty_outputs(inputs[0].device if inputs else None)
        for j, (t, v) in enumerate(zip(outputs, self.outputs)):
            self._check_tensor(t, v, "output %d" % j)
        if stream is None:
            stream = torch.cuda.current_stream()
        C.dcp_run(self._h, [t.data_ptr() for t in inputs], [t.data_ptr() for t in outputs],
                  stream.cuda_stream)
        return outputs

    def prepare(self, inputs, outputs=None):
        """Validate and marshal the buffers once; returns a callable that runs the
        program on them with one C call (for many runs on fixed buffers, e.g.
        thousands of batched instances)."""
        import ctypes
        import torch
        if len(inputs) != len(self.inputs):
            raise ValueError("expected %d inputs" % len(self.inputs))
        for i, (t, v) in enumerate(zip(inputs, self.inputs)):
            self._check_tensor(t, v, "input %d" % i)
        if outputs is None:
            outputs = self.empty_outputs(inputs[0].device if inputs else None)
        for j, (t, v) in enumerate(zip(outputs, self.outputs)):
            self._check_tensor(t, v, "output %d" % j)
        ins = C._ptrs([t.data_ptr() for t in inputs])
        outs = C._ptrs([t.data_ptr() for t in outputs])
        lib = C.load()
        h = self._h
        keep = (list(inputs), list(outputs))

        def run(stream=None):
            s = (stream or torch.cuda.current_stream()).cuda_stream
            C._check("dcp_run", lib.dcp_run(h, ins, outs, s))
            return keep[1]

        run.outputs = outputs
        return run

    def prepare_host(self, inputs, outputs):
        """``prepare`` for host buffers (numpy arrays or CPU tensors, ideally
        page-locked so the kernels access them directly): checked and
        marshalled once; the returned callable runs ``dcp_run_host``."""
        import numpy as np
        import torch
        arrs = [a.numpy() if isinstance(a, torch.Tensor) else a for a in inputs]
        outs = [o.numpy() if isinstance(o, torch.Tensor) else o for o in outputs]
        for i, (a, v) in enumerate(zip(arrs, self.inputs)):
            if (not a.flags.c_contiguous or a.shape != self.shape[v]
                    or a.dtype != _numpy_dtype(self.dtype[v])):
                raise ValueError("host input %d has the wrong shape, dtype or layout" % i)
        for j, (o, v) in enumerate(zip(outs, self.outputs)):
            if (not o.flags.c_contiguous or o.shape != self.shape[v]
                    or o.dtype != _numpy_dtype(self.dtype[v])):
                raise ValueError("host output %d has the wrong shape, dtype or layout" % j)
        if len(arrs) != len(self.inputs) or len(outs) != len(self.outputs):
            raise ValueError("expected %d inputs and %d outputs" % (len(self.inputs), len(self.outputs)))
        ins = C._ptrs([a.ctypes.data for a in arrs])
        ops = C._ptrs([o.ctypes.data for o in outs])
        lib = C.load()
        h = self._h
        keep = (arrs, outs)

        def run(stream=None):
            s = (stream or torch.cuda.current_stream()).cuda_stream
            C._check("dcp_run_host", lib.dcp_run_host(h, ins, ops, s))
            return keep[1]

        return run

    def run_host(self, inputs, outputs=None, stream=None):
        """Run on host arrays (numpy or CPU tensors); copies in and out, synchronous."""
        import numpy as np
        import torch
        arrs = []
        for i, (a, v) in enumerate(zip(inputs, self.inputs)):
            if isinstance(a, torch.Tensor):
                a = a.numpy()
            a = np.ascontiguousarray(a)
            if a.shape != self.shape[v] or a.dtype != _numpy_dtype(self.dtype[v]):
                raise ValueError("host input %d has the wrong shape or dtype" % i)
            arrs.append(a)
        if outputs is None:
            outputs = [np.empty(self.shape[v], dtype=_numpy_dtype(self.dtype[v]))
                       for v in self.outputs]
        outs = []
        for o in outputs:
            outs.append(o.numpy() if isinstance(o, torch.Tensor) else o)
        s = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
        C.dcp_run_host(self._h, [a.ctypes.data for a in arrs], [o.ctypes.data for o in outs], s)
        return outputs

    def adjoint(self, inputs, out_grads, in_grads=None, tape_budget_bytes=1 << 62, stream=None):
        """Reverse pass: cotangents of the inputs given those of the outputs."""
        import torch
        for i, (t, v) in enumerate(zip(inputs, self.inputs)):
            self._check_tensor(t, v, "input %d" % i)
        for j, (t, v) in enumerate(zip(out_grads, self.outputs)):
            self._check_tensor(t, v, "output cotangent %d" % j)
        if in_grads is None:
            in_grads = [torch.empty_like(t) for t in inputs]
        for i, (t, v) in enumerate(zip(in_grads, self.inputs)):
            self._check_tensor(t, v, "input cotangent %d" % i)
        if stream is None:
            stream = torch.cuda.current_stream()
        C.dcp_run_adjoint(self._h, [t.data_ptr() for t in inputs],
                          [t.data_ptr() for t in out_grads], [t.data_ptr() for t in in_grads],
                          tape_budget_bytes, stream.cuda_stream)
        return in_grads

    def prepare_adjoint(self, tape_budget_bytes=1 << 62):
        """Plan and compile the reverse pass without running it (no GPU needed)."""
        C.dcp_prepare_adjoint(self._h, tape_budget_bytes)
        return self.plan()

    def sync(self, stream=None):
        import torch
        s = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
        C.dcp_sync(self._h, s)

    def close(self):
        if self._h is not None:
            C.dcp_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
