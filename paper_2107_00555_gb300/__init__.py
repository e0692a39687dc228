"""dcp: a fused dataflow executor for NumPy-style array programs on GB300 (sm_103a).

Programs of elementwise maps, iterated stencils and reductions are built one
operation per call through the C ABI in ``include/dcp.h`` (or traced from
NumPy-style Python by ``program``, see ``frontend.py``), fused into few
kernels, compiled for sm_103a and run on device memory (Ziogas et al.,
"Productivity, Portability, Performance: Data-Centric Python", SC'21).
The library has no CPU fallback: loading fails loudly if libdcp.so cannot be
built or loaded.
"""
from . import _capi
from ._capi import DcpError, load
from .frontend import Array, Program, cos, exp, maximum, minimum, program, sin, sqrt, square, tanh
from .graph import Graph

__all__ = ["Graph", "DcpError", "load", "_capi", "program", "Program", "Array", "exp", "sin",
           "cos", "tanh", "sqrt", "square", "maximum", "minimum"]
