// C ABI entry points: argument validation, graph construction (one node per
// SSA statement, Sec. 2.3) and conversion of internal errors to status codes.
#include <cstdio>
#include <cstring>
#include <cmath>
#include <exception>
#include <new>

#include "dcp_internal.h"

namespace dcp {

static thread_local std::string g_last_error;

[[noreturn]] void fail(dcp_status code, const std::string& msg) { throw Error{code, msg}; }

void set_last_error(const std::string& msg) { g_last_error = msg; }

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    if (e == cudaErrorMemoryAllocation)
      fail(DCP_E_OOM, std::string(what) + ": " + cudaGetErrorString(e));
    fail(DCP_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
}

int dtype_size(int dtype) {
  switch (dtype) {
    case DCP_F32: return 4;
    case DCP_F64: return 8;
    case DCP_I32: return 4;
    case DCP_I64: return 8;
  }
  return 0;
}
bool dtype_is_float(int dtype) { return dtype == DCP_F32 || dtype == DCP_F64; }
const char* dtype_cname(int dtype) {
  switch (dtype) {
    case DCP_F32: return "float";
    case DCP_F64: return "double";
    case DCP_I32: return "int";
    case DCP_I64: return "long long";
  }
  return "?";
}
const char* dtype_name(int dtype) {
  switch (dtype) {
    case DCP_F32: return "f32";
    case DCP_F64: return "f64";
    case DCP_I32: return "i32";
    case DCP_I64: return "i64";
  }
  return "?";
}

bool op_is_unary(int op) { return op >= DCP_NEG && op <= DCP_SQUARE; }
bool op_is_binary(int op) { return op >= DCP_ADD && op <= DCP_MIN; }
bool op_is_scalar_imm(int op) { return op >= DCP_ADD_S && op <= DCP_RSUB_S; }
bool op_float_only(int op) {
  return op == DCP_EXP || op == DCP_SIN || op == DCP_COS || op == DCP_TANH || op == DCP_SQRT ||
         op == DCP_DIV;
}
const char* op_name(int op) {
  static const char* names[] = {"neg", "abs", "exp", "sin", "cos", "tanh", "sqrt", "square",
                                "add", "sub", "mul", "div", "max", "min",
                                "add_s", "mul_s", "sub_s", "rsub_s"};
  return (op >= 0 && op <= DCP_RSUB_S) ? names[op] : "?";
}
const char* red_name(int red) {
  static const char* names[] = {"sum", "max", "min", "maxabs"};
  return (red >= 0 && red <= DCP_MAXABS) ? names[red] : "?";
}

uint64_t fnv1a(const std::string& s) {
  uint64_t h = 1469598103934665603ull;
  for (unsigned char c : s) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace dcp

using namespace dcp;

struct dcp_graph_s {
  GraphImpl impl;
};

template <class F>
static dcp_status guarded(F&& f) {
  try {
    f();
    return DCP_OK;
  } catch (const Error& e) {
    g_last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return DCP_E_OOM;
  } catch (const std::exception& e) {
    g_last_error = std::string("internal error: ") + e.what();
    return DCP_E_INVALID_ARG;
  } catch (...) {
    g_last_error = "internal error";
    return DCP_E_INVALID_ARG;
  }
}

static GraphImpl& G(dcp_graph g) {
  if (!g) fail(DCP_E_INVALID_ARG, "graph handle is NULL");
  return g->impl;
}

static const Node& value(const GraphImpl& g, dcp_value v) {
  if (v < 0 || v >= (dcp_value)g.nodes.size())
    fail(DCP_E_INVALID_ARG, "value handle " + std::to_string(v) + " does not belong to this graph");
  return g.nodes[v];
}

static void check_mutable(const GraphImpl& g) {
  if (g.fused) fail(DCP_E_STATE, "graph is already fused; it can no longer be modified");
}

static void check_dtype(int dtype) {
  if (dtype != DCP_F32 && dtype != DCP_F64 && dtype != DCP_I32 && dtype != DCP_I64)
    fail(DCP_E_DTYPE, "unknown dtype " + std::to_string(dtype));
}

static int push(GraphImpl& g, Node&& n) {
  g.nodes.push_back(std::move(n));
  return (int)g.nodes.size() - 1;
}

extern "C" {

dcp_status dcp_graph_create(dcp_graph* out) {
  return guarded([&] {
    if (!out) fail(DCP_E_INVALID_ARG, "out is NULL");
    *out = new dcp_graph_s();
  });
}

dcp_status dcp_graph_destroy(dcp_graph g) {
  return guarded([&] { delete g; });
}

dcp_status dcp_add_input(dcp_graph gh, int32_t dtype, int32_t ndim, const int64_t* shape,
                         dcp_value* out) {
  return guarded([&] {
    GraphImpl& g = G(gh);
    check_mutable(g);
    if (!out) fail(DCP_E_INVALID_ARG, "out is NULL");
    check_dtype(dtype);
    if (ndim < 0 || ndim > 4) fail(DCP_E_SHAPE, "ndim must be in 0..4");
    if (ndim > 0 && !shape) fail(DCP_E_INVALID_ARG, "shape is NULL");
    Node n;
    n.kind = Kind::Input;
    n.dtype = dtype;
    for (int i = 0; i < ndim; ++i) {
      if (shape[i] < 0) fail(DCP_E_SHAPE, "negative extent");
      if (shape[i] > (int64_t(1) << 40)) fail(DCP_E_SHAPE, "extent too large");
      n.shape.push_back(shape[i]);
    }
    if (n.numel() > (int64_t(1) << 40)) fail(DCP_E_SHAPE, "array too large");
    int id = push(g, std::move(n));
    g.inputs.push_back(id);
    *out = id;
  });
}

dcp_status dcp_add_map(dcp_graph gh, int32_t op, int32_t n_in, const dcp_value* in, double imm,
                       dcp_value* out) {
  return guarded([&] {
    GraphImpl& g = G(gh);
    check_mutable(g);
    if (!out || !in) fail(DCP_E_INVALID_ARG, "NULL pointer argument");
    if (op < DCP_NEG || op > DCP_RSUB_S) fail(DCP_E_INVALID_ARG, "unknown map op " + std::to_string(op));
    int need = op_is_binary(op) ? 2 : 1;
    if (n_in != need)
      fail(DCP_E_INVALID_ARG, std::string("op ") + op_name(op) + " takes " + std::to_string(need) +
                                  " operand(s)");
    const Node& a = value(g, in[0]);
    Node n;
    n.kind = Kind::Map;
    n.op = op;
    n.imm = imm;
    n.dtype = a.dtype;
    n.in.push_back(in[0]);
    n.shape = a.shape;
    if (need == 2) {
      const Node& b = value(g, in[1]);
      if (b.dtype != a.dtype) fail(DCP_E_DTYPE, "operands of one op must share a dtype");
      if (a.shape != b.shape) {
        if (b.shape.empty()) {
          // broadcast scalar b
        } else if (a.shape.empty()) {
          n.shape = b.shape;
        } else {
          fail(DCP_E_SHAPE, "operand shapes differ (only 0-axis operands broadcast)");
        }
      }
      n.in.push_back(in[1]);
      if (a.shape.empty() && b.shape.empty()) {
        // scalar op scalar: fine, 0-axis result
      }
    }
    if (!dtype_is_float(a.dtype) && op_float_only(op))
      fail(DCP_E_DTYPE, std::string("op ") + op_name(op) + " is only defined on floating dtypes");
    if (op_is_scalar_imm(op) && !dtype_is_float(a.dtype)) {
      if (!(std::fabs(imm) < 9.2e18) || std::floor(imm) != imm)
        fail(DCP_E_INVALID_ARG, "integer ops need an integral immediate");
    }
    if (!op_is_scalar_imm(op)) n.imm = 0.0;
    *out = push(g, std::move(n));
  });
}

dcp_status dcp_add_stencil(dcp_graph gh, dcp_value vin, int32_t npoints, const int32_t* offsets,
                           const double* weights, int32_t bc, int32_t steps, dcp_value* out) {
  return guarded([&] {
    GraphImpl& g = G(gh);
    check_mutable(g);
    if (!out || !offsets || !weights) fail(DCP_E_INVALID_ARG, "NULL pointer argument");
    const Node& a = value(g, vin);
    if (!dtype_is_float(a.dtype)) fail(DCP_E_DTYPE, "stencils are defined on floating dtypes");
    int nd = a.ndim();
    if (nd < 1 || nd > 3) fail(DCP_E_SHAPE, "stencils take 1..3 axes");
    if (npoints < 1 || npoints > kMaxPoints)
      fail(DCP_E_INVALID_ARG, "npoints must be in 1..32");
    if (bc != DCP_BC_ZERO && bc != DCP_BC_PERIODIC && bc != DCP_BC_FIXED_RING)
      fail(DCP_E_INVALID_ARG, "unknown boundary rule");
    if (steps < 0) fail(DCP_E_INVALID_ARG, "steps must be >= 0");
    Node n;
    n.kind = Kind::Stencil;
    n.dtype = a.dtype;
    n.shape = a.shape;
    n.in.push_back(vin);
    n.bc = bc;
    n.steps = steps;
    for (int k = 0; k < npoints; ++k) {
      for (int d = 0; d < nd; ++d) {
        int32_t o = offsets[k * nd + d];
        if (o < -kMaxRadius || o > kMaxRadius)
          fail(DCP_E_INVALID_ARG, "stencil offsets are limited to |o| <= 4");
        n.offsets.push_back(o);
      }
      if (!std::isfinite(weights[k])) fail(DCP_E_INVALID_ARG, "stencil weights must be finite");
      n.weights.push_back(weights[k]);
    }
    if (a.numel() > 0 && bc == DCP_BC_PERIODIC) {
      // any extent >= 1 is fine under periodic wrap
    }
    *out = push(g, std::move(n));
  });
}

dcp_status dcp_add_reduce(dcp_graph gh, dcp_value vin, int32_t red, dcp_value* out) {
  return guarded([&] {
    GraphImpl& g = G(gh);
    check_mutable(g);
    if (!out) fail(DCP_E_INVALID_ARG, "out is NULL");
    const Node& a = value(g, vin);
    if (red < DCP_SUM || red > DCP_MAXABS) fail(DCP_E_INVALID_ARG, "unknown reduction");
    if (red != DCP_SUM && a.numel() == 0)
      fail(DCP_E_SHAPE, std::string(red_name(red)) + " of an empty array is undefined");
    Node n;
    n.kind = Kind::Reduce;
    n.dtype = a.dtype;
    n.op = red;
    n.in.push_back(vin);
    *out = push(g, std::move(n));
  });
}

dcp_status dcp_add_reduce_axis(dcp_graph gh, dcp_value vin, int32_t red, int32_t axis,
                               dcp_value* out) {
  return guarded([&] {
    GraphImpl& g = G(gh);
    check_mutable(g);
    if (!out) fail(DCP_E_INVALID_ARG, "out is NULL");
    const Node& a = value(g, vin);
    if (red < DCP_SUM || red > DCP_MAXABS) fail(DCP_E_INVALID_ARG, "unknown reduction");
    const int nd = a.ndim();
    if (nd == 0) fail(DCP_E_SHAPE, "a 0-axis value has no axis to reduce");
    if (axis < -nd || axis >= nd)
      fail(DCP_E_INVALID_ARG, "axis " + std::to_string(axis) + " out of range for " +
                                  std::to_string(nd) + " axes");
    if (axis < 0) axis += nd;
    if (red != DCP_SUM && a.shape[axis] == 0)
      fail(DCP_E_SHAPE, std::string(red_name(red)) + " along an empty axis is undefined");
    Node n;
    n.kind = Kind::Reduce;
    n.dtype = a.dtype;
    n.op = red;
    n.axis = axis;
    for (int d = 0; d < nd; ++d)
      if (d != axis) n.shape.push_back(a.shape[d]);
    n.in.push_back(vin);
    *out = push(g, std::move(n));
  });
}

dcp_status dcp_mark_output(dcp_graph gh, dcp_value v) {
  return guarded([&] {
    GraphImpl& g = G(gh);
    check_mutable(g);
    const Node& n = value(g, v);
    if (n.kind == Kind::Input) fail(DCP_E_INVALID_ARG, "an input cannot be marked as output");
    for (int o : g.outputs)
      if (o == v) fail(DCP_E_INVALID_ARG, "value is already an output");
    g.outputs.push_back(v);
  });
}

dcp_status dcp_fuse(dcp_graph gh, uint32_t flags, int32_t* n_kernels_out) {
  return guarded([&] {
    GraphImpl& g = G(gh);
    if (g.fused) fail(DCP_E_STATE, "graph is already fused");
    if (flags & ~uint32_t(DCP_FUSE_MAPS | DCP_FUSE_SUBGRAPH | DCP_TIME_TILE | DCP_BATCH |
                          DCP_AUTOTUNE))
      fail(DCP_E_INVALID_ARG, "unknown fuse flag");
    if (g.outputs.empty()) fail(DCP_E_STATE, "graph has no outputs");
    plan_graph(g, flags);
    compile_plan(g);
    g.fused = true;
    if (n_kernels_out) *n_kernels_out = g.n_launches;
  });
}

dcp_status dcp_run(dcp_graph gh, const void* const* inputs, void* const* outputs,
                   void* cuda_stream) {
  return guarded([&] {
    GraphImpl& g = G(gh);
    if (!g.fused) fail(DCP_E_STATE, "call dcp_fuse before dcp_run");
    if ((!inputs && !g.inputs.empty()) || !outputs) fail(DCP_E_INVALID_ARG, "NULL buffer list");
    run_graph(g, inputs, outputs, (cudaStream_t)cuda_stream);
  });
}

dcp_status dcp_run_host(dcp_graph gh, const void* const* inputs, void* const* outputs,
                        void* cuda_stream) {
  return guarded([&] {
    GraphImpl& g = G(gh);
    if (!g.fused) fail(DCP_E_STATE, "call dcp_fuse before dcp_run_host");
    if ((!inputs && !g.inputs.empty()) || !outputs) fail(DCP_E_INVALID_ARG, "NULL buffer list");
    run_graph_host(g, inputs, outputs, (cudaStream_t)cuda_stream);
  });
}

dcp_status dcp_run_adjoint(dcp_graph gh, const void* const* inputs, const void* const* out_grads,
                           void* const* in_grads, size_t tape_budget_bytes, void* cuda_stream) {
  return guarded([&] {
    GraphImpl& g = G(gh);
    if (!g.fused) fail(DCP_E_STATE, "call dcp_fuse before dcp_run_adjoint");
    if ((!inputs && !g.inputs.empty()) || !out_grads || !in_grads)
      fail(DCP_E_INVALID_ARG, "NULL buffer list");
    run_adjoint(g, inputs, out_grads, in_grads, tape_budget_bytes, (cudaStream_t)cuda_stream);
  });
}

dcp_status dcp_prepare_adjoint(dcp_graph gh, size_t tape_budget_bytes) {
  return guarded([&] {
    GraphImpl& g = G(gh);
    if (!g.fused) fail(DCP_E_STATE, "call dcp_fuse before dcp_prepare_adjoint");
    prepare_adjoint(g, tape_budget_bytes);
  });
}

dcp_status dcp_sync(dcp_graph gh, void* cuda_stream) {
  return guarded([&] {
    GraphImpl& g = G(gh);
    sync_graph(g, (cudaStream_t)cuda_stream);
  });
}

dcp_status dcp_set_option(dcp_graph gh, int32_t key, int64_t v) {
  return guarded([&] {
    GraphImpl& g = G(gh);
    switch (key) {
      case DCP_OPT_TIME_TILE_DEPTH:
      case DCP_OPT_TILE_X:
      case DCP_OPT_TILE_Y:
      case DCP_OPT_MAP_BLOCKS_PER_SM:
      case DCP_OPT_STENCIL_KERNEL:
      case DCP_OPT_STREAM_ROWS:
      case DCP_OPT_TILE_Z:
      case DCP_OPT_STREAM_PREFETCH:
      case DCP_OPT_STREAM_THREADS:
      case DCP_OPT_CELLS_PER_THREAD:
      case DCP_OPT_MAP_UNROLL:
      case DCP_OPT_DEFERRED_WEIGHT:
      case DCP_OPT_STREAM_MIN_CTAS:
      case DCP_OPT_ADJOINT_DEPTH:
        if (g.fused) fail(DCP_E_STATE, "tiling options must be set before dcp_fuse");
        break;
      case DCP_OPT_USE_GRAPH:
      case DCP_OPT_HOST_ACCESS:
        break;
      default:
        fail(DCP_E_INVALID_ARG, "unknown option key " + std::to_string(key));
    }
    if (v < 0) {
      g.options.erase(key);
      return;
    }
    if (key == DCP_OPT_TIME_TILE_DEPTH && (v < 1 || v > 64)) fail(DCP_E_INVALID_ARG, "depth must be 1..64");
    if (key == DCP_OPT_TILE_X && (v < 8 || v > 512 || v % 8)) fail(DCP_E_INVALID_ARG, "tile x must be a multiple of 8 in 8..512");
    if (key == DCP_OPT_TILE_Y && (v < 1 || v > 512)) fail(DCP_E_INVALID_ARG, "tile y must be in 1..512");
    if (key == DCP_OPT_MAP_BLOCKS_PER_SM && (v < 1 || v > 32)) fail(DCP_E_INVALID_ARG, "blocks per SM must be 1..32");
    if (key == DCP_OPT_STENCIL_KERNEL && v > 2) fail(DCP_E_INVALID_ARG, "stencil kernel form must be 0, 1 or 2");
    if (key == DCP_OPT_STREAM_ROWS && (v < 1 || v > (1 << 30))) fail(DCP_E_INVALID_ARG, "rows per work item must be >= 1");
    if (key == DCP_OPT_TILE_Z && (v < 1 || v > 1024)) fail(DCP_E_INVALID_ARG, "tile z must be in 1..1024");
    if (key == DCP_OPT_STREAM_PREFETCH && (v < 1 || v > 4)) fail(DCP_E_INVALID_ARG, "stream prefetch must be in 1..4");
    if (key == DCP_OPT_STREAM_THREADS && (v < 32 || v > 1024 || v % 32)) fail(DCP_E_INVALID_ARG, "stream threads must be a multiple of 32 in 32..1024");
    if (key == DCP_OPT_CELLS_PER_THREAD && v != 1 && v != 2) fail(DCP_E_INVALID_ARG, "cells per thread must be 1 or 2");
    if (key == DCP_OPT_MAP_UNROLL && (v < 1 || v > 8)) fail(DCP_E_INVALID_ARG, "map unroll must be in 1..8");
    if (key == DCP_OPT_DEFERRED_WEIGHT && v != 0 && v != 1) fail(DCP_E_INVALID_ARG, "deferred weight must be 0 or 1");
    if (key == DCP_OPT_STREAM_MIN_CTAS && (v < 1 || v > 32)) fail(DCP_E_INVALID_ARG, "stream min CTAs must be in 1..32");
    if (key == DCP_OPT_ADJOINT_DEPTH && v > 64) fail(DCP_E_INVALID_ARG, "adjoint depth must be in 0..64");
    g.options[key] = v;
  });
}

dcp_status dcp_plan_info(dcp_graph gh, char* buf, size_t len, size_t* needed) {
  return guarded([&] {
    GraphImpl& g = G(gh);
    std::string s = g.fused ? describe_plan(g) : std::string("{\"fused\": false}");
    if (needed) *needed = s.size() + 1;
    if (buf && len > 0) {
      size_t n = s.size() < len - 1 ? s.size() : len - 1;
      std::memcpy(buf, s.data(), n);
      buf[n] = 0;
    }
  });
}

const char* dcp_last_error(void) { return g_last_error.c_str(); }

const char* dcp_version(void) { return "dcp 0.1 (sm_103a)"; }

}  // extern "C"
