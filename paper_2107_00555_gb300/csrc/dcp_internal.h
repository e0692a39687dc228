// Internal declarations of the dcp runtime: graph IR, fused plan, codegen,
// run-time compilation and execution.  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "dcp.h"

namespace dcp {

// ---------------------------------------------------------------------------
// Errors: internal code throws dcp::Error; the C ABI layer converts it into a
// status code plus the thread-local message.
// ---------------------------------------------------------------------------
struct Error {
  dcp_status code;
  std::string msg;
};
[[noreturn]] void fail(dcp_status code, const std::string& msg);
void set_last_error(const std::string& msg);
void check_cuda(cudaError_t e, const char* what);
void check_cu(CUresult r, const char* what);

// Driver API entry points (driver.cpp), resolved through the runtime.
struct Driver {
  CUresult (*ctxGetCurrent)(CUcontext*) = nullptr;
  CUresult (*moduleLoadData)(CUmodule*, const void*) = nullptr;
  CUresult (*moduleGetFunction)(CUfunction*, CUmodule, const char*) = nullptr;
  CUresult (*funcGetAttribute)(int*, CUfunction_attribute, CUfunction) = nullptr;
  CUresult (*funcSetAttribute)(CUfunction, CUfunction_attribute, int) = nullptr;
  CUresult (*occupancy)(int*, CUfunction, int, size_t) = nullptr;
  CUresult (*launchKernel)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                           unsigned, CUstream, void**, void**) = nullptr;
  CUresult (*launchCooperative)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned,
                                unsigned, unsigned, CUstream, void**) = nullptr;
  CUresult (*getErrorString)(CUresult, const char**) = nullptr;
};
const Driver& drv();

int dtype_size(int dtype);
bool dtype_is_float(int dtype);
const char* dtype_cname(int dtype);  // C type used in generated code
const char* dtype_name(int dtype);

// ---------------------------------------------------------------------------
// Graph IR: one node per NumPy-level operation (SSA form, Sec. 2.3).
// ---------------------------------------------------------------------------
enum class Kind { Input, Map, Stencil, Reduce, AdjChain };

// One forward step of a chain whose reverse runs as one AdjChain node: the
// step's weights (the chain's common offsets) and its epilogue maps
// (unary / immediate ops, in order).
struct AdjStep {
  std::vector<double> weights;
  std::vector<std::pair<int, double>> epi;  // (op, imm)
};

struct Node {
  Kind kind = Kind::Input;
  int dtype = DCP_F32;
  std::vector<int64_t> shape;
  int op = -1;              // map op / reduce op
  std::vector<int> in;      // operand value ids
  double imm = 0.0;
  // stencil
  std::vector<int32_t> offsets;  // npts * ndim
  std::vector<double> weights;
  int bc = DCP_BC_ZERO;
  int steps = 0;
  // reduce: the reduced axis of the operand, -1 = all axes
  int axis = -1;
  // AdjChain (built by the adjoint only): in = {u_t, cotangent of u_{t+k}},
  // value = cotangent of u_t through the k = chain.size() forward steps
  // u_{i+1} = E_i(S_i u_i) (1-D / 2-D, offsets/bc/shape as for a stencil)
  std::vector<AdjStep> chain;
  int64_t numel() const {
    int64_t n = 1;
    for (auto s : shape) n *= s;
    return n;
  }
  int ndim() const { return (int)shape.size(); }
  int npts() const { return (int)weights.size(); }
};

// Internal map ops (emitted by the adjoint builder only, never by the ABI).
constexpr int kOpBcast = 100;  // y = 0-axis operand broadcast to the shape
constexpr int kOpConst = 101;  // y = imm
constexpr int kOpSign = 102;   // y = sign(x), sign(0) = 0
constexpr int kOpGt = 103;     // y = a > b ? 1 : 0
constexpr int kOpLt = 104;     // y = a < b ? 1 : 0

bool op_is_unary(int op);
bool op_is_binary(int op);
bool op_is_scalar_imm(int op);
bool op_float_only(int op);
const char* op_name(int op);
const char* red_name(int red);

// ---------------------------------------------------------------------------
// Fused plan (Sec. 3.1: greedy subgraph fusion, tiled write-conflict
// resolution, transient mitigation).
// ---------------------------------------------------------------------------
enum class GroupKind { Map, Stencil, Batch, AxisReduce, AdjTile };

// One step of an iterated stencil inside a stencil group.  `node` is the
// stencil node providing offsets/weights; `epi` the unary/immediate map nodes
// applied, in order, to the weighted sum (stencil -> map epilogue fusion).
struct StepDesc {
  int node = -1;
  std::vector<int> epi;
};

struct Group {
  GroupKind kind = GroupKind::Map;
  int dtype = DCP_F32;
  std::vector<int64_t> shape;   // iteration space
  // Map groups: members computed in registers, in topological order.
  // Stencil groups: prologue members producing `st_in` (may be empty, then
  // st_in is loaded), steps, then post members computed from `st_out`.
  std::vector<int> members;     // map node ids (map groups) / prologue members
  std::vector<int> post;        // post members (stencil groups)
  std::vector<int> loads;       // full-shape values read from memory (map / prologue)
  std::vector<int> post_loads;  // full-shape values read at the output index (stencil post)
  std::vector<int> scalars;     // 0-axis values broadcast into the expressions
  std::vector<int> stores;      // values written to memory by this group
  std::vector<int> reds;        // reduce node ids computed here
  int st_in = -1;               // stencil input value
  int st_out = -1;              // value after the last step (+ its epilogue)
  std::vector<StepDesc> steps;
  int bc = DCP_BC_ZERO;
  std::vector<int32_t> offsets;  // common offset set, padded to 3 axes (dz,dy,dx)
  int radius[3] = {0, 0, 0};
  // launch decomposition
  int depth = 1;                // stencil steps per launch
  int tile[3] = {1, 1, 1};      // output tile (z, y, x) for stencils
  int threads = 256;
  int blocks_per_sm = 4;
  int variant = 0;              // stencils: 0 = shared-memory tile, 1 = warp stream,
                                //           2 = cooperative (every step in one launch)
  int seg = 0;                  // warp stream: rows per work item (single arrays)
  int prefetch = 1;             // warp stream: rows requested ahead, in row windows (2*ry+1)
  int min_ctas = 0;             // warp stream: CTAs per SM the register budget must allow (0: any)
  int cx = 1;                   // 3-D stencils: cells per thread along x (1 or 2)
  int unroll = 2;               // map groups: 16-byte vectors per array in flight per thread
  // axis-reduce groups: the reduced axis of the iteration space `shape`
  int axis = -1;
  // batch groups: the member stencil groups (same program, different shapes)
  std::vector<int> batch_members;  // indices into Plan::groups of absorbed groups
  bool absorbed = false;           // this stencil group runs inside a batch group
};

struct Kernel {
  std::string name;
  std::string source;
  CUfunction fn = nullptr;
  int smem_bytes = 0;
  int threads = 256;
  double compile_ms = 0.0;
  int regs = 0;
};

// ---------------------------------------------------------------------------
// Run-time compilation (NVRTC -> cubin for sm_103a, Sec. 3.3) and a module
// cache keyed by the source text.
// ---------------------------------------------------------------------------
struct CompiledModule {
  CUmodule mod = nullptr;
  std::vector<char> cubin;
  double compile_ms = 0.0;
  bool from_cache = false;
};
typedef std::shared_ptr<const std::vector<char>> CubinRef;
CubinRef nvrtc_compile(const std::string& src, const std::string& name, double* ms,
                       std::string* log);
CUfunction load_function(const std::string& src, const std::string& name, double* ms, int* regs);
const char* device_header_source();     // dcp_device.cuh
const char* kernel_map_source();        // k_map.cuh
const char* kernel_stencil2d_source();  // k_stencil2d.cuh
const char* kernel_stencil3d_source();  // k_stencil3d.cuh
const char* kernel_stream_source();     // k_stencil2d_stream.cuh
const char* kernel_axis_source();       // k_axis.cuh
const char* kernel_math64_source();     // k_math64.cuh
const char* kernel_adj_source();        // k_stencil_adj.cuh
const char* kernel_coop_source();       // k_stencil2d_coop.cuh

// ---------------------------------------------------------------------------
// Graph object
// ---------------------------------------------------------------------------
struct LaunchRec;  // defined in runtime.cpp

struct GraphImpl {
  std::vector<Node> nodes;
  std::vector<int> inputs;
  std::vector<int> outputs;
  bool fused = false;
  uint32_t flags = 0;
  std::map<int, int64_t> options;
  std::vector<Group> groups;      // in execution order
  std::vector<Group> batch_store; // stencil groups packed into batch groups
  std::vector<int> value_group;   // value id -> producing group (-1 input)
  std::vector<char> materialized; // value id -> needs a device buffer
  int n_launches = 0;
  std::string plan_json;
  // runtime state (runtime.cpp)
  struct Runtime;
  std::unique_ptr<Runtime> rt;
  std::shared_ptr<struct AdjointState> adj;  // adjoint.cpp
  GraphImpl();
  ~GraphImpl();
};

void plan_graph(GraphImpl& g, uint32_t flags);      // fuse.cpp
void compile_plan(GraphImpl& g);                    // runtime.cpp
void run_graph(GraphImpl& g, const void* const* inputs, void* const* outputs, cudaStream_t s);
void run_graph_host(GraphImpl& g, const void* const* inputs, void* const* outputs,
                    cudaStream_t s);
void run_adjoint(GraphImpl& g, const void* const* inputs, const void* const* out_grads,
                 void* const* in_grads, size_t budget, cudaStream_t s);
void prepare_adjoint(GraphImpl& g, size_t budget);
void sync_graph(GraphImpl& g, cudaStream_t s);
void run_adjoint_impl(GraphImpl& g, AdjointState& st, const void* const* inputs,
                      const void* const* out_grads, void* const* in_grads, size_t budget,
                      cudaStream_t s);
void prepare_adjoint_impl(GraphImpl& g, AdjointState& st, size_t budget);
std::shared_ptr<AdjointState> new_adjoint_state();
size_t adjoint_tape_bytes(const AdjointState& st);
bool adjoint_chunked(const AdjointState& st);
std::string adjoint_launches_json(const AdjointState& st);
// kernel names of a compiled graph's launches, in execution order
std::vector<std::string> launch_kernel_names(const GraphImpl& g);
std::string describe_plan(const GraphImpl& g);

// codegen.cpp
struct CodegenOut {
  std::string name;
  std::string source;
  int smem_bytes = 0;
  int threads = 256;
  int vec = 1;     // axis reductions: elements per load
  int axmode = 0;  // axis reductions: 0 vectors along inner, 1 along the reduced axis
  // stencil launches: per step, the factor applied after the step when it
  // sums ratios to a deferred common weight (1: none), 0 for a plain sum;
  // empty when no step of the launch is deferred
  std::vector<double> defer_scales;
  // first launch of a deferred run: the largest finite |input| that run keeps
  // finite (its magnitude guard's bound); 0 when the launch has no guard
  double guard_max_input = 0.0;
};
CodegenOut gen_map_kernel(const GraphImpl& g, const Group& grp, bool vec_ok);
// Stencil launch `chunk` covers steps [s0, s1) of the group.
CodegenOut gen_stencil_kernel(const GraphImpl& g, const Group& grp, int s0, int s1);
CodegenOut gen_batch_kernel(const GraphImpl& g, const Group& grp, int s0, int s1);
CodegenOut gen_axis_kernel(const GraphImpl& g, const Group& grp, bool vec_ok);
// reverse of a chunk of a 1-D / 2-D stencil chain, forward recomputed in the tile
CodegenOut gen_adj_kernel(const GraphImpl& g, const Group& grp);
// does the reverse of epilogue chain `epi` read a value other than its output?
bool adj_needs_z(const std::vector<std::pair<int, double>>& epi);

// Steps per chunk of a deferred common-weight run of stencil node n's steps
// (0: plain weighted sum; INT32_MAX: no growth bound).
int defer_chunk_steps(const Node& n);

uint64_t fnv1a(const std::string& s);

constexpr int kMaxIO = 16;       // loads / stores / reductions per kernel

// Warp-stream stencil geometry: columns per lane and columns written per warp.
inline int stream_cols_per_lane(int dtype) { return dtype == DCP_F64 || dtype == DCP_I64 ? 2 : 4; }
inline int stream_width(const Group& G) {
  return 32 * stream_cols_per_lane(G.dtype) - 2 * G.depth * G.radius[2];
}
bool stream_eligible(const Group& G, int depth);
// can the cooperative form run this group with a ty x tx tile (steps <= 63,
// 1-D / 2-D, each ragged edge tile at least a radius wide)?
bool coop_eligible(const Group& G, int ty, int tx);
constexpr int kMaxRadius = 4;
constexpr int kMaxPoints = 32;

}  // namespace dcp
