// Execution of a fused plan: one launch per fused group (or per time-tile
// chunk of a stencil group), transients allocated once and reused (Sec. 3.1
// transient allocation mitigation: temporaries are persistent, allocated when
// the program is first run), per-group scratch for the tiled reductions, and
// optional replay of the whole run as one captured CUDA graph.
#include <algorithm>
#include <cinttypes>
#include <cstring>
#include <numeric>
#include <sstream>

#include "dcp_internal.h"

namespace dcp {

namespace {

struct MapParamsH {
  const void* ld[kMaxIO];
  void* st[kMaxIO];
  const void* sc[kMaxIO];
  void* red_out[kMaxIO];
  int64_t n;
  void* partials;
  void* ticket;
};
struct StParamsH {
  const void* ld[kMaxIO];
  const void* pld[kMaxIO];
  void* st[kMaxIO];
  const void* sc[kMaxIO];
  void* red_out[kMaxIO];
  int32_t nz, ny, nx;
  int32_t tiles_x, tiles_y, tiles_z;
  void* partials;
  void* ticket;
};
struct InstH {
  const void* in;
  void* out;
  int32_t ny, nx, tiles_x, tile0;
};
struct BatchParamsH {
  const void* inst;
  int32_t ninst;
  int32_t total_tiles;
};
static_assert(sizeof(StParamsH) == 5 * kMaxIO * 8 + 24 + 16, "stencil params layout");
static_assert(sizeof(InstH) == 32, "instance layout");

struct LaunchSpec {
  int group = -1;
  int s0 = 0, s1 = 0;  // stencil steps of this launch
  CodegenOut code;
  CodegenOut code_scalar;  // map groups: element-by-element fallback for unaligned buffers
  CUfunction fn = nullptr, fn_scalar = nullptr;
  double compile_ms = 0.0;
  int regs = 0;
  int occupancy = 0;
  int occ_scalar = 1;
};

int64_t numel(const std::vector<int64_t>& s) {
  int64_t n = 1;
  for (auto v : s) n *= v;
  return n;
}

void dims3(const std::vector<int64_t>& s, int32_t& nz, int32_t& ny, int32_t& nx) {
  int64_t d[3] = {1, 1, 1};
  for (size_t i = 0; i < s.size(); ++i) d[3 - s.size() + i] = s[i];
  for (int i = 0; i < 3; ++i)
    if (d[i] > 0x7fffffff) fail(DCP_E_SHAPE, "stencil extents must be < 2^31");
  nz = (int32_t)d[0];
  ny = (int32_t)d[1];
  nx = (int32_t)d[2];
}

}  // namespace

struct GraphImpl::Runtime {
  std::vector<LaunchSpec> launches;
  bool device_ready = false;
  int device = -1;
  int sms = 0;
  std::vector<void*> allocs;
  std::vector<void*> transient;          // per value id
  std::vector<void*> state[2];           // per group: time-tile ping-pong
  std::vector<void*> partials;           // per group
  std::vector<unsigned*> tickets;        // per group
  std::vector<int> partial_slots;        // per group: blocks that may write partials
  // batch tables, per launch
  std::vector<InstH*> host_tables;       // pinned
  std::vector<void*> dev_tables;
  std::vector<int> table_tiles;
  std::vector<std::vector<const void*>> table_key;
  cudaEvent_t table_ev = nullptr;
  std::vector<int64_t> batch_offset;     // per batch member: element offset in batch state
  void* batch_state[2] = {nullptr, nullptr};
  // host-buffer runs
  std::vector<void*> stage_in, stage_out;
  // graph replay
  cudaGraphExec_t gexec = nullptr;
  std::vector<const void*> gkey;
  ~Runtime() {
    if (device_ready) {
      int cur = -1;
      cudaGetDevice(&cur);
      if (cur != device) cudaSetDevice(device);
      cudaDeviceSynchronize();
      if (gexec) cudaGraphExecDestroy(gexec);
      for (void* p : allocs) cudaFree(p);
      for (InstH* h : host_tables) cudaFreeHost(h);
      if (table_ev) cudaEventDestroy(table_ev);
      if (cur != device && cur >= 0) cudaSetDevice(cur);
    }
  }
};

GraphImpl::GraphImpl() = default;
GraphImpl::~GraphImpl() = default;

// ---------------------------------------------------------------------------
// compile: generate + NVRTC every launch of the plan (no GPU needed)
// ---------------------------------------------------------------------------
void compile_plan(GraphImpl& g) {
  g.rt.reset(new GraphImpl::Runtime());
  auto& L = g.rt->launches;
  for (int gi = 0; gi < (int)g.groups.size(); ++gi) {
    const Group& G = g.groups[gi];
    if (G.kind == GroupKind::Map) {
      LaunchSpec ls;
      ls.group = gi;
      ls.code = gen_map_kernel(g, G, true);
      ls.code_scalar = gen_map_kernel(g, G, false);
      double ms = 0;
      nvrtc_compile(ls.code.source, ls.code.name, &ms, nullptr);
      ls.compile_ms = ms;
      L.push_back(std::move(ls));
    } else {
      int S = (int)G.steps.size();
      for (int s0 = 0; s0 < S; s0 += G.depth) {
        LaunchSpec ls;
        ls.group = gi;
        ls.s0 = s0;
        ls.s1 = std::min(S, s0 + G.depth);
        ls.code = gen_stencil_kernel(g, G, ls.s0, ls.s1);
        if (ls.code.smem_bytes > 227 * 1024)
          fail(DCP_E_UNSUPPORTED, "stencil tile needs " + std::to_string(ls.code.smem_bytes) +
                                      " bytes of shared memory; lower the tile or depth");
        double ms = 0;
        nvrtc_compile(ls.code.source, ls.code.name, &ms, nullptr);
        ls.compile_ms = ms;
        L.push_back(std::move(ls));
      }
    }
  }
  g.n_launches = (int)L.size();
}

// ---------------------------------------------------------------------------
// device state: modules, transients, scratch
// ---------------------------------------------------------------------------
static void* dalloc(GraphImpl::Runtime& rt, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  check_cuda(cudaMalloc(&p, bytes), "cudaMalloc");
  rt.allocs.push_back(p);
  return p;
}

static void ensure_device(GraphImpl& g) {
  auto& rt = *g.rt;
  int dev = -1;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  if (rt.device_ready) {
    if (dev != rt.device) fail(DCP_E_STATE, "graph was first run on another device");
    return;
  }
  check_cuda(cudaFree(nullptr), "CUDA context initialisation");
  int sms = 0;
  check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  rt.device = dev;
  rt.sms = sms;
  const int N = (int)g.nodes.size();
  rt.transient.assign(N, nullptr);
  std::vector<char> is_io(N, 0);
  for (int v : g.inputs) is_io[v] = 1;
  for (int v : g.outputs) is_io[v] = 1;
  try {
    for (auto& ls : rt.launches) {
      ls.fn = load_function(ls.code.source, ls.code.name, nullptr, &ls.regs);
      if (ls.code.smem_bytes > 48 * 1024)
        check_cu(drv().funcSetAttribute(ls.fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES,
                                    ls.code.smem_bytes),
                 "cuFuncSetAttribute(max dynamic smem)");
      int occ = 0;
      check_cu(drv().occupancy(&occ, ls.fn, ls.code.threads,
                                                           ls.code.smem_bytes),
               "occupancy query");
      if (occ < 1) fail(DCP_E_UNSUPPORTED, "kernel " + ls.code.name + " cannot be resident on an SM");
      ls.occupancy = occ;
    }
    for (int v = 0; v < N; ++v)
      if (g.materialized[v] && !is_io[v])
        rt.transient[v] = dalloc(rt, (size_t)g.nodes[v].numel() * dtype_size(g.nodes[v].dtype));
    const int NG = (int)g.groups.size();
    rt.state[0].assign(NG, nullptr);
    rt.state[1].assign(NG, nullptr);
    rt.partials.assign(NG, nullptr);
    rt.tickets.assign(NG, nullptr);
    rt.partial_slots.assign(NG, 0);
    for (int gi = 0; gi < NG; ++gi) {
      const Group& G = g.groups[gi];
      int nch = G.kind == GroupKind::Map ? 1 : ((int)G.steps.size() + G.depth - 1) / G.depth;
      if (G.kind == GroupKind::Stencil && nch > 1) {
        size_t bytes = (size_t)numel(G.shape) * dtype_size(G.dtype);
        rt.state[0][gi] = dalloc(rt, bytes);
        if (nch > 2) rt.state[1][gi] = dalloc(rt, bytes);
      }
      if (G.kind == GroupKind::Batch) {
        int64_t tot = 0;
        rt.batch_offset.clear();
        for (int m : G.batch_members) {
          rt.batch_offset.push_back(tot);
          tot += (numel(g.batch_store[m].shape) + 31) / 32 * 32;  // 128-byte aligned slices
        }
        if (nch > 1) {
          rt.batch_state[0] = dalloc(rt, (size_t)tot * dtype_size(G.dtype));
          if (nch > 2) rt.batch_state[1] = dalloc(rt, (size_t)tot * dtype_size(G.dtype));
        }
      }
      if (!G.reds.empty()) {
        int slots = 0;
        if (G.kind == GroupKind::Map) {
          slots = sms * G.blocks_per_sm;
        } else {
          // stencil reductions: one partial per CTA of the last launch
          int32_t nz, ny, nx;
          dims3(G.shape, nz, ny, nx);
          int64_t tiles = (int64_t)((nx + G.tile[2] - 1) / G.tile[2]);
          if (G.shape.size() >= 2) tiles *= (ny + G.tile[1] - 1) / G.tile[1];
          if (G.shape.size() == 3) tiles *= (nz + G.tile[0] - 1) / G.tile[0];
          slots = (int)std::max<int64_t>(1, tiles);
        }
        rt.partial_slots[gi] = slots;
        rt.partials[gi] = dalloc(rt, (size_t)slots * G.reds.size() * 8);
        rt.tickets[gi] = (unsigned*)dalloc(rt, 256);
        check_cuda(cudaMemset(rt.tickets[gi], 0, 256), "cudaMemset(ticket)");
      }
    }
    rt.host_tables.assign(rt.launches.size(), nullptr);
    rt.dev_tables.assign(rt.launches.size(), nullptr);
    rt.table_tiles.assign(rt.launches.size(), 0);
    rt.table_key.assign(rt.launches.size(), {});
    check_cuda(cudaEventCreateWithFlags(&rt.table_ev, cudaEventDisableTiming), "cudaEventCreate");
    check_cuda(cudaDeviceSynchronize(), "device set-up");
  } catch (...) {
    for (void* p : rt.allocs) cudaFree(p);
    rt.allocs.clear();
    throw;
  }
  rt.device_ready = true;
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------
static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static void launch_map(GraphImpl& g, LaunchSpec& ls, const std::vector<const void*>& ptr,
                       cudaStream_t s) {
  auto& rt = *g.rt;
  const Group& G = g.groups[ls.group];
  MapParamsH p;
  std::memset(&p, 0, sizeof p);
  bool vec = true;
  const size_t esz = dtype_size(G.dtype);
  for (size_t i = 0; i < G.loads.size(); ++i) {
    p.ld[i] = ptr[G.loads[i]];
    vec = vec && aligned16(p.ld[i]);
    if ((uintptr_t)p.ld[i] % esz) fail(DCP_E_INVALID_ARG, "buffer not aligned to its element size");
  }
  for (size_t i = 0; i < G.stores.size(); ++i) {
    p.st[i] = const_cast<void*>(ptr[G.stores[i]]);
    vec = vec && aligned16(p.st[i]);
    if ((uintptr_t)p.st[i] % esz) fail(DCP_E_INVALID_ARG, "buffer not aligned to its element size");
  }
  for (size_t i = 0; i < G.scalars.size(); ++i) p.sc[i] = ptr[G.scalars[i]];
  for (size_t i = 0; i < G.reds.size(); ++i) p.red_out[i] = const_cast<void*>(ptr[G.reds[i]]);
  p.n = numel(G.shape);
  p.partials = rt.partials[ls.group];
  p.ticket = rt.tickets[ls.group];
  if (p.n == 0 && G.reds.empty()) return;
  CUfunction fn = ls.fn;
  int per = 16 / (int)esz;
  int occ = ls.occupancy;
  if (!vec) {
    if (!ls.fn_scalar) {
      ls.fn_scalar = load_function(ls.code_scalar.source, ls.code_scalar.name, nullptr, nullptr);
      check_cu(drv().occupancy(&ls.occ_scalar, ls.fn_scalar, G.threads, 0), "occupancy query");
    }
    fn = ls.fn_scalar;
    per = 1;
    occ = ls.occ_scalar;
  }
  // one wave of resident CTAs (grid-stride loop): no partial second wave
  int64_t work = (p.n + per - 1) / per;
  int64_t blocks = (work + G.threads - 1) / G.threads;
  int64_t maxb = (int64_t)rt.sms * std::max(1, std::min(G.blocks_per_sm, occ));
  if (blocks > maxb) blocks = maxb;
  if (blocks < 1) blocks = 1;
  void* args[] = {&p};
  check_cu(drv().launchKernel(fn, (unsigned)blocks, 1, 1, G.threads, 1, 1, 0, (CUstream)s, args, nullptr),
           "cuLaunchKernel(map)");
}

static void launch_stencil(GraphImpl& g, LaunchSpec& ls, const std::vector<const void*>& ptr,
                           cudaStream_t s) {
  auto& rt = *g.rt;
  const Group& G = g.groups[ls.group];
  const int S = (int)G.steps.size();
  const bool first = ls.s0 == 0, last = ls.s1 == S;
  const int chunk = ls.s0 / G.depth;
  StParamsH p;
  std::memset(&p, 0, sizeof p);
  if (first) {
    if (!G.members.empty()) {
      for (size_t i = 0; i < G.loads.size(); ++i) p.ld[i] = ptr[G.loads[i]];
    } else {
      p.ld[0] = ptr[G.st_in];
    }
  } else {
    p.ld[0] = rt.state[(chunk - 1) % 2][ls.group];
  }
  if (last) {
    for (size_t i = 0; i < G.stores.size(); ++i) p.st[i] = const_cast<void*>(ptr[G.stores[i]]);
    for (size_t i = 0; i < G.post_loads.size(); ++i) p.pld[i] = ptr[G.post_loads[i]];
    for (size_t i = 0; i < G.reds.size(); ++i) p.red_out[i] = const_cast<void*>(ptr[G.reds[i]]);
  } else {
    p.st[0] = rt.state[chunk % 2][ls.group];
  }
  for (size_t i = 0; i < G.scalars.size(); ++i) p.sc[i] = ptr[G.scalars[i]];
  dims3(G.shape, p.nz, p.ny, p.nx);
  if ((int64_t)p.nz * p.ny * p.nx == 0) return;
  const int nd = (int)G.shape.size();
  const int TX = G.tile[2], TY = nd == 1 ? 1 : G.tile[1];
  p.tiles_x = (p.nx + TX - 1) / TX;
  p.tiles_y = (p.ny + TY - 1) / TY;
  p.tiles_z = nd == 3 ? (p.nz + G.tile[0] - 1) / G.tile[0] : 1;
  p.partials = rt.partials[ls.group];
  p.ticket = rt.tickets[ls.group];
  int64_t gx = (int64_t)p.tiles_x * p.tiles_y;
  if (gx > 0x7fffffff) fail(DCP_E_SHAPE, "grid too large");
  void* args[] = {&p};
  check_cu(drv().launchKernel(ls.fn, (unsigned)gx, (unsigned)p.tiles_z, 1, ls.code.threads, 1, 1,
                          ls.code.smem_bytes, (CUstream)s, args, nullptr),
           "cuLaunchKernel(stencil)");
}

static void launch_batch(GraphImpl& g, size_t li, LaunchSpec& ls,
                         const std::vector<const void*>& ptr, cudaStream_t s) {
  auto& rt = *g.rt;
  const Group& G = g.groups[ls.group];
  const int S = (int)G.steps.size();
  const bool first = ls.s0 == 0, last = ls.s1 == S;
  const int chunk = ls.s0 / G.depth;
  const size_t esz = dtype_size(G.dtype);
  const int nm = (int)G.batch_members.size();
  // key: the caller pointers this table depends on
  std::vector<const void*> key;
  for (int m : G.batch_members) {
    key.push_back(ptr[g.batch_store[m].st_in]);
    key.push_back(ptr[g.batch_store[m].st_out]);
  }
  if (!rt.dev_tables[li] || rt.table_key[li] != key) {
    if (!rt.host_tables[li]) {
      check_cuda(cudaMallocHost((void**)&rt.host_tables[li], sizeof(InstH) * nm), "cudaMallocHost");
      rt.dev_tables[li] = dalloc(rt, sizeof(InstH) * nm);
    } else {
      check_cuda(cudaEventSynchronize(rt.table_ev), "cudaEventSynchronize");
    }
    // members ordered by tile count, largest first, for load balance
    std::vector<int> order(nm);
    std::iota(order.begin(), order.end(), 0);
    auto tiles_of = [&](int k) {
      const Group& M = g.batch_store[G.batch_members[k]];
      int64_t ny = M.shape[0], nx = M.shape[1];
      return ((nx + G.tile[2] - 1) / G.tile[2]) * ((ny + G.tile[1] - 1) / G.tile[1]);
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return tiles_of(a) > tiles_of(b); });
    int64_t t0 = 0;
    for (int j = 0; j < nm; ++j) {
      int k = order[j];
      const Group& M = g.batch_store[G.batch_members[k]];
      InstH& I = rt.host_tables[li][j];
      const size_t off = (size_t)rt.batch_offset[k] * esz;
      I.in = first ? ptr[M.st_in] : (const char*)rt.batch_state[(chunk - 1) % 2] + off;
      I.out = last ? const_cast<void*>(ptr[M.st_out]) : (char*)rt.batch_state[chunk % 2] + off;
      I.ny = (int32_t)M.shape[0];
      I.nx = (int32_t)M.shape[1];
      I.tiles_x = (int32_t)((I.nx + G.tile[2] - 1) / G.tile[2]);
      I.tile0 = (int32_t)t0;
      t0 += tiles_of(k);
    }
    if (t0 > 0x7fffffff) fail(DCP_E_SHAPE, "batch has too many tiles");
    rt.table_tiles[li] = (int)t0;
    check_cuda(cudaMemcpyAsync(rt.dev_tables[li], rt.host_tables[li], sizeof(InstH) * nm,
                               cudaMemcpyHostToDevice, s),
               "cudaMemcpyAsync(batch table)");
    check_cuda(cudaEventRecord(rt.table_ev, s), "cudaEventRecord");
    rt.table_key[li] = key;
  }
  BatchParamsH p{rt.dev_tables[li], nm, rt.table_tiles[li]};
  if (p.total_tiles == 0) return;
  int64_t grid = std::min<int64_t>(p.total_tiles, (int64_t)rt.sms * ls.occupancy);
  void* args[] = {&p};
  check_cu(drv().launchKernel(ls.fn, (unsigned)grid, 1, 1, ls.code.threads, 1, 1, ls.code.smem_bytes,
                          (CUstream)s, args, nullptr),
           "cuLaunchKernel(batch)");
}

static std::vector<const void*> bind(GraphImpl& g, const void* const* inputs,
                                     void* const* outputs) {
  auto& rt = *g.rt;
  std::vector<const void*> ptr(g.nodes.size(), nullptr);
  for (int v = 0; v < (int)g.nodes.size(); ++v) ptr[v] = rt.transient[v];
  for (size_t i = 0; i < g.inputs.size(); ++i) {
    const Node& n = g.nodes[g.inputs[i]];
    if (!inputs[i] && n.numel() > 0) fail(DCP_E_INVALID_ARG, "input " + std::to_string(i) + " is NULL");
    ptr[g.inputs[i]] = inputs[i];
  }
  for (size_t j = 0; j < g.outputs.size(); ++j) {
    const Node& n = g.nodes[g.outputs[j]];
    if (!outputs[j] && (n.numel() > 0 || n.kind == Kind::Reduce))
      fail(DCP_E_INVALID_ARG, "output " + std::to_string(j) + " is NULL");
    ptr[g.outputs[j]] = outputs[j];
  }
  return ptr;
}

static void launch_all(GraphImpl& g, const std::vector<const void*>& ptr, cudaStream_t s) {
  auto& rt = *g.rt;
  for (size_t li = 0; li < rt.launches.size(); ++li) {
    LaunchSpec& ls = rt.launches[li];
    const Group& G = g.groups[ls.group];
    if (G.kind == GroupKind::Map) launch_map(g, ls, ptr, s);
    else if (G.kind == GroupKind::Stencil) launch_stencil(g, ls, ptr, s);
    else launch_batch(g, li, ls, ptr, s);
  }
}

void run_graph(GraphImpl& g, const void* const* inputs, void* const* outputs, cudaStream_t s) {
  ensure_device(g);
  auto& rt = *g.rt;
  std::vector<const void*> ptr = bind(g, inputs, outputs);
  auto it = g.options.find(DCP_OPT_USE_GRAPH);
  bool use_graph = it != g.options.end() && it->second == 1;
  if (!use_graph) {
    launch_all(g, ptr, s);
    return;
  }
  // CUDA-graph replay: the run is captured once per set of caller pointers.
  // A new pointer set is first run eagerly, which refreshes the batch tables
  // outside the capture, and then captured; later runs replay the graph.
  std::vector<const void*> key(ptr.begin(), ptr.end());
  if (!rt.gexec || key != rt.gkey) {
    if (rt.gexec) {
      cudaGraphExecDestroy(rt.gexec);
      rt.gexec = nullptr;
    }
    // run once eagerly so that any table upload happens outside the capture
    launch_all(g, ptr, s);
    cudaStream_t cs = nullptr;
    check_cuda(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate");
    cudaGraph_t graph = nullptr;
    check_cuda(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    try {
      launch_all(g, ptr, cs);
    } catch (...) {
      cudaStreamEndCapture(cs, &graph);
      if (graph) cudaGraphDestroy(graph);
      cudaStreamDestroy(cs);
      throw;
    }
    check_cuda(cudaStreamEndCapture(cs, &graph), "cudaStreamEndCapture");
    cudaError_t e = cudaGraphInstantiate(&rt.gexec, graph, 0);
    cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    check_cuda(e, "cudaGraphInstantiate");
    rt.gkey = key;
    return;  // this run already executed eagerly
  }
  check_cuda(cudaGraphLaunch(rt.gexec, s), "cudaGraphLaunch");
}

void run_graph_host(GraphImpl& g, const void* const* inputs, void* const* outputs,
                    cudaStream_t s) {
  ensure_device(g);
  auto& rt = *g.rt;
  if (rt.stage_in.empty() && !g.inputs.empty()) {
    for (int v : g.inputs)
      rt.stage_in.push_back(dalloc(rt, (size_t)g.nodes[v].numel() * dtype_size(g.nodes[v].dtype)));
  }
  if (rt.stage_out.empty()) {
    for (int v : g.outputs)
      rt.stage_out.push_back(dalloc(rt, (size_t)g.nodes[v].numel() * dtype_size(g.nodes[v].dtype)));
  }
  for (size_t i = 0; i < g.inputs.size(); ++i) {
    const Node& n = g.nodes[g.inputs[i]];
    size_t bytes = (size_t)n.numel() * dtype_size(n.dtype);
    if (bytes && !inputs[i]) fail(DCP_E_INVALID_ARG, "host input is NULL");
    if (bytes)
      check_cuda(cudaMemcpyAsync(rt.stage_in[i], inputs[i], bytes, cudaMemcpyHostToDevice, s),
                 "cudaMemcpyAsync(H2D)");
  }
  run_graph(g, (const void* const*)rt.stage_in.data(), rt.stage_out.data(), s);
  for (size_t j = 0; j < g.outputs.size(); ++j) {
    const Node& n = g.nodes[g.outputs[j]];
    size_t bytes = (size_t)n.numel() * dtype_size(n.dtype);
    if (bytes && !outputs[j]) fail(DCP_E_INVALID_ARG, "host output is NULL");
    if (bytes)
      check_cuda(cudaMemcpyAsync(outputs[j], rt.stage_out[j], bytes, cudaMemcpyDeviceToHost, s),
                 "cudaMemcpyAsync(D2H)");
  }
  check_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize");
}

void sync_graph(GraphImpl& g, cudaStream_t s) {
  (void)g;
  check_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  check_cuda(cudaGetLastError(), "asynchronous CUDA error");
}

// ---------------------------------------------------------------------------
// plan description (JSON)
// ---------------------------------------------------------------------------
std::string describe_plan(const GraphImpl& g) {
  std::ostringstream os;
  os << "{\"fused\": true, \"flags\": " << g.flags << ", \"n_launches\": " << g.n_launches
     << ", \"groups\": [";
  for (size_t gi = 0; gi < g.groups.size(); ++gi) {
    const Group& G = g.groups[gi];
    if (gi) os << ", ";
    const char* kind = G.kind == GroupKind::Map ? "map" : (G.kind == GroupKind::Stencil ? "stencil" : "batch");
    os << "{\"kind\": \"" << kind << "\", \"dtype\": \"" << dtype_name(G.dtype) << "\", \"shape\": [";
    for (size_t i = 0; i < G.shape.size(); ++i) os << (i ? ", " : "") << G.shape[i];
    os << "], \"members\": " << G.members.size() << ", \"post\": " << G.post.size()
       << ", \"loads\": " << G.loads.size() + G.post_loads.size() << ", \"scalars\": " << G.scalars.size()
       << ", \"stores\": " << G.stores.size() << ", \"reductions\": " << G.reds.size()
       << ", \"steps\": " << G.steps.size() << ", \"depth\": " << G.depth << ", \"tile\": ["
       << G.tile[0] << ", " << G.tile[1] << ", " << G.tile[2] << "]";
    if (G.kind == GroupKind::Batch) os << ", \"instances\": " << G.batch_members.size();
    int epi = 0;
    for (const StepDesc& s : G.steps) epi += (int)s.epi.size();
    os << ", \"epilogue_ops\": " << epi << "}";
  }
  os << "], \"launches\": [";
  if (g.rt) {
    for (size_t li = 0; li < g.rt->launches.size(); ++li) {
      const LaunchSpec& ls = g.rt->launches[li];
      os << (li ? ", " : "") << "{\"group\": " << ls.group << ", \"kernel\": \"" << ls.code.name
         << "\", \"steps\": [" << ls.s0 << ", " << ls.s1 << "], \"smem\": " << ls.code.smem_bytes
         << ", \"threads\": " << ls.code.threads << ", \"compile_ms\": " << ls.compile_ms
         << ", \"regs\": " << ls.regs << ", \"occupancy\": " << ls.occupancy << "}";
    }
  }
  os << "], \"transient_bytes\": ";
  int64_t tb = 0;
  std::vector<char> is_io(g.nodes.size(), 0);
  for (int v : g.inputs) is_io[v] = 1;
  for (int v : g.outputs) is_io[v] = 1;
  for (size_t v = 0; v < g.nodes.size(); ++v)
    if (g.materialized.size() > v && g.materialized[v] && !is_io[v])
      tb += g.nodes[v].numel() * dtype_size(g.nodes[v].dtype);
  os << tb << "}";
  return os.str();
}

void run_adjoint(GraphImpl& g, const void* const* inputs, const void* const* out_grads,
                 void* const* in_grads, size_t budget, cudaStream_t s) {
  ensure_device(g);
  if (!g.adj) g.adj = new_adjoint_state();
  run_adjoint_impl(g, *g.adj, inputs, out_grads, in_grads, budget, s);
}

}  // namespace dcp
