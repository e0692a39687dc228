// Execution of a fused plan: one launch per fused group (or per time-tile
// chunk of a stencil group), transients allocated once and reused (Sec. 3.1
// transient allocation mitigation: temporaries are persistent, allocated when
// the program is first run), per-group scratch for the tiled reductions
// (whole-array and axis), optional replay of the whole run as one captured
// CUDA graph, runs on host buffers (in place when page-locked), host-side
// fault injection for tests, and the autotuner that times candidate kernel
// forms, tile shapes and time-tile depths of every stencil group on the
// first run.
#include <algorithm>
#include <array>
#include <cinttypes>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
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
  int32_t seg, pad_;
  void* partials;
  void* ticket;
  void* guard;
};
// Cooperative stencil form: the stencil parameters plus the exchange
// arrays, the per-tile flags, the epoch counter and the error word.
struct CoopParamsH {
  StParamsH s;
  void* xb[2];
  void* flags;
  void* ctr;
  void* err;
};
struct AxParamsH {
  const void* ld[kMaxIO];
  const void* sc[kMaxIO];
  void* out[kMaxIO];
  void* partials;
  void* tickets;
  int64_t outer, R, inner;
  int64_t rchunk;
  int64_t ntiles;
  int32_t TO, TI, TR, S;
};
static_assert(sizeof(AxParamsH) == 3 * kMaxIO * 8 + 16 + 40 + 16, "axis params layout");
struct InstH {
  const void* in;
  void* out;
  int32_t ny, nx, tiles_x, tile0;
};
struct BatchParamsH {
  const void* inst;
  int32_t ninst;
  int32_t total_tiles;
  int32_t seg;
  int32_t pad_;
  void* guard;
};
static_assert(sizeof(StParamsH) == 5 * kMaxIO * 8 + 32 + 24, "stencil params layout");
static_assert(sizeof(CoopParamsH) == sizeof(StParamsH) + 5 * 8, "cooperative params layout");
static_assert(sizeof(BatchParamsH) == 32, "batch params layout");
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

// Batch instance table of one launch (chunk) of a batch group.
struct Table {
  InstH* host = nullptr;  // pinned
  void* dev = nullptr;
  int tiles = 0;
  std::vector<const void*> key;
};

struct GroupRT {
  void* state[2] = {nullptr, nullptr};  // time-tile ping-pong (stencil) / slabs (batch)
  void* partials = nullptr;
  int partial_slots = 0;
  unsigned* ticket = nullptr;
  unsigned* tickets = nullptr;   // axis reductions: one per block tile
  int64_t ntickets = 0;
  std::vector<int64_t> offsets;  // batch: element offset of each member in a slab
  std::map<int, Table> tables;   // batch: per chunk
  // magnitude guard of a deferred run: the largest finite |input| bit pattern
  // its first launch saw, and the bound that keeps the run finite (0: none)
  unsigned long long* guard = nullptr;
  double guard_bound = 0.0;
  // cooperative form: per-tile flags, [epoch, CTAs finished], error word
  unsigned* coop_flags = nullptr;
  int64_t coop_ntiles = 0;
  unsigned* coop_ctr = nullptr;
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

int group_nd(const Group& G) { return G.kind == GroupKind::Batch ? 2 : (int)G.shape.size(); }

}  // namespace

struct GraphImpl::Runtime {
  std::vector<LaunchSpec> launches;  // grouped by group, in execution order
  bool device_ready = false;
  bool tuned = false;
  int device = -1;
  int sms = 0;
  std::vector<void*> allocs;
  std::vector<InstH*> pinned;
  std::vector<void*> transient;  // per value id
  std::vector<GroupRT> grt;      // per group
  cudaEvent_t table_ev = nullptr;
  bool table_ev_used = false;
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
      for (InstH* h : pinned) cudaFreeHost(h);
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
static std::vector<LaunchSpec> build_group_launches(GraphImpl& g, int gi) {
  std::vector<LaunchSpec> L;
  const Group& G = g.groups[gi];
  if (G.kind == GroupKind::AxisReduce) {
    LaunchSpec ls;
    ls.group = gi;
    ls.code = gen_axis_kernel(g, G, true);
    ls.code_scalar = gen_axis_kernel(g, G, false);
    nvrtc_compile(ls.code.source, ls.code.name, &ls.compile_ms, nullptr);
    L.push_back(std::move(ls));
    return L;
  }
  if (G.kind == GroupKind::AdjTile) {
    LaunchSpec ls;
    ls.group = gi;
    ls.s1 = G.depth;
    ls.code = gen_adj_kernel(g, G);
    if (ls.code.smem_bytes > 227 * 1024)
      fail(DCP_E_UNSUPPORTED, "reverse stencil tile needs " + std::to_string(ls.code.smem_bytes) +
                                  " bytes of shared memory; lower the tile or the reverse depth");
    nvrtc_compile(ls.code.source, ls.code.name, &ls.compile_ms, nullptr);
    L.push_back(std::move(ls));
    return L;
  }
  if (G.kind == GroupKind::Map) {
    LaunchSpec ls;
    ls.group = gi;
    ls.code = gen_map_kernel(g, G, true);
    ls.code_scalar = gen_map_kernel(g, G, false);
    nvrtc_compile(ls.code.source, ls.code.name, &ls.compile_ms, nullptr);
    L.push_back(std::move(ls));
    return L;
  }
  const int S = (int)G.steps.size();
  for (int s0 = 0; s0 < S; s0 += G.depth) {
    LaunchSpec ls;
    ls.group = gi;
    ls.s0 = s0;
    ls.s1 = std::min(S, s0 + G.depth);
    ls.code = gen_stencil_kernel(g, G, ls.s0, ls.s1);
    if (ls.code.smem_bytes > 227 * 1024)
      fail(DCP_E_UNSUPPORTED, "stencil tile needs " + std::to_string(ls.code.smem_bytes) +
                                  " bytes of shared memory; lower the tile or depth");
    nvrtc_compile(ls.code.source, ls.code.name, &ls.compile_ms, nullptr);
    L.push_back(std::move(ls));
  }
  return L;
}

void compile_plan(GraphImpl& g) {
  g.rt.reset(new GraphImpl::Runtime());
  for (int gi = 0; gi < (int)g.groups.size(); ++gi) {
    std::vector<LaunchSpec> L = build_group_launches(g, gi);
    for (auto& ls : L) g.rt->launches.push_back(std::move(ls));
  }
  g.n_launches = (int)g.rt->launches.size();
}

// ---------------------------------------------------------------------------
// device state: modules, transients, scratch
// ---------------------------------------------------------------------------
// Host-side fault injection for tests (DCP_FAULT=alloc or DCP_FAULT=launch):
// the named operation fails with the status a real failure returns, before
// any device work, so the error paths run without faulting a GPU.
static void maybe_inject(const char* what, dcp_status code) {
  const char* f = std::getenv("DCP_FAULT");
  if (f && std::strcmp(f, what) == 0)
    fail(code, std::string("injected ") + what + " failure (DCP_FAULT)");
}

static void* dalloc(GraphImpl::Runtime& rt, size_t bytes) {
  maybe_inject("alloc", DCP_E_OOM);
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  check_cuda(cudaMalloc(&p, bytes), "cudaMalloc");
  rt.allocs.push_back(p);
  return p;
}

static void load_launch(LaunchSpec& ls) {
  ls.fn = load_function(ls.code.source, ls.code.name, nullptr, &ls.regs);
  if (ls.code.smem_bytes > 48 * 1024)
    check_cu(drv().funcSetAttribute(ls.fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES,
                                    ls.code.smem_bytes),
             "cuFuncSetAttribute(max dynamic smem)");
  int occ = 0;
  check_cu(drv().occupancy(&occ, ls.fn, ls.code.threads, ls.code.smem_bytes), "occupancy query");
  if (occ < 1) fail(DCP_E_UNSUPPORTED, "kernel " + ls.code.name + " cannot be resident on an SM");
  ls.occupancy = occ;
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
    for (auto& ls : rt.launches) load_launch(ls);
    for (int v = 0; v < N; ++v)
      if (g.materialized[v] && !is_io[v])
        rt.transient[v] = dalloc(rt, (size_t)g.nodes[v].numel() * dtype_size(g.nodes[v].dtype));
    const int NG = (int)g.groups.size();
    rt.grt.assign(NG, GroupRT());
    for (int gi = 0; gi < NG; ++gi) {
      const Group& G = g.groups[gi];
      GroupRT& R = rt.grt[gi];
      if (G.kind == GroupKind::Batch) {
        int64_t tot = 0;
        for (int m : G.batch_members) {
          R.offsets.push_back(tot);
          tot += (numel(g.batch_store[m].shape) + 31) / 32 * 32;  // 128-byte aligned slices
        }
      }
      if (!G.reds.empty()) {
        R.ticket = (unsigned*)dalloc(rt, 256);
        check_cuda(cudaMemset(R.ticket, 0, 256), "cudaMemset(ticket)");
      }
      if (G.kind == GroupKind::Stencil || G.kind == GroupKind::Batch) {
        R.guard = (unsigned long long*)dalloc(rt, 256);
        check_cuda(cudaMemset(R.guard, 0, 256), "cudaMemset(guard)");
      }
    }
    check_cuda(cudaEventCreateWithFlags(&rt.table_ev, cudaEventDisableTiming), "cudaEventCreate");
    check_cuda(cudaDeviceSynchronize(), "device set-up");
  } catch (...) {
    for (void* p : rt.allocs) cudaFree(p);
    rt.allocs.clear();
    throw;
  }
  rt.device_ready = true;
}

// Scratch that depends on the launch shape, allocated on first need.
static void* group_state(GraphImpl& g, int gi, int which) {
  auto& rt = *g.rt;
  GroupRT& R = rt.grt[gi];
  if (!R.state[which]) {
    const Group& G = g.groups[gi];
    size_t elems = 0;
    if (G.kind == GroupKind::Batch) {
      for (size_t k = 0; k < G.batch_members.size(); ++k)
        elems = std::max<size_t>(elems, (size_t)R.offsets[k] +
                                            (size_t)numel(g.batch_store[G.batch_members[k]].shape));
    } else {
      elems = (size_t)numel(G.shape);
    }
    R.state[which] = dalloc(rt, elems * dtype_size(G.dtype));
  }
  return R.state[which];
}

static void* group_partials(GraphImpl& g, int gi, int64_t slots) {
  auto& rt = *g.rt;
  GroupRT& R = rt.grt[gi];
  if (slots < 1) slots = 1;
  if (!R.partials || R.partial_slots < slots) {
    R.partials = dalloc(rt, (size_t)slots * g.groups[gi].reds.size() * 8);
    R.partial_slots = (int)slots;
  }
  return R.partials;
}

// Zeroed tickets of an axis-reduction group (cleared on the launch stream;
// every launch leaves them zero again).
static unsigned* group_tickets(GraphImpl& g, int gi, int64_t n, cudaStream_t s) {
  auto& rt = *g.rt;
  GroupRT& R = rt.grt[gi];
  if (n < 1) n = 1;
  if (!R.tickets || R.ntickets < n) {
    R.tickets = (unsigned*)dalloc(rt, (size_t)n * sizeof(unsigned));
    check_cuda(cudaMemsetAsync(R.tickets, 0, (size_t)n * sizeof(unsigned), s), "cudaMemsetAsync(tickets)");
    R.ntickets = n;
  }
  return R.tickets;
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------
static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static int64_t pow2ceil(int64_t v) {
  int64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Axis reduction: the (outer, R, inner) view of the iteration space, a
// power-of-two thread layout along (outer, R, inner) that keeps consecutive
// threads on the contiguous axis, and an R split when the tiles alone would
// not fill the GPU.
static void launch_axis(GraphImpl& g, LaunchSpec& ls, const std::vector<const void*>& ptr,
                        cudaStream_t s) {
  auto& rt = *g.rt;
  const Group& G = g.groups[ls.group];
  AxParamsH p;
  std::memset(&p, 0, sizeof p);
  const size_t esz = dtype_size(G.dtype);
  bool vec = ls.code.vec > 1;
  for (size_t i = 0; i < G.loads.size(); ++i) {
    p.ld[i] = ptr[G.loads[i]];
    vec = vec && aligned16(p.ld[i]);
    if ((uintptr_t)p.ld[i] % esz) fail(DCP_E_INVALID_ARG, "buffer not aligned to its element size");
  }
  for (size_t i = 0; i < G.scalars.size(); ++i) p.sc[i] = ptr[G.scalars[i]];
  for (size_t i = 0; i < G.reds.size(); ++i) {
    p.out[i] = const_cast<void*>(ptr[G.reds[i]]);
    if ((uintptr_t)p.out[i] % esz) fail(DCP_E_INVALID_ARG, "buffer not aligned to its element size");
  }
  int64_t outer = 1, inner = 1;
  for (int d = 0; d < G.axis; ++d) outer *= G.shape[d];
  for (int d = G.axis + 1; d < (int)G.shape.size(); ++d) inner *= G.shape[d];
  const int64_t R = G.shape[G.axis];
  if (outer * inner == 0) return;
  CUfunction fn = ls.fn;
  int occ = ls.occupancy;
  if (!vec && ls.code.vec > 1) {
    if (!ls.fn_scalar) {
      ls.fn_scalar = load_function(ls.code_scalar.source, ls.code_scalar.name, nullptr, nullptr);
      check_cu(drv().occupancy(&ls.occ_scalar, ls.fn_scalar, ls.code_scalar.threads, 0),
               "occupancy query");
    }
    fn = ls.fn_scalar;
    occ = ls.occ_scalar;
  }
  const int64_t V = vec ? ls.code.vec : 1;
  const bool along_inner = ls.code.axmode == 0;
  const int threads = ls.code.threads;
  const int64_t target = (int64_t)rt.sms * std::max(1, occ);
  // threads along inner cover V adjacent indices each when vectors run along inner
  int64_t TI = along_inner ? std::min<int64_t>(pow2ceil((inner + V - 1) / V), threads) : 1;
  // rows of up to 4096 contiguous elements: at most a warp per row (shuffle
  // tree, several rows per CTA); otherwise as many threads as fit
  const int64_t trmax = (inner == 1 && R <= 4096) ? 32 : threads / TI;
  const int64_t rv = along_inner ? 1 : V;  // elements of R per thread and step
  int64_t TR = std::min<int64_t>(pow2ceil(std::max<int64_t>((R + rv - 1) / rv, 1)), trmax);
  auto tiles_of = [&](int64_t ti, int64_t tr) {
    const int64_t to = threads / (ti * tr);
    const int64_t span = ti * (along_inner ? V : 1);
    return (outer + to - 1) / to * ((inner + span - 1) / span);
  };
  // fewer than about four waves of tiles: move threads from inner to R (down
  // to a warp along inner, a 32*V-element contiguous span per load) while R
  // has work for them; fewer splits of R follow
  while (along_inner && TI > 32 && tiles_of(TI, TR) < 4 * target && R >= TR * 16) {
    TI >>= 1;
    TR <<= 1;
  }
  const int64_t TO = threads / (TI * TR);
  const int64_t ntiles = (inner + TI * (along_inner ? V : 1) - 1) / (TI * (along_inner ? V : 1));
  const int64_t base = (outer + TO - 1) / TO * ntiles;
  int64_t S = 1;
  if (base < target && R > TR * rv * 32)
    S = std::min<int64_t>({(target + base - 1) / base, (R + TR * rv * 32 - 1) / (TR * rv * 32), 65535});
  // splits start on a vector boundary of R
  int64_t rchunk = std::max<int64_t>(1, (R + S - 1) / S);
  rchunk = (rchunk + rv - 1) / rv * rv;
  S = std::max<int64_t>(1, (R + rchunk - 1) / rchunk);
  const int64_t grid = base;  // one CTA per tile (and per split of R)
  if (grid > 0x7fffffff) fail(DCP_E_SHAPE, "axis reduction grid too large");
  p.outer = outer;
  p.R = R;
  p.inner = inner;
  p.rchunk = S == 1 ? std::max<int64_t>(R, 1) : rchunk;
  p.ntiles = ntiles;
  p.TO = (int32_t)TO;
  p.TI = (int32_t)TI;
  p.TR = (int32_t)TR;
  p.S = (int32_t)S;
  if (S > 1) {
    p.partials = group_partials(g, ls.group, S * outer * inner);
    p.tickets = group_tickets(g, ls.group, base, s);
  }
  void* args[] = {&p};
  check_cu(drv().launchKernel(fn, (unsigned)grid, (unsigned)S, 1, threads, 1, 1, 0, (CUstream)s,
                              args, nullptr),
           "cuLaunchKernel(axis reduction)");
}

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
  if (!G.reds.empty()) {
    p.partials = group_partials(g, ls.group, blocks);
    p.ticket = rt.grt[ls.group].ticket;
  }
  void* args[] = {&p};
  check_cu(drv().launchKernel(fn, (unsigned)blocks, 1, 1, G.threads, 1, 1, 0, (CUstream)s, args,
                              nullptr),
           "cuLaunchKernel(map)");
}

// Guard word of a launch that checks its input (first launch of a deferred
// run): cleared on the launch stream (so a captured graph clears it too).
static void* arm_guard(GraphImpl& g, const LaunchSpec& ls, cudaStream_t s) {
  if (!(ls.code.guard_max_input > 0.0)) return nullptr;
  GroupRT& R = g.rt->grt[ls.group];
  R.guard_bound = ls.code.guard_max_input;
  check_cuda(cudaMemsetAsync(R.guard, 0, sizeof(unsigned long long), s), "cudaMemsetAsync(guard)");
  return R.guard;
}

static void launch_coop(GraphImpl& g, LaunchSpec& ls, const StParamsH& sp, int64_t tiles,
                        cudaStream_t s);

static void launch_stencil(GraphImpl& g, LaunchSpec& ls, const std::vector<const void*>& ptr,
                           cudaStream_t s) {
  auto& rt = *g.rt;
  const Group& G = g.groups[ls.group];
  const int S = (int)G.steps.size();
  const bool first = ls.s0 == 0, last = ls.s1 == S;
  const int chunk = ls.s0 / G.depth;
  StParamsH p;
  std::memset(&p, 0, sizeof p);
  dims3(G.shape, p.nz, p.ny, p.nx);
  if ((int64_t)p.nz * p.ny * p.nx == 0) return;
  if (first) {
    if (!G.members.empty()) {
      for (size_t i = 0; i < G.loads.size(); ++i) p.ld[i] = ptr[G.loads[i]];
    } else {
      p.ld[0] = ptr[G.st_in];
    }
  } else {
    p.ld[0] = group_state(g, ls.group, (chunk - 1) % 2);
  }
  if (last) {
    for (size_t i = 0; i < G.stores.size(); ++i) p.st[i] = const_cast<void*>(ptr[G.stores[i]]);
    for (size_t i = 0; i < G.post_loads.size(); ++i) p.pld[i] = ptr[G.post_loads[i]];
    for (size_t i = 0; i < G.reds.size(); ++i) p.red_out[i] = const_cast<void*>(ptr[G.reds[i]]);
  } else {
    p.st[0] = group_state(g, ls.group, chunk % 2);
  }
  for (size_t i = 0; i < G.scalars.size(); ++i) p.sc[i] = ptr[G.scalars[i]];
  const int nd = (int)G.shape.size();
  int64_t gx;
  if (G.variant == 1) {
    // warp stream: one warp per (strip, row segment) work item, warps stride
    const int W = stream_width(G);
    int64_t items = (int64_t)((p.nx + W - 1) / W) * ((p.ny + G.seg - 1) / G.seg);
    const int wpb = ls.code.threads / 32;
    int64_t warps = std::min<int64_t>(items, (int64_t)rt.sms * ls.occupancy * wpb);
    gx = std::max<int64_t>(1, (warps + wpb - 1) / wpb);
    p.tiles_x = p.tiles_y = p.tiles_z = 1;
    p.seg = G.seg;
  } else {
    const int TX = G.tile[2], TY = nd == 1 ? 1 : G.tile[1];
    p.tiles_x = (p.nx + TX - 1) / TX;
    p.tiles_y = (p.ny + TY - 1) / TY;
    p.tiles_z = nd == 3 ? (p.nz + G.tile[0] - 1) / G.tile[0] : 1;
    gx = (int64_t)p.tiles_x * p.tiles_y;
  }
  if (gx > 0x7fffffff) fail(DCP_E_SHAPE, "grid too large");
  if (last && !G.reds.empty()) {
    p.partials = group_partials(g, ls.group, gx * p.tiles_z);
    p.ticket = rt.grt[ls.group].ticket;
  }
  p.guard = arm_guard(g, ls, s);
  if (G.variant == 2) {
    launch_coop(g, ls, p, gx, s);
    return;
  }
  void* args[] = {&p};
  check_cu(drv().launchKernel(ls.fn, (unsigned)gx, (unsigned)p.tiles_z, 1, ls.code.threads, 1, 1,
                              ls.code.smem_bytes, (CUstream)s, args, nullptr),
           "cuLaunchKernel(stencil)");
}

// Cooperative form: one launch runs every step; neighbouring tiles
// exchange their border rings through the group's two state arrays.
static void launch_coop(GraphImpl& g, LaunchSpec& ls, const StParamsH& sp, int64_t tiles,
                        cudaStream_t s) {
  auto& rt = *g.rt;
  GroupRT& R = rt.grt[ls.group];
  if (tiles > (int64_t)rt.sms * ls.occupancy)
    fail(DCP_E_UNSUPPORTED, "the cooperative stencil form needs every tile resident: " +
                                std::to_string(tiles) + " tiles, " +
                                std::to_string((int64_t)rt.sms * ls.occupancy) + " resident CTAs");
  if (!R.coop_ctr) {
    R.coop_ctr = (unsigned*)dalloc(rt, 256);  // [0] epoch, [1] finished CTAs, [2] error word
    check_cuda(cudaMemset(R.coop_ctr, 0, 256), "cudaMemset(coop counters)");
  }
  if (R.coop_ntiles < tiles) {
    // a new flag table starts from epoch 0 with every flag 0 (behind every
    // target), both reset in stream order after the launches before it
    R.coop_flags = (unsigned*)dalloc(rt, (size_t)tiles * sizeof(unsigned));
    check_cuda(cudaMemsetAsync(R.coop_flags, 0, (size_t)tiles * sizeof(unsigned), s),
               "cudaMemsetAsync(flags)");
    check_cuda(cudaMemsetAsync(R.coop_ctr, 0, 2 * sizeof(unsigned), s), "cudaMemsetAsync(epoch)");
    R.coop_ntiles = tiles;
  }
  CoopParamsH p;
  std::memset(&p, 0, sizeof p);
  p.s = sp;
  p.xb[0] = group_state(g, ls.group, 0);
  p.xb[1] = group_state(g, ls.group, 1);
  p.flags = R.coop_flags;
  p.ctr = R.coop_ctr;
  p.err = R.coop_ctr + 2;
  void* args[] = {&p};
  check_cu(drv().launchCooperative(ls.fn, (unsigned)tiles, 1, 1, ls.code.threads, 1, 1,
                                   ls.code.smem_bytes, (CUstream)s, args),
           "cuLaunchCooperativeKernel(stencil)");
}

static void launch_batch(GraphImpl& g, LaunchSpec& ls, const std::vector<const void*>& ptr,
                         cudaStream_t s) {
  auto& rt = *g.rt;
  const Group& G = g.groups[ls.group];
  GroupRT& R = rt.grt[ls.group];
  const int S = (int)G.steps.size();
  const bool first = ls.s0 == 0, last = ls.s1 == S;
  const int chunk = ls.s0 / G.depth;
  const size_t esz = dtype_size(G.dtype);
  const int nm = (int)G.batch_members.size();
  // the table depends on the caller pointers and on the tile shape
  std::vector<const void*> key;
  key.push_back((const void*)(intptr_t)G.tile[1]);
  key.push_back((const void*)(intptr_t)G.tile[2]);
  key.push_back((const void*)(intptr_t)G.depth);
  key.push_back((const void*)(intptr_t)G.variant);
  key.push_back((const void*)(intptr_t)G.seg);
  for (int m : G.batch_members) {
    key.push_back(ptr[g.batch_store[m].st_in]);
    key.push_back(ptr[g.batch_store[m].st_out]);
  }
  Table& T = R.tables[chunk];
  if (!T.dev || T.key != key) {
    if (!T.host) {
      check_cuda(cudaMallocHost((void**)&T.host, sizeof(InstH) * nm), "cudaMallocHost");
      rt.pinned.push_back(T.host);
      T.dev = dalloc(rt, sizeof(InstH) * nm);
    } else if (rt.table_ev_used) {
      // the previous upload of this pinned table must have been consumed
      check_cuda(cudaEventSynchronize(rt.table_ev), "cudaEventSynchronize");
    }
    const void* in_slab = first ? nullptr : group_state(g, ls.group, (chunk - 1) % 2);
    void* out_slab = last ? nullptr : group_state(g, ls.group, chunk % 2);
    // members ordered by tile count, largest first, for load balance
    // work items of a member: tiles (tile kernel) or column strips (stream kernel)
    auto tiles_of = [&](int k) {
      const Group& M = g.batch_store[G.batch_members[k]];
      int64_t ny = M.shape[0], nx = M.shape[1];
      if (G.variant == 1)
        return ((nx + stream_width(G) - 1) / stream_width(G)) * ((ny + G.seg - 1) / G.seg);
      return ((nx + G.tile[2] - 1) / G.tile[2]) * ((ny + G.tile[1] - 1) / G.tile[1]);
    };
    std::vector<int> order(nm);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return tiles_of(a) > tiles_of(b); });
    int64_t t0 = 0;
    for (int j = 0; j < nm; ++j) {
      int k = order[j];
      const Group& M = g.batch_store[G.batch_members[k]];
      InstH& I = T.host[j];
      const size_t off = (size_t)R.offsets[k] * esz;
      I.in = first ? ptr[M.st_in] : (const char*)in_slab + off;
      I.out = last ? const_cast<void*>(ptr[M.st_out]) : (char*)out_slab + off;
      I.ny = (int32_t)M.shape[0];
      I.nx = (int32_t)M.shape[1];
      I.tiles_x = (int32_t)(G.variant == 1 ? (I.nx + stream_width(G) - 1) / stream_width(G)
                                           : (I.nx + G.tile[2] - 1) / G.tile[2]);
      I.tile0 = (int32_t)t0;
      t0 += tiles_of(k);
    }
    if (t0 > 0x7fffffff) fail(DCP_E_SHAPE, "batch has too many tiles");
    T.tiles = (int)t0;
    check_cuda(cudaMemcpyAsync(T.dev, T.host, sizeof(InstH) * nm, cudaMemcpyHostToDevice, s),
               "cudaMemcpyAsync(batch table)");
    check_cuda(cudaEventRecord(rt.table_ev, s), "cudaEventRecord");
    rt.table_ev_used = true;
    T.key = key;
  }
  BatchParamsH p{T.dev, nm, T.tiles, G.seg, 0, nullptr};
  if (p.total_tiles == 0) return;
  p.guard = arm_guard(g, ls, s);
  int64_t grid;
  if (G.variant == 1) {
    const int wpb = ls.code.threads / 32;
    grid = std::min<int64_t>((p.total_tiles + wpb - 1) / wpb, (int64_t)rt.sms * ls.occupancy);
  } else {
    grid = std::min<int64_t>(p.total_tiles, (int64_t)rt.sms * ls.occupancy);
  }
  void* args[] = {&p};
  check_cu(drv().launchKernel(ls.fn, (unsigned)grid, 1, 1, ls.code.threads, 1, 1,
                              ls.code.smem_bytes, (CUstream)s, args, nullptr),
           "cuLaunchKernel(batch)");
}

// Time-tiled reverse of a stencil chain chunk: one CTA per output tile.
static void launch_adj(GraphImpl& g, LaunchSpec& ls, const std::vector<const void*>& ptr,
                       cudaStream_t s) {
  const Group& G = g.groups[ls.group];
  StParamsH p;
  std::memset(&p, 0, sizeof p);
  dims3(G.shape, p.nz, p.ny, p.nx);
  if ((int64_t)p.nz * p.ny * p.nx == 0) return;
  p.ld[0] = ptr[G.loads[0]];
  p.ld[1] = ptr[G.loads[1]];
  p.st[0] = const_cast<void*>(ptr[G.st_out]);
  const int TX = G.tile[2], TY = G.shape.size() == 1 ? 1 : G.tile[1];
  p.tiles_x = (p.nx + TX - 1) / TX;
  p.tiles_y = (p.ny + TY - 1) / TY;
  p.tiles_z = 1;
  const int64_t gx = (int64_t)p.tiles_x * p.tiles_y;
  if (gx > 0x7fffffff) fail(DCP_E_SHAPE, "grid too large");
  void* args[] = {&p};
  check_cu(drv().launchKernel(ls.fn, (unsigned)gx, 1, 1, ls.code.threads, 1, 1,
                              ls.code.smem_bytes, (CUstream)s, args, nullptr),
           "cuLaunchKernel(reverse stencil)");
}

static void launch_one(GraphImpl& g, LaunchSpec& ls, const std::vector<const void*>& ptr,
                       cudaStream_t s) {
  maybe_inject("launch", DCP_E_CUDA);
  const Group& G = g.groups[ls.group];
  if (G.kind == GroupKind::Map) launch_map(g, ls, ptr, s);
  else if (G.kind == GroupKind::AxisReduce) launch_axis(g, ls, ptr, s);
  else if (G.kind == GroupKind::Stencil) launch_stencil(g, ls, ptr, s);
  else if (G.kind == GroupKind::AdjTile) launch_adj(g, ls, ptr, s);
  else launch_batch(g, ls, ptr, s);
}

static void launch_group(GraphImpl& g, int gi, const std::vector<const void*>& ptr,
                         cudaStream_t s) {
  for (auto& ls : g.rt->launches)
    if (ls.group == gi) launch_one(g, ls, ptr, s);
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
    if (!outputs[j] && (n.numel() > 0 || (n.kind == Kind::Reduce && n.axis < 0)))
      fail(DCP_E_INVALID_ARG, "output " + std::to_string(j) + " is NULL");
    ptr[g.outputs[j]] = outputs[j];
  }
  return ptr;
}

static void launch_all(GraphImpl& g, const std::vector<const void*>& ptr, cudaStream_t s) {
  for (auto& ls : g.rt->launches) launch_one(g, ls, ptr, s);
}

// ---------------------------------------------------------------------------
// Autotuner (DCP_AUTOTUNE).  On the first run every stencil / batch group is
// timed under candidate (depth, tile) choices on the caller's buffers, in
// execution order (so its inputs are already valid), and keeps the fastest.
// All candidates perform identical per-step arithmetic, so the tuning run's
// outputs are the program's outputs.  Choices are cached per group signature
// in memory and, if DCP_TUNE_CACHE names a file, on disk.
// ---------------------------------------------------------------------------
namespace {
// A tuned configuration: depth, tz, ty, tx, and for 3-D stencils the cells
// per thread along x, for 2-D tile kernels the threads per CTA (32 or more;
// smaller values mean the default 256) (stream kernels: tz = -1, ty = rows
// per item, tx = prefetch depth).
typedef std::array<int, 5> TuneCfg;
std::mutex g_tune_mu;
std::map<std::string, TuneCfg> g_tune_cache;  // signature -> configuration
bool g_tune_loaded = false;

void tune_cache_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* f = std::getenv("DCP_TUNE_CACHE");
  if (!f || !*f) return;
  std::ifstream in(f);
  std::string line;
  while (std::getline(in, line)) {
    std::istringstream ls(line);
    std::string key;
    TuneCfg c = {1, 1, 1, 1, 1};
    if (!(ls >> key >> c[0] >> c[1] >> c[2] >> c[3])) continue;
    if (!(ls >> c[4])) c[4] = 1;  // entries without the fifth field
    g_tune_cache[key] = c;
  }
}

void tune_cache_store(const std::string& key, const TuneCfg& v) {
  g_tune_cache[key] = v;
  const char* f = std::getenv("DCP_TUNE_CACHE");
  if (!f || !*f) return;
  std::ofstream out(f, std::ios::app);
  out << key << " " << v[0] << " " << v[1] << " " << v[2] << " " << v[3] << " " << v[4] << "\n";
}

std::string group_signature(const GraphImpl& g, const Group& G, int device_sms) {
  std::ostringstream os;
  os << "sm" << device_sms << "|k" << (int)G.kind << "|t" << G.dtype << "|bc" << G.bc << "|s";
  if (G.kind == GroupKind::Batch) {
    int64_t cells = 0;
    for (int m : G.batch_members) cells += numel(g.batch_store[m].shape);
    os << "B" << G.batch_members.size() << "x" << cells;
  } else {
    for (auto v : G.shape) os << v << "x";
  }
  os << "|n" << G.steps.size() << "|o";
  for (auto o : G.offsets) os << o << ",";
  os << "|p" << G.members.size() << "," << G.post.size() << "," << G.reds.size();
  for (const StepDesc& s : G.steps) os << "," << s.epi.size();
  char h[32];
  std::snprintf(h, sizeof h, "%016" PRIx64, fnv1a(os.str()));
  return h;
}

std::vector<TuneCfg> tune_candidates(const Group& G, int sms) {
  std::vector<TuneCfg> c;
  const int S = (int)G.steps.size();
  const int nd = group_nd(G);
  if (nd == 3) {
    // one cell per thread (256-thread tiles) and paired cells along x
    const std::array<int, 3> tiles[] = {{32, 8, 32}, {64, 8, 32}, {16, 8, 32},
                                        {32, 4, 64}, {32, 16, 32}, {64, 4, 64}};
    for (const auto& t : tiles) c.push_back({1, t[0], t[1], t[2], 1});
    const std::array<int, 3> pair_tiles[] = {{16, 8, 32}, {32, 8, 32}, {16, 16, 32},
                                             {32, 16, 32}, {16, 8, 64}, {32, 4, 64}};
    if (G.radius[2] <= 2)
      for (const auto& t : pair_tiles) c.push_back({1, t[0], t[1], t[2], 2});
    return c;
  }
  std::vector<int> depths;
  for (int d : {1, 2, 3, 4, 5, 8, 10})
    if (d <= S) depths.push_back(d);
  std::vector<std::array<int, 2>> tiles;
  if (nd == 1) tiles = {{1, 256}, {1, 512}, {1, 1024}};
  else if (G.dtype == DCP_F32) tiles = {{32, 64}, {64, 64}, {16, 128}, {32, 128}, {64, 32}};
  else tiles = {{32, 32}, {16, 64}, {32, 64}, {64, 32}, {16, 32}, {16, 16}, {8, 32}};
  // small binary64 grids are bound by the FP64 pipes of the SMs they occupy:
  // tile shapes whose count is at most one or two per SM balance that work
  // (e.g. 152 tiles of 14 x 32 on a 256 x 256 grid)
  size_t balanced = 0;
  if (nd == 2 && G.kind != GroupKind::Batch && G.dtype == DCP_F64 && sms > 0) {
    const int64_t ny = G.shape[0], nx = G.shape[1];
    for (int per_sm : {1, 2})
      for (int tx : {16, 32, 64}) {
        const int64_t tiles_x = (nx + tx - 1) / tx;
        const int64_t rows = (int64_t)per_sm * sms / tiles_x;
        if (rows < 1) continue;
        const int64_t ty = (ny + rows - 1) / rows;
        if (ty >= 4 && ty <= 256 && tiles_x * ((ny + ty - 1) / ty) * 2 > (int64_t)per_sm * sms) {
          tiles.push_back({(int)ty, tx});
          ++balanced;
        }
      }
  }
  const size_t base_tiles = tiles.size() - balanced;
  for (int d : depths)
    for (size_t i = 0; i < tiles.size(); ++i) {
      const auto& t = tiles[i];
      int ry = nd == 1 ? 0 : G.radius[1], rx = G.radius[2];
      long smem = 2L * (t[0] + 2 * d * ry) * (t[1] + 2 * d * rx) * dtype_size(G.dtype);
      if (smem > 160 * 1024) continue;
      c.push_back({d, 1, t[0], t[1], 1});
      // the balanced tiles also with 512 and 1024 threads: one cell per
      // thread keeps hundreds of independent FP64 chains in flight per SM,
      // which a latency-bound small grid needs
      if (i >= base_tiles)
        for (int th : {512, 1024}) c.push_back({d, 1, t[0], t[1], th});
    }
  // (the cooperative form, tz slot = -2, is not a candidate: on the 256^2
  // f64 average its neighbour exchanges through L2 cost about 3.5 us per
  // step, nearly twice the time per step of two time-tiled launches)
  // warp-stream variant (tz slot = -1 marks it; ty slot = rows per work item,
  // 0 = planner's; tx slot = row windows requested ahead)
  for (int d : {1, 2, 3, 4, 5, 6, 8, 10})
    if (d <= S && stream_eligible(G, d))
      for (int pf : {1, 2}) {
        if (G.kind == GroupKind::Batch) {
          // last slot: CTAs per SM the register budget must allow (more
          // resident warps to hide the row loads' latency, fewer registers)
          for (int seg : {32, 64, 128}) c.push_back({d, -1, seg, pf, 1});
        } else {
          c.push_back({d, -1, 0, pf, 1});
          // small arrays: short row segments spread the strips over more warps
          const int64_t ny = G.shape.size() == 2 ? G.shape[0] : 1;
          if (ny <= 1024)
            for (int seg : {8, 16, 32})
              if (seg < ny) c.push_back({d, -1, seg, pf, 1});
        }
      }
  return c;
}

void apply_config(GraphImpl& g, int gi, const TuneCfg& cfg) {
  Group& G = g.groups[gi];
  G.depth = cfg[0];
  G.variant = cfg[1] == -1 ? 1 : (cfg[1] == -2 ? 2 : 0);
  G.tile[0] = cfg[1] < 0 ? 1 : cfg[1];
  G.tile[1] = cfg[2];
  G.tile[2] = cfg[3];
  G.cx = cfg[4] == 2 && G.tile[2] % 2 == 0 && G.radius[2] <= 2 ? 2 : 1;
  if (G.variant == 1) {
    auto th = g.options.find(DCP_OPT_STREAM_THREADS);
    G.threads = th == g.options.end() ? 64 : (int)th->second;
    G.prefetch = cfg[3] > 0 ? cfg[3] : 1;
    G.min_ctas = cfg[4] > 1 ? cfg[4] : 0;
    if (G.kind == GroupKind::Batch) {
      G.seg = cfg[2] > 0 ? cfg[2] : 64;
    } else {
      int64_t ny = G.shape.size() == 2 ? G.shape[0] : 1, nx = G.shape.back();
      int64_t strips = (nx + stream_width(G) - 1) / stream_width(G);
      int64_t seg = cfg[2] > 0 ? cfg[2]
                               : std::max<int64_t>((ny * strips + 2431) / 2432,
                                                   8 * G.depth * std::max(1, G.radius[1]));
      G.seg = (int)std::min<int64_t>(std::max<int64_t>(seg, 1), std::max<int64_t>(ny, 1));
    }
  } else {
    G.threads = group_nd(G) == 3 || cfg[4] < 32 ? 256 : cfg[4];
  }
  std::vector<LaunchSpec> L = build_group_launches(g, gi);
  for (auto& ls : L) load_launch(ls);
  if (G.variant == 2) {
    // every tile must be resident at once
    const int nd = group_nd(G);
    const int64_t ny = nd == 2 ? G.shape[0] : 1, nx = G.shape.back();
    const int64_t tiles = ((ny + G.tile[1] - 1) / G.tile[1]) * ((nx + G.tile[2] - 1) / G.tile[2]);
    if (tiles > (int64_t)g.rt->sms * L[0].occupancy)
      fail(DCP_E_UNSUPPORTED, "cooperative candidate does not fit the resident CTAs");
  }
  auto& all = g.rt->launches;
  std::vector<LaunchSpec> merged;
  bool placed = false;
  for (auto& ls : all) {
    if (ls.group == gi) {
      if (!placed) {
        for (auto& n : L) merged.push_back(std::move(n));
        placed = true;
      }
      continue;
    }
    merged.push_back(std::move(ls));
  }
  all = std::move(merged);
  g.rt->grt[gi].tables.clear();
}
}  // namespace

static void autotune(GraphImpl& g, const std::vector<const void*>& ptr, cudaStream_t s) {
  auto& rt = *g.rt;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_cache_load();
  cudaEvent_t e0, e1;
  check_cuda(cudaEventCreate(&e0), "cudaEventCreate");
  check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
  for (int gi = 0; gi < (int)g.groups.size(); ++gi) {
    const Group& G = g.groups[gi];
    // (a cooperative group runs as the option asked: it is not a candidate form)
    if (G.kind == GroupKind::Map || G.kind == GroupKind::AxisReduce ||
        G.kind == GroupKind::AdjTile || G.variant == 2) {
      launch_group(g, gi, ptr, s);
      continue;
    }
    std::string key = group_signature(g, G, rt.sms);
    auto hit = g_tune_cache.find(key);
    if (hit != g_tune_cache.end()) {
      apply_config(g, gi, hit->second);
      launch_group(g, gi, ptr, s);
      continue;
    }
    TuneCfg best = {G.depth, G.variant == 1 ? -1 : (G.variant == 2 ? -2 : G.tile[0]),
                    G.variant == 1 ? G.seg : G.tile[1], G.variant == 1 ? G.prefetch : G.tile[2],
                    G.variant == 2 ? G.threads : G.cx};
    float best_ms = 1e30f;
    for (const auto& cfg : tune_candidates(G, rt.sms)) {
      try {
        apply_config(g, gi, cfg);
      } catch (const Error&) {
        continue;  // a candidate that cannot be compiled or made resident is skipped
      }
      launch_group(g, gi, ptr, s);  // warm-up (and table upload)
      check_cuda(cudaEventRecord(e0, s), "cudaEventRecord");
      for (int r = 0; r < 3; ++r) launch_group(g, gi, ptr, s);
      check_cuda(cudaEventRecord(e1, s), "cudaEventRecord");
      check_cuda(cudaEventSynchronize(e1), "cudaEventSynchronize");
      float ms = 0.f;
      check_cuda(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
      if (ms < best_ms) {
        best_ms = ms;
        best = cfg;
      }
    }
    apply_config(g, gi, best);
    launch_group(g, gi, ptr, s);
    tune_cache_store(key, best);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g.n_launches = (int)rt.launches.size();
}

void run_graph(GraphImpl& g, const void* const* inputs, void* const* outputs, cudaStream_t s) {
  ensure_device(g);
  auto& rt = *g.rt;
  std::vector<const void*> ptr = bind(g, inputs, outputs);
  if ((g.flags & DCP_AUTOTUNE) && !rt.tuned) {
    autotune(g, ptr, s);
    rt.tuned = true;
    return;  // the tuning run computed this run's outputs
  }
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

// Device-visible address of a page-locked host buffer, or nullptr when the
// buffer is pageable (then it must be staged through device memory).
static void* mapped_address(const void* host) {
  if (!host) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of an unknown pointer
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return a.devicePointer;
}

// After the stream is idle: reports a deferred run whose input exceeded the
// magnitude its scaled state keeps finite (the guard word is then cleared).
static void check_guards(GraphImpl& g) {
  if (!g.rt || !g.rt->device_ready) return;
  auto& rt = *g.rt;
  for (size_t gi = 0; gi < rt.grt.size(); ++gi) {
    GroupRT& R = rt.grt[gi];
    if (R.coop_ctr) {
      unsigned err = 0;
      check_cuda(cudaMemcpy(&err, R.coop_ctr + 2, sizeof err, cudaMemcpyDeviceToHost),
                 "cudaMemcpy(coop error word)");
      if (err) {
        check_cuda(cudaMemset(R.coop_ctr + 2, 0, sizeof err), "cudaMemset(coop error word)");
        fail(DCP_E_TIMEOUT, "a cooperative stencil launch gave up waiting for a neighbouring tile; "
                            "its results are not valid");
      }
    }
    if (!R.guard || !(R.guard_bound > 0.0)) continue;
    unsigned long long bits = 0;
    check_cuda(cudaMemcpy(&bits, R.guard, sizeof bits, cudaMemcpyDeviceToHost), "cudaMemcpy(guard)");
    const bool f32 = g.groups[gi].dtype == DCP_F32;
    double seen;
    if (f32) {
      uint32_t b = (uint32_t)bits;
      float f;
      std::memcpy(&f, &b, 4);
      seen = f;
    } else {
      std::memcpy(&seen, &bits, 8);
    }
    if (seen > R.guard_bound) {
      check_cuda(cudaMemset(R.guard, 0, sizeof bits), "cudaMemset(guard)");
      char msg[320];
      std::snprintf(msg, sizeof msg,
                    "a stencil input of magnitude %.3g exceeds %.3g, the largest the deferred "
                    "common weight keeps finite for this stencil (its scaled state grows within a "
                    "chunk of steps); results may have overflowed: set DCP_OPT_DEFERRED_WEIGHT = 0 "
                    "before dcp_fuse for the plain weighted sum",
                    seen, R.guard_bound);
      fail(DCP_E_UNSUPPORTED, msg);
    }
  }
}

void run_graph_host(GraphImpl& g, const void* const* inputs, void* const* outputs,
                    cudaStream_t s) {
  ensure_device(g);
  auto& rt = *g.rt;
  // Zero-copy: when every host buffer is page-locked, the kernels read the
  // inputs and write the outputs in host memory directly (over the chip-to-
  // chip link on Grace systems), which avoids the staging copies.
  auto it = g.options.find(DCP_OPT_HOST_ACCESS);
  const bool allow_direct = it == g.options.end() || it->second != 0;
  if (allow_direct) {
    std::vector<const void*> din(g.inputs.size(), nullptr);
    std::vector<void*> dout(g.outputs.size(), nullptr);
    bool ok = true;
    for (size_t i = 0; i < g.inputs.size() && ok; ++i) {
      if (g.nodes[g.inputs[i]].numel() == 0) continue;
      din[i] = mapped_address(inputs[i]);
      ok = din[i] != nullptr;
    }
    for (size_t j = 0; j < g.outputs.size() && ok; ++j) {
      dout[j] = mapped_address(outputs[j]);
      ok = dout[j] != nullptr || g.nodes[g.outputs[j]].numel() == 0;
    }
    if (ok) {
      run_graph(g, din.data(), dout.data(), s);
      check_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize");
      check_guards(g);
      return;
    }
  }
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
  check_guards(g);
}

void sync_graph(GraphImpl& g, cudaStream_t s) {
  check_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  check_cuda(cudaGetLastError(), "asynchronous CUDA error");
  check_guards(g);
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
    const char* kind = G.kind == GroupKind::Map
                           ? "map"
                           : (G.kind == GroupKind::Stencil
                                  ? "stencil"
                                  : (G.kind == GroupKind::AxisReduce
                                         ? "axis_reduce"
                                         : (G.kind == GroupKind::AdjTile ? "reverse_tile"
                                                                         : "batch")));
    os << "{\"kind\": \"" << kind << "\", \"dtype\": \"" << dtype_name(G.dtype) << "\", \"shape\": [";
    for (size_t i = 0; i < G.shape.size(); ++i) os << (i ? ", " : "") << G.shape[i];
    os << "], \"members\": " << G.members.size() << ", \"post\": " << G.post.size()
       << ", \"loads\": " << G.loads.size() + G.post_loads.size() << ", \"scalars\": " << G.scalars.size()
       << ", \"stores\": " << G.stores.size() << ", \"reductions\": " << G.reds.size()
       << ", \"steps\": " << G.steps.size() << ", \"depth\": " << G.depth << ", \"tile\": ["
       << G.tile[0] << ", " << G.tile[1] << ", " << G.tile[2] << "]";
    if (G.kind == GroupKind::Batch) os << ", \"instances\": " << G.batch_members.size();
    if (G.kind == GroupKind::AxisReduce) os << ", \"axis\": " << G.axis;
    if (G.kind == GroupKind::Stencil && G.shape.size() == 3) os << ", \"cells_per_thread\": " << G.cx;
    if (G.kind != GroupKind::Map && G.kind != GroupKind::AxisReduce && G.kind != GroupKind::AdjTile)
      os << ", \"kernel_form\": \"" << (G.variant == 1 ? "stream" : (G.variant == 2 ? "coop" : "tile")) << "\", \"seg\": " << G.seg
         << ", \"prefetch\": " << G.prefetch << ", \"threads\": " << G.threads
         << ", \"min_ctas\": " << G.min_ctas;
    int epi = 0;
    for (const StepDesc& s : G.steps) epi += (int)s.epi.size();
    if (G.kind == GroupKind::AdjTile)
      for (const AdjStep& s : g.nodes[G.st_out].chain) epi += (int)s.epi.size();
    os << ", \"epilogue_ops\": " << epi << "}";
  }
  os << "], \"launches\": [";
  if (g.rt) {
    for (size_t li = 0; li < g.rt->launches.size(); ++li) {
      const LaunchSpec& ls = g.rt->launches[li];
      os << (li ? ", " : "") << "{\"group\": " << ls.group << ", \"kernel\": \"" << ls.code.name
         << "\", \"steps\": [" << ls.s0 << ", " << ls.s1 << "], \"smem\": " << ls.code.smem_bytes
         << ", \"threads\": " << ls.code.threads << ", \"compile_ms\": " << ls.compile_ms
         << ", \"regs\": " << ls.regs << ", \"occupancy\": " << ls.occupancy;
      if (!ls.code.defer_scales.empty()) {
        os << ", \"deferred_scales\": [";
        for (size_t i = 0; i < ls.code.defer_scales.size(); ++i) {
          char num[32];
          std::snprintf(num, sizeof num, "%.17g", ls.code.defer_scales[i]);
          os << (i ? ", " : "") << num;
        }
        os << "]";
      }
      os << "}";
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
  os << tb;
  if (g.adj)
    os << ", \"adjoint\": {\"tape_bytes\": " << adjoint_tape_bytes(*g.adj) << ", \"checkpointed\": "
       << (adjoint_chunked(*g.adj) ? "true" : "false")
       << ", \"launches\": " << adjoint_launches_json(*g.adj) << "}";
  os << "}";
  return os.str();
}

std::vector<std::string> launch_kernel_names(const GraphImpl& g) {
  std::vector<std::string> out;
  if (g.rt)
    for (const auto& ls : g.rt->launches) out.push_back(ls.code.name);
  return out;
}

void run_adjoint(GraphImpl& g, const void* const* inputs, const void* const* out_grads,
                 void* const* in_grads, size_t budget, cudaStream_t s) {
  ensure_device(g);
  if (!g.adj) g.adj = new_adjoint_state();
  run_adjoint_impl(g, *g.adj, inputs, out_grads, in_grads, budget, s);
}

void prepare_adjoint(GraphImpl& g, size_t budget) {
  if (!g.adj) g.adj = new_adjoint_state();
  prepare_adjoint_impl(g, *g.adj, budget);
}

}  // namespace dcp
