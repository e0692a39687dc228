// Code generation (Sec. 3.3: the GPU backend emits CUDA for every fused
// scope): each fused group becomes one hand-written skeleton from kernels/
// specialised with the group's expression DAG, stencil weights, tile shape
// and boundary rule.  The expression is emitted as straight-line code in
// registers; constants are emitted bit-exactly.
#include <cfloat>
#include <cinttypes>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <sstream>

#include "dcp_internal.h"

namespace dcp {

namespace {

// Variable names in generated code are numbered per kernel in order of first
// use, not by graph node id, so that structurally identical groups (e.g. the
// same program on many arrays) generate identical sources and share one
// compiled module.
thread_local std::map<int, int>* t_names = nullptr;

struct NameScope {
  std::map<int, int> names;
  std::map<int, int>* prev;
  NameScope() : prev(t_names) { t_names = &names; }
  ~NameScope() { t_names = prev; }
};

std::string var(int v) {
  if (!t_names) return "v" + std::to_string(v);
  auto it = t_names->find(v);
  int id;
  if (it == t_names->end()) {
    id = (int)t_names->size();
    (*t_names)[v] = id;
  } else {
    id = it->second;
  }
  return "v" + std::to_string(id);
}

std::string imm_literal(int dtype, double imm) {
  char buf[96];
  switch (dtype) {
    case DCP_F32: {
      float f = (float)imm;
      uint32_t b;
      std::memcpy(&b, &f, 4);
      std::snprintf(buf, sizeof buf, "__int_as_float(0x%08" PRIx32 ")", b);
      break;
    }
    case DCP_F64: {
      uint64_t b;
      std::memcpy(&b, &imm, 8);
      std::snprintf(buf, sizeof buf, "__longlong_as_double(0x%016" PRIx64 "ll)", b);
      break;
    }
    case DCP_I32: {
      int64_t i = (int64_t)imm;
      uint32_t b = (uint32_t)(uint64_t)i;
      std::snprintf(buf, sizeof buf, "((int)0x%08" PRIx32 "u)", b);
      break;
    }
    default: {
      int64_t i = (int64_t)imm;
      std::snprintf(buf, sizeof buf, "((long long)0x%016" PRIx64 "ull)", (uint64_t)i);
      break;
    }
  }
  return buf;
}

// Weight literal in the group's dtype (stencils are floating).
std::string weight_literal(int dtype, double w) { return imm_literal(dtype, w); }

// C expression of map op `op` (dtype, immediate) applied to operand
// expressions.
std::string op_expr(int op, int dtype, double imm_v, const std::string& a, const std::string& b) {
  std::string imm = imm_literal(dtype, imm_v);
  switch (op) {
    case kOpBcast: return a;
    case kOpConst: return imm;
    case kOpSign: return "dcp_sign(" + a + ")";
    case kOpGt: return "dcp_gt(" + a + ", " + b + ")";
    case kOpLt: return "dcp_lt(" + a + ", " + b + ")";
    case DCP_NEG: return "dcp_neg(" + a + ")";
    case DCP_ABS: return "dcp_abs(" + a + ")";
    case DCP_EXP: return (dtype == DCP_F64 ? "dcp_exp64(" : "dcp_exp(") + a + ")";
    case DCP_SIN: return (dtype == DCP_F64 ? "dcp_sin64(" : "dcp_sin(") + a + ")";
    case DCP_COS: return (dtype == DCP_F64 ? "dcp_cos64(" : "dcp_cos(") + a + ")";
    case DCP_TANH: return "dcp_tanh(" + a + ")";
    case DCP_SQRT: return "dcp_sqrt(" + a + ")";
    case DCP_SQUARE: return "dcp_square(" + a + ")";
    case DCP_ADD: return "dcp_add(" + a + ", " + b + ")";
    case DCP_SUB: return "dcp_sub(" + a + ", " + b + ")";
    case DCP_MUL: return "dcp_mul(" + a + ", " + b + ")";
    case DCP_DIV: return "dcp_div(" + a + ", " + b + ")";
    case DCP_MAX: return "dcp_max(" + a + ", " + b + ")";
    case DCP_MIN: return "dcp_min(" + a + ", " + b + ")";
    case DCP_ADD_S: return "dcp_add(" + a + ", " + imm + ")";
    case DCP_MUL_S: return "dcp_mul(" + a + ", " + imm + ")";
    case DCP_SUB_S: return "dcp_sub(" + a + ", " + imm + ")";
    case DCP_RSUB_S: return "dcp_sub(" + imm + ", " + a + ")";
  }
  fail(DCP_E_INVALID_ARG, "codegen: unknown op");
}

// C expression of map node v applied to operand expressions.
std::string map_expr(const GraphImpl& g, int v, const std::string& a, const std::string& b) {
  const Node& n = g.nodes[v];
  if (n.kind == Kind::Stencil) return a;  // zero-step stencil: identity
  return op_expr(n.op, n.dtype, n.imm, a, b);
}

void emit_members(std::ostringstream& os, const GraphImpl& g, const std::vector<int>& members) {
  for (int v : members) {
    const Node& n = g.nodes[v];
    std::string a = n.in.empty() ? "" : var(n.in[0]);
    std::string b = n.in.size() > 1 ? var(n.in[1]) : "";
    os << "  const DCP_T " << var(v) << " = " << map_expr(g, v, a, b) << ";\n";
  }
}

std::string red_op_fn(const GraphImpl& g, const std::vector<int>& reds) {
  std::ostringstream os;
  os << "__device__ __forceinline__ constexpr int dcp_red_op(int r) { return ";
  for (size_t i = 0; i < reds.size(); ++i) os << "r == " << i << " ? " << g.nodes[reds[i]].op << " : ";
  os << "0; }\n";
  return os.str();
}

// A kernel's name hashes its generated prefix together with the
// hand-written skeletons it includes, so the name (and the compiled-module
// caches keyed by the source) changes exactly when one of them changes.
uint64_t skeleton_hash(const std::string& body) {
  std::string text = device_header_source();
  const std::pair<const char*, const char*> skel[] = {
      {"k_map.cuh", kernel_map_source()},
      {"k_stencil2d.cuh", kernel_stencil2d_source()},
      {"k_stencil3d.cuh", kernel_stencil3d_source()},
      {"k_stencil2d_stream.cuh", kernel_stream_source()},
      {"k_axis.cuh", kernel_axis_source()},
      {"k_math64.cuh", kernel_math64_source()},
      {"k_stencil_adj.cuh", kernel_adj_source()},
      {"k_stencil2d_coop.cuh", kernel_coop_source()}};
  for (const auto& k : skel)
    if (body.find(std::string("#include \"") + k.first + "\"") != std::string::npos) text += k.second;
  return fnv1a(text);
}

std::string finish(const std::string& prefix, const std::string& b) {
  // binary64 exp / sin / cos come from k_math64.cuh; it is included only by
  // kernels that call them, so other kernels' sources (and names) do not
  // depend on it
  std::string body = b;
  const std::string dev = "#include \"dcp_device.cuh\"\n";
  const size_t at = body.find(dev);
  if (at != std::string::npos && (body.find("dcp_exp64(") != std::string::npos ||
                                  body.find("dcp_sin64(") != std::string::npos ||
                                  body.find("dcp_cos64(") != std::string::npos))
    body.insert(at + dev.size(), "#include \"k_math64.cuh\"\n");
  char name[64];
  std::snprintf(name, sizeof name, "%s_%016" PRIx64, prefix.c_str(),
                fnv1a(body) ^ skeleton_hash(body));
  return std::string("#define DCP_KNAME ") + name + "\n" + body;
}

std::string kname_of(const std::string& src) {
  const char* p = std::strstr(src.c_str(), "#define DCP_KNAME ");
  std::string s(p + std::strlen("#define DCP_KNAME "));
  return s.substr(0, s.find('\n'));
}

}  // namespace

CodegenOut gen_map_kernel(const GraphImpl& g, const Group& G, bool vec_ok) {
  NameScope names;
  std::ostringstream os;
  const int T = G.dtype;
  int vec = vec_ok ? 16 / dtype_size(T) : 1;
  os << "// dcp fused map kernel: " << G.members.size() << " ops, " << G.loads.size() << " loads, "
     << G.stores.size() << " stores, " << G.reds.size() << " reductions\n";
  os << "#define DCP_T " << dtype_cname(T) << "\n";
  os << "#define DCP_VEC " << vec << "\n#define DCP_UNROLL " << (vec > 1 ? G.unroll : 1) << "\n";
  os << "#define DCP_NLOAD " << G.loads.size() << "\n#define DCP_NSTORE " << G.stores.size()
     << "\n#define DCP_NSCALAR " << G.scalars.size() << "\n#define DCP_NRED " << G.reds.size()
     << "\n#define DCP_THREADS " << G.threads << "\n";
  os << red_op_fn(g, G.reds);
  os << "#include \"dcp_device.cuh\"\n";
  os << "__device__ __forceinline__ void dcp_body(const DCP_T* ld, const DCP_T* sc, DCP_T* st, "
        "DCP_T* rv) {\n";
  for (size_t i = 0; i < G.loads.size(); ++i)
    os << "  const DCP_T " << var(G.loads[i]) << " = ld[" << i << "];\n";
  for (size_t i = 0; i < G.scalars.size(); ++i)
    os << "  const DCP_T " << var(G.scalars[i]) << " = sc[" << i << "];\n";
  emit_members(os, g, G.members);
  for (size_t i = 0; i < G.stores.size(); ++i) os << "  st[" << i << "] = " << var(G.stores[i]) << ";\n";
  for (size_t i = 0; i < G.reds.size(); ++i)
    os << "  rv[" << i << "] = " << var(g.nodes[G.reds[i]].in[0]) << ";\n";
  os << "  (void)ld; (void)sc; (void)st; (void)rv;\n}\n";
  os << "#include \"k_map.cuh\"\n";
  CodegenOut out;
  out.source = finish(vec > 1 ? "dcp_map_v" : "dcp_map_s", os.str());
  out.name = kname_of(out.source);
  out.threads = G.threads;
  out.smem_bytes = 0;
  return out;
}

// Axis reduction (k_axis.cuh): the reduced operands, with the fused
// prologue maps, at a flat index of the iteration space.
CodegenOut gen_axis_kernel(const GraphImpl& g, const Group& G, bool vec_ok) {
  NameScope names;
  std::ostringstream os;
  const int T = G.dtype;
  int64_t inner = 1;
  for (int d = G.axis + 1; d < (int)G.shape.size(); ++d) inner *= G.shape[d];
  const int64_t R = G.shape[G.axis];
  // 16-byte vectors along the contiguous axis when the shape allows it and
  // the reduction tree's shared memory stays within 32 KB
  const int axmode = inner > 1 ? 0 : 1;
  int vec = vec_ok ? 16 / dtype_size(T) : 1;
  if ((axmode == 0 ? inner : R) % vec != 0 || (int)G.reds.size() * vec > 16) vec = 1;
  os << "// dcp axis reduction kernel: " << G.members.size() << " prologue ops, " << G.loads.size()
     << " loads, " << G.reds.size() << " reductions along axis " << G.axis << "\n";
  os << "#define DCP_T " << dtype_cname(T) << "\n#define DCP_THREADS " << G.threads
     << "\n#define DCP_NRED " << G.reds.size() << "\n#define DCP_NLOAD " << G.loads.size()
     << "\n#define DCP_NSCALAR " << G.scalars.size() << "\n#define DCP_VEC " << vec
     << "\n#define DCP_AXMODE " << axmode << "\n";
  os << red_op_fn(g, G.reds);
  os << "#include \"dcp_device.cuh\"\n";
  os << "__device__ __forceinline__ void dcp_body(const DCP_T* ld, const DCP_T* sc, DCP_T* rv) {\n";
  for (size_t i = 0; i < G.loads.size(); ++i)
    os << "  const DCP_T " << var(G.loads[i]) << " = ld[" << i << "];\n";
  for (size_t i = 0; i < G.scalars.size(); ++i)
    os << "  const DCP_T " << var(G.scalars[i]) << " = sc[" << i << "];\n";
  emit_members(os, g, G.members);
  for (size_t i = 0; i < G.reds.size(); ++i)
    os << "  rv[" << i << "] = " << var(g.nodes[G.reds[i]].in[0]) << ";\n";
  os << "  (void)ld; (void)sc;\n}\n";
  os << "#include \"k_axis.cuh\"\n";
  CodegenOut out;
  out.source = finish("dcp_axis", os.str());
  out.name = kname_of(out.source);
  out.threads = G.threads;
  out.smem_bytes = 0;
  out.vec = vec;
  out.axmode = axmode;
  return out;
}

namespace {

// Functions shared by 2-D and 3-D stencil sources: input (prologue), post.
void emit_stencil_io(std::ostringstream& os, const GraphImpl& g, const Group& G, bool first,
                     bool last) {
  os << "__device__ __forceinline__ DCP_T dcp_input(const DcpStParamsT<DCP_T>& p, const DCP_T* sc, "
        "long long gi) {\n";
  if (first && !G.members.empty()) {
    for (size_t i = 0; i < G.loads.size(); ++i)
      os << "  const DCP_T " << var(G.loads[i]) << " = p.ld[" << i << "][gi];\n";
    for (size_t i = 0; i < G.scalars.size(); ++i)
      os << "  const DCP_T " << var(G.scalars[i]) << " = sc[" << i << "];\n";
    emit_members(os, g, G.members);
    os << "  (void)sc;\n  return " << var(G.st_in) << ";\n}\n";
  } else {
    os << "  (void)sc;\n  return p.ld[0][gi];\n}\n";
  }
  os << "__device__ __forceinline__ void dcp_post(const DcpStParamsT<DCP_T>& p, const DCP_T* sc, "
        "long long gi, DCP_T v, DCP_T* st, DCP_T* rv) {\n";
  if (last) {
    os << "  const DCP_T " << var(G.st_out) << " = v;\n";
    for (size_t i = 0; i < G.post_loads.size(); ++i)
      os << "  const DCP_T " << var(G.post_loads[i]) << " = p.pld[" << i << "][gi];\n";
    for (size_t i = 0; i < G.scalars.size(); ++i)
      os << "  const DCP_T " << var(G.scalars[i]) << " = sc[" << i << "];\n";
    emit_members(os, g, G.post);
    for (size_t i = 0; i < G.stores.size(); ++i)
      os << "  st[" << i << "] = " << var(G.stores[i]) << ";\n";
    for (size_t i = 0; i < G.reds.size(); ++i)
      os << "  rv[" << i << "] = " << var(g.nodes[G.reds[i]].in[0]) << ";\n";
  }
  os << "  (void)p; (void)sc; (void)gi; (void)v; (void)st; (void)rv;\n}\n";
}

// Deferred common weight of a linear run of binary64 stencil steps.  A step
// u' = sum_k w_k u[p + o_k] whose weights are all exact multiples
// w_k = f r_k of one weight f (r_k = 1 at f's own points) is computed as
// w' = sum_k r_k w[p + o_k] on the scaled state w = u / f^t, and f^m is
// applied once at the end of every chunk of m steps.  The sum then starts
// from a point of ratio 1 with no multiply, so a p-point step takes p - 1
// FP64 operations instead of p (6 instead of 7 for the 7-point heat
// stencil, where 0.4 = 4 * 0.1 exactly; 4 adds instead of 5 operations for
// the 5-point average).  Only binary64 steps, which the FP64 pipe bounds,
// take this form.  A run is the consecutive steps of a group with equal
// weights (one stencil node, or a fused chain of equal ones), no epilogue
// map before its last step, a zero or periodic boundary (a fixed ring would
// need its border rescaled every step) and at least two steps.  Chunks are
// at most D steps with (sum |r_k|)^D <= 2^32, so the scaled state stays
// within 2^32 of the unscaled state's bound; f^m is the product of m
// roundings of f, applied with one more rounding.  Each step's arithmetic
// depends only on its place in its run, so every kernel form, tile shape,
// time-tile depth and split into launches computes the same bits.
//
// binary32 steps keep the plain sum: the float32 stencils are bound by
// instruction issue and memory latency, not by their arithmetic, and the
// deferred form measured no faster on the batched workload (slower at some
// time-tile depths).
struct Defer {
  bool on = false;
  std::vector<int> order;     // point order: a ratio-1 point first
  std::vector<double> ratio;  // r_k = w_k / f, exact
  double scale = 1.0;         // multiply after this step (1.0: none)
  double max_input = 0.0;     // largest finite |input| the run keeps finite
};

bool defer_ratios(const std::vector<double>& w, std::vector<double>& ratio, double& f_out,
                  double& gsum) {
  const int P = (int)w.size();
  double f = 0.0;
  int best = 0;
  for (int k = 0; k < P; ++k) {  // f: the most frequent nonzero weight
    if (w[k] == 0.0) continue;
    int c = 0;
    for (int j = 0; j < P; ++j) c += w[j] == w[k];
    if (c > best) best = c, f = w[k];
  }
  if (f == 0.0 || !std::isfinite(f)) return false;
  ratio.assign(P, 0.0);
  gsum = 0.0;
  for (int k = 0; k < P; ++k) {
    const double r = w[k] / f;
    if (!std::isfinite(r) || std::fma(r, f, -w[k]) != 0.0) return false;  // exact
    ratio[k] = r;
    gsum += std::fabs(r);
  }
  f_out = f;
  return true;
}

}  // namespace

// Longest chunk (steps between two applications of f^m) of a deferred run of
// stencil node n's steps; 0 when its steps keep the plain weighted sum.
// Unbounded growth limits (sum |r_k| <= 1) give INT32_MAX.
int defer_chunk_steps(const Node& n) {
  if (n.dtype != DCP_F64 || (n.bc != DCP_BC_ZERO && n.bc != DCP_BC_PERIODIC)) return 0;
  std::vector<double> r;
  double f = 0.0, gsum = 0.0;
  if (!defer_ratios(n.weights, r, f, gsum)) return 0;
  if (gsum <= 1.0) return INT32_MAX;
  const int D = (int)std::floor(32.0 / std::log2(gsum));
  return D >= 2 ? D : 0;
}

namespace {

Defer plan_defer(const GraphImpl& g, const Group& G, int s) {
  Defer d;
  const Node& n = g.nodes[G.steps[s].node];
  if (n.dtype != DCP_F64 || (n.bc != DCP_BC_ZERO && n.bc != DCP_BC_PERIODIC)) return d;
  auto opt = g.options.find(DCP_OPT_DEFERRED_WEIGHT);
  if (opt != g.options.end() && opt->second == 0) return d;
  const int S = (int)G.steps.size();
  // steps of the group share their offsets; a run also needs the same
  // weights and boundary
  auto same = [&](int t) {
    const Node& m = g.nodes[G.steps[t].node];
    return m.bc == n.bc && m.weights == n.weights;
  };
  int a = s;
  while (a > 0 && same(a - 1) && G.steps[a - 1].epi.empty()) --a;
  int b = s + 1;
  while (b < S && same(b) && G.steps[b - 1].epi.empty()) ++b;
  const int L = b - a;
  if (L < 2) return d;
  std::vector<double> r;
  double f = 0.0, gsum = 0.0;
  if (!defer_ratios(n.weights, r, f, gsum)) return d;
  const int Dmax = defer_chunk_steps(n);
  if (Dmax == 0) return d;
  const int D = std::min(L, Dmax);
  if (D < 2) return d;
  auto power = [f](int m) {
    double F = 1.0;
    for (int t = 0; t < m; ++t) F *= f;
    return std::isnormal(F) ? F : 0.0;
  };
  if (power(D) == 0.0 || (L % D != 0 && power(L % D) == 0.0)) return d;
  const int i = s - a;
  const int m = (i + 1) % D == 0 ? D : (s == b - 1 ? (i + 1) % D : 0);
  d.on = true;
  d.ratio = r;
  for (int k = 0; k < (int)r.size(); ++k)
    if (r[k] == 1.0) {
      d.order.push_back(k);
      break;
    }
  for (int k = 0; k < (int)r.size(); ++k)
    if (k != d.order[0]) d.order.push_back(k);
  d.scale = m > 0 ? power(m) : 1.0;
  // the scaled state of a chunk of D steps is at most (sum |r_k|)^D times the
  // largest |input| (sum |r_k| <= 1: no growth)
  const double growth = gsum <= 1.0 ? 1.0 : std::pow(gsum, (double)D);
  d.max_input = DBL_MAX / growth;
  return d;
}

// Multipliers of the binary64 weighted sums, held in registers.  On GB300 a
// binary64 fused multiply-add whose multiplier is a register of its own
// issues at the FP64 pipe's full rate (2 per clock per SM), while an add, a
// multiply, or fused multiply-adds that all share one multiplier issue at
// 1.68 (the library's FP64 probe).  So the terms of a sum are fused
// multiply-adds by multipliers kept in distinct registers -- an add becomes
// x * 1 + acc, which rounds exactly like acc + x -- loaded at kernel start
// from a small table in device memory (values the compiler cannot fold
// back into immediates).  Up to kMax slots (registers); beyond that, terms
// reuse slots holding the same value.  binary32 sums keep immediates.
struct MulRegs {
  static constexpr int kMax = 8;
  bool on = false;
  std::vector<double> vals;
  int next = 0;
  std::string get(int T, double w) {
    if (!on) return weight_literal(T, w);
    auto same = [w](double v) { return std::memcmp(&v, &w, sizeof v) == 0; };
    if ((int)vals.size() < kMax) {
      vals.push_back(w);
      return "km[" + std::to_string(vals.size() - 1) + "]";
    }
    for (int t = 0; t < kMax; ++t) {
      const int i = (next + t) % kMax;
      if (same(vals[i])) {
        next = i + 1;
        return "km[" + std::to_string(i) + "]";
      }
    }
    return weight_literal(T, w);
  }
  // The table the kernel loads its multiplier registers from.
  std::string table() const {
    std::ostringstream os;
    const int n = vals.empty() ? 1 : (int)vals.size();
    os << "#define DCP_NK " << n << "\n__device__ double dcp_km[DCP_NK] = {";
    for (int i = 0; i < n; ++i) {
      char buf[48];
      std::snprintf(buf, sizeof buf, "%a", vals.empty() ? 1.0 : vals[i]);  // exact
      os << (i ? ", " : "") << buf;
    }
    os << "};\n";
    return os.str();
  }
};

// One term of a weighted sum into accumulator a (declared by the first).
// Deferred sums: the first point is copied, the others are fused
// multiply-adds (ratio 1: x * 1 + acc, the same rounding as acc + x).
void emit_term(std::ostringstream& os, int T, const std::string& a, const std::string& x, double w,
               bool first, bool deferred, MulRegs& km) {
  if (deferred) {
    if (first) os << "  DCP_T " << a << " = " << x << ";\n";
    else if (w == 1.0 && !km.on) os << "  " << a << " = dcp_add(" << a << ", " << x << ");\n";
    else if (w == 1.0)
      os << "  " << a << " = dcp_fma_rn(" << x << ", " << km.get(T, 1.0) << ", " << a << ");\n";
    else os << "  " << a << " = dcp_fma_rn(" << weight_literal(T, w) << ", " << x << ", " << a << ");\n";
    return;
  }
  if (first) os << "  DCP_T " << a << " = dcp_mul_rn(" << weight_literal(T, w) << ", " << x << ");\n";
  else os << "  " << a << " = dcp_fma_rn(" << km.get(T, w) << ", " << x << ", " << a << ");\n";
}

// Epilogue chain of one step as a function of the weighted sum.
std::string epi_body(const GraphImpl& g, const StepDesc& s) {
  std::ostringstream os;
  std::string cur = "v";
  int k = 0;
  for (int e : s.epi) {
    std::string nv = "e" + std::to_string(k++);
    os << "  const DCP_T " << nv << " = " << map_expr(g, e, cur, "") << ";\n";
    cur = nv;
  }
  os << "  return " << cur << ";\n";
  return os.str();
}

}  // namespace

// Warp-stream form (k_stencil2d_stream.cuh) of a 1-D / 2-D stencil launch.
static CodegenOut gen_stream_kernel(const GraphImpl& g, const Group& G, int s0, int s1) {
  NameScope names;
  const bool batch = G.kind == GroupKind::Batch;
  const int nd = batch ? 2 : (int)G.shape.size();
  const int T = G.dtype;
  const int nsteps = s1 - s0;
  const bool first = s0 == 0, last = s1 == (int)G.steps.size();
  const int C = stream_cols_per_lane(T);
  const int ry = nd == 1 ? 0 : G.radius[1], rx = G.radius[2];
  const int NR = 2 * ry + 1;
  const int RXA = rx > 0 ? rx : 1;
  std::ostringstream os;
  os << "// dcp warp-stream stencil kernel: " << nsteps << " steps per launch, bc " << G.bc << ", "
     << nd << "-D" << (batch ? ", batched" : "") << "\n";
  os << "#define DCP_T " << dtype_cname(T) << "\n#define DCP_C " << C << "\n";
  os << "#define DCP_THREADS " << G.threads << "\n#define DCP_BC " << G.bc << "\n";
  os << "#define DCP_LAST " << (last ? 1 : 0) << "\n#define DCP_BATCH " << (batch ? 1 : 0) << "\n";
  os << "#define DCP_NSTORE " << (last ? (int)G.stores.size() : 1) << "\n#define DCP_NRED "
     << (last ? (int)G.reds.size() : 0) << "\n#define DCP_NSCALAR " << G.scalars.size() << "\n";
  os << "#define DCP_RX " << rx << "\n#define DCP_RY " << ry << "\n#define DCP_NSTEPS " << nsteps
     << "\n#define DCP_PDM " << G.prefetch << "\n";
  const Defer guard = first ? plan_defer(g, G, 0) : Defer();
  os << "#define DCP_GUARD " << (guard.on ? 1 : 0) << "\n";
  if (G.min_ctas > 0) os << "#define DCP_MINB " << G.min_ctas << "\n";
  os << red_op_fn(g, last ? G.reds : std::vector<int>{});
  os << "#include \"dcp_device.cuh\"\n";
  if (!batch) emit_stencil_io(os, g, G, first, last);
  std::ostringstream decls;  // declarations that need the multiplier count
  decls << "template <int S> __device__ __forceinline__ void dcp_level(const DCP_T (&up)[" << NR
        << "][" << C << "], const DCP_T (&lf)[" << NR << "][" << RXA << "], const DCP_T (&rt)["
        << NR << "][" << RXA << "], DCP_T (&out)[" << C << "], const DCP_T (&km)[DCP_NK]);\n";
  os << "template <int S> __device__ __forceinline__ DCP_T dcp_epi(DCP_T v);\n";
  // which rows of each step read a neighbour column to the left / right
  // (only those rows are exchanged between lanes)
  std::vector<unsigned> lmask(nsteps, 0u), rmask(nsteps, 0u);
  for (int s = 0; s < nsteps; ++s) {
    const Node& sn = g.nodes[G.steps[s0 + s].node];
    for (int k = 0; k < sn.npts(); ++k) {
      const int row = ry + G.offsets[k * 3 + 1], dx = G.offsets[k * 3 + 2];
      if (dx < 0) lmask[s] |= 1u << row;
      if (dx > 0) rmask[s] |= 1u << row;
    }
  }
  auto mask_fn = [&](const char* name, const std::vector<unsigned>& m) {
    os << "__device__ __forceinline__ constexpr bool " << name << "(int s, int d) {\n"
       << "  constexpr unsigned m[" << nsteps << "] = {";
    for (int s = 0; s < nsteps; ++s) os << (s ? ", " : "") << m[s] << "u";
    os << "};\n  return (m[s] >> d) & 1u;\n}\n";
  };
  mask_fn("dcp_uses_lf", lmask);
  mask_fn("dcp_uses_rt", rmask);
  std::vector<double> scales;
  MulRegs km;
  km.on = T == DCP_F64;
  std::ostringstream sums;  // emitted after the multiplier table they use
  for (int s = 0; s < nsteps; ++s) {
    std::ostringstream& os = sums;
    const StepDesc& sd = G.steps[s0 + s];
    const Node& sn = g.nodes[sd.node];
    os << "template <> __device__ __forceinline__ void dcp_level<" << s << ">(const DCP_T (&up)[" << NR
       << "][" << C << "], const DCP_T (&lf)[" << NR << "][" << RXA << "], const DCP_T (&rt)[" << NR
       << "][" << RXA << "], DCP_T (&out)[" << C << "], const DCP_T (&km)[DCP_NK]) {\n";
    os << "  (void)lf; (void)rt; (void)km;\n";
    const Defer df = plan_defer(g, G, s0 + s);
    if (df.on) os << "  // deferred common weight: the ratios w_k / f\n";
    scales.push_back(df.on ? df.scale : 0.0);
    for (int c = 0; c < C; ++c) {
      const std::string a = "a" + std::to_string(c);
      for (int i = 0; i < sn.npts(); ++i) {
        const int k = df.on ? df.order[i] : i;
        int dy = G.offsets[k * 3 + 1], dx = G.offsets[k * 3 + 2];
        int cc = c + dx, row = ry + dy;
        std::string x;
        if (cc < 0) x = "lf[" + std::to_string(row) + "][" + std::to_string(rx + cc) + "]";
        else if (cc >= C) x = "rt[" + std::to_string(row) + "][" + std::to_string(cc - C) + "]";
        else x = "up[" + std::to_string(row) + "][" + std::to_string(cc) + "]";
        emit_term(os, T, a, x, df.on ? df.ratio[k] : sn.weights[k], i == 0, df.on, km);
      }
      if (df.scale != 1.0) os << "  " << a << " = dcp_mul_rn(" << weight_literal(T, df.scale) << ", " << a << ");\n";
      os << "  out[" << c << "] = " << a << ";\n";
    }
    os << "}\n";
    os << "template <> __device__ __forceinline__ DCP_T dcp_epi<" << s << ">(DCP_T v) {\n"
       << epi_body(g, sd) << "}\n";
  }
  os << km.table() << decls.str() << sums.str();
  os << "#include \"k_stencil2d_stream.cuh\"\n";
  CodegenOut out;
  out.threads = G.threads;
  out.smem_bytes = 0;
  for (double x : scales)
    if (x != 0.0) out.defer_scales = scales;
  out.guard_max_input = guard.on ? guard.max_input : 0.0;
  out.source = finish(batch ? "dcp_bstream" : "dcp_stream", os.str());
  out.name = kname_of(out.source);
  return out;
}

CodegenOut gen_stencil_kernel(const GraphImpl& g, const Group& G, int s0, int s1) {
  if (G.variant == 1) return gen_stream_kernel(g, G, s0, s1);
  NameScope names;
  const bool batch = G.kind == GroupKind::Batch;
  const int nd = batch ? 2 : (int)G.shape.size();
  const int T = G.dtype;
  const int nsteps = s1 - s0;
  const bool first = s0 == 0, last = s1 == (int)G.steps.size();
  std::ostringstream os;
  os << "// dcp stencil kernel: " << nsteps << " steps per launch, bc " << G.bc << ", " << nd
     << "-D" << (batch ? ", batched" : "") << "\n";
  // 3-D: paired cells along x when requested and the tile allows it; rows of
  // the plane are then stored from an even offset so every pair is aligned
  const int rz = G.radius[0], ry = G.radius[1], rx = G.radius[2];
  const int CX3 = nd == 3 && G.cx == 2 && G.tile[2] % 2 == 0 && rx <= 2 ? 2 : 1;
  const int threads = nd == 3 ? G.tile[2] * G.tile[1] / CX3 : G.threads;
  os << "#define DCP_T " << dtype_cname(T) << "\n";
  os << "#define DCP_THREADS " << threads << "\n#define DCP_BC " << G.bc << "\n";
  os << "#define DCP_LAST " << (last ? 1 : 0) << "\n#define DCP_BATCH " << (batch ? 1 : 0) << "\n";
  int nstore = last ? (int)G.stores.size() : 1;
  int nred = last ? (int)G.reds.size() : 0;
  os << "#define DCP_NSTORE " << nstore << "\n#define DCP_NRED " << nred << "\n#define DCP_NSCALAR "
     << G.scalars.size() << "\n";
  const Defer guard = first ? plan_defer(g, G, 0) : Defer();
  os << "#define DCP_GUARD " << (guard.on ? 1 : 0) << "\n";
  os << red_op_fn(g, last ? G.reds : std::vector<int>{});
  os << "#include \"dcp_device.cuh\"\n";
  CodegenOut out;
  out.threads = threads;
  out.guard_max_input = guard.on ? guard.max_input : 0.0;
  // cooperative form: every step in one launch, a halo of one radius
  const bool coop = G.variant == 2 && nd <= 2 && !batch;
  if (coop && (!first || !last))
    fail(DCP_E_UNSUPPORTED, "the cooperative stencil form runs every step in one launch");
  if (nd <= 2) {
    const int TX = G.tile[2], TY = nd == 1 ? 1 : G.tile[1];
    const int RY = nd == 1 ? 0 : ry;
    const int hs = coop ? 1 : nsteps;  // halo width in radii
    const int PW = TX + 2 * hs * rx, PH = TY + 2 * hs * RY;
    os << "#define DCP_TX " << TX << "\n#define DCP_TY " << TY << "\n#define DCP_RX " << rx
       << "\n#define DCP_RY " << RY << "\n#define DCP_NSTEPS " << nsteps << "\n";
    if (!batch) emit_stencil_io(os, g, G, first, last);
    os << "template <int S> __device__ __forceinline__ DCP_T dcp_epi(DCP_T v);\n";
    std::vector<double> scales;
    MulRegs km;
    km.on = T == DCP_F64;
    std::ostringstream sums;  // emitted after the multiplier table they use
    for (int s = 0; s < nsteps; ++s) {
      std::ostringstream& os = sums;
      const StepDesc& sd = G.steps[s0 + s];
      const Node& sn = g.nodes[sd.node];
      os << "template <> __device__ __forceinline__ DCP_T dcp_sum<" << s
         << ">(const DCP_T* A, int c, const DCP_T (&km)[DCP_NK]) {\n  (void)km;\n";
      const Defer df = plan_defer(g, G, s0 + s);
      if (df.on) os << "  // deferred common weight: the ratios w_k / f\n";
      scales.push_back(df.on ? df.scale : 0.0);
      for (int i = 0; i < sn.npts(); ++i) {
        const int k = df.on ? df.order[i] : i;
        int dy = G.offsets[k * 3 + 1], dx = G.offsets[k * 3 + 2];
        int off = dy * PW + dx;
        std::string x = "A[c + (" + std::to_string(off) + ")]";
        emit_term(os, T, "acc", x, df.on ? df.ratio[k] : sn.weights[k], i == 0, df.on, km);
      }
      if (df.scale != 1.0) os << "  acc = dcp_mul_rn(" << weight_literal(T, df.scale) << ", acc);\n";
      os << "  return acc;\n}\n";
      os << "template <> __device__ __forceinline__ DCP_T dcp_epi<" << s << ">(DCP_T v) {\n"
         << epi_body(g, sd) << "}\n";
    }
    os << km.table();
    os << "template <int S> __device__ __forceinline__ DCP_T dcp_sum(const DCP_T* A, int c, "
          "const DCP_T (&km)[DCP_NK]);\n";
    os << sums.str();
    if (coop) {
      // host-side fault injection (DCP_FAULT=coop_wait): every neighbour wait
      // gives up after 1000 polls, so the bounded-wait error path runs
      // without a fault or a hang
      const char* f = std::getenv("DCP_FAULT");
      if (f && std::strcmp(f, "coop_wait") == 0)
        os << "#define DCP_SPIN_LIMIT 1000\n#define DCP_WAIT_SKEW 4096u\n";
    }
    os << (coop ? "#include \"k_stencil2d_coop.cuh\"\n" : "#include \"k_stencil2d.cuh\"\n");
    out.smem_bytes = 2 * PW * PH * dtype_size(T);
    for (double x : scales)
      if (x != 0.0) out.defer_scales = scales;
  } else {
    if (nsteps != 1) fail(DCP_E_UNSUPPORTED, "3-D stencil launches run one step each");
    const int TX = G.tile[2], TY = G.tile[1], TZ = G.tile[0];
    const int CX = CX3;
    const int AX = CX == 2 ? (rx + 1) / 2 * 2 : rx;
    const int PW = TX + 2 * AX, PH = TY + 2 * ry;
    os << "#define DCP_TX " << TX << "\n#define DCP_TY " << TY << "\n#define DCP_TZ " << TZ
       << "\n#define DCP_RX " << rx << "\n#define DCP_RY " << ry << "\n#define DCP_RZ " << rz
       << "\n#define DCP_CX " << CX << "\n#define DCP_AX " << AX << "\n";
    emit_stencil_io(os, g, G, first, last);
    const StepDesc& sd = G.steps[s0];
    const Node& sn = g.nodes[sd.node];
    MulRegs km;
    km.on = T == DCP_F64;
    std::ostringstream sums;  // emitted after the multiplier table it uses
    sums << "__device__ __forceinline__ void dcp_sum3(const DCP_T* const* pl, int c, DCP_T (&v)["
         << CX << "], const DCP_T (&km)[DCP_NK]) {\n  (void)km;\n";
    const Defer df = plan_defer(g, G, s0);
    std::vector<int> order(sn.npts());
    for (int k = 0; k < sn.npts(); ++k) order[k] = df.on ? df.order[k] : k;
    auto wt = [&](int k) { return df.on ? df.ratio[k] : sn.weights[k]; };
    if (df.on) sums << "  // deferred common weight: the ratios w_k / f\n";
    if (df.on) out.defer_scales = {df.scale};
    if (CX == 1) {
      for (int i = 0; i < sn.npts(); ++i) {
        const int k = order[i];
        int dz = G.offsets[k * 3], dy = G.offsets[k * 3 + 1], dx = G.offsets[k * 3 + 2];
        std::string x = "pl[" + std::to_string(dz + rz) + "][c + (" + std::to_string(dy * PW + dx) + ")]";
        emit_term(sums, T, "acc", x, wt(k), i == 0, df.on, km);
      }
      if (df.scale != 1.0) sums << "  acc = dcp_mul_rn(" << weight_literal(T, df.scale) << ", acc);\n";
      sums << "  v[0] = acc;\n";
    } else {
      // one aligned pair load per distinct (plane, pair index) the two cells read
      auto floor_div2 = [](int o) { return o >= 0 ? o / 2 : -((-o + 1) / 2); };
      std::map<std::pair<int, int>, std::string> pairs;
      sums << "  typedef typename DcpVec2<DCP_T>::type T2;\n";
      for (int k = 0; k < sn.npts(); ++k)
        for (int j = 0; j < 2; ++j) {
          int dz = G.offsets[k * 3], dy = G.offsets[k * 3 + 1], dx = G.offsets[k * 3 + 2];
          int q = floor_div2(dy * PW + dx + j);
          auto key = std::make_pair(dz + rz, q);
          if (pairs.count(key)) continue;
          std::string nm = "p" + std::to_string(pairs.size());
          pairs[key] = nm;
          sums << "  const T2 " << nm << " = *reinterpret_cast<const T2*>(pl[" << key.first
               << "] + c + (" << 2 * q << "));\n";
        }
      for (int j = 0; j < 2; ++j) {
        std::string a = "a" + std::to_string(j);
        for (int i = 0; i < sn.npts(); ++i) {
          const int k = order[i];
          int dz = G.offsets[k * 3], dy = G.offsets[k * 3 + 1], dx = G.offsets[k * 3 + 2];
          int o = dy * PW + dx + j, q = floor_div2(o);
          std::string x = pairs[std::make_pair(dz + rz, q)] + (o - 2 * q == 0 ? ".x" : ".y");
          emit_term(sums, T, a, x, wt(k), i == 0, df.on, km);
        }
        if (df.scale != 1.0)
          sums << "  " << a << " = dcp_mul_rn(" << weight_literal(T, df.scale) << ", " << a << ");\n";
        sums << "  v[" << j << "] = a" << j << ";\n";
      }
    }
    sums << "}\n";
    os << km.table() << sums.str();
    os << "__device__ __forceinline__ DCP_T dcp_epi3(DCP_T v) {\n" << epi_body(g, sd) << "}\n";
    os << "#include \"k_stencil3d.cuh\"\n";
    out.smem_bytes = (2 * rz + 2) * PW * PH * dtype_size(T);
  }
  out.source = finish(batch ? "dcp_batch" : (nd == 3 ? "dcp_st3d" : (coop ? "dcp_coop" : "dcp_st2d")),
                      os.str());
  out.name = kname_of(out.source);
  return out;
}

CodegenOut gen_batch_kernel(const GraphImpl& g, const Group& G, int s0, int s1) {
  return gen_stencil_kernel(g, G, s0, s1);
}


// ---------------------------------------------------------------------------
// Time-tiled reverse pass of a 1-D / 2-D stencil chain (k_stencil_adj.cuh).
// ---------------------------------------------------------------------------
namespace {

// Which forward value the reverse rule of a unary / immediate op reads:
// 1 its operand X, 2 its result Y, 0 neither.  The rules are those of the
// adjoint's per-op reverse maps, so the fused reverse rounds alike.
int vjp_reads(int op) {
  switch (op) {
    case DCP_ABS: case DCP_SIN: case DCP_COS: case DCP_SQUARE: return 1;
    case DCP_EXP: case DCP_TANH: case DCP_SQRT: return 2;
    case DCP_NEG: case DCP_ADD_S: case DCP_SUB_S: case DCP_MUL_S: case DCP_RSUB_S: return 0;
  }
  fail(DCP_E_UNSUPPORTED, std::string("adjoint: no reverse rule for epilogue op ") + op_name(op));
}

// Cotangent of the operand of op from the cotangent a of its result (the
// same expressions as the per-op reverse maps of the adjoint builder).
std::string vjp_expr(int op, double imm, int T, const std::string& a, const std::string& X,
                     const std::string& Y) {
  switch (op) {
    case DCP_NEG: return op_expr(DCP_NEG, T, 0, a, "");
    case DCP_ABS: return op_expr(DCP_MUL, T, 0, op_expr(kOpSign, T, 0, X, ""), a);
    case DCP_EXP: return op_expr(DCP_MUL, T, 0, Y, a);
    case DCP_SIN: return op_expr(DCP_MUL, T, 0, op_expr(DCP_COS, T, 0, X, ""), a);
    case DCP_COS:
      return op_expr(DCP_MUL, T, 0, op_expr(DCP_NEG, T, 0, op_expr(DCP_SIN, T, 0, X, ""), ""), a);
    case DCP_TANH:
      return op_expr(DCP_MUL, T, 0,
                     op_expr(DCP_RSUB_S, T, 1.0, op_expr(DCP_SQUARE, T, 0, Y, ""), ""), a);
    case DCP_SQRT: return op_expr(DCP_DIV, T, 0, op_expr(DCP_MUL_S, T, 0.5, a, ""), Y);
    case DCP_SQUARE:
      return op_expr(DCP_MUL, T, 0, op_expr(DCP_MUL_S, T, 2.0, X, ""), a);
    case DCP_ADD_S: case DCP_SUB_S: return a;
    case DCP_MUL_S: return op_expr(DCP_MUL_S, T, imm, a, "");
    case DCP_RSUB_S: return op_expr(DCP_NEG, T, 0, a, "");
  }
  fail(DCP_E_UNSUPPORTED, std::string("adjoint: no reverse rule for epilogue op ") + op_name(op));
}

}  // namespace

bool adj_needs_z(const std::vector<std::pair<int, double>>& epi) {
  const int m = (int)epi.size();
  for (int j = 0; j < m; ++j) {
    const int r = vjp_reads(epi[j].first);
    if (r == 1) return true;               // the operand: z or an intermediate
    if (r == 2 && j + 1 < m) return true;  // an intermediate result
  }
  return false;
}

CodegenOut gen_adj_kernel(const GraphImpl& g, const Group& G) {
  NameScope names;
  const Node& n = g.nodes[G.st_out];
  const int T = G.dtype;
  const int K = (int)n.chain.size();
  const int nd = (int)G.shape.size();
  const int ry = nd == 1 ? 0 : G.radius[1], rx = G.radius[2];
  const int TX = G.tile[2], TY = nd == 1 ? 1 : G.tile[1];
  const int PW = TX + 4 * K * rx, PH = TY + 4 * K * ry;
  bool needz = false;
  for (const AdjStep& st : n.chain) needz = needz || adj_needs_z(st.epi);
  std::ostringstream os;
  os << "// dcp time-tiled reverse stencil kernel: " << K << " steps per launch, bc " << G.bc << ", "
     << nd << "-D\n";
  os << "#define DCP_T " << dtype_cname(T) << "\n#define DCP_THREADS " << G.threads
     << "\n#define DCP_BC " << G.bc << "\n#define DCP_TX " << TX << "\n#define DCP_TY " << TY
     << "\n#define DCP_RX " << rx << "\n#define DCP_RY " << ry << "\n#define DCP_K " << K
     << "\n#define DCP_NEEDZ " << (needz ? 1 : 0) << "\n";
  os << "#include \"dcp_device.cuh\"\n";
  MulRegs km;
  km.on = T == DCP_F64;
  std::ostringstream fn;  // emitted after the multiplier table they use
  for (int s = 0; s < K; ++s) {
    const AdjStep& st = n.chain[s];
    const int P = (int)st.weights.size();
    for (int dir = 0; dir < 2; ++dir) {  // 0: forward sum, 1: transposed sum
      fn << "template <> __device__ __forceinline__ DCP_T " << (dir ? "dcp_bsum<" : "dcp_fsum<") << s
         << ">(const DCP_T* A, int c, const DCP_T (&km)[DCP_NK]) {\n  (void)km;\n";
      for (int k = 0; k < P; ++k) {
        const int sg = dir ? -1 : 1;
        const int dy = sg * G.offsets[k * 3 + 1], dx = sg * G.offsets[k * 3 + 2];
        emit_term(fn, T, "acc", "A[c + (" + std::to_string(dy * PW + dx) + ")]", st.weights[k],
                  k == 0, false, km);
      }
      fn << "  return acc;\n}\n";
    }
    // forward epilogue
    fn << "template <> __device__ __forceinline__ DCP_T dcp_fepi<" << s << ">(DCP_T v) {\n";
    std::string cur = "v";
    for (size_t j = 0; j < st.epi.size(); ++j) {
      std::string nv = "e" + std::to_string(j);
      fn << "  const DCP_T " << nv << " = " << op_expr(st.epi[j].first, T, st.epi[j].second, cur, "")
         << ";\n";
      cur = nv;
    }
    fn << "  return " << cur << ";\n}\n";
    // reverse of the epilogue: intermediates recomputed from z when read
    fn << "template <> __device__ __forceinline__ DCP_T dcp_vjp<" << s
       << ">(DCP_T g, DCP_T z, DCP_T u) {\n  (void)z; (void)u;\n";
    const int m = (int)st.epi.size();
    std::vector<std::string> val(m + 1);  // val[0] = z, val[j] = result of op j-1
    val[0] = "z";
    const bool need = adj_needs_z(st.epi);
    for (int j = 0; j < m; ++j) {
      if (need && j + 1 < m) {
        val[j + 1] = "f" + std::to_string(j);
        fn << "  const DCP_T " << val[j + 1] << " = "
           << op_expr(st.epi[j].first, T, st.epi[j].second, val[j], "") << ";\n";
      }
    }
    if (m > 0) val[m] = "u";
    std::string a = "g";
    for (int j = m - 1; j >= 0; --j) {
      std::string nv = "a" + std::to_string(j);
      fn << "  const DCP_T " << nv << " = "
         << vjp_expr(st.epi[j].first, st.epi[j].second, T, a, val[j], val[j + 1]) << ";\n";
      a = nv;
    }
    fn << "  return " << a << ";\n}\n";
  }
  os << km.table();
  os << "template <int S> __device__ __forceinline__ DCP_T dcp_fsum(const DCP_T* A, int c, const "
        "DCP_T (&km)[DCP_NK]);\n"
     << "template <int S> __device__ __forceinline__ DCP_T dcp_bsum(const DCP_T* A, int c, const "
        "DCP_T (&km)[DCP_NK]);\n"
     << "template <int S> __device__ __forceinline__ DCP_T dcp_fepi(DCP_T v);\n"
     << "template <int S> __device__ __forceinline__ DCP_T dcp_vjp(DCP_T g, DCP_T z, DCP_T u);\n";
  os << fn.str();
  os << "#include \"k_stencil_adj.cuh\"\n";
  CodegenOut out;
  out.threads = G.threads;
  out.smem_bytes = (K + 1 + (needz ? K : 0)) * PW * PH * dtype_size(T);
  out.source = finish("dcp_adj", os.str());
  out.name = kname_of(out.source);
  return out;
}

}  // namespace dcp
