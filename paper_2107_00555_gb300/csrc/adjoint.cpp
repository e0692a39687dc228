// Reverse pass (adjoint) of a program.
//
// The reverse of a program is itself a dataflow program: each node's
// vector-Jacobian product is emitted as elementwise maps (and, for a stencil
// S, the transposed stencil S^T: the same weights at negated offsets), built
// as a new graph and fused and compiled by the same planner and kernel
// skeletons as any forward program.  For the iterated tanh-stencil chain,
// for example, every reverse step  g_t = S^T (g_{t+1} * (1 - u_{t+1}^2))
// becomes one time-step kernel whose prologue evaluates the map at every
// cell of its halo tile.
//
// Forward values the reverse pass needs are either recomputed inside the
// reverse kernels (pure elementwise functions of inputs) or read from a
// tape: values downstream of a stencil or a reduction in the same segment
// are stored by a forward run (the "tape").  When the tape fits the caller's
// budget the whole program is one segment.  Otherwise the program is cut
// into segments of ceil(sqrt(S)) stencil nodes; the forward run stores only
// the values live across segment boundaries (checkpoints), and each segment
// is recomputed from its checkpoint just before its reverse pass.
#include <algorithm>
#include <cmath>
#include <map>
#include <set>

#include <sstream>

#include "dcp_internal.h"

namespace dcp {

namespace {

// Buffer of a sub-graph input/output as seen by the driver.
enum class BK { Fwd, Cot, OutGrad };
struct Bind {
  BK kind;
  int v;    // parent value (Fwd, Cot) or output index (OutGrad)
  int ver;  // Cot: accumulation version
};

struct Sub {
  std::unique_ptr<GraphImpl> g;
  std::vector<Bind> in, out;
};

int b_node(GraphImpl& g, Node&& n) {
  g.nodes.push_back(std::move(n));
  return (int)g.nodes.size() - 1;
}

int b_input(GraphImpl& g, int dtype, const std::vector<int64_t>& shape) {
  Node n;
  n.kind = Kind::Input;
  n.dtype = dtype;
  n.shape = shape;
  int id = b_node(g, std::move(n));
  g.inputs.push_back(id);
  return id;
}

int b_map(GraphImpl& g, int op, std::vector<int> in, double imm = 0.0) {
  Node n;
  n.kind = Kind::Map;
  n.op = op;
  n.imm = imm;
  n.in = in;
  n.dtype = g.nodes[in[0]].dtype;
  n.shape = g.nodes[in[0]].shape;
  if (in.size() > 1 && n.shape.empty()) n.shape = g.nodes[in[1]].shape;
  return b_node(g, std::move(n));
}

int b_bcast(GraphImpl& g, int scalar, const std::vector<int64_t>& shape) {
  Node n;
  n.kind = Kind::Map;
  n.op = kOpBcast;
  n.in = {scalar};
  n.dtype = g.nodes[scalar].dtype;
  n.shape = shape;
  return b_node(g, std::move(n));
}

int b_const(GraphImpl& g, int dtype, const std::vector<int64_t>& shape, double v) {
  Node n;
  n.kind = Kind::Map;
  n.op = kOpConst;
  n.imm = v;
  n.dtype = dtype;
  n.shape = shape;
  return b_node(g, std::move(n));
}

int b_reduce_sum(GraphImpl& g, int v) {
  Node n;
  n.kind = Kind::Reduce;
  n.op = DCP_SUM;
  n.in = {v};
  n.dtype = g.nodes[v].dtype;
  return b_node(g, std::move(n));
}

int b_stencil(GraphImpl& g, int v, const Node& fw, bool transpose) {
  Node n = fw;
  n.in = {v};
  n.shape = g.nodes[v].shape;
  n.dtype = g.nodes[v].dtype;
  if (transpose)
    for (auto& o : n.offsets) o = -o;
  return b_node(g, std::move(n));
}

struct Planner {
  const GraphImpl& F;
  std::vector<std::vector<int>> users;
  std::vector<char> is_out;
  std::vector<int> out_index;
  int N = 0;

  explicit Planner(const GraphImpl& f) : F(f) {
    N = (int)F.nodes.size();
    users.assign(N, {});
    for (int v = 0; v < N; ++v)
      for (int a : F.nodes[v].in) users[a].push_back(v);
    is_out.assign(N, 0);
    out_index.assign(N, -1);
    for (size_t j = 0; j < F.outputs.size(); ++j) {
      is_out[F.outputs[j]] = 1;
      out_index[F.outputs[j]] = (int)j;
    }
  }

  // Values downstream of a stencil or reduction inside [n0, v] (taped when needed).
  bool derived_from_heavy(int v, int n0, std::map<int, bool>& memo) const {
    if (v < n0) return false;
    auto it = memo.find(v);
    if (it != memo.end()) return it->second;
    const Node& n = F.nodes[v];
    bool r = false;
    if (n.kind == Kind::Stencil || n.kind == Kind::Reduce) r = true;
    else if (n.kind == Kind::Map)
      for (int a : n.in) r = r || derived_from_heavy(a, n0, memo);
    memo[v] = r;
    return r;
  }
};

// Builds the reverse program of segment [n0, n1).  `ver` holds, per parent
// value, how many cotangent contributions exist so far (segments are built
// in reverse order); it is updated for the live-in values of this segment.
struct ReverseBuilder {
  const Planner& P;
  const GraphImpl& F;
  int n0, n1;
  Sub sub;
  GraphImpl* R;
  std::map<int, int> fwd;      // parent value -> R value (forward)
  std::map<int, int> cot;      // parent value -> R value (cotangent; may be 0-axis broadcast)
  std::map<int, bool> heavy;
  std::set<int> tape;          // parent values of this segment read from the tape

  ReverseBuilder(const Planner& p, int a, int b) : P(p), F(p.F), n0(a), n1(b) {
    sub.g.reset(new GraphImpl());
    R = sub.g.get();
  }

  // A chain of 1-D / 2-D one-step stencil nodes u_{i+1} = E_i(S_i u_i)
  // (E_i: the unary / immediate maps following S_i) inside this segment,
  // every intermediate read only by the next node.  Its reverse runs as
  // time-tiled chunks (AdjChain nodes) that recompute the forward states
  // inside each tile from every K-th state.
  struct Chain {
    std::vector<int> st;                // stencil nodes, in order
    std::vector<std::vector<int>> epi;  // epilogue map nodes of each
    int in = -1;                        // u_0
    int last = -1;                      // node whose value is the chain's result
    int K = 0;                          // reverse steps per launch
  };
  std::map<int, Chain> chains;  // keyed by `last`

  bool single_internal_user(int v, int& u) const {
    if (P.is_out[v] || P.users[v].size() != 1) return false;
    u = P.users[v][0];
    return u < n1;
  }

  bool chain_stencil(int v, const Node& like) const {
    const Node& n = F.nodes[v];
    return n.kind == Kind::Stencil && n.steps == 1 && n.ndim() >= 1 && n.ndim() <= 2 &&
           (n.bc == DCP_BC_ZERO || n.bc == DCP_BC_PERIODIC) && n.dtype == like.dtype &&
           n.shape == like.shape && n.bc == like.bc && n.offsets == like.offsets;
  }

  static bool epilogue_op(int op) {
    switch (op) {
      case DCP_NEG: case DCP_ABS: case DCP_EXP: case DCP_SIN: case DCP_COS: case DCP_TANH:
      case DCP_SQRT: case DCP_SQUARE: case DCP_ADD_S: case DCP_SUB_S: case DCP_MUL_S:
      case DCP_RSUB_S: return true;
    }
    return false;
  }

  void find_chains() {
    auto it = F.options.find(DCP_OPT_ADJOINT_DEPTH);
    std::set<int> seen;
    for (int v = n0; v < n1; ++v) {
      const Node& head = F.nodes[v];
      if (seen.count(v) || !chain_stencil(v, head)) continue;
      // reverse steps per launch (DCP_OPT_ADJOINT_DEPTH; default off: the
      // recomputation trades device-memory traffic and tape for FP32 / FP64
      // work, which pays only where memory bounds the per-step reverse)
      const int64_t K = it != F.options.end() ? it->second : 0;
      if (K < 1) continue;
      Chain c;
      c.in = head.in[0];
      c.K = (int)K;
      int s = v;
      for (;;) {
        seen.insert(s);
        c.st.push_back(s);
        c.epi.emplace_back();
        int x = s, u = -1;
        while (single_internal_user(x, u)) {
          const Node& m = F.nodes[u];
          if (m.kind != Kind::Map || !epilogue_op(m.op) || m.shape != head.shape ||
              m.dtype != head.dtype)
            break;
          c.epi.back().push_back(u);
          x = u;
        }
        c.last = x;
        if (!single_internal_user(x, u) || !chain_stencil(u, head)) break;
        s = u;
      }
      // worth it only where a step before the last has an epilogue (a chain
      // that is linear up to its last step reverses as a transposed stencil
      // chain, time tiled as such); binary64 steps without an epilogue may
      // run on a deferred common weight in the forward pass, which the
      // recomputation does not reproduce
      bool nonlinear = false, all_epi = true;
      for (size_t i = 0; i < c.epi.size(); ++i) {
        nonlinear = nonlinear || (i + 1 < c.epi.size() && !c.epi[i].empty());
        all_epi = all_epi && !c.epi[i].empty();
      }
      if (!nonlinear || (head.dtype == DCP_F64 && !all_epi)) continue;
      chains[c.last] = c;
    }
  }

  // Reverse of chain c, given the cotangent `a` of its result: chunks of K
  // steps from the end; each reads its first state (input or tape) and the
  // cotangent of its last, and yields the cotangent of its first.
  void chain_vjp(const Chain& c, int a) {
    const Node& head = F.nodes[c.st[0]];
    const int K = c.K;
    const int m = (int)c.st.size();
    int cot_v = full(a, head.shape);
    for (int b = m; b > 0;) {
      const int s0 = ((b - 1) / K) * K;  // chunks start at multiples of K
      const int ua = s0 == 0 ? c.in : (c.epi[s0 - 1].empty() ? c.st[s0 - 1] : c.epi[s0 - 1].back());
      Node n;
      n.kind = Kind::AdjChain;
      n.dtype = head.dtype;
      n.shape = head.shape;
      n.bc = head.bc;
      n.offsets = head.offsets;
      n.weights = head.weights;
      n.steps = b - s0;
      for (int i = s0; i < b; ++i) {
        AdjStep st;
        st.weights = F.nodes[c.st[i]].weights;
        for (int e : c.epi[i]) st.epi.emplace_back(F.nodes[e].op, F.nodes[e].imm);
        n.chain.push_back(st);
      }
      n.in = {fwd_value(ua), cot_v};
      cot_v = b_node(*R, std::move(n));
      b = s0;
    }
    acc(c.in, cot_v);
  }

  int fwd_value(int v) {
    auto it = fwd.find(v);
    if (it != fwd.end()) return it->second;
    const Node& n = F.nodes[v];
    int r;
    bool from_memory = v < n0 || n.kind == Kind::Input || P.derived_from_heavy(v, n0, heavy);
    if (from_memory) {
      r = b_input(*R, n.dtype, n.shape);
      sub.in.push_back(Bind{BK::Fwd, v, 0});
      if (v >= n0 && n.kind != Kind::Input) tape.insert(v);
    } else if (n.kind == Kind::Map) {
      std::vector<int> ops;
      for (int a : n.in) ops.push_back(fwd_value(a));
      Node m = n;
      m.in = ops;
      r = b_node(*R, std::move(m));
    } else {  // zero-step stencil: identity of its operand
      r = fwd_value(n.in[0]);
    }
    fwd[v] = r;
    return r;
  }

  // full-shape value of a cotangent that may be a 0-axis broadcast
  int full(int c, const std::vector<int64_t>& shape) {
    if (R->nodes[c].shape.empty() && !shape.empty()) return b_bcast(*R, c, shape);
    return c;
  }

  void acc(int v, int c) {
    const Node& n = F.nodes[v];
    if (!dtype_is_float(n.dtype)) return;
    if (n.shape.empty() && !R->nodes[c].shape.empty()) c = b_reduce_sum(*R, c);
    auto it = cot.find(v);
    if (it == cot.end()) {
      cot[v] = c;
      return;
    }
    int a = it->second;
    // both 0-axis or one broadcast: the add broadcasts
    cot[v] = b_map(*R, DCP_ADD, {full(a, n.shape), c});
  }

  void map_vjp(int v, int a) {
    const Node& n = F.nodes[v];
    const int x = n.in[0];
    const int z = n.in.size() > 1 ? n.in[1] : -1;
    auto X = [&] { return fwd_value(x); };
    auto Z = [&] { return fwd_value(z); };
    auto Y = [&] { return fwd_value(v); };
    switch (n.op) {
      case DCP_NEG: acc(x, b_map(*R, DCP_NEG, {a})); break;
      case DCP_ABS: acc(x, b_map(*R, DCP_MUL, {b_map(*R, kOpSign, {X()}), a})); break;
      case DCP_EXP: acc(x, b_map(*R, DCP_MUL, {Y(), a})); break;
      case DCP_SIN: acc(x, b_map(*R, DCP_MUL, {b_map(*R, DCP_COS, {X()}), a})); break;
      case DCP_COS:
        acc(x, b_map(*R, DCP_MUL, {b_map(*R, DCP_NEG, {b_map(*R, DCP_SIN, {X()})}), a}));
        break;
      case DCP_TANH:
        acc(x, b_map(*R, DCP_MUL, {b_map(*R, DCP_RSUB_S, {b_map(*R, DCP_SQUARE, {Y()})}, 1.0), a}));
        break;
      case DCP_SQRT: acc(x, b_map(*R, DCP_DIV, {b_map(*R, DCP_MUL_S, {a}, 0.5), Y()})); break;
      case DCP_SQUARE: acc(x, b_map(*R, DCP_MUL, {b_map(*R, DCP_MUL_S, {X()}, 2.0), a})); break;
      case DCP_ADD: acc(x, a); acc(z, a); break;
      case DCP_SUB: acc(x, a); acc(z, b_map(*R, DCP_NEG, {a})); break;
      case DCP_MUL:
        acc(x, b_map(*R, DCP_MUL, {Z(), a}));
        acc(z, b_map(*R, DCP_MUL, {X(), a}));
        break;
      case DCP_DIV: {
        int zz = Z();
        acc(x, b_map(*R, DCP_DIV, {a, zz}));
        acc(z, b_map(*R, DCP_NEG, {b_map(*R, DCP_DIV, {b_map(*R, DCP_MUL, {X(), a}),
                                                       b_map(*R, DCP_SQUARE, {zz})})}));
        break;
      }
      case DCP_MAX:
      case DCP_MIN: {
        int m = b_map(*R, n.op == DCP_MAX ? kOpGt : kOpLt, {X(), Z()});
        int cx = b_map(*R, DCP_MUL, {m, a});
        acc(x, cx);
        acc(z, b_map(*R, DCP_MUL, {b_map(*R, DCP_RSUB_S, {m}, 1.0), a}));
        break;
      }
      case DCP_ADD_S:
      case DCP_SUB_S: acc(x, a); break;
      case DCP_MUL_S: acc(x, b_map(*R, DCP_MUL_S, {a}, n.imm)); break;
      case DCP_RSUB_S: acc(x, b_map(*R, DCP_NEG, {a})); break;
      default: fail(DCP_E_UNSUPPORTED, "adjoint: op not differentiable");
    }
  }

  void build(std::map<int, int>& ver) {
    find_chains();
    // seeds: cotangents of values of this segment that are outputs or read later
    for (int v = n0; v < n1; ++v) {
      const Node& n = F.nodes[v];
      if (!dtype_is_float(n.dtype) || n.kind == Kind::Input) continue;
      bool later = false;
      for (int u : P.users[v])
        if (u >= n1) later = true;
      if (P.is_out[v]) {
        int c = b_input(*R, n.dtype, n.shape);
        sub.in.push_back(Bind{BK::OutGrad, P.out_index[v], 0});
        acc(v, c);
      }
      if (later && ver[v] > 0) {
        int c = b_input(*R, n.dtype, n.shape);
        sub.in.push_back(Bind{BK::Cot, v, ver[v]});
        acc(v, c);
      }
    }
    // live-in values carrying earlier contributions start from them
    // (program inputs count as live-in wherever they are read)
    std::set<int> livein;
    for (int v = n0; v < n1; ++v)
      for (int a : F.nodes[v].in)
        if ((a < n0 || F.nodes[a].kind == Kind::Input) && dtype_is_float(F.nodes[a].dtype))
          livein.insert(a);
    for (int v = n1 - 1; v >= n0; --v) {
      auto it = cot.find(v);
      if (it == cot.end()) continue;
      const Node& n = F.nodes[v];
      int a = it->second;
      auto ch = chains.find(v);
      if (ch != chains.end()) {
        chain_vjp(ch->second, a);
        continue;
      }
      switch (n.kind) {
        case Kind::AdjChain:
        case Kind::Input: break;
        case Kind::Map: map_vjp(v, a); break;
        case Kind::Stencil:
          if (n.steps == 0) {
            acc(n.in[0], a);
            break;
          }
          if (n.bc == DCP_BC_FIXED_RING)
            fail(DCP_E_UNSUPPORTED, "adjoint of fixed-ring stencils is not implemented");
          acc(n.in[0], b_stencil(*R, full(a, n.shape), n, true));
          break;
        case Kind::Reduce:
          if (n.op != DCP_SUM) fail(DCP_E_UNSUPPORTED, "adjoint supports sum reductions only");
          acc(n.in[0], a);
          break;
      }
    }
    // outputs: cotangents of live-in values (accumulated onto earlier contributions)
    for (int v : livein) {
      auto it = cot.find(v);
      if (it == cot.end()) continue;
      int c = full(it->second, F.nodes[v].shape);
      if (ver[v] > 0) {
        int prev = b_input(*R, F.nodes[v].dtype, F.nodes[v].shape);
        sub.in.push_back(Bind{BK::Cot, v, ver[v]});
        c = b_map(*R, DCP_ADD, {prev, c});
      }
      // an output may not be an input of the same graph: copy through a map
      if (R->nodes[c].kind == Kind::Input) c = b_map(*R, DCP_ADD_S, {c}, 0.0);
      // a value marked twice as output is not allowed; add a copy if needed
      if (std::find(R->outputs.begin(), R->outputs.end(), c) != R->outputs.end())
        c = b_map(*R, DCP_ADD_S, {c}, 0.0);
      R->outputs.push_back(c);
      ver[v] += 1;
      sub.out.push_back(Bind{BK::Cot, v, ver[v]});
    }
  }
};

// Forward sub-program of [n0, n1) with the given outputs; inputs are the
// values defined before n0 that the kept nodes read.
Sub forward_segment(const GraphImpl& F, int n0, int n1, const std::vector<int>& outs) {
  Sub s;
  s.g.reset(new GraphImpl());
  GraphImpl& G = *s.g;
  std::map<int, int> m;
  std::set<int> need(outs.begin(), outs.end());
  // keep only what the outputs need
  std::vector<char> keep(F.nodes.size(), 0);
  std::vector<int> stack(outs.begin(), outs.end());
  while (!stack.empty()) {
    int v = stack.back();
    stack.pop_back();
    if (keep[v]) continue;
    keep[v] = 1;
    if (v < n0 || F.nodes[v].kind == Kind::Input) continue;
    for (int a : F.nodes[v].in) stack.push_back(a);
  }
  for (int v = 0; v < n1; ++v) {
    if (!keep[v]) continue;
    const Node& n = F.nodes[v];
    if (v < n0 || n.kind == Kind::Input) {
      m[v] = b_input(G, n.dtype, n.shape);
      s.in.push_back(Bind{BK::Fwd, v, 0});
      continue;
    }
    Node c = n;
    for (auto& a : c.in) a = m.at(a);
    m[v] = b_node(G, std::move(c));
  }
  for (int v : outs) {
    G.outputs.push_back(m.at(v));
    s.out.push_back(Bind{BK::Fwd, v, 0});
  }
  return s;
}

size_t bytes_of(const Node& n) { return (size_t)n.numel() * dtype_size(n.dtype); }

}  // namespace

struct AdjointPlan {
  bool chunked = false;
  size_t tape_bytes = 0;
  // tape values that are not checkpoints live in one arena; in checkpointed
  // mode the segments reuse it (one segment's tape at a time)
  std::map<int, size_t> tape_offset;
  size_t arena_bytes = 0;
  Sub forward;                 // stores the tape (full) or the checkpoints (chunked)
  std::vector<Sub> seg_fwd;    // chunked: recompute segment tapes
  std::vector<Sub> seg_rev;    // reverse programs, in execution order
  std::vector<int> input_ver;  // final cotangent version of each program input
};

void plan_adjoint(const GraphImpl& F, size_t budget, AdjointPlan& out) {
  for (const Node& n : F.nodes) {
    if (!dtype_is_float(n.dtype))
      fail(DCP_E_UNSUPPORTED, "the adjoint is defined for floating programs only");
    if (n.kind == Kind::Reduce && n.axis >= 0)
      fail(DCP_E_UNSUPPORTED, "the adjoint of axis reductions is not implemented");
  }
  Planner P(F);
  const int N = P.N;
  // segment boundaries: before every k-th stencil node
  std::vector<int> stencils;
  for (int v = 0; v < N; ++v)
    if (F.nodes[v].kind == Kind::Stencil && F.nodes[v].steps > 0) stencils.push_back(v);

  auto build = [&](std::vector<int> bounds, AdjointPlan& plan) {
    // bounds: increasing node positions, first 0, last N
    const int C = (int)bounds.size() - 1;
    std::map<int, int> ver;
    std::vector<Sub> rev(C);
    std::vector<std::set<int>> tapes(C);
    std::set<int> ckpt;  // forward values needed across segments (non-inputs)
    for (int c = C - 1; c >= 0; --c) {
      ReverseBuilder rb(P, bounds[c], bounds[c + 1]);
      rb.build(ver);
      for (const Bind& b : rb.sub.in)
        if (b.kind == BK::Fwd && b.v < bounds[c] && F.nodes[b.v].kind != Kind::Input) ckpt.insert(b.v);
      tapes[c] = rb.tape;
      rev[c] = std::move(rb.sub);
    }
    plan.seg_rev.clear();
    for (int c = C - 1; c >= 0; --c) plan.seg_rev.push_back(std::move(rev[c]));
    plan.input_ver.clear();
    for (int v : F.inputs) plan.input_ver.push_back(ver[v]);
    plan.seg_fwd.clear();
    plan.tape_offset.clear();
    plan.arena_bytes = 0;
    size_t bytes = 0;
    auto place = [&](const std::set<int>& vals) {
      size_t off = 0;
      for (int v : vals) {
        if (ckpt.count(v)) continue;
        plan.tape_offset[v] = off;
        off += (bytes_of(F.nodes[v]) + 255) / 256 * 256;
      }
      plan.arena_bytes = std::max(plan.arena_bytes, off);
    };
    if (C == 1) {
      std::vector<int> outs(tapes[0].begin(), tapes[0].end());
      for (int v : outs) bytes += bytes_of(F.nodes[v]);
      plan.forward = outs.empty() ? Sub() : forward_segment(F, 0, N, outs);
      place(tapes[0]);
    } else {
      // checkpoints also include what segment recomputation reads
      std::vector<Sub> segf(C);
      size_t maxtape = 0;
      for (int c = 0; c < C; ++c) {
        std::vector<int> outs(tapes[c].begin(), tapes[c].end());
        size_t tb = 0;
        for (int v : outs) tb += bytes_of(F.nodes[v]);
        maxtape = std::max(maxtape, tb);
        if (!outs.empty()) {
          segf[c] = forward_segment(F, bounds[c], bounds[c + 1], outs);
          for (const Bind& b : segf[c].in)
            if (F.nodes[b.v].kind != Kind::Input) ckpt.insert(b.v);
        }
      }
      std::vector<int> outs(ckpt.begin(), ckpt.end());
      for (int v : outs) bytes += bytes_of(F.nodes[v]);
      bytes += maxtape;
      plan.forward = outs.empty() ? Sub() : forward_segment(F, 0, N, outs);
      for (int c = C - 1; c >= 0; --c) plan.seg_fwd.push_back(std::move(segf[c]));
      for (int c = 0; c < C; ++c) place(tapes[c]);
    }
    plan.tape_bytes = bytes;
  };

  build({0, N}, out);
  out.chunked = false;
  if (out.tape_bytes <= budget || stencils.size() < 2) {
    if (out.tape_bytes > budget) fail(DCP_E_OOM, "the adjoint tape does not fit the budget");
    return;
  }
  const int S = (int)stencils.size();
  const int K = (int)std::ceil(std::sqrt((double)S));
  // A cut before stencil node stencils[i] keeps the forward values bitwise
  // those of the unsegmented run when it falls on a chunk end of a deferred
  // common-weight run: the run of equal one-input steps that the full-tape
  // forward fuses is then split where it applies f^m anyway, so both halves
  // round exactly like the whole.  Cuts move forward to the next such place
  // (node boundaries between different chains always qualify).
  auto chained = [&](int p, int q) {  // q's steps continue p's run
    const Node& a = F.nodes[p];
    const Node& b = F.nodes[q];
    return b.in.size() == 1 && b.in[0] == p && P.users[p].size() == 1 && !P.is_out[p] &&
           a.weights == b.weights && a.offsets == b.offsets && a.bc == b.bc &&
           a.dtype == b.dtype && defer_chunk_steps(a) > 0;
  };
  auto aligned = [&](int i) {
    if (!chained(stencils[i - 1], stencils[i])) return true;
    const int D = defer_chunk_steps(F.nodes[stencils[i]]);
    long long steps = 0;
    int j = i - 1;
    for (;;) {
      steps += F.nodes[stencils[j]].steps;
      if (j == 0 || !chained(stencils[j - 1], stencils[j])) break;
      --j;
    }
    // an unbounded run applies f^L once at its end: no cut inside it is free
    return D != INT32_MAX && steps % D == 0;
  };
  auto segment = [&](bool align) {
    std::vector<int> bounds{0};
    for (int i = K; i < S; i += K) {
      if (align)
        while (i < S && !aligned(i)) ++i;
      if (i < S) bounds.push_back(stencils[i]);
    }
    bounds.push_back(N);
    return bounds;
  };
  AdjointPlan ch;
  std::vector<int> bounds = segment(true);
  if (bounds.size() > 2) {
    build(bounds, ch);
  }
  if (bounds.size() <= 2 || ch.tape_bytes > budget) {
    // no aligned cut fits the budget: cut every K stencil nodes (forward
    // values may then differ from the full tape's in their last bits)
    bounds = segment(false);
    build(bounds, ch);
  }
  ch.chunked = true;
  if (ch.tape_bytes > budget)
    fail(DCP_E_OOM, "even sqrt(T) checkpointing needs " + std::to_string(ch.tape_bytes) +
                        " bytes of tape, above the budget");
  out = std::move(ch);
}

// ---------------------------------------------------------------------------
// execution
// ---------------------------------------------------------------------------
struct AdjointState {
  size_t budget = 0;
  bool built = false;
  AdjointPlan plan;
  void* arena = nullptr;
  std::map<std::pair<int, int>, void*> bufs;  // (kind*2^20 + value, parity) -> device buffer
  std::vector<void*> allocs;
  ~AdjointState() {
    for (void* p : allocs) cudaFree(p);
  }
  void* buffer(int tag, int v, int parity, size_t bytes) {
    auto key = std::make_pair(tag * (1 << 24) + v, parity);
    auto it = bufs.find(key);
    if (it != bufs.end()) return it->second;
    void* p = nullptr;
    check_cuda(cudaMalloc(&p, bytes ? bytes : 16), "cudaMalloc(adjoint)");
    allocs.push_back(p);
    bufs[key] = p;
    return p;
  }
};

// Sub-programs are planned with the parent program's fusion flags, so the
// reverse pass of an op-by-op program is op-by-op too.
static void fuse_sub(Sub& s, uint32_t flags, const std::map<int, int64_t>& options) {
  if (!s.g) return;
  s.g->options = options;  // the program's tiling and launch options apply to its reverse pass
  plan_graph(*s.g, flags & (DCP_FUSE_MAPS | DCP_FUSE_SUBGRAPH | DCP_TIME_TILE));
  compile_plan(*s.g);
  s.g->fused = true;
}

// Plans the reverse pass for `budget` and compiles its kernels (no device
// work); a plan for the same budget is kept.
void prepare_adjoint_impl(GraphImpl& g, AdjointState& st, size_t budget) {
  if (st.built && st.budget == budget) return;
  AdjointPlan p;
  plan_adjoint(g, budget, p);
  fuse_sub(p.forward, g.flags, g.options);
  for (Sub& x : p.seg_fwd) fuse_sub(x, g.flags, g.options);
  for (Sub& x : p.seg_rev) fuse_sub(x, g.flags, g.options);
  st.plan = std::move(p);
  st.budget = budget;
  st.built = true;
  if (st.arena) {
    cudaFree(st.arena);
    st.allocs.erase(std::find(st.allocs.begin(), st.allocs.end(), st.arena));
    st.arena = nullptr;
  }
}

void run_adjoint_impl(GraphImpl& g, AdjointState& st, const void* const* inputs,
                      const void* const* out_grads, void* const* in_grads, size_t budget,
                      cudaStream_t s) {
  prepare_adjoint_impl(g, st, budget);
  if (st.plan.arena_bytes && !st.arena) {
    check_cuda(cudaMalloc(&st.arena, st.plan.arena_bytes), "cudaMalloc(adjoint tape)");
    st.allocs.push_back(st.arena);
  }
  std::map<int, int> input_index;
  for (size_t i = 0; i < g.inputs.size(); ++i) input_index[g.inputs[i]] = (int)i;
  auto resolve = [&](const Bind& b) -> void* {
    const Node& n = g.nodes[b.kind == BK::OutGrad ? g.outputs[b.v] : b.v];
    size_t bytes = bytes_of(n);
    switch (b.kind) {
      case BK::OutGrad: {
        if (!out_grads[b.v]) fail(DCP_E_INVALID_ARG, "output cotangent is NULL");
        return const_cast<void*>(out_grads[b.v]);
      }
      case BK::Fwd: {
        auto it = input_index.find(b.v);
        if (it != input_index.end()) return const_cast<void*>(inputs[it->second]);
        auto t = st.plan.tape_offset.find(b.v);
        if (t != st.plan.tape_offset.end()) return (char*)st.arena + t->second;
        return st.buffer(0, b.v, 0, bytes);
      }
      case BK::Cot:
        return st.buffer(1, b.v, b.ver & 1, bytes);
    }
    return nullptr;
  };
  auto run_sub = [&](Sub& x) {
    if (!x.g) return;
    std::vector<void*> in, out;
    for (const Bind& b : x.in) in.push_back(resolve(b));
    for (const Bind& b : x.out) out.push_back(resolve(b));
    run_graph(*x.g, (const void* const*)in.data(), out.data(), s);
  };
  run_sub(st.plan.forward);
  const size_t C = st.plan.seg_rev.size();
  for (size_t c = 0; c < C; ++c) {
    if (st.plan.chunked) run_sub(st.plan.seg_fwd[c]);
    run_sub(st.plan.seg_rev[c]);
  }
  for (size_t i = 0; i < g.inputs.size(); ++i) {
    const Node& n = g.nodes[g.inputs[i]];
    size_t bytes = bytes_of(n);
    if (!in_grads[i]) fail(DCP_E_INVALID_ARG, "input cotangent buffer is NULL");
    int ver = st.plan.input_ver[i];
    if (ver == 0) {
      check_cuda(cudaMemsetAsync(in_grads[i], 0, bytes, s), "cudaMemsetAsync");
    } else {
      void* src = st.buffer(1, g.inputs[i], ver & 1, bytes);
      check_cuda(cudaMemcpyAsync(in_grads[i], src, bytes, cudaMemcpyDeviceToDevice, s),
                 "cudaMemcpyAsync(cotangent)");
    }
  }
}

std::shared_ptr<AdjointState> new_adjoint_state() { return std::make_shared<AdjointState>(); }
size_t adjoint_tape_bytes(const AdjointState& st) { return st.plan.tape_bytes; }
bool adjoint_chunked(const AdjointState& st) { return st.plan.chunked; }

// The reverse pass's kernels in execution order (JSON array).
std::string adjoint_launches_json(const AdjointState& st) {
  std::ostringstream os;
  os << "[";
  bool first = true;
  auto add = [&](const Sub& x, const char* phase) {
    if (!x.g) return;
    for (const std::string& k : launch_kernel_names(*x.g)) {
      os << (first ? "" : ", ") << "{\"phase\": \"" << phase << "\", \"kernel\": \"" << k
         << "\"}";
      first = false;
    }
  };
  if (st.built) {
    add(st.plan.forward, "forward");
    for (size_t c = 0; c < st.plan.seg_rev.size(); ++c) {
      if (st.plan.chunked) add(st.plan.seg_fwd[c], "recompute");
      add(st.plan.seg_rev[c], "reverse");
    }
  }
  os << "]";
  return os.str();
}

}  // namespace dcp
