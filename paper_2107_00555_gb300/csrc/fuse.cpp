// Planning passes over the SSA graph (Sec. 3.1 auto-optimisation):
//  * map fusion -- greedy merging of elementwise maps that share an iteration
//    space into one expression DAG evaluated in registers (Sec. 3.1, "greedy
//    subgraph fusion": fuse the largest contiguous subgraphs over the same
//    iteration space, checking that what a map consumes is a subset of what
//    the fused scope produces);
//  * subgraph fusion -- reductions become epilogues of the kernel that
//    produces their operand (tiled write-conflict resolution, Sec. 3.1);
//    an axis reduction takes the elementwise maps producing its operand as
//    the prologue of its own kernel, and reductions along the same axis of
//    that prologue share the kernel;
//    elementwise maps feeding a stencil become its prologue, evaluated at
//    every cell the stencil tile reads; unary maps after a stencil step
//    become that step's epilogue; maps after the last step become a post
//    stage; consecutive stencils with the same neighbourhood chain into one
//    group that can be time tiled;
//  * transient mitigation -- a value gets a device buffer only if it is a
//    program output or is read by another kernel (Sec. 3.1: temporaries are
//    persistent and fused-away temporaries are never allocated);
//  * batching -- independent stencil groups running the same step program
//    on different shapes are packed into one launch (the side-by-side
//    connected components of Sec. 2.4 state fusion).
#include <algorithm>
#include <cmath>
#include <set>
#include <sstream>

#include "dcp_internal.h"

namespace dcp {

namespace {

struct Planner {
  GraphImpl& g;
  uint32_t flags;
  std::vector<std::vector<int>> users;
  std::vector<char> live, is_out;

  std::vector<Group>& batch_store;
  Planner(GraphImpl& gi, uint32_t f) : g(gi), flags(f), batch_store(gi.batch_store) {}

  bool fmaps() const { return flags & DCP_FUSE_MAPS; }
  bool fsub() const { return flags & DCP_FUSE_SUBGRAPH; }

  int live_users(int v) const {
    int c = 0;
    for (int u : users[v])
      if (live[u]) ++c;
    return c;
  }

  bool in_vec(const std::vector<int>& a, int v) const {
    return std::find(a.begin(), a.end(), v) != a.end();
  }

  // Is `v` computed in registers by group `gi` (member, stencil output, post)?
  bool computed_in(int gi, int v) const {
    const Group& G = g.groups[gi];
    if (G.kind == GroupKind::Map || G.kind == GroupKind::AxisReduce) return in_vec(G.members, v);
    if (G.kind == GroupKind::Stencil) return v == G.st_out || in_vec(G.post, v);
    if (G.kind == GroupKind::AdjTile) return v == G.st_out;
    return false;
  }

  // Value available in memory before group gi runs (an input, or produced by
  // an earlier group).
  bool available_before(int v, int gi) const {
    int pg = g.value_group[v];
    return pg < 0 || pg < gi;
  }

  void add_operand(Group& G, int gi, int a) {
    if (computed_in(gi, a)) return;
    const Node& n = g.nodes[a];
    bool scalar = n.shape.empty() && !G.shape.empty();
    std::vector<int>& dst = scalar ? G.scalars : (G.kind == GroupKind::Stencil ? G.post_loads : G.loads);
    if (!in_vec(dst, a)) dst.push_back(a);
  }

  void plan() {
    const int N = (int)g.nodes.size();
    users.assign(N, {});
    for (int v = 0; v < N; ++v)
      for (int a : g.nodes[v].in) users[a].push_back(v);
    is_out.assign(N, 0);
    for (int o : g.outputs) is_out[o] = 1;
    // liveness: everything an output depends on
    live.assign(N, 0);
    std::vector<int> stack(g.outputs.begin(), g.outputs.end());
    while (!stack.empty()) {
      int v = stack.back();
      stack.pop_back();
      if (live[v]) continue;
      live[v] = 1;
      for (int a : g.nodes[v].in) stack.push_back(a);
    }
    g.groups.clear();
    g.value_group.assign(N, -1);

    for (int v = 0; v < N; ++v) {
      if (!live[v]) continue;
      const Node& n = g.nodes[v];
      switch (n.kind) {
        case Kind::Input: break;
        case Kind::Map: plan_map(v); break;
        case Kind::Reduce: plan_reduce(v); break;
        case Kind::Stencil: plan_stencil(v); break;
        case Kind::AdjChain: plan_adj(v); break;
      }
    }
    if (flags & DCP_BATCH) plan_batch();
    finalize();
  }

  void plan_map(int v) {
    const Node& n = g.nodes[v];
    // (1) stencil step epilogue: a unary / immediate map of a stencil group's
    //     current output, which nothing else reads.
    if (fsub() && (op_is_unary(n.op) || op_is_scalar_imm(n.op))) {
      int a = n.in[0];
      int gi = g.value_group[a];
      if (gi >= 0 && gi == (int)g.groups.size() - 1) {
        Group& G = g.groups[gi];
        if (G.kind == GroupKind::Stencil && G.st_out == a && G.post.empty() && G.reds.empty() &&
            !is_out[a] && live_users(a) == 1 && !G.steps.empty()) {
          G.steps.back().epi.push_back(v);
          G.st_out = v;
          g.value_group[v] = gi;
          return;
        }
      }
    }
    // (2) join a group that computes one of the operands.
    int best = -1;
    if (fmaps() || fsub()) {
      for (int a : n.in) {
        int gi = g.value_group[a];
        if (gi < 0 || !computed_in(gi, a)) continue;
        const Group& G = g.groups[gi];
        if (G.shape != n.shape) continue;
        if (G.kind == GroupKind::Map && !fmaps()) continue;
        if (G.kind == GroupKind::Stencil && !fsub()) continue;
        if (G.kind == GroupKind::Batch || G.kind == GroupKind::AxisReduce ||
            G.kind == GroupKind::AdjTile)
          continue;
        bool ok = true;
        for (int b : n.in)
          if (!computed_in(gi, b) && !available_before(b, gi)) ok = false;
        if (ok && gi > best) best = gi;
      }
    }
    // (3) no producer group qualifies (e.g. every operand is a program input):
    //     extend the contiguous subgraph, i.e. join the latest group if it is
    //     a map group over the same iteration space.
    if (best < 0 && fmaps() && !n.shape.empty() && !g.groups.empty()) {
      int gi = (int)g.groups.size() - 1;
      const Group& G = g.groups[gi];
      if (G.kind == GroupKind::Map && G.shape == n.shape) {
        bool ok = true;
        for (int b : n.in)
          if (!computed_in(gi, b) && !available_before(b, gi)) ok = false;
        if (ok) best = gi;
      }
    }
    if (best >= 0) {
      Group& G = g.groups[best];
      if (G.kind == GroupKind::Map) G.members.push_back(v);
      else G.post.push_back(v);
      g.value_group[v] = best;
      for (int a : n.in) add_operand(G, best, a);
      return;
    }
    Group G;
    G.kind = GroupKind::Map;
    G.dtype = n.dtype;
    G.shape = n.shape;
    G.members.push_back(v);
    g.groups.push_back(G);
    int gi = (int)g.groups.size() - 1;
    g.value_group[v] = gi;
    for (int a : n.in) add_operand(g.groups[gi], gi, a);
  }

  // Axis reduction (tiled write-conflict resolution with one partial per
  // remaining index): joins the axis-reduce group computing its operand, or
  // the latest one over the same space and axis; otherwise starts a group
  // that takes the producer map group as its prologue when every value of
  // that group is consumed inside it or by reductions along the same axis.
  void plan_axis_reduce(int v) {
    const Node& n = g.nodes[v];
    int a = n.in[0];
    const Node& an = g.nodes[a];
    auto same_space = [&](const Group& G) {
      return G.kind == GroupKind::AxisReduce && G.shape == an.shape && G.axis == n.axis &&
             G.dtype == an.dtype;
    };
    int gi = g.value_group[a];
    if (gi >= 0 && g.groups[gi].kind == GroupKind::AxisReduce && computed_in(gi, a)) {
      Group& G = g.groups[gi];
      if (!same_space(G) || (int)G.reds.size() >= kMaxIO)
        fail(DCP_E_UNSUPPORTED, "too many reductions of one fused prologue");
      G.reds.push_back(v);
      g.value_group[v] = gi;
      return;
    }
    if (fsub() && !g.groups.empty()) {
      int li = (int)g.groups.size() - 1;
      Group& G = g.groups[li];
      if (same_space(G) && (int)G.reds.size() < kMaxIO && available_before(a, li)) {
        G.reds.push_back(v);
        g.value_group[v] = li;
        add_operand(G, li, a);
        return;
      }
    }
    Group R;
    R.kind = GroupKind::AxisReduce;
    R.dtype = an.dtype;
    R.shape = an.shape;
    R.axis = n.axis;
    bool absorbed = false;
    if (fsub() && gi >= 0 && gi == (int)g.groups.size() - 1 &&
        g.groups[gi].kind == GroupKind::Map && computed_in(gi, a)) {
      const Group& M = g.groups[gi];
      bool ok = M.reds.empty() && M.shape == an.shape;
      int nred = 0;
      for (int m : M.members) {
        if (is_out[m] || g.nodes[m].kind != Kind::Map) ok = false;
        for (int u : users[m]) {
          if (!live[u] || in_vec(M.members, u)) continue;
          const Node& un = g.nodes[u];
          if (un.kind == Kind::Reduce && un.axis == n.axis) ++nred;
          else ok = false;
        }
      }
      if (ok && nred <= kMaxIO) {
        R.members = M.members;
        R.loads = M.loads;
        R.scalars = M.scalars;
        g.groups.pop_back();
        absorbed = true;
      }
    }
    if (!absorbed) R.loads.push_back(a);
    R.reds.push_back(v);
    g.groups.push_back(R);
    int ri = (int)g.groups.size() - 1;
    g.value_group[v] = ri;
    for (int m : R.members) g.value_group[m] = ri;
  }

  void plan_reduce(int v) {
    const Node& n = g.nodes[v];
    if (n.axis >= 0) {
      plan_axis_reduce(v);
      return;
    }
    int a = n.in[0];
    int gi = g.value_group[a];
    if (fsub() && gi >= 0 && computed_in(gi, a) && g.groups[gi].kind != GroupKind::Batch &&
        g.groups[gi].kind != GroupKind::AxisReduce && g.groups[gi].kind != GroupKind::AdjTile &&
        (int)g.groups[gi].reds.size() < kMaxIO) {
      g.groups[gi].reds.push_back(v);
      g.value_group[v] = gi;
      return;
    }
    Group G;
    G.kind = GroupKind::Map;
    G.dtype = g.nodes[a].dtype;
    G.shape = g.nodes[a].shape;
    G.loads.push_back(a);
    G.reds.push_back(v);
    g.groups.push_back(G);
    g.value_group[v] = (int)g.groups.size() - 1;
  }

  static std::vector<int32_t> pad_offsets(const Node& n) {
    std::vector<int32_t> o;
    int nd = n.ndim();
    for (int k = 0; k < n.npts(); ++k)
      for (int d = 0; d < 3; ++d) {
        int src = d - (3 - nd);
        o.push_back(src >= 0 ? n.offsets[k * nd + src] : 0);
      }
    return o;
  }

  void plan_stencil(int v) {
    const Node& n = g.nodes[v];
    int a = n.in[0];
    if (n.steps == 0) {  // identity: a copy kernel
      Group G;
      G.kind = GroupKind::Map;
      G.dtype = n.dtype;
      G.shape = n.shape;
      G.members.push_back(v);
      G.loads.push_back(a);
      g.groups.push_back(G);
      g.value_group[v] = (int)g.groups.size() - 1;
      return;
    }
    std::vector<int32_t> offs = pad_offsets(n);
    int gi = g.value_group[a];
    // stencil -> stencil: extend the chain (time tiling candidate)
    if (fsub() && gi >= 0 && gi == (int)g.groups.size() - 1) {
      Group& G = g.groups[gi];
      if (G.kind == GroupKind::Stencil && G.st_out == a && G.post.empty() && G.reds.empty() &&
          !is_out[a] && live_users(a) == 1 && G.bc == n.bc && G.offsets == offs &&
          G.dtype == n.dtype) {
        for (int t = 0; t < n.steps; ++t) G.steps.push_back(StepDesc{v, {}});
        G.st_out = v;
        g.value_group[v] = gi;
        return;
      }
    }
    Group S;
    S.kind = GroupKind::Stencil;
    S.dtype = n.dtype;
    S.shape = n.shape;
    S.bc = n.bc;
    S.offsets = offs;
    for (int d = 0; d < 3; ++d) {
      int r = 0;
      for (int k = 0; k < n.npts(); ++k) r = std::max(r, std::abs(offs[k * 3 + d]));
      S.radius[d] = r;
    }
    // map -> stencil prologue: the producer map group is the latest group, has
    // no reductions, and none of its values is read outside this stencil.
    if (fsub() && gi >= 0 && gi == (int)g.groups.size() - 1 &&
        g.groups[gi].kind == GroupKind::Map && computed_in(gi, a)) {
      Group& M = g.groups[gi];
      bool ok = M.reds.empty() && M.shape == n.shape;
      for (int m : M.members) {
        if (is_out[m]) ok = false;
        for (int u : users[m])
          if (live[u] && u != v && !in_vec(M.members, u)) ok = false;
        if (g.nodes[m].kind != Kind::Map) ok = false;
      }
      if (ok) {
        S.members = M.members;
        S.loads = M.loads;
        S.scalars = M.scalars;
        g.groups.pop_back();
      }
    }
    S.st_in = a;
    for (int t = 0; t < n.steps; ++t) S.steps.push_back(StepDesc{v, {}});
    S.st_out = v;
    g.groups.push_back(S);
    int si = (int)g.groups.size() - 1;
    g.value_group[v] = si;
    for (int m : S.members) g.value_group[m] = si;
  }

  // Reverse of a chunk of a stencil chain (built by the adjoint): one group
  // reading u_t and the cotangent of u_{t+k} from memory, storing the
  // cotangent of u_t.
  void plan_adj(int v) {
    const Node& n = g.nodes[v];
    Group A;
    A.kind = GroupKind::AdjTile;
    A.dtype = n.dtype;
    A.shape = n.shape;
    A.bc = n.bc;
    A.offsets = pad_offsets(n);
    for (int d = 0; d < 3; ++d) {
      int r = 0;
      for (int k = 0; k < n.npts(); ++k) r = std::max(r, std::abs(A.offsets[k * 3 + d]));
      A.radius[d] = r;
    }
    A.loads = {n.in[0], n.in[1]};
    A.st_in = n.in[0];
    A.st_out = v;
    A.depth = (int)n.chain.size();
    A.members.push_back(v);
    g.groups.push_back(A);
    g.value_group[v] = (int)g.groups.size() - 1;
  }

  // Pack independent stencil groups that run one step program into batches.
  void plan_batch() {
    std::map<std::string, std::vector<int>> classes;
    for (int gi = 0; gi < (int)g.groups.size(); ++gi) {
      Group& G = g.groups[gi];
      if (G.kind != GroupKind::Stencil || !G.members.empty() || !G.post.empty() ||
          !G.reds.empty() || G.shape.size() != 2)
        continue;
      if (!is_out[G.st_out] || live_users(G.st_out) != 0) continue;
      if (g.value_group[G.st_in] >= 0) continue;  // batch members read program inputs
      std::ostringstream key;
      key.precision(17);
      key << G.dtype << "|" << G.bc << "|";
      for (auto o : G.offsets) key << o << ",";
      for (const StepDesc& s : G.steps) {
        key << "[";
        for (double w : g.nodes[s.node].weights) key << w << ",";
        for (int e : s.epi) key << g.nodes[e].op << ":" << g.nodes[e].imm << ",";
        key << "]";
      }
      classes[key.str()].push_back(gi);
    }
    for (auto& kv : classes) {
      if (kv.second.size() < 2) continue;
      Group B = g.groups[kv.second.front()];
      B.kind = GroupKind::Batch;
      B.shape.clear();
      B.batch_members = kv.second;
      for (int gi : kv.second) g.groups[gi].absorbed = true;
      g.groups.push_back(B);
    }
  }

  void finalize() {
    // Drop absorbed groups, keeping execution order; batch groups run where
    // they were appended (after every member's producers).
    std::vector<Group> out;
    std::vector<int> remap(g.groups.size(), -1);
    for (int gi = 0; gi < (int)g.groups.size(); ++gi) {
      if (g.groups[gi].absorbed) continue;
      remap[gi] = (int)out.size();
      out.push_back(g.groups[gi]);
    }
    // store the absorbed groups' descriptions inside the batch for codegen
    std::vector<Group> all = g.groups;
    for (Group& G : out)
      if (G.kind == GroupKind::Batch) {
        std::vector<int> members = G.batch_members;
        G.batch_members.clear();
        for (int m : members) {
          G.batch_members.push_back((int)batch_store.size());
          batch_store.push_back(all[m]);
        }
      }
    g.groups = out;
    const int N = (int)g.nodes.size();
    for (int v = 0; v < N; ++v)
      if (g.value_group[v] >= 0) g.value_group[v] = remap[g.value_group[v]];
    // batch: member values belong to the batch group
    for (int gi = 0; gi < (int)g.groups.size(); ++gi)
      if (g.groups[gi].kind == GroupKind::Batch)
        for (int m : g.groups[gi].batch_members) {
          const Group& M = batch_store[m];
          g.value_group[M.st_out] = gi;
          for (const StepDesc& s : M.steps) {
            g.value_group[s.node] = gi;
            for (int e : s.epi) g.value_group[e] = gi;
          }
        }

    // Materialisation: a value computed by group G is stored when it is an
    // output or read by a live node outside G.
    g.materialized.assign(N, 0);
    for (int v = 0; v < N; ++v)
      if (g.nodes[v].kind == Kind::Input) g.materialized[v] = 1;
    for (int gi = 0; gi < (int)g.groups.size(); ++gi) {
      Group& G = g.groups[gi];
      G.stores.clear();
      std::vector<int> cand;
      if (G.kind == GroupKind::Map) cand = G.members;
      if (G.kind == GroupKind::Stencil) {
        cand.push_back(G.st_out);
        cand.insert(cand.end(), G.post.begin(), G.post.end());
      }
      if (G.kind == GroupKind::AdjTile) cand.push_back(G.st_out);
      for (int v : cand) {
        bool need = is_out[v];
        for (int u : users[v])
          if (live[u] && g.value_group[u] != gi) need = true;
        // in a stencil group, the stencil output feeds post members in registers
        if (need) {
          G.stores.push_back(v);
          g.materialized[v] = 1;
        }
      }
      for (int r : G.reds) g.materialized[r] = 1;
      if (G.kind == GroupKind::Batch) {
        for (int m : G.batch_members) g.materialized[batch_store[m].st_out] = 1;
      }
      if ((int)G.loads.size() > kMaxIO || (int)G.post_loads.size() > kMaxIO ||
          (int)G.stores.size() > kMaxIO || (int)G.scalars.size() > kMaxIO)
        fail(DCP_E_UNSUPPORTED, "a fused group exceeds 16 loads/stores; split the program");
    }
    // Launch shapes
    int nl = 0;
    for (Group& G : g.groups) {
      if (G.kind == GroupKind::Map) {
        G.threads = 256;
        G.blocks_per_sm = (int)opt(DCP_OPT_MAP_BLOCKS_PER_SM, 8);
        G.unroll = (int)opt(DCP_OPT_MAP_UNROLL, 2);
        nl += 1;
      } else if (G.kind == GroupKind::AxisReduce) {
        G.threads = 256;
        nl += 1;
      } else if (G.kind == GroupKind::AdjTile) {
        // output tile; the halo is 2 k r (the forward k steps grow the
        // region the reverse k steps consume)
        const bool one_d = G.shape.size() == 1;
        G.tile[0] = 1;
        G.tile[1] = one_d ? 1 : (int)opt(DCP_OPT_TILE_Y, G.dtype == DCP_F32 ? 32 : 16);
        G.tile[2] = (int)opt(DCP_OPT_TILE_X, one_d ? 512 : 32);
        G.threads = 256;
        nl += 1;
      } else {
        choose_stencil_tiling(G);
        int S = (int)G.steps.size();
        nl += (S + G.depth - 1) / G.depth;
      }
    }
    g.n_launches = nl;
  }

  int64_t opt(int key, int64_t def) const {
    auto it = g.options.find(key);
    return it == g.options.end() ? def : it->second;
  }

  void choose_stencil_tiling(Group& G) {
    choose_stencil_tiling_impl(G);
    // the warp-stream kernel when it applies (zero / fixed-ring boundary, 1-D
    // or 2-D, radius <= 2); the shared-memory tile kernel otherwise
    int var = stream_eligible(G, G.depth) ? 1 : 0;
    auto it = g.options.find(DCP_OPT_STENCIL_KERNEL);
    if (it != g.options.end()) var = (it->second == 1 && stream_eligible(G, G.depth)) ? 1 : 0;
    if (it != g.options.end() && it->second == 2 && G.kind == GroupKind::Stencil &&
        G.shape.size() <= 2) {
      // cooperative form: every step in one launch on the tile the options
      // (or the defaults) give
      G.depth = (int)G.steps.size();
      if (!coop_eligible(G, G.tile[1], G.tile[2]))
        fail(DCP_E_UNSUPPORTED, "the cooperative stencil form needs at most 63 steps and edge "
                                "tiles at least a radius wide");
      var = 2;
      // one thread per tile cell (64..1024): the tile's cells are independent
      // chains, which a latency-bound small grid needs in flight
      const int cells = (G.shape.size() == 1 ? 1 : G.tile[1]) * G.tile[2];
      G.threads = std::min(1024, std::max(64, (cells + 31) / 32 * 32));
    }
    G.variant = var;
    if (var == 1) {
      G.threads = (int)opt(DCP_OPT_STREAM_THREADS, 64);
      G.prefetch = (int)opt(DCP_OPT_STREAM_PREFETCH, 1);
      G.min_ctas = (int)opt(DCP_OPT_STREAM_MIN_CTAS, 0);
      if (G.kind == GroupKind::Batch) {
        G.seg = 64;  // rows per work item: short, uniform items balance the batch
      } else {
        // rows per work item: enough items to fill the GPU, and at least
        // 8 * depth * radius rows so warm-up rows stay a small fraction
        int64_t ny = G.shape.size() == 2 ? G.shape[0] : 1;
        int64_t nx = G.shape.back();
        int64_t strips = (nx + stream_width(G) - 1) / stream_width(G);
        int64_t target_items = 152 * 16;
        int64_t seg = (ny * strips + target_items - 1) / target_items;
        seg = std::max<int64_t>(seg, 8 * G.depth * std::max(1, G.radius[1]));
        G.seg = (int)std::min<int64_t>(std::max<int64_t>(seg, 1), std::max<int64_t>(ny, 1));
      }
      auto so = g.options.find(DCP_OPT_STREAM_ROWS);
      if (so != g.options.end()) G.seg = (int)so->second;
    }
  }

  void choose_stencil_tiling_impl(Group& G) {
    int S = (int)G.steps.size();
    bool tt = flags & DCP_TIME_TILE;
    int nd = G.kind == GroupKind::Batch ? 2 : (int)G.shape.size();
    int depth = 1;
    if (tt && nd <= 2) depth = std::min(S, G.dtype == DCP_F32 ? 4 : 2);
    depth = (int)opt(DCP_OPT_TIME_TILE_DEPTH, depth);
    if (nd == 3) depth = 1;  // 3-D kernels stream planes one step at a time
    depth = std::max(1, std::min(depth, S));
    G.depth = depth;
    if (nd == 3) {
      G.tile[0] = (int)opt(DCP_OPT_TILE_Z, 16);  // z chunk
      G.tile[1] = (int)opt(DCP_OPT_TILE_Y, 8);
      G.tile[2] = (int)opt(DCP_OPT_TILE_X, 32);
      // two cells per thread along x (two independent FP64 chains per
      // thread, aligned pair loads) where the tile and radius allow it
      const bool pairs_ok = G.tile[2] % 2 == 0 && G.radius[2] <= 2;
      G.cx = pairs_ok ? (int)opt(DCP_OPT_CELLS_PER_THREAD, 2) : 1;
      G.threads = 256;
    } else {
      G.tile[0] = 1;
      G.tile[1] = (int)opt(DCP_OPT_TILE_Y, 32);
      G.tile[2] = (int)opt(DCP_OPT_TILE_X, G.dtype == DCP_F32 ? 64 : 32);
      G.threads = 256;
    }
  }

};

}  // namespace

bool coop_eligible(const Group& G, int ty, int tx) {
  const int nd = (int)G.shape.size();
  if (G.kind != GroupKind::Stencil || nd > 2 || G.steps.empty() || G.steps.size() > 63) return false;
  const int64_t ny = nd == 2 ? G.shape[0] : 1, nx = G.shape.back();
  if (nd == 1) ty = 1;
  const int ry = nd == 2 ? G.radius[1] : 0, rx = G.radius[2];
  if (ty < std::max(1, ry) || tx < std::max(1, rx) || ny < 1 || nx < 1) return false;
  // the halo must come from the adjacent tiles only
  const int64_t ey = ny % ty, ex = nx % tx;
  if ((ey != 0 && ey < ry) || (ex != 0 && ex < rx)) return false;
  if (ny < ry || nx < rx) return false;
  return true;
}

bool stream_eligible(const Group& G, int depth) {
  const int nd = G.kind == GroupKind::Batch ? 2 : (int)G.shape.size();
  if (nd > 2 || G.bc == DCP_BC_PERIODIC) return false;
  if (G.radius[1] > 2 || G.radius[2] > 2) return false;
  const int C = stream_cols_per_lane(G.dtype);
  if (G.radius[2] > C) return false;
  return 32 * C - 2 * depth * G.radius[2] >= 8;
}

void plan_graph(GraphImpl& g, uint32_t flags) {
  g.flags = flags;
  g.batch_store.clear();
  Planner p(g, flags);
  p.plan();
}

}  // namespace dcp
