#include "program.hpp"

#include <algorithm>
#include <cmath>
#include <functional>
#include <map>

namespace qtn {

namespace {

std::vector<int> set_and(const std::vector<int>& a, const std::vector<int>& b) {
  std::vector<int> r;
  std::set_intersection(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(r));
  return r;
}
std::vector<int> set_minus(const std::vector<int>& a, const std::vector<int>& b) {
  std::vector<int> r;
  std::set_difference(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(r));
  return r;
}

// First-fit allocator over a linear arena of elements.
struct Arena {
  std::map<uint32_t, uint32_t> used;  // offset -> size
  uint32_t high = 0;
  uint32_t alloc(uint32_t size) {
    uint32_t at = 0;
    for (const auto& [off, sz] : used) {
      if (off >= at + size) break;
      at = std::max(at, off + sz);
    }
    used[at] = size;
    high = std::max(high, at + size);
    return at;
  }
  void release(uint32_t off) { used.erase(off); }
};

}  // namespace

std::string compile_program(const Network& net, const Plan& plan_in, bool c_reuses_operands,
                            Program* out) {
  Plan plan = plan_in;
  const int L = plan.n_leaves;
  Program pg;
  pg.n = net.n;
  pg.p = net.p;
  pg.k = (int)plan.cuts.size();

  // A network of one tensor has no merge: multiply it by a constant 1.
  bool unit_leaf = false;
  if (plan.merges.empty()) {
    unit_leaf = true;
    plan.tensors.insert(plan.tensors.begin() + L, std::vector<int>{});
    // shift intermediate ids (there are none) and add the merge
    plan.merges.push_back({0, L, L + 1});
    plan.tensors.push_back(plan.tensors[0]);  // rank of leaf 0 must be 0 here
    if (!plan.tensors[0].empty()) return "single-tensor network must be closed";
  }
  const int n_leaves = L + (unit_leaf ? 1 : 0);
  const int T = (int)plan.tensors.size();
  auto is_leaf = [&](int t) { return t < n_leaves; };

  // Contraction tree.
  std::vector<int> producer(T, -1);
  for (size_t j = 0; j < plan.merges.size(); ++j) producer[plan.merges[j].c] = (int)j;
  const int root = plan.merges.back().c;
  auto elems = [&](int t) -> double { return is_leaf(t) ? 0.0 : std::ldexp(1.0, (int)plan.tensors[t].size()); };

  // Peak arena need of each subtree, visiting the needier child first.
  std::vector<double> need(T, 0.0);
  std::vector<char> first_is_a(T, 1);
  for (const Merge& m : plan.merges) {
    double sa = elems(m.a), sb = elems(m.b), sc = elems(m.c);
    double ab = std::max({need[m.a], sa + need[m.b], sa + sb + sc});
    double ba = std::max({need[m.b], sb + need[m.a], sa + sb + sc});
    first_is_a[m.c] = ab <= ba;
    need[m.c] = std::min(ab, ba);
  }
  std::vector<int> order;  // merge ids in execution order
  std::function<void(int)> visit = [&](int t) {
    if (producer[t] < 0) return;
    const Merge& m = plan.merges[producer[t]];
    if (first_is_a[t]) {
      visit(m.a);
      visit(m.b);
    } else {
      visit(m.b);
      visit(m.a);
    }
    order.push_back(producer[t]);
  };
  visit(root);
  if (order.size() != plan.merges.size()) return "contraction tree is not connected to its root";

  // Canonical lists per merge, and the storage layout of every operand.
  struct Canon {
    std::vector<int> m, n, k;
  };
  std::vector<Canon> canon(plan.merges.size());
  std::vector<std::vector<int>> layout(T);
  for (size_t j = 0; j < plan.merges.size(); ++j) {
    const Merge& mg = plan.merges[j];
    const auto& A = plan.tensors[mg.a];
    const auto& B = plan.tensors[mg.b];
    Canon& c = canon[j];
    c.k = set_and(A, B);
    c.m = set_minus(A, B);
    c.n = set_minus(B, A);
    if (c.m.size() + c.k.size() > 16 || c.n.size() + c.k.size() > 16 || c.m.size() + c.n.size() > 16)
      return "a tensor of rank > 16 is beyond the on-chip executors";
    layout[mg.a] = c.m;
    layout[mg.a].insert(layout[mg.a].end(), c.k.begin(), c.k.end());
    layout[mg.b] = c.k;
    layout[mg.b].insert(layout[mg.b].end(), c.n.begin(), c.n.end());
  }

  // Leaves: [open legs in consumer order | cut legs by cut number].
  std::vector<int> cut_no(net.indices.size(), -1);
  for (size_t j = 0; j < plan.cuts.size(); ++j) cut_no[plan.cuts[j]] = (int)j;
  pg.leaves.resize(n_leaves);
  uint32_t leaf_off = 0;
  for (int t = 0; t < n_leaves; ++t) {
    DevLeaf lf{};
    lf.base = leaf_off;
    for (int b = 0; b < 8; ++b) lf.slot_of_bit[b] = -1;
    if (unit_leaf && t == L) {
      lf.gate = -1;
      lf.rank_nc = 0;
      lf.ncut = 0;
    } else {
      const Gate& g = net.gates[t];
      lf.gate = (int16_t)t;
      const auto& lay = layout[t];
      lf.rank_nc = (uint8_t)lay.size();
      int pos = 0;
      for (int ix : lay) {
        int slot = -1;
        for (int s = 0; s < 4; ++s)
          if (g.leg[s] == ix) slot = s;
        if (slot < 0) return "leaf layout refers to an index the gate does not carry";
        lf.slot_of_bit[pos++] = (int8_t)slot;
      }
      std::vector<std::pair<int, int>> cuts_here;  // (cut number, slot)
      for (int s = 0; s < 4; ++s)
        if (g.leg[s] >= 0 && cut_no[g.leg[s]] >= 0) cuts_here.push_back({cut_no[g.leg[s]], s});
      std::sort(cuts_here.begin(), cuts_here.end());
      if ((int)cuts_here.size() > kMaxLeafCuts) return "too many cut legs on one gate";
      lf.ncut = (uint8_t)cuts_here.size();
      for (size_t j = 0; j < cuts_here.size(); ++j) {
        lf.cut_bit[j] = (uint8_t)cuts_here[j].first;
        lf.slot_of_bit[pos++] = (int8_t)cuts_here[j].second;
      }
    }
    pg.max_rank = std::max(pg.max_rank, (int)lf.rank_nc);
    leaf_off += 1u << (lf.rank_nc + lf.ncut);
    pg.leaves[t] = lf;
  }
  pg.leaf_elems = leaf_off;

  Arena arena;
  pg.c_reuses_operands = c_reuses_operands;
  std::vector<uint32_t> to_release;
  std::vector<uint32_t> where(T, 0);
  for (int j : order) {
    const Merge& mg = plan.merges[j];
    const Canon& c = canon[j];
    DevStep st{};
    int64_t a_block = -1;
    st.ma = (uint8_t)c.m.size();
    st.nb = (uint8_t)c.n.size();
    st.kb = (uint8_t)c.k.size();
    st.flags = 0;
    if (is_leaf(mg.a)) {
      st.flags |= STEP_A_LEAF;
      st.a = (uint16_t)mg.a;
    } else {
      st.a = where[mg.a];
      a_block = (int64_t)where[mg.a];
    }
    if (is_leaf(mg.b)) {
      st.flags |= STEP_B_LEAF;
      st.b = (uint16_t)mg.b;
    } else {
      st.b = where[mg.b];
      to_release.push_back(where[mg.b]);
    }
    int rc = (int)(c.m.size() + c.n.size());
    pg.width = std::max(pg.width, (int)(c.m.size() + c.n.size() + c.k.size()));
    pg.max_rank = std::max(pg.max_rank, rc);
    pg.macs_per_slice += std::ldexp(1.0, (int)(c.m.size() + c.n.size() + c.k.size()));
    // A is read completely before the first store of C; B is streamed while
    // C is written, so only A's block may be reused by C.
    if (a_block >= 0) {
      if (c_reuses_operands) arena.release((uint32_t)a_block);
      else to_release.push_back((uint32_t)a_block);
    }
    if (mg.c == root) {
      st.flags |= STEP_ROOT;
      st.c = 0;
    } else {
      uint32_t off = arena.alloc(1u << rc);
      where[mg.c] = off;
      st.c = off;
      // canonical C bit b is index (b < |m| ? m[b] : n[b - |m|]); its storage
      // bit is its position in C's consumer layout.
      std::vector<int> canon_ix = c.m;
      canon_ix.insert(canon_ix.end(), c.n.begin(), c.n.end());
      const auto& lay = layout[mg.c];
      for (int b = 0; b < rc; ++b) {
        auto it = std::find(lay.begin(), lay.end(), canon_ix[b]);
        if (it == lay.end()) return "consumer layout misses an index";
        st.w[b] = (uint16_t)(1u << (it - lay.begin()));
      }
    }
    for (uint32_t r : to_release) arena.release(r);
    to_release.clear();
    pg.steps.push_back(st);
  }
  pg.arena_elems = std::max<uint32_t>(arena.high, 1);

  pg.gate_q.resize(2 * net.gates.size());
  pg.gate_layer.resize(net.gates.size());
  pg.gate_in_h.resize(2 * net.gates.size());
  pg.gate_out_kind.resize(2 * net.gates.size());
  for (size_t g = 0; g < net.gates.size(); ++g) {
    for (int w = 0; w < 2; ++w) {
      pg.gate_q[2 * g + w] = net.gates[g].q[w];
      pg.gate_in_h[2 * g + w] = net.gates[g].in_h[w];
      pg.gate_out_kind[2 * g + w] = net.gates[g].out_kind[w];
    }
    pg.gate_layer[g] = (int8_t)net.gates[g].layer;
  }
  *out = std::move(pg);
  return "";
}

}  // namespace qtn
