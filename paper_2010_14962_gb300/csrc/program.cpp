#include "program.hpp"

#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <numeric>

namespace qtn {

namespace {

using Set = std::vector<int>;  // sorted ids: real index i < I, inner class c as I + c

Set set_and(const Set& a, const Set& b) {
  Set r;
  std::set_intersection(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(r));
  return r;
}
Set set_minus(const Set& a, const Set& b) {
  Set r;
  std::set_difference(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(r));
  return r;
}
Set set_or(const Set& a, const Set& b) {
  Set r;
  std::set_union(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(r));
  return r;
}
Set concat(const Set& a, const Set& b) {
  Set r = a;
  r.insert(r.end(), b.begin(), b.end());
  return r;
}

// First-fit allocator over a linear arena of elements.
struct Arena {
  std::map<uint64_t, uint64_t> used;  // offset -> size
  uint64_t high = 0;
  uint64_t alloc(uint64_t size) {
    uint64_t at = 0;
    for (const auto& [off, sz] : used) {
      if (off >= at + size) break;
      at = std::max(at, off + sz);
    }
    used[at] = size;
    high = std::max(high, at + size);
    return at;
  }
  void release(uint64_t off) { used.erase(off); }
};

int find_root(std::vector<int>& parent, int x) {
  while (parent[x] != x) x = parent[x] = parent[parent[x]];
  return x;
}

}  // namespace

std::vector<int> cut_classes(const Network& net, const std::vector<int>& cuts, int* n_classes) {
  const int k = (int)cuts.size();
  std::vector<int> cut_no(net.indices.size(), -1);
  for (int j = 0; j < k; ++j) cut_no[cuts[j]] = j;
  std::vector<int> parent(k);
  std::iota(parent.begin(), parent.end(), 0);
  // The in and out segment of a wire through a diagonal gate (ket slots w,
  // 2 + w; in the density form also the bra slots 4 + w, 6 + w).
  for (const Gate& g : net.gates)
    for (int d = 0; d < (g.kind != GATE_ZZ ? 0 : net.density ? 8 : 4); d += 4)
      for (int w = 0; w < 2; ++w) {
        if (g.out_kind[w] != OUT_PLAIN || g.leg[d + w] < 0 || g.leg[d + 2 + w] < 0) continue;
        int a = cut_no[g.leg[d + w]], b = cut_no[g.leg[d + 2 + w]];
        if (a >= 0 && b >= 0) parent[find_root(parent, a)] = find_root(parent, b);
      }
  std::map<int, int> id;
  std::vector<int> cls(k);
  for (int j = 0; j < k; ++j) {
    int r = find_root(parent, j);
    auto it = id.find(r);
    if (it == id.end()) it = id.emplace(r, (int)id.size()).first;
    cls[j] = it->second;
  }
  *n_classes = (int)id.size();
  return cls;
}

std::string compile_program(const Network& net, const Plan& plan_in, const ProgramOptions& opt, Program* out) {
  Plan plan = plan_in;
  const int L = plan.n_leaves;
  const int I = (int)net.indices.size();
  const int K = (int)plan.cuts.size();
  Program pg;
  pg.n = net.n;
  pg.p = net.p;
  pg.k = K;
  pg.density = net.density;

  // Classes and their outer / inner positions.
  std::vector<int> cls = opt.cut_class;
  if (cls.empty()) {
    cls.resize(K);
    std::iota(cls.begin(), cls.end(), 0);
  }
  if ((int)cls.size() != K) return "cut_class must have one entry per cut";
  pg.n_classes = K ? *std::max_element(cls.begin(), cls.end()) + 1 : 0;
  std::vector<int> cls_pos(pg.n_classes, -1);
  std::vector<char> is_inner(pg.n_classes, 0);
  for (int c = 0; c < pg.n_classes; ++c) is_inner[c] = c < (int)opt.inner.size() && opt.inner[c];
  for (int c = 0; c < pg.n_classes; ++c) {
    if (is_inner[c]) {
      cls_pos[c] = (int)pg.inner_class.size();
      pg.inner_class.push_back(c);
    } else {
      cls_pos[c] = (int)pg.outer_class.size();
      pg.outer_class.push_back(c);
    }
  }
  pg.n_inner = (int)pg.inner_class.size();
  pg.n_outer = (int)pg.outer_class.size();
  if (pg.n_outer > 62) return "too many outer slice classes";
  std::vector<int> cut_no(I, -1);
  for (int j = 0; j < K; ++j) cut_no[plan.cuts[j]] = j;

  // A network of one tensor has no merge: multiply it by a constant 1.
  bool unit_leaf = false;
  if (plan.merges.empty()) {
    unit_leaf = true;
    plan.tensors.insert(plan.tensors.begin() + L, Set{});
    plan.merges.push_back({0, L, L + 1});
    plan.tensors.push_back(plan.tensors[0]);
    if (!plan.tensors[0].empty()) return "single-tensor network must be closed";
  }
  const int n_leaves = L + (unit_leaf ? 1 : 0);
  const int T = (int)plan.tensors.size();
  auto is_leaf = [&](int t) { return t < n_leaves; };
  auto leaf_gate = [&](int t) -> const Gate* { return (unit_leaf && t == L) ? nullptr : &net.gates[t]; };

  // Full index set of every tensor: real open indices + inner classes below it.
  std::vector<Set> full(T);
  for (int t = 0; t < n_leaves; ++t) {
    Set f = plan.tensors[t];
    if (const Gate* g = leaf_gate(t))
      for (int s = 0; s < kMaxLegs; ++s)
        if (g->leg[s] >= 0 && cut_no[g->leg[s]] >= 0 && is_inner[cls[cut_no[g->leg[s]]]])
          f.push_back(I + cls[cut_no[g->leg[s]]]);
    std::sort(f.begin(), f.end());
    f.erase(std::unique(f.begin(), f.end()), f.end());
    full[t] = f;
  }
  struct Canon {
    Set m, n, k, b;
  };
  std::vector<Canon> canon(plan.merges.size());
  for (size_t j = 0; j < plan.merges.size(); ++j) {
    const Merge& mg = plan.merges[j];
    const Set& A = full[mg.a];
    const Set& B = full[mg.b];
    Canon& c = canon[j];
    // Shared real indices are summed unless the result keeps them (an index
    // held by a third tensor, graphical-model form): those are batch bits.
    Set shared = set_and(A, B);
    const Set& kept = plan.tensors[mg.c];
    for (int x : shared)
      (x < I && !std::binary_search(kept.begin(), kept.end(), x) ? c.k : c.b).push_back(x);
    c.m = set_minus(A, B);
    c.n = set_minus(B, A);
    Set vC = set_or(set_minus(A, c.k), set_minus(B, c.k));
    full[mg.c] = vC;
    const int max_rank = opt.wide ? kWideMaxRank : kMaxRank;
    if ((int)(c.m.size() + c.k.size() + c.b.size()) > max_rank ||
        (int)(c.n.size() + c.k.size() + c.b.size()) > max_rank || (int)vC.size() > max_rank)
      return opt.wide ? "a tensor of rank > 34 is beyond the wide executor"
                      : "a tensor of rank > 16 is beyond the on-chip executors";
  }

  // Contraction tree, DFS order visiting the needier child first.
  std::vector<int> producer(T, -1);
  for (size_t j = 0; j < plan.merges.size(); ++j) producer[plan.merges[j].c] = (int)j;
  const int root = plan.merges.back().c;
  auto elems = [&](int t) -> double { return is_leaf(t) ? 0.0 : std::ldexp(1.0, (int)full[t].size()); };
  std::vector<double> need(T, 0.0);
  std::vector<char> first_is_a(T, 1);
  for (const Merge& m : plan.merges) {
    double sa = elems(m.a), sb = elems(m.b), sc = elems(m.c);
    double ab = std::max({need[m.a], sa + need[m.b], sa + sb + sc});
    double ba = std::max({need[m.b], sb + need[m.a], sa + sb + sc});
    first_is_a[m.c] = ab <= ba;
    need[m.c] = std::min(ab, ba);
  }
  std::vector<int> order;
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

  // Storage layout of each operand: its consumer's canonical order.
  std::vector<Set> layout(T);
  for (size_t j = 0; j < plan.merges.size(); ++j) {
    const Merge& mg = plan.merges[j];
    const Canon& c = canon[j];
    layout[mg.a] = concat(concat(c.m, c.k), c.b);
    layout[mg.b] = concat(concat(c.k, c.n), c.b);
  }

  // Leaves: [consumer layout | outer classes of the cut legs].
  pg.leaves.resize(n_leaves);
  uint32_t leaf_off = 0;
  for (int t = 0; t < n_leaves; ++t) {
    DevLeaf lf{};
    lf.base = leaf_off;
    const Gate* g = leaf_gate(t);
    if (!g) {
      lf.gate = -1;
    } else {
      lf.gate = (int16_t)t;
      int pos = 0;
      auto slots_of = [&](int id) -> uint8_t {
        uint8_t mask = 0;
        for (int s = 0; s < kMaxLegs; ++s) {
          int ix = g->leg[s];
          if (ix < 0) continue;
          if (id < I ? ix == id : (cut_no[ix] >= 0 && cls[cut_no[ix]] == id - I)) mask |= (uint8_t)(1u << s);
        }
        return mask;
      };
      for (int id : layout[t]) {
        uint8_t mask = slots_of(id);
        if (!mask) return "leaf layout refers to an index the gate does not carry";
        lf.slot_mask[pos++] = mask;
      }
      lf.rank_nc = (uint8_t)pos;
      std::vector<std::pair<int, int>> outer;  // (outer position, class)
      for (int s = 0; s < kMaxLegs; ++s) {
        int ix = g->leg[s];
        if (ix < 0 || cut_no[ix] < 0) continue;
        int c = cls[cut_no[ix]];
        if (!is_inner[c]) outer.push_back({cls_pos[c], c});
      }
      std::sort(outer.begin(), outer.end());
      outer.erase(std::unique(outer.begin(), outer.end()), outer.end());
      if ((int)outer.size() > kMaxLeafCuts || pos + (int)outer.size() > 8) return "too many cut legs on one gate";
      lf.ncut = (uint8_t)outer.size();
      for (size_t j = 0; j < outer.size(); ++j) {
        lf.cut_bit[j] = (uint8_t)outer[j].first;
        lf.slot_mask[pos++] = slots_of(I + outer[j].second);
      }
    }
    pg.max_rank = std::max(pg.max_rank, (int)lf.rank_nc);
    leaf_off += 1u << (lf.rank_nc + lf.ncut);
    pg.leaves[t] = lf;
  }

  // Hoisting: merges reached by no outer-class cut leg.
  std::vector<char> dep_outer(T, 0), pro(plan.merges.size(), 0), exported(T, 0);
  for (int t = 0; t < n_leaves; ++t) dep_outer[t] = pg.leaves[t].ncut > 0;
  for (const Merge& m : plan.merges) dep_outer[m.c] = dep_outer[m.a] || dep_outer[m.b];
  const bool hoist = opt.hoist && pg.n_outer > 0;
  std::vector<int> consumer(T, -1);
  for (size_t j = 0; j < plan.merges.size(); ++j) {
    consumer[plan.merges[j].a] = (int)j;
    consumer[plan.merges[j].b] = (int)j;
    if (hoist && !dep_outer[plan.merges[j].c]) pro[j] = 1;
  }
  std::vector<int> leaf_id(T, -1);  // leaves and pseudo-leaves
  for (int t = 0; t < n_leaves; ++t) leaf_id[t] = t;
  for (size_t j = 0; j < plan.merges.size(); ++j) {
    const int c = plan.merges[j].c;
    if (pro[j] && consumer[c] >= 0 && !pro[consumer[c]]) {
      exported[c] = 1;
      DevLeaf lf{};
      lf.base = leaf_off;
      lf.gate = -2;
      lf.rank_nc = (uint8_t)layout[c].size();
      lf.ncut = 0;
      if ((uint64_t)leaf_off + (1ull << lf.rank_nc) > 0xffffffffull) return "leaf table beyond 2^32 elements";
      leaf_off += 1u << lf.rank_nc;
      leaf_id[c] = (int)pg.leaves.size();
      pg.leaves.push_back(lf);
    }
  }
  pg.leaf_elems = leaf_off;

  // Item steps and prologue steps by level (stable: DFS order within a
  // level).  For the items, leaves and hoisted results are level 0.
  std::vector<int> item_order, pro_order;
  for (int j : order) (pro[j] ? pro_order : item_order).push_back(j);
  std::vector<int> level_of(plan.merges.size(), 0);
  if (opt.levels) {
    std::vector<int> lev_t(T, 0);
    for (const std::vector<int>* seq : {&pro_order, &item_order}) {
      for (int j : *seq) {
        const Merge& mg = plan.merges[j];
        auto lv = [&](int t) { return (is_leaf(t) || (!pro[j] && exported[t])) ? 0 : lev_t[t]; };
        lev_t[mg.c] = 1 + std::max(lv(mg.a), lv(mg.b));
        level_of[j] = lev_t[mg.c];
      }
    }
    std::stable_sort(pro_order.begin(), pro_order.end(), [&](int x, int y) { return level_of[x] < level_of[y]; });
    if (opt.level_budget == 0)
      std::stable_sort(item_order.begin(), item_order.end(),
                       [&](int x, int y) { return level_of[x] < level_of[y]; });
  }
  // Memory-bounded levels (level_budget > 0): list scheduling along the
  // depth-first order.  Each level takes, in depth-first order, every step
  // whose operands are ready (leaves, hoisted results, earlier levels) while
  // its result still fits in the arena budget (the first ready step always
  // does); a level's inputs are freed when it ends.  The allocation is
  // simulated with the same first-fit arena and the same calls as the
  // emission below, so the emitted program has exactly this arena.
  std::vector<int> item_level;  // level of each item step, in emission order
  constexpr size_t kLevelWindow = 12;
  if (opt.levels && opt.level_budget > 0) {
    std::vector<int> rem = item_order, bseq;
    Arena sim;
    std::vector<uint64_t> at(T, 0);
    std::vector<char> avail(T, 0), taken(plan.merges.size(), 0);
    for (int t = 0; t < T; ++t) avail[t] = is_leaf(t) || exported[t];
    int lev = 0;
    while (!rem.empty()) {
      std::vector<uint64_t> rel;
      std::vector<int> outs, keep;
      bool took = false;
      for (size_t q = 0; q < rem.size(); ++q) {
        const int j = rem[q];
        const Merge& mg = plan.merges[j];
        // Look ahead only a few remaining steps: results taken far ahead of
        // their depth-first turn stay alive long and raise the arena.
        if (q >= kLevelWindow || !avail[mg.a] || !avail[mg.b]) {
          keep.push_back(j);
          continue;
        }
        if (mg.c != root) {
          const Canon& c = canon[j];
          const uint64_t size = 1ull << (c.m.size() + c.n.size() + c.b.size());
          const uint64_t off = sim.alloc(size);
          if (took && off + size > opt.level_budget) {
            sim.release(off);
            keep.push_back(j);
            continue;
          }
          at[mg.c] = off;
        }
        took = true;
        bseq.push_back(j);
        item_level.push_back(lev);
        if (!(is_leaf(mg.a) || exported[mg.a])) rel.push_back(at[mg.a]);
        if (!(is_leaf(mg.b) || exported[mg.b])) rel.push_back(at[mg.b]);
        outs.push_back(mg.c);
      }
      for (uint64_t r : rel) sim.release(r);
      for (int t : outs) avail[t] = 1;
      rem.swap(keep);
      ++lev;
    }
    item_order = bseq;
  }

  std::vector<uint64_t> where(T, 0);
  auto emit = [&](bool prologue_pass, bool c_reuses_a, std::vector<DevStep>* out, std::vector<WideStep>* wout,
                  uint64_t* arena_high, double* macs) -> std::string {
    Arena arena;
    const bool by_level = opt.levels;
    const bool bounded = by_level && !prologue_pass && opt.level_budget > 0;
    std::vector<uint64_t> level_release;  // inputs freed when their level ends
    const std::vector<int>& seq = prologue_pass ? pro_order : item_order;
    auto level_at = [&](size_t si) { return bounded ? item_level[si] : level_of[seq[si]]; };
    for (size_t si = 0; si < seq.size(); ++si) {
      const int j = seq[si];
      if ((bool)pro[j] != prologue_pass) continue;
      const Merge& mg = plan.merges[j];
      const Canon& c = canon[j];
      DevStep st{};
      WideStep ws{};
      st.ma = (uint8_t)c.m.size();
      st.nb = (uint8_t)c.n.size();
      st.kb = (uint8_t)c.k.size();
      st.bb = (uint8_t)c.b.size();
      std::vector<uint64_t> to_release;
      int64_t a_block = -1;
      auto as_leaf = [&](int t) { return is_leaf(t) || (!prologue_pass && exported[t]); };
      if (as_leaf(mg.a)) {
        st.flags |= STEP_A_LEAF;
        ws.a = (uint64_t)leaf_id[mg.a];
      } else {
        ws.a = where[mg.a];
        a_block = (int64_t)where[mg.a];
      }
      if (as_leaf(mg.b)) {
        st.flags |= STEP_B_LEAF;
        ws.b = (uint64_t)leaf_id[mg.b];
      } else {
        ws.b = where[mg.b];
        to_release.push_back(where[mg.b]);
      }
      st.a = (uint32_t)ws.a;
      st.b = (uint32_t)ws.b;
      const int rc = (int)(c.m.size() + c.n.size() + c.b.size());
      const int wd = rc + (int)c.k.size();
      pg.width = std::max(pg.width, wd);
      pg.max_rank = std::max(pg.max_rank, rc);
      *macs += std::ldexp(1.0, wd);
      // A is read completely before the first store of C; B may be read
      // while C is written, so only A's block may be reused by C.  Within a
      // level nothing is reused: its merges run at the same time.
      if (a_block >= 0) {
        if (c_reuses_a && !by_level) arena.release((uint64_t)a_block);
        else to_release.push_back((uint64_t)a_block);
      }
      const Set canon_ix = concat(concat(c.m, c.n), c.b);
      if (mg.c == root) {
        st.flags |= STEP_ROOT;
        st.c = 0;
        for (int id : canon_ix) {
          if (id < I) return "the root keeps a real index open";
          pg.root_class.push_back(id - I);
        }
      } else {
        if (prologue_pass && exported[mg.c]) {
          st.flags |= STEP_EXPORT;
          ws.c = (uint64_t)leaf_id[mg.c];
        } else {
          const uint64_t off = arena.alloc(1ull << rc);
          where[mg.c] = off;
          ws.c = off;
        }
        st.c = (uint32_t)ws.c;
        const Set& lay = layout[mg.c];
        for (int b = 0; b < rc; ++b) {
          auto it = std::find(lay.begin(), lay.end(), canon_ix[b]);
          if (it == lay.end()) return "consumer layout misses an index";
          ws.wpos[b] = (uint8_t)(it - lay.begin());
          if (!opt.wide) st.w[b] = (uint16_t)(1u << (it - lay.begin()));
        }
      }
      if (by_level) {
        level_release.insert(level_release.end(), to_release.begin(), to_release.end());
        const bool level_ends = si + 1 == seq.size() || level_at(si + 1) != level_at(si);
        if (level_ends) {
          for (uint64_t r : level_release) arena.release(r);
          level_release.clear();
        }
      } else {
        for (uint64_t r : to_release) arena.release(r);
      }
      ws.ma = st.ma;
      ws.nb = st.nb;
      ws.kb = st.kb;
      ws.bb = st.bb;
      ws.flags = st.flags;
      if (opt.wide) wout->push_back(ws);
      else out->push_back(st);
    }
    *arena_high = std::max<uint64_t>(arena.high, 1);
    return "";
  };
  uint64_t pro_high = 0, item_high = 0;
  std::string err = emit(true, false, &pg.prologue, &pg.wide_prologue, &pro_high, &pg.macs_prologue);
  if (err.empty())
    err = emit(false, opt.c_reuses_a, &pg.steps, &pg.wide_steps, &item_high, &pg.macs_per_item);
  if (!err.empty()) return err;
  if (opt.wide) {
    if (opt.levels) return "wide programs have no levels";
    pg.wide_arena_elems = item_high;
    pg.wide_pro_arena_elems = pg.wide_prologue.empty() ? 0 : pro_high;
  } else {
    if (item_high > 0xffffffffull || pro_high > 0xffffffffull) return "arena beyond 2^32 elements";
    pg.arena_elems = (uint32_t)item_high;
    pg.pro_arena_elems = (uint32_t)pro_high;
  }
  if (pg.prologue.empty()) pg.pro_arena_elems = 0;
  if (opt.levels) {
    // Level of emitted step i: its depth, or its bounded level.
    std::vector<int> item_lv(pg.steps.size()), pro_lv(pg.prologue.size());
    for (size_t i = 0; i < pg.steps.size(); ++i)
      item_lv[i] = opt.level_budget > 0 ? item_level[i] : level_of[item_order[i]];
    for (size_t i = 0; i < pg.prologue.size(); ++i) pro_lv[i] = level_of[pro_order[i]];
    auto tables = [&](const std::vector<DevStep>& steps, const std::vector<int>& seq, std::vector<DevLevel>* levels,
                      std::vector<uint32_t>* out_start) -> std::string {
      out_start->assign(2 * steps.size(), 0);
      for (size_t i = 0; i < steps.size(); ++i) {
        const DevStep& st = steps[i];
        const int rc = st.ma + st.nb + st.bb;
        // Four-output table: the root's outputs are summed, not stored, so
        // its sum over k is split too.
        const int split = (st.flags & STEP_ROOT) ? std::min<int>(st.kb, kRootSplitLog2) : 0;
        if (i == 0 || seq[i] != seq[i - 1]) {
          if (levels->size() >= 0xffff) return "too many levels";
          levels->push_back(DevLevel{(uint16_t)i, 0, {0, 0}});
        }
        DevLevel& lv = levels->back();
        for (int u = 0; u < 2; ++u) {
          const uint32_t units = 1u << std::max(0, rc + (u ? split - kLevelUnitLog2 : 0));
          // Executors index (unit, item) pairs of a level in 32 bits, <= 32 items.
          if ((uint64_t)lv.units[u] + units > (1ull << 26)) return "level too large";
          (*out_start)[2 * i + u] = lv.units[u];
          lv.units[u] += units;
        }
        ++lv.count;
      }
      return "";
    };
    err = tables(pg.steps, item_lv, &pg.levels, &pg.out_start);
    if (err.empty()) err = tables(pg.prologue, pro_lv, &pg.pro_levels, &pg.pro_out_start);
    if (!err.empty()) return err;
    auto nibbles = [](const std::vector<DevStep>& steps, std::vector<uint16_t>* out) {
      out->assign(steps.size() * kPosNibEntries, 0);
      for (size_t i = 0; i < steps.size(); ++i) {
        const DevStep& st = steps[i];
        const int rc = st.ma + st.nb + st.bb;
        if (st.flags & STEP_ROOT) continue;
        for (int g = 0; g < 4; ++g)
          for (int v = 0; v < 16; ++v) {
            uint32_t pos = 0;
            for (int b = 0; b < 4; ++b)
              if (((v >> b) & 1) && 4 * g + b < rc) pos += st.w[4 * g + b];
            (*out)[i * kPosNibEntries + 16 * g + v] = (uint16_t)pos;
          }
      }
    };
    nibbles(pg.steps, &pg.pos_nib);
    nibbles(pg.prologue, &pg.pro_pos_nib);
  }

  pg.gate_q.resize(2 * net.gates.size());
  pg.gate_layer.resize(net.gates.size());
  pg.gate_in_h.resize(2 * net.gates.size());
  pg.gate_out_kind.resize(2 * net.gates.size());
  pg.gate_kind.resize(net.gates.size());
  for (size_t g = 0; g < net.gates.size(); ++g) {
    for (int w = 0; w < 2; ++w) {
      pg.gate_q[2 * g + w] = net.gates[g].q[w];
      pg.gate_in_h[2 * g + w] = net.gates[g].in_h[w];
      pg.gate_out_kind[2 * g + w] = net.gates[g].out_kind[w];
    }
    pg.gate_layer[g] = (int8_t)net.gates[g].layer;
    pg.gate_kind[g] = net.gates[g].kind;
  }
  *out = std::move(pg);
  return "";
}

ProgramOptions choose_batched(const Network& net, const Plan& plan, uint32_t smem_elems, uint64_t min_items) {
  ProgramOptions opt;
  int nc = 0;
  opt.cut_class = cut_classes(net, plan.cuts, &nc);
  opt.inner.assign(nc, 0);
  auto per_slice = [&](const ProgramOptions& o, Program* pg) -> double {
    if (!compile_program(net, plan, o, pg).empty()) return -1.0;
    if (pg->arena_elems + pg->leaf_elems > smem_elems) return -1.0;
    return pg->macs_per_item / std::ldexp(1.0, pg->n_inner);
  };
  Program cur;
  double best = per_slice(opt, &cur);
  int n_inner = 0;
  while (true) {
    if (std::ldexp(1.0, nc - n_inner - 1) < (double)min_items) break;
    int pick = -1;
    double pick_cost = best;
    for (int c = 0; c < nc; ++c) {
      if (opt.inner[c]) continue;
      ProgramOptions trial = opt;
      trial.inner[c] = 1;
      Program pg;
      double v = per_slice(trial, &pg);
      if (v >= 0 && v < pick_cost * 0.97) {
        pick_cost = v;
        pick = c;
      }
    }
    if (pick < 0) break;
    opt.inner[pick] = 1;
    best = pick_cost;
    ++n_inner;
  }
  return opt;
}

}  // namespace qtn
