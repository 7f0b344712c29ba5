#include "plan.hpp"
#include "program.hpp"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <limits>

namespace qtn {

int Bits::count() const {
  int c = 0;
  for (uint64_t x : w) c += __builtin_popcountll(x);
  return c;
}

std::vector<int> Bits::list() const {
  std::vector<int> r;
  for (size_t i = 0; i < w.size(); ++i) {
    uint64_t x = w[i];
    while (x) {
      r.push_back((int)(i * 64 + __builtin_ctzll(x)));
      x &= x - 1;
    }
  }
  return r;
}

double Plan::log2_flops_total() const {
  return (double)cuts.size() + std::log2(8.0 * macs);
}

double Cost::log2_flops_total() const { return (double)k + std::log2(8.0 * macs); }

namespace {

// Runs the elimination of every non-cut index, by min-fill or by a given
// order, merging the two tensors that hold the eliminated index.  Fills
// `plan` (when non-null) with the merge list and tensor index sets, and
// always fills `cost`.
// With `min_degree` the index whose merged bag is smallest is taken (no fill
// computation: a cheap estimate); `bag_sizes` (optional) receives |A u B| of
// every merge.
std::string eliminate_hyper(const Network& net, const std::vector<char>& is_cut,
                            const std::vector<int>* given_order, Plan* plan, Cost* cost, bool min_degree,
                            std::vector<int>* bag_sizes);

std::string eliminate(const Network& net, const std::vector<char>& is_cut,
                      const std::vector<int>* given_order, Plan* plan, Cost* cost, bool min_degree = false,
                      std::vector<int>* bag_sizes = nullptr) {
  if (net.gm) return eliminate_hyper(net, is_cut, given_order, plan, cost, min_degree, bag_sizes);
  const int I = (int)net.indices.size();
  const int L = (int)net.gates.size();
  const int W = (I + 63) / 64;
  std::vector<Bits> T;
  T.reserve(2 * L);
  for (int g = 0; g < L; ++g) {
    Bits b(I);
    for (int s = 0; s < kMaxLegs; ++s) {
      int e = net.gates[g].leg[s];
      if (e >= 0 && !is_cut[e]) b.set(e);
    }
    T.push_back(std::move(b));
  }
  std::vector<int> rank(L);
  for (int g = 0; g < L; ++g) rank[g] = T[g].count();
  std::vector<std::array<int, 2>> where(I);
  std::vector<char> alive_i(I, 0);
  int n_alive = 0;
  for (int e = 0; e < I; ++e) {
    where[e] = {net.indices[e].tensor[0], net.indices[e].tensor[1]};
    if (!is_cut[e]) {
      alive_i[e] = 1;
      n_alive++;
    }
  }
  std::vector<Bits> adj(I, Bits(I));
  for (int g = 0; g < L; ++g)
    for (int u : T[g].list())
      for (int j = 0; j < W; ++j) adj[u].w[j] |= T[g].w[j];
  std::vector<char> alive_t(L, 1);

  int width = 0, max_rank = 0;
  double macs = 0, live = 0, peak = 0;
  for (int g = 0; g < L; ++g) {
    live += std::ldexp(1.0, rank[g]);
    max_rank = std::max(max_rank, rank[g]);
  }
  peak = live;
  if (plan) {
    plan->merges.clear();
    plan->order.clear();
  }
  size_t order_pos = 0;
  std::vector<uint64_t> onlyA(W), onlyB(W);

  auto merge = [&](int t1, int t2) {
    Bits C(I);
    int u_size = 0;
    for (int j = 0; j < W; ++j) {
      C.w[j] = T[t1].w[j] ^ T[t2].w[j];
      u_size += __builtin_popcountll(T[t1].w[j] | T[t2].w[j]);
    }
    int c = (int)T.size();
    int rc = C.count();
    if (bag_sizes) bag_sizes->push_back(u_size);
    width = std::max(width, u_size);
    max_rank = std::max(max_rank, rc);
    macs += std::ldexp(1.0, u_size);
    live += std::ldexp(1.0, rc);
    peak = std::max(peak, live);
    live -= std::ldexp(1.0, rank[t1]) + std::ldexp(1.0, rank[t2]);
    for (int j = 0; j < W; ++j) {
      uint64_t s = T[t1].w[j] & T[t2].w[j];
      while (s) {
        int u = j * 64 + __builtin_ctzll(s);
        s &= s - 1;
        alive_i[u] = 0;
        n_alive--;
      }
    }
    for (int u : C.list()) {
      for (int h = 0; h < 2; ++h)
        if (where[u][h] == t1 || where[u][h] == t2) where[u][h] = c;
      for (int j = 0; j < W; ++j) adj[u].w[j] |= C.w[j];
    }
    alive_t[t1] = alive_t[t2] = 0;
    alive_t.push_back(1);
    rank.push_back(rc);
    T.push_back(std::move(C));
    if (plan) plan->merges.push_back({t1, t2, c});
    return c;
  };

  while (n_alive > 0) {
    int best = -1;
    if (given_order) {
      while (order_pos < given_order->size() && !alive_i[(*given_order)[order_pos]]) order_pos++;
      if (order_pos == given_order->size()) return "order does not cover every non-cut index";
      best = (*given_order)[order_pos++];
    } else if (min_degree) {
      int best_size = 1 << 30;
      for (int e = 0; e < I; ++e) {
        if (!alive_i[e]) continue;
        const Bits& A = T[where[e][0]];
        const Bits& B = T[where[e][1]];
        int size = 0;
        for (int j = 0; j < W; ++j) size += __builtin_popcountll(A.w[j] | B.w[j]);
        if (size < best_size) {
          best_size = size;
          best = e;
        }
      }
    } else {
      long best_fill = std::numeric_limits<long>::max();
      int best_size = 0;
      for (int e = 0; e < I; ++e) {
        if (!alive_i[e]) continue;
        const Bits& A = T[where[e][0]];
        const Bits& B = T[where[e][1]];
        int size = 0;
        for (int j = 0; j < W; ++j) {
          onlyA[j] = A.w[j] & ~B.w[j];
          onlyB[j] = B.w[j] & ~A.w[j];
          size += __builtin_popcountll(A.w[j] | B.w[j]);
        }
        long fill = 0;
        for (int j = 0; j < W && fill <= best_fill; ++j) {
          uint64_t x = onlyA[j];
          while (x) {
            int u = j * 64 + __builtin_ctzll(x);
            x &= x - 1;
            for (int h = 0; h < W; ++h)
              fill += __builtin_popcountll(onlyB[h] & ~adj[u].w[h]);
          }
        }
        if (fill < best_fill || (fill == best_fill && size < best_size)) {
          best_fill = fill;
          best_size = size;
          best = e;
        }
      }
    }
    if (plan) plan->order.push_back(best);
    merge(where[best][0], where[best][1]);
  }
  // Every remaining live tensor is a scalar (one per connected component,
  // plus leaves whose legs were all cut): multiply them together.
  std::vector<int> rest;
  for (int t = 0; t < (int)T.size(); ++t)
    if (alive_t[t]) rest.push_back(t);
  int acc = rest[0];
  for (size_t i = 1; i < rest.size(); ++i) acc = merge(acc, rest[i]);

  if (cost) {
    cost->width = width;
    cost->max_rank = max_rank;
    cost->macs = macs;
    cost->peak_elems = peak;
  }
  if (plan) {
    plan->n_indices = I;
    plan->n_leaves = L;
    plan->tensors.resize(T.size());
    for (size_t t = 0; t < T.size(); ++t) plan->tensors[t] = T[t].list();
    plan->width = width;
    plan->max_rank = max_rank;
    plan->macs = macs;
    plan->peak_elems = peak;
  }
  return "";
}

// The same elimination when an index may be held by more than two tensors
// (graphical-model form: a variable shared by the diagonal gates of its
// layer).  Eliminating index e merges all tensors that hold it, two at a
// time (lowest ids first); a merge sums every index no other live tensor
// holds, so e is summed by the last merge.  Min-fill counts the pairs of
// e's neighbours that are not yet adjacent.
std::string eliminate_hyper(const Network& net, const std::vector<char>& is_cut,
                            const std::vector<int>* given_order, Plan* plan, Cost* cost, bool min_degree,
                            std::vector<int>* bag_sizes) {
  const int I = (int)net.indices.size();
  const int L = (int)net.gates.size();
  const int W = (I + 63) / 64;
  std::vector<Bits> T;
  T.reserve(3 * L);
  std::vector<std::vector<int>> hold(I);
  for (int g = 0; g < L; ++g) {
    Bits b(I);
    for (int s = 0; s < kMaxLegs; ++s) {
      const int e = net.gates[g].leg[s];
      if (e >= 0 && !is_cut[e] && !b.get(e)) {
        b.set(e);
        hold[e].push_back(g);
      }
    }
    T.push_back(std::move(b));
  }
  std::vector<char> alive_i(I, 0);
  int n_alive = 0;
  for (int e = 0; e < I; ++e)
    if (!is_cut[e]) {
      if (hold[e].size() < 2) return "an index is held by fewer than two tensors";
      alive_i[e] = 1;
      n_alive++;
    }
  std::vector<int> rank(L);
  for (int g = 0; g < L; ++g) rank[g] = T[g].count();
  std::vector<Bits> adj(I, Bits(I));
  for (int g = 0; g < L; ++g)
    for (int u : T[g].list())
      for (int j = 0; j < W; ++j) adj[u].w[j] |= T[g].w[j];
  std::vector<char> alive_t(L, 1);
  int width = 0, max_rank = 0;
  double macs = 0, live = 0, peak = 0;
  for (int g = 0; g < L; ++g) {
    live += std::ldexp(1.0, rank[g]);
    max_rank = std::max(max_rank, rank[g]);
  }
  peak = live;
  if (plan) {
    plan->merges.clear();
    plan->order.clear();
  }

  auto merge = [&](int t1, int t2) {
    Bits C(I);
    int u_size = 0;
    for (int j = 0; j < W; ++j) {
      C.w[j] = T[t1].w[j] | T[t2].w[j];
      u_size += __builtin_popcountll(C.w[j]);
    }
    const int c = (int)T.size();
    for (int u : C.list()) {
      std::vector<int>& h = hold[u];
      h.erase(std::remove_if(h.begin(), h.end(), [&](int t) { return t == t1 || t == t2; }), h.end());
      if (h.empty()) {  // only the merged tensor holds u: summed here
        C.clear(u);
        alive_i[u] = 0;
        n_alive--;
      } else {
        h.push_back(c);
      }
    }
    const int rc = C.count();
    if (bag_sizes) bag_sizes->push_back(u_size);
    width = std::max(width, u_size);
    max_rank = std::max(max_rank, rc);
    macs += std::ldexp(1.0, u_size);
    live += std::ldexp(1.0, rc);
    peak = std::max(peak, live);
    live -= std::ldexp(1.0, rank[t1]) + std::ldexp(1.0, rank[t2]);
    for (int u : C.list())
      for (int j = 0; j < W; ++j) adj[u].w[j] |= C.w[j];
    alive_t[t1] = alive_t[t2] = 0;
    alive_t.push_back(1);
    rank.push_back(rc);
    T.push_back(std::move(C));
    if (plan) plan->merges.push_back({t1, t2, c});
    return c;
  };

  size_t order_pos = 0;
  Bits nb(I);
  while (n_alive > 0) {
    int best = -1;
    if (given_order) {
      while (order_pos < given_order->size() && !alive_i[(*given_order)[order_pos]]) order_pos++;
      if (order_pos == given_order->size()) return "order does not cover every non-cut index";
      best = (*given_order)[order_pos++];
    } else {
      long best_fill = std::numeric_limits<long>::max();
      int best_size = 1 << 30;
      for (int e = 0; e < I; ++e) {
        if (!alive_i[e]) continue;
        for (int j = 0; j < W; ++j) nb.w[j] = 0;
        for (int t : hold[e])
          for (int j = 0; j < W; ++j) nb.w[j] |= T[t].w[j];
        const int size = nb.count();
        long fill = 0;
        if (!min_degree) {
          nb.clear(e);
          for (int u : nb.list()) {
            for (int j = 0; j < W; ++j) fill += __builtin_popcountll(nb.w[j] & ~adj[u].w[j]);
            if (fill / 2 > best_fill) break;
          }
          fill /= 2;
        }
        if (fill < best_fill || (fill == best_fill && size < best_size)) {
          best_fill = fill;
          best_size = size;
          best = e;
        }
      }
    }
    if (plan) plan->order.push_back(best);
    std::vector<int> h = hold[best];
    std::sort(h.begin(), h.end());
    int acc = h[0];
    for (size_t i = 1; i < h.size(); ++i) acc = merge(acc, h[i]);
  }
  std::vector<int> rest;
  for (int t = 0; t < (int)T.size(); ++t)
    if (alive_t[t]) rest.push_back(t);
  int acc = rest[0];
  for (size_t i = 1; i < rest.size(); ++i) acc = merge(acc, rest[i]);

  if (cost) {
    cost->width = width;
    cost->max_rank = max_rank;
    cost->macs = macs;
    cost->peak_elems = peak;
  }
  if (plan) {
    plan->n_indices = I;
    plan->n_leaves = L;
    plan->tensors.resize(T.size());
    for (size_t t = 0; t < T.size(); ++t) plan->tensors[t] = T[t].list();
    plan->width = width;
    plan->max_rank = max_rank;
    plan->macs = macs;
    plan->peak_elems = peak;
  }
  return "";
}

std::string check_cuts(const Network& net, const std::vector<int>& cuts, std::vector<char>* is_cut) {
  const int I = (int)net.indices.size();
  is_cut->assign(I, 0);
  for (int c : cuts) {
    if (c < 0 || c >= I) return "cut index out of range";
    if ((*is_cut)[c]) return "duplicate cut index";
    (*is_cut)[c] = 1;
  }
  return "";
}

}  // namespace

std::string make_plan(const Network& net, const std::vector<int>& cuts,
                      const std::vector<int>& order, Plan* out) {
  std::vector<char> is_cut;
  std::string err = check_cuts(net, cuts, &is_cut);
  if (!err.empty()) return err;
  if ((int)cuts.size() > 62) return "at most 62 cut indices are supported";
  if (!order.empty()) {
    std::vector<char> seen(net.indices.size(), 0);
    size_t expect = 0;
    for (size_t e = 0; e < net.indices.size(); ++e) expect += !is_cut[e];
    if (order.size() != expect) return "order must list every non-cut index exactly once";
    for (int e : order) {
      if (e < 0 || e >= (int)net.indices.size() || is_cut[e] || seen[e])
        return "order must be a permutation of the non-cut indices";
      seen[e] = 1;
    }
  }
  Plan p;
  p.cuts = cuts;
  Cost c;
  err = eliminate(net, is_cut, order.empty() ? nullptr : &order, &p, &c);
  if (!err.empty()) return err;
  *out = std::move(p);
  return "";
}

Cost min_degree_cost(const Network& net, const std::vector<int>& cuts, std::vector<int>* bag_sizes) {
  std::vector<char> is_cut;
  Cost c{};
  c.k = (int)cuts.size();
  if (!check_cuts(net, cuts, &is_cut).empty()) {
    c.width = 1 << 20;
    c.macs = std::numeric_limits<double>::infinity();
    return c;
  }
  eliminate(net, is_cut, nullptr, nullptr, &c, true, bag_sizes);
  return c;
}

Cost plan_cost(const Network& net, const std::vector<int>& cuts) {
  std::vector<char> is_cut;
  Cost c{};
  c.k = (int)cuts.size();
  if (!check_cuts(net, cuts, &is_cut).empty()) {
    c.width = 1 << 20;
    c.macs = std::numeric_limits<double>::infinity();
    return c;
  }
  eliminate(net, is_cut, nullptr, nullptr, &c);
  return c;
}

namespace {
bool better(const Cost& a, const Cost& b) {
  if (a.width != b.width) return a.width < b.width;
  return a.log2_flops_total() < b.log2_flops_total();
}
}  // namespace

std::vector<int> greedy_cuts(const Network& net, int k, const std::vector<int>& start) {
  std::vector<int> cuts = start;
  const int I = (int)net.indices.size();
  while ((int)cuts.size() < k && (int)cuts.size() < I) {
    Plan p;
    make_plan(net, cuts, {}, &p);
    std::vector<char> cand(I, 0), is_cut(I, 0);
    for (int c : cuts) is_cut[c] = 1;
    for (const Merge& m : p.merges) {
      const auto& A = p.tensors[m.a];
      const auto& B = p.tensors[m.b];
      std::vector<int> U;
      std::set_union(A.begin(), A.end(), B.begin(), B.end(), std::back_inserter(U));
      if ((int)U.size() == p.width)
        for (int u : U) cand[u] = 1;
    }
    int best = -1;
    Cost best_cost{};
    for (int e = 0; e < I; ++e) {
      if (!cand[e] || is_cut[e]) continue;
      std::vector<int> trial = cuts;
      trial.push_back(e);
      Cost c = plan_cost(net, trial);
      if (best < 0 || better(c, best_cost)) {
        best = e;
        best_cost = c;
      }
    }
    if (best < 0) {  // no bag left to shrink: cut the lowest unused index
      for (int e = 0; e < I && best < 0; ++e)
        if (!is_cut[e]) best = e;
    }
    cuts.push_back(best);
  }
  return cuts;
}

double default_fitness(const Network& net, const std::vector<int>& cuts, void*) {
  Cost c = plan_cost(net, cuts);
  // Width first (the paper's tree width), then total log2 flops (< 128).
  return (double)c.width + c.log2_flops_total() / 128.0;
}

double flops_fitness(const Network& net, const std::vector<int>& cuts, void*) {
  return plan_cost(net, cuts).log2_flops_total();
}

double nonzero_flops_fitness(const Network& net, const std::vector<int>& cuts, void* width_cap) {
  // Slices of cut classes that disagree are exactly zero and never run:
  // 2^classes slices of 8 * macs flops each; a width above the cap costs 8
  // (log2) per extra index.
  const Cost c = plan_cost(net, cuts);
  int n_classes = 0;
  cut_classes(net, cuts, &n_classes);
  const int cap = width_cap ? *static_cast<const int*>(width_cap) : c.width;
  return std::log2(8.0 * c.macs) + n_classes + 8.0 * std::max(0, c.width - cap);
}

namespace {
// Portable bounded draw (the same stream on every platform).
struct Rng {
  std::mt19937_64 g;
  explicit Rng(uint64_t s) : g(s) {}
  int below(int n) {
    uint64_t lim = std::numeric_limits<uint64_t>::max() - std::numeric_limits<uint64_t>::max() % (uint64_t)n;
    uint64_t x;
    do x = g(); while (x >= lim);
    return (int)(x % (uint64_t)n);
  }
};

int draw_absent(Rng& rng, int I, const std::vector<int>& ind) {
  for (;;) {
    int e = rng.below(I);
    if (std::find(ind.begin(), ind.end(), e) == ind.end()) return e;
  }
}

// Replace one copy of each repeated element by a random absent index.
void repair(Rng& rng, int I, std::vector<int>& ind) {
  for (size_t i = 0; i < ind.size(); ++i)
    for (size_t j = 0; j < i; ++j)
      if (ind[i] == ind[j]) {
        ind[i] = draw_absent(rng, I, ind);
        break;
      }
}
}  // namespace

GAResult genetic_cuts(const Network& net, int M, const GAOptions& opt,
                      const std::vector<std::vector<int>>& seeds, FitnessFn fitness, void* ctx) {
  const int I = (int)net.indices.size();
  GAResult res;
  Rng rng(opt.seed);
  const int N = std::max(opt.N, 1);
  M = std::min(M, I);
  // Population: the given seeds first, random M-subsets for the rest.
  std::vector<std::vector<int>> P;
  for (const auto& s : seeds)
    if ((int)P.size() < N && (int)s.size() == M) P.push_back(s);
  while ((int)P.size() < N) {
    std::vector<int> ind;
    while ((int)ind.size() < M) ind.push_back(draw_absent(rng, I, ind));
    P.push_back(ind);
  }
  std::vector<double> fit(N);
  auto evaluate_and_sort = [&]() {
    for (int i = 0; i < N; ++i) {
      fit[i] = fitness(net, P[i], ctx);
      res.evaluations++;
    }
    std::vector<int> idx(N);
    for (int i = 0; i < N; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return fit[a] < fit[b]; });
    std::vector<std::vector<int>> P2(N);
    std::vector<double> f2(N);
    for (int i = 0; i < N; ++i) {
      P2[i] = P[idx[i]];
      f2[i] = fit[idx[i]];
    }
    P.swap(P2);
    fit.swap(f2);
    res.best_fitness_per_generation.push_back(fit[0]);
  };
  const int tail = M / 2;
  int t = 0;
  const auto t_start = std::chrono::steady_clock::now();
  do {
    evaluate_and_sort();                                // Step 1
    for (int i = 1; i + 1 < N; i += 2) {                // Step 2
      for (int j = M - tail; j < M; ++j) std::swap(P[i][j], P[i + 1][j]);
      repair(rng, I, P[i]);
      repair(rng, I, P[i + 1]);
    }
    if (N > 1 && M > 0) {                               // Step 3
      int who = 1 + rng.below(N - 1);
      int pos = rng.below(M);
      P[who][pos] = draw_absent(rng, I, P[who]);
    }
    ++t;                                                // Step 4
    if (opt.time_budget_s > 0 &&
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count() > opt.time_budget_s)
      break;
  } while (t <= opt.T);
  evaluate_and_sort();                                  // Step 5
  res.best = P[0];
  return res;
}

}  // namespace qtn
