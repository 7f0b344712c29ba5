#include "surrogate.hpp"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <numeric>
#include <random>
#include <set>
#include <thread>

namespace qtn {

namespace {

struct Rng {
  std::mt19937_64 g;
  explicit Rng(uint64_t s) : g(s) {}
  uint64_t next() { return g(); }
  int below(int n) {
    const uint64_t lim = UINT64_MAX - UINT64_MAX % (uint64_t)n;
    uint64_t x;
    do x = g(); while (x >= lim);
    return (int)(x % (uint64_t)n);
  }
  double uniform() { return (double)(g() >> 11) * (1.0 / 9007199254740992.0); }
};

uint64_t mix(uint64_t a, uint64_t b) {
  uint64_t z = a * 0x9E3779B97F4A7C15ull + b + 0x632BE59BD9B4E019ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Connected simple 3-regular graph (configuration model with rejection).
std::vector<int32_t> random_cubic(int n, Rng& rng) {
  for (;;) {
    std::vector<int> stubs;
    for (int i = 0; i < n; ++i)
      for (int d = 0; d < 3; ++d) stubs.push_back(i);
    for (int i = (int)stubs.size() - 1; i > 0; --i) std::swap(stubs[i], stubs[rng.below(i + 1)]);
    std::set<std::pair<int, int>> seen;
    bool ok = true;
    std::vector<int32_t> e;
    for (size_t i = 0; i < stubs.size(); i += 2) {
      int a = std::min(stubs[i], stubs[i + 1]), b = std::max(stubs[i], stubs[i + 1]);
      if (a == b || !seen.insert({a, b}).second) {
        ok = false;
        break;
      }
      e.push_back(a);
      e.push_back(b);
    }
    if (!ok) continue;
    std::vector<int> parent(n);
    std::iota(parent.begin(), parent.end(), 0);
    std::function<int(int)> find = [&](int x) { return parent[x] == x ? x : parent[x] = find(parent[x]); };
    for (size_t i = 0; i < e.size(); i += 2) parent[find(e[i])] = find(e[i + 1]);
    int root = find(0);
    bool conn = true;
    for (int i = 0; i < n && conn; ++i) conn = find(i) == root;
    if (conn) return e;
  }
}

double quantile(std::vector<int> v, double q) {
  if (v.empty()) return 0;
  std::sort(v.begin(), v.end());
  size_t i = (size_t)std::min<double>((double)v.size() - 1, std::floor(q * (double)(v.size() - 1) + 0.5));
  return v[i];
}

std::vector<int> random_cuts(int I, int k, Rng& rng) {
  std::vector<int> all(I);
  std::iota(all.begin(), all.end(), 0);
  for (int i = 0; i < k; ++i) std::swap(all[i], all[i + rng.below(I - i)]);
  all.resize(k);
  return all;
}

double md_log2_flops(const Network& net, const std::vector<int>& cuts) {
  return min_degree_cost(net, cuts, nullptr).log2_flops_total();
}

}  // namespace

void surrogate_features(const Network& net, const std::vector<int>& cuts, float* f) {
  for (int i = 0; i < kSurrogateFeatures; ++i) f[i] = 0.f;
  const int I = (int)net.indices.size(), L = (int)net.gates.size(), k = (int)cuts.size();
  std::vector<char> is_cut(I, 0);
  for (int c : cuts) is_cut[c] = 1;
  int ncls = 0;
  if (k) {
    // cut classes: in/out segments of one wire through a diagonal gate
    std::vector<int> parent(k);
    std::iota(parent.begin(), parent.end(), 0);
    std::map<int, int> cut_no;
    for (int j = 0; j < k; ++j) cut_no[cuts[j]] = j;
    std::function<int(int)> find = [&](int x) { return parent[x] == x ? x : parent[x] = find(parent[x]); };
    for (const Gate& g : net.gates)
      for (int w = 0; w < 2; ++w)
        if (g.out_kind[w] == OUT_PLAIN && g.leg[w] >= 0 && g.leg[2 + w] >= 0 && is_cut[g.leg[w]] &&
            is_cut[g.leg[2 + w]])
          parent[find(cut_no[g.leg[w]])] = find(cut_no[g.leg[2 + w]]);
    std::set<int> roots;
    for (int j = 0; j < k; ++j) roots.insert(find(j));
    ncls = (int)roots.size();
  }
  f[0] = net.n / 128.f;
  f[1] = net.p / 4.f;
  f[2] = k / 32.f;
  f[3] = I / 512.f;
  f[4] = L / 512.f;
  f[5] = ncls / 32.f;
  std::vector<int> per_gate(L, 0), deg_after(L, 0);
  for (int g = 0; g < L; ++g)
    for (int s = 0; s < kMaxLegs; ++s) {
      int ix = net.gates[g].leg[s];
      if (ix < 0) continue;
      if (is_cut[ix]) per_gate[g]++;
      else deg_after[g]++;
    }
  for (int g = 0; g < L; ++g) {
    f[6 + std::min(per_gate[g], 4)] += 1.f / L;
    f[18 + std::min(deg_after[g], 4)] += 1.f / L;
  }
  if (k) {
    for (int c : cuts) {
      const Index& ix = net.indices[c];
      int zz = 0;
      for (const Gate& g : net.gates) zz += (g.q[0] == ix.qubit) + (g.q[1] == ix.qubit);
      double r = zz > 2 ? (double)ix.pos / (double)(zz - 2) : 0.0;
      f[11 + std::min(5, (int)(r * 6.0))] += 1.f / k;
    }
    int shared = 0;
    for (int g = 0; g < L; ++g) shared += per_gate[g] >= 2;
    f[17] = (float)shared / (float)k;
  }
  // components of the gate graph left after cutting
  std::vector<int> parent(L);
  std::iota(parent.begin(), parent.end(), 0);
  std::function<int(int)> find = [&](int x) { return parent[x] == x ? x : parent[x] = find(parent[x]); };
  for (int e = 0; e < I; ++e)
    if (!is_cut[e]) parent[find(net.indices[e].tensor[0])] = find(net.indices[e].tensor[1]);
  std::map<int, int> comp;
  for (int g = 0; g < L; ++g) comp[find(g)]++;
  int largest = 0;
  for (auto& [r, c] : comp) largest = std::max(largest, c);
  f[23] = comp.size() / 16.f;
  f[24] = (float)largest / (float)L;
  // min-degree elimination
  std::vector<int> bags;
  Cost c = min_degree_cost(net, cuts, &bags);
  f[25] = c.width / 32.f;
  f[26] = (float)(c.log2_flops_total() / 64.0);
  f[27] = (float)(std::log2(c.peak_elems * 8.0) / 64.0);
  f[28] = c.max_rank / 32.f;
  const double qs[8] = {0.10, 0.25, 0.50, 0.75, 0.90, 0.95, 0.99, 1.0};
  for (int i = 0; i < 8; ++i) f[29 + i] = (float)(quantile(bags, qs[i]) / 32.0);
  if (!bags.empty()) {
    int at_w = 0, near_w = 0;
    for (int b : bags) {
      at_w += b == c.width;
      near_w += b >= c.width - 2;
      f[39 + std::min(5, c.width - b)] += 1.f / (float)bags.size();
    }
    f[37] = (float)at_w / (float)bags.size();
    f[38] = (float)near_w / (float)bags.size();
  }
  f[45] = (float)(net.n * net.p) / 512.f;
  f[46] = k ? (float)ncls / (float)k : 1.f;
  f[47] = 1.f;
}

void surrogate_labels(const Network& net, const std::vector<int>& cuts, float* out) {
  Cost c = plan_cost(net, cuts);
  out[0] = (float)c.log2_flops_total();
  out[1] = (float)std::log2(c.peak_elems * 8.0);
}

void surrogate_dataset(int count, int n_lo, int n_hi, int p_lo, int p_hi, int k_lo, int k_hi, uint64_t seed,
                       int threads, float* X, float* Y) {
  auto one = [&](int i) {
    Rng rng(mix(seed, (uint64_t)i));
    const int n = 2 * (n_lo / 2 + rng.below(std::max(1, n_hi / 2 - n_lo / 2 + 1)));
    const int p = p_lo + rng.below(p_hi - p_lo + 1);
    std::vector<int32_t> e = random_cubic(n, rng);
    std::vector<double> ga(p, 0.5), be(p, 0.5);
    Network net;
    build_network(n, p, e.data(), (int)e.size() / 2, ga.data(), be.data(), &net);
    const int I = (int)net.indices.size();
    const int k = std::min(I - 1, k_lo + rng.below(k_hi - k_lo + 1));
    std::vector<int> cuts = random_cuts(I, k, rng);
    if (rng.uniform() < 0.6 && k > 0) {
      // improve by random single swaps under the min-degree estimate, so the
      // set resembles what a search visits
      double cur = md_log2_flops(net, cuts);
      const int steps = 4 + rng.below(40);
      for (int s = 0; s < steps; ++s) {
        std::vector<int> t = cuts;
        int pos = rng.below(k);
        int cand;
        do cand = rng.below(I); while (std::find(t.begin(), t.end(), cand) != t.end());
        t[pos] = cand;
        double v = md_log2_flops(net, t);
        if (v <= cur) {
          cur = v;
          cuts = t;
        }
      }
    }
    surrogate_features(net, cuts, X + (size_t)i * kSurrogateFeatures);
    surrogate_labels(net, cuts, Y + (size_t)i * kSurrogateTargets);
  };
  threads = std::max(1, threads);
  std::vector<std::thread> pool;
  for (int t = 0; t < threads; ++t)
    pool.emplace_back([&, t]() {
      for (int i = t; i < count; i += threads) one(i);
    });
  for (auto& th : pool) th.join();
}

SurrogateSearchResult surrogate_genetic_cuts(const Network& net, int M, int T, int N, int top, uint64_t seed,
                                             const std::vector<std::vector<int>>& seeds, const PredictFn& predict) {
  const int I = (int)net.indices.size();
  M = std::min(M, I);
  N = std::max(N, 2);
  top = std::max(top, 1);
  Rng rng(seed);
  SurrogateSearchResult res;
  std::map<std::vector<int>, double> exact;  // sorted set -> exact fitness
  auto exact_of = [&](const std::vector<int>& ind) {
    std::vector<int> key = ind;
    std::sort(key.begin(), key.end());
    auto it = exact.find(key);
    if (it != exact.end()) return it->second;
    Cost c = plan_cost(net, ind);
    double v = c.log2_flops_total();
    exact[key] = v;
    res.exact_evaluations++;
    if (res.best.empty() || v < res.best_exact) {
      res.best = ind;
      res.best_exact = v;
    }
    return v;
  };
  auto draw_absent = [&](const std::vector<int>& ind) {
    for (;;) {
      int e = rng.below(I);
      if (std::find(ind.begin(), ind.end(), e) == ind.end()) return e;
    }
  };
  auto repair = [&](std::vector<int>& ind) {
    for (size_t i = 0; i < ind.size(); ++i)
      for (size_t j = 0; j < i; ++j)
        if (ind[i] == ind[j]) {
          ind[i] = draw_absent(ind);
          break;
        }
  };
  std::vector<std::vector<int>> P;
  for (const auto& s : seeds)
    if ((int)P.size() < N && (int)s.size() == M) P.push_back(s);
  while ((int)P.size() < N) {
    std::vector<int> ind;
    while ((int)ind.size() < M) ind.push_back(draw_absent(ind));
    P.push_back(ind);
  }
  for (size_t i = 0; i < P.size() && i < seeds.size(); ++i) exact_of(P[i]);
  std::vector<float> X((size_t)N * kSurrogateFeatures), Y((size_t)N * kSurrogateTargets);
  const int tail = M / 2;
  for (int t = 0; t <= T; ++t) {
    // Step 1 with the surrogate: predicted log2 total flops, then sort
    for (int i = 0; i < N; ++i) surrogate_features(net, P[i], X.data() + (size_t)i * kSurrogateFeatures);
    predict(X.data(), N, Y.data());
    res.surrogate_evaluations += N;
    std::vector<int> idx(N);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int a, int b) { return Y[(size_t)a * kSurrogateTargets] < Y[(size_t)b * kSurrogateTargets]; });
    std::vector<std::vector<int>> S(N);
    for (int i = 0; i < N; ++i) S[i] = P[idx[i]];
    // the exact counter scores the most promising individuals
    for (int i = 0; i < std::min(top, N); ++i) exact_of(S[i]);
    // elitism by the exact counter: the best exact set stays first
    S[0] = res.best;
    res.best_per_generation.push_back(res.best_exact);
    // Step 2: crossover of adjacent pairs, the best excluded
    for (int i = 1; i + 1 < N; i += 2) {
      for (int j = M - tail; j < M; ++j) std::swap(S[i][j], S[i + 1][j]);
      repair(S[i]);
      repair(S[i + 1]);
    }
    // Step 3: mutation (every individual but the best, to explore widely)
    for (int i = 1; i < N; ++i) {
      int pos = rng.below(M);
      S[i][pos] = draw_absent(S[i]);
    }
    P.swap(S);
  }
  return res;
}

}  // namespace qtn
