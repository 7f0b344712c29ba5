#include "network.hpp"

#include <algorithm>
#include <cstdio>
#include <set>

namespace qtn {

std::string build_network(int n, int p, const int32_t* edges, int m,
                          const double* gamma, const double* beta, Network* out) {
  if (n < 2) return "n must be >= 2";
  if (p < 1) return "p must be >= 1";
  if (m < 1 || edges == nullptr) return "the graph needs at least one edge";
  if (gamma == nullptr || beta == nullptr) return "gamma and beta must be given";
  Network net;
  net.n = n;
  net.p = p;
  std::set<std::array<int, 2>> seen;
  std::vector<int> deg(n, 0);
  for (int e = 0; e < m; ++e) {
    int a = edges[2 * e], b = edges[2 * e + 1];
    if (a < 0 || b < 0 || a >= n || b >= n || a == b) {
      char buf[96];
      snprintf(buf, sizeof buf, "edge %d = (%d, %d) is not a pair of distinct qubits", e, a, b);
      return buf;
    }
    std::array<int, 2> key{std::min(a, b), std::max(a, b)};
    if (!seen.insert(key).second) {
      char buf[96];
      snprintf(buf, sizeof buf, "edge %d = (%d, %d) is a duplicate", e, a, b);
      return buf;
    }
    deg[a]++;
    deg[b]++;
  }
  for (int q = 0; q < n; ++q)
    if (deg[q] == 0) {
      char buf[96];
      snprintf(buf, sizeof buf, "qubit %d has no ZZ gate", q);
      return buf;
    }
  net.edges.assign(seen.begin(), seen.end());  // lexicographic gate order
  net.gamma.assign(gamma, gamma + p);
  net.beta.assign(beta, beta + p);

  // Per qubit: the (gate, out slot) whose out leg is still open, and how many
  // ZZ gates have acted on it so far.
  std::vector<int> open_gate(n, -1), open_slot(n, -1), count(n, 0);
  for (int l = 0; l < p; ++l) {
    for (const auto& e : net.edges) {
      Gate g{};
      g.layer = l;
      g.q[0] = e[0];
      g.q[1] = e[1];
      int gid = (int)net.gates.size();
      for (int w = 0; w < 2; ++w) {
        int q = e[w];
        g.leg[w] = -1;
        g.leg[2 + w] = -1;
        g.leg[4 + w] = -1;
        g.leg[6 + w] = -1;
        g.out_kind[w] = OUT_PLAIN;
        if (open_gate[q] < 0) {
          g.in_h[w] = 1;
        } else {
          g.in_h[w] = 0;
          Index ix;
          ix.tensor[0] = open_gate[q];
          ix.slot[0] = open_slot[q];
          ix.tensor[1] = gid;
          ix.slot[1] = w;
          ix.qubit = q;
          ix.pos = count[q] - 1;
          int iid = (int)net.indices.size();
          net.indices.push_back(ix);
          net.gates[open_gate[q]].leg[open_slot[q]] = iid;
          g.leg[w] = iid;
        }
        open_gate[q] = gid;
        open_slot[q] = 2 + w;
        count[q]++;
      }
      net.gates.push_back(g);
    }
    // Mixer RX(2 beta_l): absorbed on the open out leg of every wire.
    for (int q = 0; q < n; ++q) {
      Gate& g = net.gates[open_gate[q]];
      int w = open_slot[q] - 2;
      g.out_kind[w] = (l == p - 1) ? OUT_FINAL : OUT_RX;
    }
  }
  *out = std::move(net);
  return "";
}

std::vector<std::vector<int>> leaf_index_lists(const Network& net) {
  std::vector<std::vector<int>> r(net.gates.size());
  for (size_t g = 0; g < net.gates.size(); ++g)
    for (int s = 0; s < kMaxLegs; ++s)
      if (net.gates[g].leg[s] >= 0) r[g].push_back(net.gates[g].leg[s]);
  return r;
}

Network density_network(const Network& a) {
  Network d = a;
  d.density = true;
  const int I = (int)a.indices.size();
  for (int i = 0; i < I; ++i) {
    Index bra = a.indices[i];
    bra.slot[0] += 4;
    bra.slot[1] += 4;
    d.indices.push_back(bra);
  }
  for (Gate& g : d.gates)
    for (int s = 0; s < 4; ++s) g.leg[4 + s] = g.leg[s] >= 0 ? g.leg[s] + I : -1;
  return d;
}

std::string build_gm_network(int n, int p, const int32_t* edges, int m, const double* gamma, const double* beta,
                             Network* out) {
  Network base;
  std::string err = build_network(n, p, edges, m, gamma, beta, &base);  // validation, edge order
  if (!err.empty()) return err;
  Network net;
  net.n = n;
  net.p = p;
  net.gm = true;
  net.edges = base.edges;
  net.gamma = base.gamma;
  net.beta = base.beta;
  auto var = [&](int l, int q) { return l * n + q; };  // z_q^(l + 1)
  for (int l = 0; l < p; ++l)
    for (const auto& e : net.edges) {
      Gate g{};
      g.kind = GATE_GM_ZZ;
      g.layer = l;
      g.q[0] = e[0];
      g.q[1] = e[1];
      for (int s = 0; s < kMaxLegs; ++s) g.leg[s] = -1;
      g.leg[0] = var(l, e[0]);
      g.leg[1] = var(l, e[1]);
      net.gates.push_back(g);
    }
  for (int l = 0; l < p; ++l)
    for (int q = 0; q < n; ++q) {
      Gate g{};
      g.kind = GATE_GM_RX;
      g.layer = l;
      g.q[0] = g.q[1] = q;
      for (int s = 0; s < kMaxLegs; ++s) g.leg[s] = -1;
      g.leg[0] = var(l, q);
      g.leg[1] = l + 1 < p ? var(l + 1, q) : -1;
      net.gates.push_back(g);
    }
  net.indices.resize((size_t)n * p);
  for (int i = 0; i < n * p; ++i) {
    Index& ix = net.indices[i];
    ix.qubit = i % n;
    ix.pos = i / n;
    ix.tensor[0] = ix.tensor[1] = -1;
    ix.slot[0] = ix.slot[1] = -1;
  }
  for (int g = 0; g < (int)net.gates.size(); ++g)
    for (int s = 0; s < 2; ++s) {
      const int e = net.gates[g].leg[s];
      if (e < 0) continue;
      Index& ix = net.indices[e];
      const int h = ix.tensor[0] < 0 ? 0 : ix.tensor[1] < 0 ? 1 : -1;
      if (h >= 0) {
        ix.tensor[h] = g;
        ix.slot[h] = s;
      }
    }
  *out = std::move(net);
  return "";
}

}  // namespace qtn
