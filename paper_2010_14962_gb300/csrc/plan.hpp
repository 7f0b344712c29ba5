// Contraction planning on the host: elimination orders over tensor indices,
// the exact cost counter, and cut-set (edge-cutting) search.
//
// Paper mapping: Sec. II.B ties the memory and time of a contraction to the
// largest intermediate tensor, i.e. to the width of the tree decomposition an
// elimination order induces; Sec. III.A fixes the values of m cut edges and
// sums the 2^m (here: dimension 2) sliced networks (Eq. 2); Sec. III.B /
// Algorithm 1 searches the cut set with a genetic algorithm.
#pragma once
#include <cstdint>
#include <random>
#include <string>
#include <vector>

#include "network.hpp"

namespace qtn {

// Index set of one tensor as a fixed-width bitset.
struct Bits {
  std::vector<uint64_t> w;
  Bits() = default;
  explicit Bits(int nbits) : w((nbits + 63) / 64, 0) {}
  void set(int i) { w[i >> 6] |= 1ull << (i & 63); }
  void clear(int i) { w[i >> 6] &= ~(1ull << (i & 63)); }
  bool get(int i) const { return (w[i >> 6] >> (i & 63)) & 1; }
  int count() const;
  std::vector<int> list() const;
};

// One pairwise contraction (Eq. 1): tensors a and b merge into c; the indices
// they share are summed, the others stay open.
struct Merge {
  int a, b, c;
};

// A contraction plan for one sliced network.  Tensor ids: 0..L-1 are the
// leaves (gate tensors with cut indices removed), L.. are intermediates in
// the order they are created.  `tensors[t]` is the sorted index set of t.
struct Plan {
  int n_indices = 0;
  int n_leaves = 0;
  std::vector<int> cuts;                     // slice bit j <-> index cuts[j]
  std::vector<int> order;                    // eliminated indices, in order
  std::vector<std::vector<int>> tensors;     // index sets (open indices)
  std::vector<Merge> merges;                 // root = merges.back().c
  // Exact cost (per slice unless stated).
  int width = 0;          // max |A u B| over merges (bag size of the order)
  int max_rank = 0;       // max rank of any tensor
  double macs = 0;        // complex multiply-adds per slice
  double peak_elems = 0;  // max sum of 2^rank over simultaneously live tensors
  double log2_flops_total() const;  // log2(2^k * 8 * macs)
};

// Plans the contraction of `net` with index set `cuts` fixed.  If `order` is
// non-empty it must list every non-cut index exactly once (an index already
// summed by an earlier merge is skipped); otherwise min-fill chooses it
// (ties: fill, then bag size, then lowest id).  Returns "" or an error.
std::string make_plan(const Network& net, const std::vector<int>& cuts,
                      const std::vector<int>& order, Plan* out);

// Same as make_plan but only the cost fields are filled (no tensor lists).
struct Cost {
  int width;
  int max_rank;
  double macs;
  double peak_elems;
  int k;
  double log2_flops_total() const;
};
Cost plan_cost(const Network& net, const std::vector<int>& cuts);

// Cheap estimate of the same: elimination by smallest merged bag (min
// degree, no fill computation); `bag_sizes` (optional) gets |A u B| per merge.
Cost min_degree_cost(const Network& net, const std::vector<int>& cuts, std::vector<int>* bag_sizes);

// Greedy cut search: k times, cut the index (taken from the widest bags of
// the current min-fill order) that gives the smallest (width, total flops).
std::vector<int> greedy_cuts(const Network& net, int k,
                             const std::vector<int>& start = {});

// Genetic search of Algorithm 1 (Sec. III.B).  Individuals are sets of M
// cut indices; fitness = (width, total log2 flops) from `fitness`.
struct GAOptions {
  int T = 4;          // maximum iteration counter (loop runs until t > T)
  int N = 11;         // population size
  uint64_t seed = 1;
  double time_budget_s = 0;  // stop after the generation that exceeds it (0: none)
};
struct GAResult {
  std::vector<int> best;
  std::vector<double> best_fitness_per_generation;  // scalarised fitness
  int evaluations = 0;
};
using FitnessFn = double (*)(const Network&, const std::vector<int>&, void*);
double default_fitness(const Network& net, const std::vector<int>& cuts, void*);
double flops_fitness(const Network& net, const std::vector<int>& cuts, void*);  // log2 total flops
// log2 flops of the structurally non-zero slices (2^classes x per-slice), plus
// a penalty for a width above *(const int*)width_cap.
double nonzero_flops_fitness(const Network& net, const std::vector<int>& cuts, void* width_cap);
GAResult genetic_cuts(const Network& net, int M, const GAOptions& opt,
                      const std::vector<std::vector<int>>& seeds,
                      FitnessFn fitness, void* ctx);

}  // namespace qtn
