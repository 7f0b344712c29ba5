// Learned cost surrogate for the cut search: features of a (network, cut set)
// pair that cost far less than planning it, training data labelled by the
// exact counter, and a genetic search (Algorithm 1, Sec. III.B) whose fitness
// is the surrogate's prediction, with the exact counter deciding among the
// individuals it keeps.
#pragma once
#include <cstdint>
#include <functional>
#include <vector>

#include "network.hpp"
#include "plan.hpp"

namespace qtn {

constexpr int kSurrogateFeatures = 48;
constexpr int kSurrogateTargets = 2;  // log2 total flops, log2 peak bytes (complex64)

// Features of cutting `cuts` out of `net`: sizes, the cut pattern, the gate
// graph left after cutting, and the bag sizes of a min-degree elimination
// (no fill computation).
void surrogate_features(const Network& net, const std::vector<int>& cuts, float* out);

// Exact labels (min-fill plan): log2 total flops and log2 peak bytes.
void surrogate_labels(const Network& net, const std::vector<int>& cuts, float* out);

// `count` random samples: connected 3-regular graphs with n in [n_lo, n_hi]
// (even), p in {p_lo..p_hi}, k in [k_lo, k_hi] cuts drawn uniformly or from
// the large bags of a min-degree elimination.  Sample i depends only on
// (seed, i).  X: count x kSurrogateFeatures, Y: count x kSurrogateTargets.
void surrogate_dataset(int count, int n_lo, int n_hi, int p_lo, int p_hi, int k_lo, int k_hi, uint64_t seed,
                       int threads, float* X, float* Y);

// Predicts rows of targets for a batch of feature rows (n x features).
using PredictFn = std::function<void(const float* X, int n, float* Y)>;

struct SurrogateSearchResult {
  std::vector<int> best;                 // best cut set by the exact counter
  double best_exact = 0;                 // its fitness (width + log2 flops / 128)
  std::vector<double> best_per_generation;
  int exact_evaluations = 0;
  int surrogate_evaluations = 0;
};

// Algorithm 1 with the surrogate as fitness: a population of N sets of M
// cuts, T+1 generations of evaluate / sort / crossover of adjacent pairs
// (the best kept) / one mutation per individual; each generation the `top`
// best by prediction are evaluated exactly, and the best exact one is kept
// (elitism by the exact counter).  Seeds (e.g. the greedy set) join the
// initial population.
SurrogateSearchResult surrogate_genetic_cuts(const Network& net, int M, int T, int N, int top, uint64_t seed,
                                             const std::vector<std::vector<int>>& seeds, const PredictFn& predict);

}  // namespace qtn
