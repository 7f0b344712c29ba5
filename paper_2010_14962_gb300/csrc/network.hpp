// Host-side tensor network of a QAOA amplitude <x|C|0^n>.
//
// The circuit is mapped to an undirected graph as in the paper's Sec. II.A
// (Fig. 1): every gate is a vertex, every wire segment an edge (tensor index).
// Edges carry dimension 2 (amplitude form) instead of the paper's
// dimension-4 density-operator basis.  Rank <= 2 tensors (H|0>, the RX mixers
// and the <x_i| projections) are absorbed into the neighbouring ZZ gate, so
// only the p * |E| ZZ tensors remain as vertices; their values are produced
// on the device in FP64 from (gamma, beta, x).
#pragma once
#include <array>
#include <cstdint>
#include <string>
#include <vector>

namespace qtn {

// Role of the "out" side of a ZZ gate's wire leg.
enum OutKind : int8_t {
  OUT_PLAIN = 0,  // leg continues to the next ZZ gate of the same layer
  OUT_RX = 1,     // mixer RX(2 beta_l) of this layer absorbed on the leg
  OUT_FINAL = 2,  // <x_q| RX(2 beta_p) absorbed: leg closed
};

// One ZZ(gamma_l) gate on qubits (q[0], q[1]).  Leg slots are
// 0 = in q0, 1 = in q1, 2 = out q0, 3 = out q1.  A slot holds the id of the
// index (wire segment) it connects to, or -1 if the wire end was absorbed.
// In the density form (Sec. II.A with dimension-4 edges) the vertex is the
// gate's superoperator G (x) conj(G): slots 4..7 are the bra copies of
// slots 0..3 (each dimension-4 edge is a ket bit and a bra bit).
constexpr int kMaxLegs = 8;
struct Gate {
  int layer;
  int q[2];
  int leg[kMaxLegs];
  int8_t in_h[2];    // 1 if H|0> (unnormalised [1,1]) is absorbed on the in leg
  int8_t out_kind[2];
};

// A wire segment between two consecutive ZZ gates on qubit `qubit`; it is the
// segment that follows the `pos`-th ZZ gate (0-based) acting on that qubit.
struct Index {
  int tensor[2];  // gate ids of the endpoints (tensor[0] is the earlier gate)
  int slot[2];    // leg slots on those gates
  int qubit;
  int pos;
};

struct Network {
  int n = 0, p = 0;
  std::vector<std::array<int, 2>> edges;  // sorted lexicographically, i < j
  std::vector<double> gamma, beta;
  std::vector<Gate> gates;
  std::vector<Index> indices;
  // Density form: indices [I/2, I) are the bra copies of [0, I/2); the
  // network's scalar is <x| rho |x> = |a(x)|^2 (times 2^-n unnormalised).
  bool density = false;
};

// Builds the network; returns an empty string on success, else a message.
std::string build_network(int n, int p, const int32_t* edges, int m,
                          const double* gamma, const double* beta, Network* out);

// The density form of an amplitude network: same vertices, every edge of
// dimension 4 (ket bit i, bra bit i + I).
Network density_network(const Network& amplitude);

// Index sets of every leaf (gate) tensor, in leg-slot order, absorbed legs
// dropped.
std::vector<std::vector<int>> leaf_index_lists(const Network& net);

}  // namespace qtn
