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

// Vertex kinds.  GATE_ZZ: a ZZ gate with its absorbed pieces, legs as above.
// The graphical-model form shares one index among all diagonal gates that
// act on a qubit between two mixers (the basis value z_q^(l) of qubit q in
// layer l): GATE_GM_ZZ is the factor exp(-i gamma_l s_i s_j) on legs 0, 1 =
// z_i^(l), z_j^(l); GATE_GM_RX is <z_q^(l+1)| RX(2 beta_l) |z_q^(l)> on legs
// 0 = z_q^(l), 1 = z_q^(l+1) (-1 in the last layer: the row is x_q).
enum GateKind : int8_t { GATE_ZZ = 0, GATE_GM_ZZ = 1, GATE_GM_RX = 2 };

struct Gate {
  int layer;
  int q[2];
  int leg[kMaxLegs];
  int8_t in_h[2];    // 1 if H|0> (unnormalised [1,1]) is absorbed on the in leg
  int8_t out_kind[2];
  int8_t kind = GATE_ZZ;
};

// A wire segment between two consecutive ZZ gates on qubit `qubit`; it is the
// segment that follows the `pos`-th ZZ gate (0-based) acting on that qubit.
// In the graphical-model form: the variable z_qubit^(pos + 1), held by every
// factor of its layer on that qubit (tensor / slot: the first two holders).
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
  // Graphical-model form: an index may be held by more than two tensors.
  bool gm = false;
};

// Builds the network; returns an empty string on success, else a message.
std::string build_network(int n, int p, const int32_t* edges, int m,
                          const double* gamma, const double* beta, Network* out);

// The density form of an amplitude network: same vertices, every edge of
// dimension 4 (ket bit i, bra bit i + I).
Network density_network(const Network& amplitude);

// The graphical-model form of the same circuit: n * p variables z_q^(l)
// (index (l - 1) * n + q), p * m ZZ factors (layer-major, edge order) then
// p * n mixer factors (layer-major, qubit order).  Same validation and the
// same amplitude as build_network.
std::string build_gm_network(int n, int p, const int32_t* edges, int m, const double* gamma, const double* beta,
                             Network* out);

// Index sets of every leaf (gate) tensor, in leg-slot order, absorbed legs
// dropped.
std::vector<std::vector<int>> leaf_index_lists(const Network& net);

}  // namespace qtn
