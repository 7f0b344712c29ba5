// Step program: a contraction plan lowered to the flat form the device
// kernels interpret.
//
// Every pairwise merge C = A * B (Eq. 1) is executed in a canonical form:
//   A stored as [m | k], B as [k | n], C computed as [m | n],
// where m = A's free indices, n = B's free indices, k = shared (summed)
// indices; bit 0 is the fastest.  Each tensor is stored in the canonical
// order of the merge that consumes it, so operand loads are contiguous and
// only the producer's store is permuted (per-merge bit weights).
//
// Leaves (gate tensors) live in a per-amplitude leaf table built on the device
// in FP64 and rounded to the working precision.  A leaf's cut legs are its
// highest bits, so the sub-block of slice s (Sec. III.A: the cut edges fixed
// to the bits of s) is the contiguous block at offset
//   sum_j bit(s, cut_bit_j) << (rank_nc + j).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "network.hpp"
#include "plan.hpp"

namespace qtn {

constexpr int kMaxLeafCuts = 4;

// Leaf table entry; also carries what the leaf-build kernel needs.
struct DevLeaf {
  uint32_t base;       // element offset in the leaf table
  uint8_t rank_nc;     // legs kept open (low bits)
  uint8_t ncut;        // cut legs (high bits), <= kMaxLeafCuts
  uint8_t cut_bit[kMaxLeafCuts];  // slice bit fixing each cut leg
  int16_t gate;        // gate id (-1: the constant scalar 1)
  int8_t slot_of_bit[8];           // gate leg slot (0..3) at each layout bit
};

enum StepFlags : uint8_t {
  STEP_A_LEAF = 1,
  STEP_B_LEAF = 2,
  STEP_ROOT = 4,  // C is the slice's scalar result
};

constexpr int kMaxRank = 16;

// One merge.  The canonical C element o = m + (n << ma) is stored at arena
// offset c + sum_b bit(o, b) * w[b] (w: bit weights of C's storage layout).
struct DevStep {
  uint8_t ma, nb, kb;  // log2 sizes of m, n, k
  uint8_t flags;
  uint32_t a, b;       // leaf id or arena element offset
  uint32_t c;          // arena element offset of C
  uint16_t w[kMaxRank];
};
static_assert(sizeof(DevStep) == 48, "DevStep layout");

struct Program {
  int n = 0, p = 0, k = 0;
  std::vector<DevLeaf> leaves;
  std::vector<DevStep> steps;
  uint32_t leaf_elems = 0;           // elements in one leaf table
  uint32_t arena_elems = 0;          // per-slice arena (elements)
  bool c_reuses_operands = false;    // arena lets C overlap A (never B)
  int width = 0;                     // max ma + nb + kb
  int max_rank = 0;                  // max tensor rank in the program
  double macs_per_slice = 0;         // sum 2^(ma+nb+kb)
  // Gate data for the leaf-build kernel.
  std::vector<int32_t> gate_q;       // 2 per gate
  std::vector<int8_t> gate_layer;
  std::vector<int8_t> gate_in_h;     // 2 per gate
  std::vector<int8_t> gate_out_kind; // 2 per gate
};

// Lowers `plan` (merges over `net`) to a program.  With `c_reuses_operands`
// the arena lets a merge's result overwrite its A operand (for executors that
// read A completely before the first store of C; B may still be read while C
// is written).  Returns "" or an error.
std::string compile_program(const Network& net, const Plan& plan, bool c_reuses_operands,
                            Program* out);

}  // namespace qtn
