// Step program: a contraction plan lowered to the flat form the device
// executors interpret.
//
// Every pairwise merge C = A * B (Eq. 1) is executed in a canonical form
//   A stored as [m | k | b], B as [k | n | b], C computed as [m | n | b],
// where k = indices shared by A and B (summed), b = batch bits shared by A
// and B (kept), m = the rest of A, n = the rest of B; bit 0 is the fastest.
// Each tensor is stored in the canonical order of the merge that consumes
// it, so operand loads are contiguous and only the producer's store is
// permuted (per-merge bit weights).
//
// Slices (Sec. III.A, Eq. 2).  The k cut indices are grouped into classes:
// two cuts that are the input and output segment of one wire through a
// diagonal ZZ gate can only take equal values in a non-zero slice, so they
// form one class and the other slices (exactly zero) are never enumerated
// by the batched executor.  Classes are either "outer" (fixed per work item:
// the leaf sub-block is selected by an offset) or "inner" (carried as an
// open batch index through the merges of one work item, so each merge runs
// once per distinct value of the inner bits it depends on; the root then
// holds one scalar per inner assignment, i.e. per slice).  With no inner
// class and one class per cut this is the plain per-slice contraction.
//
// Leaves (gate tensors) live in a per-bit-string leaf table built on the
// device in FP64 and rounded to the working precision.  A leaf's outer-class
// bits are its highest bits, so the sub-block of a work item is the
// contiguous block at offset sum_j bit(item, cut_bit_j) << (rank_nc + j).
//
// Hoisting: a merge whose subtree holds no leaf with an outer-class cut leg
// has the same value in every work item.  Such merges form the prologue,
// run once per bit string; the ones consumed by per-item merges write their
// result into the leaf table as "pseudo-leaves" (gate -2), which the item
// steps read like leaves.
//
// Levels (optional): the item steps are ordered by their depth in the
// contraction tree (a merge's level is one more than the deepest merge that
// produces one of its operands).  Merges of one level are independent, so
// an executor can run all of them at once, with one barrier per level
// instead of one per merge; the arena is then allocated per level (a
// level's results never overlap the tensors it reads).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "network.hpp"
#include "plan.hpp"

namespace qtn {

constexpr int kMaxLeafCuts = 4;
constexpr int kMaxRank = 16;

// Leaf table entry; also carries what the leaf-build kernel needs.
struct DevLeaf {
  uint32_t base;       // element offset in the leaf table
  uint8_t rank_nc;     // layout bits read by the consumer (low bits)
  uint8_t ncut;        // outer-class bits (high bits), <= kMaxLeafCuts
  uint8_t cut_bit[kMaxLeafCuts];  // item bit fixing each high bit
  int16_t gate;        // gate id (-1: the constant scalar 1)
  uint8_t slot_mask[8];           // gate leg slots (bit s = slot s) of each layout bit
};
static_assert(sizeof(DevLeaf) == 20, "DevLeaf layout");

enum StepFlags : uint8_t {
  STEP_A_LEAF = 1,
  STEP_B_LEAF = 2,
  STEP_ROOT = 4,    // C is the work item's result: summed, not stored
  STEP_EXPORT = 8,  // prologue step: C is written to the leaf table as leaf `c`
};

// One merge.  The canonical C element o = m + (n << ma) + (b << (ma + nb))
// is stored at arena offset c + sum_i bit(o, i) * w[i].  The first four
// bytes (ma, nb, kb, bb) are read by the executors as one 32-bit word.
struct DevStep {
  uint8_t ma, nb, kb, bb;  // log2 sizes of m, n, k, b
  uint8_t flags, pad0, pad1, pad2;
  uint32_t a, b;           // leaf id or arena element offset
  uint32_t c;              // arena element offset of C
  uint16_t w[kMaxRank];
};
static_assert(sizeof(DevStep) == 52, "DevStep layout");

// One level of a level-ordered program: steps [first, first + count), whose
// output units (in step order) form one flat range.  A unit is 2^u
// consecutive outputs of a step (all of them if it has fewer), so a step of
// rank rc has 2^max(0, rc - u) units; tables are kept for u = 0 (one output
// per unit) and u = 2 (four).  In the four-output table the root step
// counts rc + min(kb, 2): its outputs are summed, not stored, so its sum over
// k is split into up to four independent parts (entries of their own; the
// 16-byte types, whose table is the first, keep one compensated FP64 add per
// output).
constexpr int kLevelUnitLog2 = 2;
constexpr int kRootSplitLog2 = 2;
constexpr int kPosNibEntries = 64;  // per step: 4 nibbles x 16 values (ranks <= 16)
constexpr int kLevelUnit = 1 << kLevelUnitLog2;
struct DevLevel {
  uint16_t first, count;
  uint32_t units[2];  // [0]: single outputs, [1]: units of kLevelUnit
};
static_assert(sizeof(DevLevel) == 12, "DevLevel layout");

// One merge of a wide program (intermediates in global memory, ranks up to
// kWideMaxRank): the same canonical form as DevStep, with 64-bit arena
// offsets and, per canonical output bit, its bit position in the consumer's
// layout (the store weight is 1 << wpos).
constexpr int kWideMaxRank = 34;
struct WideStep {
  uint8_t ma, nb, kb, bb, flags;
  uint64_t a, b, c;  // leaf id or arena element offset (c: leaf id when exported)
  uint8_t wpos[kWideMaxRank];
};

struct ProgramOptions {
  bool levels = false;            // order item steps by tree level (see above)
  // With levels: 0 = levels by depth (fewest barriers); else the item steps
  // keep their depth-first order and consecutive independent steps share a
  // level while the arena stays within this many elements (memory-bounded).
  uint32_t level_budget = 0;
  bool c_reuses_a = false;        // C may overwrite A's arena block
  bool hoist = true;              // run outer-class-invariant merges once per bit string
  std::vector<int> cut_class;     // class of each cut (size k); empty = one class per cut
  std::vector<char> inner;        // per class: carried as a batch index
  // Wide program: tensors up to kWideMaxRank in a global-memory arena;
  // emits wide_steps / wide_prologue instead of steps / prologue.
  bool wide = false;
};

struct Program {
  int n = 0, p = 0, k = 0;
  bool density = false;              // leaves are G (x) conj(G)
  int n_classes = 0;                 // slice classes (non-zero slices = 2^n_classes)
  int n_outer = 0, n_inner = 0;      // outer / inner classes
  std::vector<int> outer_class;      // outer bit position -> class
  std::vector<int> inner_class;      // inner bit position -> class
  std::vector<int> root_class;       // class of each canonical bit of the root's output
  std::vector<DevLeaf> leaves;
  std::vector<DevStep> steps;        // per work item
  std::vector<DevLevel> levels;      // level-ordered programs only
  std::vector<uint32_t> out_start;   // per step: first unit in its level's range, 2 per step (as DevLevel::units)
  std::vector<DevLevel> pro_levels;  // the same for the prologue
  std::vector<uint32_t> pro_out_start;
  // Level-ordered programs: store offsets by nibble, 64 per step: entry
  // [16 g + v] = the offset of output bits 4g..4g+3 equal to v (sum of the
  // step's bit weights), so pos(o) = sum_g entry[16 g + nibble_g(o)].
  std::vector<uint16_t> pos_nib, pro_pos_nib;
  std::vector<DevStep> prologue;     // once per bit string: merges that no outer class reaches
  std::vector<WideStep> wide_steps, wide_prologue;  // wide programs only
  uint64_t wide_arena_elems = 0, wide_pro_arena_elems = 0;
  uint32_t pro_arena_elems = 0;      // prologue arena (elements)
  double macs_prologue = 0;          // per bit string
  uint32_t leaf_elems = 0;           // elements in one leaf table
  uint32_t arena_elems = 0;          // per-item arena (elements)
  int width = 0;                     // max ma + nb + kb + bb
  int max_rank = 0;                  // max tensor rank (with batch bits)
  double macs_per_item = 0;          // sum 2^(ma+nb+kb+bb)
  // Gate data for the leaf-build kernel.
  std::vector<int32_t> gate_q;       // 2 per gate
  std::vector<int8_t> gate_layer;
  std::vector<int8_t> gate_in_h;     // 2 per gate
  std::vector<int8_t> gate_out_kind; // 2 per gate
  std::vector<int8_t> gate_kind;     // GateKind per gate
};

// Lowers `plan` (merges over `net`) to a program.  Returns "" or an error.
std::string compile_program(const Network& net, const Plan& plan, const ProgramOptions& opt, Program* out);

// Classes of the plan's cuts: cuts that are the in and out segment of one
// wire through a ZZ gate whose out leg is plain (a diagonal delta) must take
// equal values in every non-zero slice.  Returns the class of each cut and
// sets *n_classes.
std::vector<int> cut_classes(const Network& net, const std::vector<int>& cuts, int* n_classes);

// Chooses inner classes greedily (largest MAC saving first) while the
// program's arena + leaf table fit `smem_elems` elements and at least
// `min_items` work items remain per bit string.
ProgramOptions choose_batched(const Network& net, const Plan& plan, uint32_t smem_elems, uint64_t min_items);

}  // namespace qtn
