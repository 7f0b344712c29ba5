// Per-plan specialised level executor: the level program of one plan is
// turned into CUDA source in which every merge (Eq. 1) is straight-line code
// with its shape, operand offsets, leaf sub-block selection and store
// permutation as constants, compiled at run time by NVRTC for the current
// device and launched like the interpreted level executor (same arguments,
// same results, same fixed-order sums).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "program.hpp"

namespace qtn {

// Launch shape and schedule of the specialised kernel.  A block walks its
// share of the slices in chunks.  Single-phase: every level of the program
// runs on 2^log2_items items at a time.  Two-phase: the levels below
// `split_level` (the many small merges on the leaf side of the contraction
// tree) run on 2^log2_forest items at a time in arenas that hold only what
// those levels touch; the tensors they pass to the later levels are parked
// in a per-block global scratch area (L2-resident) and reloaded, two items'
// worth at a time, into full arenas for the remaining levels.  The autotuner
// times both forms.
struct JitLevelShape {
  int threads = 0;         // threads per block
  int blocks_per_sm = 1;   // shared memory sized for this many blocks per SM
  int log2_items = 0;      // items per pass of the full-arena levels
  uint32_t arena_stride = 0;
  size_t smem = 0;         // dynamic shared memory per block
  // two-phase schedule (split_level == 0: single-phase)
  int split_level = 0;
  int log2_forest = 0;            // items per pass of the levels below split_level
  uint32_t forest_stride = 0;     // elements between their arenas
  uint32_t cross_elems = 0;       // elements parked per item
  size_t scratch_elems_per_block = 0;
  double est_cost = 0, est_cost_single = 0;  // estimated slot-steps per item
};

// Whether the run-time compiler could be loaded (libnvrtc of the toolkit).
bool jit_available(std::string* why);

// Launch shape of the specialised kernel of level program `pg` for elements
// of `elem_bytes`, `threads` per block and `blocks_per_sm` blocks sharing an
// SM, single-phase or (two_phase) the two-phase schedule with the fewest
// estimated slot-steps per item; false if not even one item fits, or no
// two-phase schedule does.
bool jit_level_shape(const Program& pg, int elem_bytes, int threads, int blocks_per_sm, bool two_phase,
                     JitLevelShape* out);

// The same for `bps` blocks per SM and `cap` bytes of shared memory per
// block (no device query).
bool jit_level_schedule(const Program& pg, int elem_bytes, int threads, int bps, size_t cap, bool two_phase,
                        JitLevelShape* out);

// Tensors a two-phase schedule with split level `split` parks: (arena
// offset, elements, offset in the per-item park area) each, and the arena
// extent of the levels below `split`.  False if an arena operand has no
// writer (not a valid level program).
struct JitCrossing {
  uint32_t off, size, at;
};
bool jit_crossings(const Program& pg, size_t split, std::vector<JitCrossing>* out, uint32_t* extent);

// CUDA source of the specialised kernel ("qtn_level_jit"); empty (and *err
// set) if the program has a form the generator does not handle.
std::string jit_level_source(const Program& pg, Arith a, const JitLevelShape& sh, std::string* err);

// Compiles `src` for the current device, loads it and returns the kernel
// handle (usable with cudaLaunchKernel) with its shared-memory cap raised to
// `smem`.  False and *err on failure.
bool jit_compile(const std::string& src, size_t smem, const void** kernel, std::string* err, size_t pro_smem = 0,
                 const void** prologue = nullptr);

// The generated source also holds "qtn_prologue_jit" when the program has
// hoisted merges in levels: one block of kJitPrologueThreads per bit string,
// jit_prologue_smem bytes of dynamic shared memory, writing the pseudo-leaves
// of each bit string's leaf table (what prologue_level_kernel computes).
constexpr int kJitPrologueThreads = 1024;
size_t jit_prologue_smem(const Program& pg, int elem_bytes);
cudaError_t jit_prologue_launch(const void* kernel, int nx, size_t smem, void* leaf_tables, cudaStream_t stream);

// Launches a kernel made by jit_compile: grid = blocks_per_x * nx blocks;
// `scratch` holds scratch_elems_per_block elements per block (two-phase
// schedule; may be null otherwise).
cudaError_t jit_level_launch(const void* kernel, const JitLevelShape& sh, int nx, int blocks_per_x,
                             const void* leaf_tables, Partial* partials, void* scratch, uint64_t slice_lo,
                             uint64_t slice_hi, cudaStream_t stream);

}  // namespace qtn
