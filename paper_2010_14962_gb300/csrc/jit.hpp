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

#include "kernels.cuh"
#include "program.hpp"

namespace qtn {

struct JitLevelShape {
  int threads = 0;         // threads per block
  int blocks_per_sm = 1;   // shared memory sized for this many blocks per SM
  int log2_items = 0;      // items per block = 2^log2_items
  uint32_t arena_stride = 0;
  size_t smem = 0;         // dynamic shared memory per block
};

// Whether the run-time compiler could be loaded (libnvrtc of the toolkit).
bool jit_available(std::string* why);

// Launch shape of the specialised kernel of level program `pg` for elements
// of `elem_bytes`, `threads` per block and `blocks_per_sm` blocks sharing an
// SM; false if not even one item fits.
bool jit_level_shape(const Program& pg, int elem_bytes, int threads, int blocks_per_sm, JitLevelShape* out);

// CUDA source of the specialised kernel ("qtn_level_jit"); empty (and *err
// set) if the program has a form the generator does not handle.
std::string jit_level_source(const Program& pg, Arith a, const JitLevelShape& sh, std::string* err);

// Compiles `src` for the current device, loads it and returns the kernel
// handle (usable with cudaLaunchKernel) with its shared-memory cap raised to
// `smem`.  False and *err on failure.
bool jit_compile(const std::string& src, size_t smem, const void** kernel, std::string* err);

// Launches a kernel made by jit_compile: grid = blocks_per_x * nx blocks.
cudaError_t jit_level_launch(const void* kernel, const JitLevelShape& sh, int nx, int blocks_per_x,
                             const void* leaf_tables, Partial* partials, uint64_t slice_lo, uint64_t slice_hi,
                             cudaStream_t stream);

}  // namespace qtn
