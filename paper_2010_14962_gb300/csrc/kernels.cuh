// Device side of the sliced contraction: launch interface shared by the
// C-ABI layer and the kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "program.hpp"

namespace qtn {

// Lane: one work item per thread; Block: one item per block, a barrier per
// merge; Warp: one item per warp; Level: 2^log2_items items per block, all
// merges of one tree level (of all those items) at once, a barrier per level;
// LevelJit: the same as Level, run by a kernel generated for the program
// (jit.hpp) instead of the interpreter; Wide: intermediates in global memory,
// one launch per merge and group of items (wide.hpp).
enum class Executor : int { Lane = 0, Block = 1, Warp = 2, Level = 3, LevelJit = 4, Wide = 5 };
struct WideState;

// Arithmetic of the merges: complex128, complex64, double-float complex64
// (FP32X2), and complex64 storage with products rounded as the tensor cores
// would (TF32; BF16 / TF32 split in two, 3 products; BF16 split in three,
// 6 products), FP32 accumulation.
enum class Arith : int { F64, F32, F32X2, TF32, BF16X3, TF32X3, BF16X6 };
int arith_elem_bytes(Arith a);

// Compensated (Kahan) partial sum of complex slice results: the running sums
// (re, im) and their compensations (cre, cim).
struct alignas(16) Partial {
  double re, im, cre, cim;
  __host__ __device__ static Partial make(double a, double b, double c, double d) { return Partial{a, b, c, d}; }
};

// Device copy of one plan's program.
struct DeviceProgram {
  int n = 0, p = 0, k = 0;
  int n_leaves = 0, n_steps = 0;
  uint32_t leaf_elems = 0;
  uint32_t arena_elems = 0;  // of the executor's program
  Executor exec = Executor::Lane;
  const DevLeaf* leaves = nullptr;
  const DevStep* steps = nullptr;
  const DevStep* pro_steps = nullptr;  // hoisted merges, once per bit string
  int n_pro_steps = 0;
  uint32_t pro_arena_elems = 0;
  const int32_t* gate_q = nullptr;
  const int8_t* gate_layer = nullptr;
  const int8_t* gate_in_h = nullptr;
  const int8_t* gate_out_kind = nullptr;
  const double* gamma = nullptr;
  const double* trig = nullptr;  // p x (cos gamma, sin gamma, cos beta, sin beta), once per program; may be null
  const double* beta = nullptr;
  int density = 0;  // leaves are G (x) conj(G) (density form)
  const int8_t* gate_kind = nullptr;  // GateKind per gate
  // Level executor only.
  const DevLevel* levels = nullptr;
  const uint32_t* out_start = nullptr;
  int n_levels = 0;
  const DevLevel* pro_levels = nullptr;  // level-ordered prologue (1024-thread blocks)
  const uint32_t* pro_out_start = nullptr;
  int n_pro_levels = 0;
  const uint16_t* pos_nib = nullptr;      // store offsets by nibble (level programs)
  const uint16_t* pro_pos_nib = nullptr;
  int block_threads = 256;  // threads per block (512 or 1024)
  int blocks_per_sm = 1;    // shared memory is sized for this many blocks per SM
  // LevelJit only: the generated kernel (for one arithmetic) and its shape.
  const void* jit_kernel = nullptr;
  int jit_log2_items = 0;
  size_t jit_smem = 0;
  size_t jit_scratch_bytes = 0;  // per block (two-phase schedule), else 0
  const void* jit_prologue = nullptr;  // generated prologue kernel, if any
  size_t jit_pro_smem = 0;
  // Wide only: the device state for the arithmetic and bit-string count of
  // the coming launch (set by the caller before exec_shape / launch).
  WideState* wide = nullptr;
};

// One launch sequence: leaf tables for nx bit strings, the slice range
// [slice_lo, slice_hi) of each, per-block Kahan partials, and the final sum.
struct LaunchBuffers {
  void* leaf_tables = nullptr;   // nx * leaf_elems elements (float2 / double2)
  Partial* partials = nullptr;   // nx * blocks_per_x
  int* err = nullptr;            // set non-zero by a kernel that met a bad step
  void* jit_scratch = nullptr;   // grid blocks * the generated kernel's per-block scratch
};

// Grid shape and dynamic shared memory of the executor for `prog`, `nx` bit
// strings and arithmetic `arith`.  Returns false if the program does not fit
// on chip (or the executor has no kernel for that arithmetic).
struct ExecShape {
  int threads = 0;
  int blocks_per_x = 0;
  int log2_items = 0;          // Level executor: items per block = 2^log2_items
  uint32_t arena_stride = 0;   // Level executor: elements between item arenas
  size_t smem = 0;
  size_t pro_smem = 0;  // prologue kernel (one block of 256 threads per bit string)
};
bool exec_shape(const DeviceProgram& prog, Arith arith, int nx, uint64_t slices_per_x, ExecShape* out);

// Enqueues leaf build + execution + finalisation on `stream`.
//   d_x       : nx * n bit bytes (device)
//   d_out     : nx double2 (scaled amplitude), may be null
//   d_raw     : nx Partial (unscaled Kahan sum and compensation), may be null
//   d_slices  : nx * (slice_hi - slice_lo) double2, may be null
//   ev0, ev1  : optional events recorded just before / after the executor
//   d_gamma, d_beta : optional nx * p angles (device), one set per bit
//               string; null: the program's angles for all
// The per-layer trig table of a program's fixed angles (device sincos).
cudaError_t launch_trig_table(const double* d_gamma, const double* d_beta, int p, double* d_out, cudaStream_t stream);

// The double-float arithmetic check (qtn_arith_check): count complex dot
// products of K terms each (device arrays), scalar and merge-loop forms.
cudaError_t launch_arith_check(const double2* d_a, const double2* d_b, int count, int K, double2* d_scalar,
                               double2* d_merge, cudaStream_t stream);

cudaError_t launch_contraction(const DeviceProgram& prog, Arith arith, const uint8_t* d_x, int nx,
                               uint64_t slice_lo, uint64_t slice_hi, const LaunchBuffers& buf,
                               const ExecShape& shape, double scale, double2* d_out, Partial* d_raw,
                               double2* d_slices, cudaStream_t stream, cudaEvent_t ev0 = nullptr,
                               cudaEvent_t ev1 = nullptr, const double* d_gamma = nullptr,
                               const double* d_beta = nullptr);

// One job of a multi-job launch (device array; pointers are device pointers).
struct JobDesc {
  const DevLeaf* leaves;
  const DevStep* steps;
  const DevStep* pro_steps;
  const int32_t* gate_q;
  const int8_t* gate_layer;
  const int8_t* gate_in_h;
  const int8_t* gate_out_kind;
  const int8_t* gate_kind;
  const double* gamma;
  const double* beta;
  const uint8_t* x;   // n bit bytes
  void* leaf_table;   // leaf_elems elements
  int n, n_leaves, n_steps, n_pro_steps;
  uint32_t leaf_elems, arena_elems, pro_arena_elems;
  uint32_t leaf_start;   // first block of this job in the leaf launch
  uint32_t first_chunk, n_chunks;
  double scale;
  // Level programs (multi_level_kernel) only.
  const DevLevel* levels;
  const uint32_t* out_start;
  int n_levels;
  const DevLevel* pro_levels;
  const uint32_t* pro_out_start;
  int n_pro_levels;
  const uint16_t* pos_nib;
  const uint16_t* pro_pos_nib;
  int log2_items;          // items per block = 2^log2_items; chunks are multiples of it
  uint32_t arena_stride;   // elements between item arenas
  int density;             // leaves are G (x) conj(G) (density form)
};
// A range of work items of one job.
struct ChunkDesc {
  uint32_t job, pad;
  uint64_t lo, hi;
};

// Shared memory of the block executor for a program.
size_t block_smem_bytes(int n_steps, int n_leaves, uint32_t leaf_elems, uint32_t arena_elems, Arith a, int threads);
// Shared memory of the level executor for a program and `items` items per block.
size_t level_smem_bytes(int n_steps, int n_levels, int n_leaves, uint32_t leaf_elems, uint32_t arena_stride,
                        int items, Arith a, int threads);
// Threads per block of the multi-job level executor and of level prologues.
constexpr int kMultiLevelThreads = 1024;
constexpr int kLevelPrologueThreads = 1024;

// Enqueues the multi-job sequence (leaf tables, prologues, persistent
// executor over `n_chunks` chunks, per-job finalisation into d_out[njobs]).
// exec_smem / pro_smem: the largest shared memory any job needs.  `level`:
// every job carries a level program (multi_level_kernel, 1024 threads);
// otherwise block programs (multi_exec_kernel, 256 threads).  Each block,
// before it takes a chunk, stops if *d_cancel (host-mapped, may be null) is
// non-zero or more than budget_ns (0: no limit) have passed since it started;
// a stop sets *d_status (device, must be 0 at launch) to 1 and the remaining
// chunks are skipped (the per-job results are then incomplete).
cudaError_t launch_multi(Arith a, const JobDesc* d_jobs, int njobs, uint32_t total_leaves, const ChunkDesc* d_chunks,
                         uint32_t n_chunks, unsigned* d_counter, Partial* d_chunk_partials, double2* d_out,
                         size_t exec_smem, size_t pro_smem, bool level, const volatile int* d_cancel,
                         unsigned* d_status, uint64_t budget_ns, cudaStream_t stream);

// Largest tensor rank the lane executor accepts.
constexpr int kLaneMaxRank = 5;

}  // namespace qtn
