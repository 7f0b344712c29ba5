// Wide executor: the elimination steps of one plan with intermediates in
// global memory (HBM / L2), for plans whose per-slice tensors do not fit in
// shared memory (ranks up to kWideMaxRank).  Each merge (Eq. 1) is one
// launch over a group of work items (slices, Sec. III.A), with the kernel
// chosen per step shape by an autotuner: a SIMT kernel for any shape, or
// the tensor-core kernel (tcgen05, TF32 operands, FP32 accumulation in
// tensor memory) where the merge is a dense complex GEMM and the arithmetic
// allows it.  The root of every item (its slice scalar) is a dot product
// reduced in FP64 (Kahan) per block; the per-block partials of all items of
// a bit string are summed in fixed order by the common finalisation.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "kernels.cuh"
#include "program.hpp"

namespace qtn {

enum class WideKernel : int { Simt = 0, Simt4 = 1, Tc = 2 };
const char* wide_kernel_name(WideKernel k);

// Shape key of one merge launch: log2 sizes, items in the launch, arithmetic.
using WideShapeKey = std::tuple<int, int, int, int, uint64_t, int>;

// Process-wide autotuning record of the wide executor: the fastest kernel
// per merge shape (and all timings), kept across plans.
struct WideTuneEntry {
  WideKernel best;
  std::vector<std::pair<WideKernel, float>> ms;
};
std::map<WideShapeKey, WideTuneEntry>& wide_tune_table();
// Loads / saves the table as JSON lines (path from QTN_WIDE_TUNE_CACHE if
// set); missing or unreadable files are ignored.
void wide_tune_load();
void wide_tune_save();

// Device state of one wide program for one arithmetic and bit-string count.
struct WideState {
  const Program* prog = nullptr;
  Arith arith = Arith::F64;
  int nx = 0;
  uint64_t items_per_x = 0;   // work items (outer-class assignments) per bit string
  uint64_t group = 0;         // items per pass (arena slots)
  int root_blocks = 1;        // blocks per item of the root reduction
  void* d_arena = nullptr;    // group * wide_arena_elems elements
  void* d_pro_arena = nullptr;
  std::vector<WideKernel> step_kernel;  // per item step (autotuned)
  std::vector<WideKernel> pro_kernel;   // per prologue step
  // Per item step: the candidates' times (ms per launch of `group` items,
  // CUDA events) from the tuning; empty where the kernel was forced.
  std::vector<std::vector<std::pair<WideKernel, float>>> step_ms;
  bool tuned = false;
  std::string tune_log;       // the kernel chosen per tuned shape
  int force_mode = -1;        // kernel override in force when tuned (qtn_wide_set_kernel)
  int* d_own_err = nullptr;   // error word used when the caller passes none
  float* d_tc_ws = nullptr;   // split-K partials of tensor-core merges
  uint64_t tc_ws_floats = 0;
  ~WideState();
};

// The kernel override in force (qtn_wide_set_kernel): -1 = autotuned.
int wide_force_mode();
// Whether `ws` must be tuned (again) before its next launch is captured.
bool wide_needs_tuning(const WideState* ws);

// Whether step `st` can run on the tensor-core kernel with arithmetic `a`.
bool wide_tc_eligible(const WideStep& st, Arith a);

// Allocates the arenas of `ws` (group sized to `budget_bytes`) for nx bit
// strings; the leaf tables are the caller's.
cudaError_t wide_prepare(WideState* ws, const Program& prog, Arith a, int nx, uint64_t budget_bytes);

// Times the eligible kernels of every distinct step shape of `ws` on the
// real operands (leaf tables already built on `stream`), records the fastest
// per shape (process-wide, keyed by shape) and synchronises the stream.
cudaError_t wide_tune(WideState* ws, void* leaf_tables, uint64_t slice_lo, uint64_t slice_hi, cudaStream_t stream,
                      std::string* log);

// Enqueues the wide steps for nx bit strings whose leaf tables (built by the
// caller) are at leaf_tables: prologue (once per bit string, results into the
// leaf tables), then items [slice_lo, slice_hi) of every bit string in groups;
// writes root partials (items x root_blocks per bit string, in item order) to
// partials, and, if d_slices is given, each item's value (unscaled).
cudaError_t wide_launch(WideState* ws, void* leaf_tables, uint64_t slice_lo, uint64_t slice_hi, Partial* partials,
                        double2* d_slices, int* d_err, cudaStream_t stream);

}  // namespace qtn
