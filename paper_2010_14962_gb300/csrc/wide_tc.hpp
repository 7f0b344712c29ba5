// Tensor-core merge of the wide executor: a dense complex merge (Eq. 1),
// C[m, n, b] = sum_k A[m, k, b] B[k, n, b] per work item, as real GEMMs on
// tcgen05 (kind::tf32, FP32 accumulation in tensor memory) in the 2x2 block
// form [Cr Ci] = [Ar Ai] [[Br, Bi], [-Bi, Br]] (one real GEMM of M x 2K by
// 2K x 2N per complex M x K by K x N).  Operands are staged through shared
// memory in the no-swizzle K-major core-matrix layout, split into TF32 high
// and low parts when three products are asked for (hi*hi + hi*lo + lo*hi).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "program.hpp"

namespace qtn {

// Where an operand of work item g lives: the item's arena slot (arena +
// g * arena_stride + off), or a leaf table entry of the item's bit string
// (leaf_tables + xi * leaf_elems + base + the sub-block of the item's outer
// cut values: bit cut_bit[j] of the item index at position rank_nc + j).
struct WideOperandRef {
  int leaf;
  uint64_t off;
  uint32_t base;
  uint8_t rank_nc, ncut, cut_bit[kMaxLeafCuts];
};

struct WideTcArgs {
  WideOperandRef A, B;
  int c_export;                // 1: C goes to the bit string's leaf table at c_off
  uint64_t c_off;
  const float2* arena;         // item slots
  uint64_t arena_stride;       // elements between item slots
  const float2* leaf_tables;
  uint32_t leaf_elems;         // elements per bit string's leaf table
  uint64_t item_lo, n_items, items_per_x, slice_lo;
  int prologue;                // items are bit strings
  int ma, nb, kb, bb;
  uint8_t wpos[kWideMaxRank];  // store bit positions of the canonical output bits
  int* err;                    // set non-zero if a bounded wait gave up
  float* ws;                   // split-K partials (device), or null
  uint64_t ws_floats;          // its capacity
};

// Shapes the kernel takes: a side of at least 128 (the tile's rows), the
// other side at least 8, and at least 4 summed entries.
bool wide_tc_shape_ok(int ma, int nb, int kb, int bb);

// Floats of split-K workspace the launch of this shape over n_items items
// would use with the device's SM count (0: no split).
uint64_t wide_tc_workspace_floats(int ma, int nb, int kb, int bb, uint64_t n_items);

// products: 1 (TF32) or 3 (split TF32).  Merges with few output tiles and a
// long sum are split along K over several CTAs (when a.ws holds the
// partials); a second kernel adds each output's partials in split order
// (FP64) and stores the result.
cudaError_t wide_tc_launch(const WideTcArgs& a, int products, cudaStream_t stream);

}  // namespace qtn
