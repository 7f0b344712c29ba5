// Sliced tensor-network contraction on sm_103a.
//
//   leaf_build_kernel   evaluates every gate tensor of the network once per
//                       bit string in FP64 (sincos of gamma_l, beta_l) and
//                       rounds it to the working precision (Sec. II.A: the
//                       tensors of the circuit's vertices).
//   lane_exec_kernel    one slice per GPU thread.  All slices share one step
//                       program (Sec. III.A: the subnetworks have identical
//                       topology, only the fixed cut values differ), so a warp
//                       runs 32 slices in lock step; each thread keeps its
//                       intermediates in a private column of shared memory
//                       and every merge (Eq. 1) is a fully unrolled
//                       register-resident product specialised on its shape.
//   block_exec_kernel   one work item per thread block: a slice, or (batched
//                       programs) a sub-cube of slices whose inner cut classes
//                       are carried as batch bits, so each merge runs once per
//                       distinct value of the bits it depends on; threads
//                       split the output elements of each merge.
//   finalize_kernel     fixed-order compensated FP64 sum of the per-block
//                       partial sums over slices (Eq. 2) and the 2^{-n/2}
//                       normalisation of the unnormalised H|0> = (1, 1).
#include "kernels.cuh"

#include <cuda_bf16.h>

#include "jit.hpp"
#include "wide.hpp"

#include <algorithm>
#include <type_traits>

namespace qtn {
namespace {

struct ExecParams {
  const DevStep* steps;
  const DevLeaf* leaves;
  const void* leaf_tables;
  Partial* partials;
  double2* slices;  // optional per-slice output
  uint64_t slice_lo, slice_hi;
  uint32_t leaf_elems;
  uint32_t arena_elems;
  int n_steps, n_leaves;
  int blocks_per_x;  // blocks per bit string; blockIdx.x = xi * blocks_per_x + b
};

#include "arith.cuh"

#include "rounding.cuh"

// Offset of slice s's sub-block inside a leaf: cut legs are the high bits.
__device__ __forceinline__ uint32_t leaf_offset(const DevLeaf& L, uint64_t s) {
  uint32_t off = L.base;
  for (int j = 0; j < L.ncut; ++j) off += (uint32_t)((s >> L.cut_bit[j]) & 1u) << (L.rank_nc + j);
  return off;
}

// Copies `bytes` (multiple of 4) from global to shared memory.
__device__ __forceinline__ void copy_words(void* dst, const void* src, size_t bytes) {
  const uint32_t* s = static_cast<const uint32_t*>(src);
  uint32_t* d = static_cast<uint32_t*>(dst);
  for (size_t i = threadIdx.x; i < bytes / 4; i += blockDim.x) d[i] = s[i];
}

struct SmemLayout {
  size_t leaves, table, arena, red, total;
};
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ inline SmemLayout smem_layout(int n_steps, int n_leaves, uint32_t leaf_elems,
                                                  uint32_t arena_elems, int elem_bytes, int threads,
                                                  bool per_thread_arena) {
  SmemLayout L;
  L.leaves = align16((size_t)n_steps * sizeof(DevStep));
  L.table = L.leaves + align16((size_t)n_leaves * sizeof(DevLeaf));
  L.arena = L.table + align16((size_t)leaf_elems * elem_bytes);
  size_t arena_bytes = (size_t)arena_elems * elem_bytes * (per_thread_arena ? threads : 1);
  L.red = L.arena + align16(arena_bytes);
  L.total = L.red + (size_t)threads * sizeof(Partial);
  return L;
}

// ------------------------------------------------------------ leaf build --

// Value of ZZ gate g (with its absorbed H|0>, RX and <x| pieces) at leg
// values v[0..3] (in q0, in q1, out q0, out q1; -1 on absorbed legs); t =
// (cos gamma_l, sin gamma_l, cos beta_l, sin beta_l) of the gate's layer.
__device__ __forceinline__ void gate_value(int g, const int* v, const int32_t* __restrict__ gate_q,
                                           const int8_t* __restrict__ gate_in_h,
                                           const int8_t* __restrict__ gate_out_kind, const double* t,
                                           const uint8_t* __restrict__ xrow, double& re, double& im) {
  const double cg = t[0], sg = t[1], cb = t[2], sb = t[3];
  re = 0.0;
  im = 0.0;
  // T = sum over the wire values (u0, u1) inside the diagonal ZZ gate of
  //   exp(-i gamma s0 s1) * prod_w [in leg: delta] * [out leg: delta or
  //   RX(2 beta)[out, u] or <x_q|RX(2 beta)|u>];  absorbed H|0> = (1, 1).
  for (int u0 = 0; u0 < 2; ++u0)
    for (int u1 = 0; u1 < 2; ++u1) {
      const int u[2] = {u0, u1};
      const double sgn = (double)((1 - 2 * u0) * (1 - 2 * u1));
      double tre = cg, tim = -sgn * sg;
      bool ok = true;
      for (int w = 0; w < 2; ++w) {
        if (!gate_in_h[2 * g + w] && v[w] != u[w]) ok = false;
        const int kind = gate_out_kind[2 * g + w];
        if (kind == OUT_PLAIN) {
          if (v[2 + w] != u[w]) ok = false;
        } else {
          const int row = (kind == OUT_RX) ? v[2 + w] : (int)xrow[gate_q[2 * g + w]];
          if (row != u[w]) {  // multiply by -i sin(beta)
            const double nre = tim * sb, nim = -tre * sb;
            tre = nre;
            tim = nim;
          } else {
            tre *= cb;
            tim *= cb;
          }
        }
      }
      if (ok) {
        re += tre;
        im += tim;
      }
    }
}

// Value of a graphical-model factor at leg values v[0], v[1]: the ZZ phase
// exp(-i gamma_l s_0 s_1) (s = 1 - 2 z), or the mixer entry
// <z_out| RX(2 beta_l) |z_in> = cos beta_l or -i sin beta_l, with z_out =
// x_q on the last layer (leg 1 absent); t as for gate_value.
__device__ __forceinline__ void gm_factor_value(int g, int kind, const int* v, const int32_t* __restrict__ gate_q,
                                                const double* t, const uint8_t* __restrict__ xrow, double& re,
                                                double& im) {
  if (kind == GATE_GM_ZZ) {
    const double sgn = (double)((1 - 2 * v[0]) * (1 - 2 * v[1]));
    re = t[0];
    im = -sgn * t[1];
  } else {
    const int out = v[1] >= 0 ? v[1] : (int)xrow[gate_q[2 * g]];
    if (out == v[0]) {
      re = t[2];
      im = 0.0;
    } else {
      re = 0.0;
      im = -t[3];
    }
  }
}

// Entry e of leaf L (FP64 evaluation, rounded by V's conversion); t = the
// trig values of its gate's layer (cos gamma, sin gamma, cos beta, sin beta).
// In the density form (Sec. II.A, dimension-4 edges) the leaf is the
// superoperator G (x) conj(G): slots 0..3 carry the ket bits, slots 4..7 the
// bra bits.
template <class V>
__device__ __forceinline__ V leaf_entry_trig(const DevLeaf& L, int e, const int32_t* __restrict__ gate_q,
                                             const int8_t* __restrict__ gate_in_h,
                                             const int8_t* __restrict__ gate_out_kind,
                                             const int8_t* __restrict__ gate_kind, const double* t,
                                             const uint8_t* __restrict__ xrow, bool density) {
  const int r = L.rank_nc + L.ncut;
  double re = 1.0, im = 0.0;
  if (L.gate >= 0) {
    const int g = L.gate;
    int v[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
    for (int b = 0; b < r; ++b)
      for (int sl = 0; sl < 8; ++sl)
        if ((L.slot_mask[b] >> sl) & 1) v[sl] = (e >> b) & 1;
    const int kind = gate_kind[g];
    if (kind != GATE_ZZ) {
      gm_factor_value(g, kind, v, gate_q, t, xrow, re, im);
      return CplxOps<V>::from(re, im);
    }
    gate_value(g, v, gate_q, gate_in_h, gate_out_kind, t, xrow, re, im);
    if (density) {
      double bre, bim;
      gate_value(g, v + 4, gate_q, gate_in_h, gate_out_kind, t, xrow, bre, bim);
      const double pre = re * bre + im * bim, pim = im * bre - re * bim;  // (re + i im) * conj(bre + i bim)
      re = pre;
      im = pim;
    }
  }
  return CplxOps<V>::from(re, im);
}

// The same with the layer's trig values computed here.
template <class V>
__device__ __forceinline__ V leaf_entry(const DevLeaf& L, int e, const int32_t* __restrict__ gate_q,
                                        const int8_t* __restrict__ gate_layer, const int8_t* __restrict__ gate_in_h,
                                        const int8_t* __restrict__ gate_out_kind, const int8_t* __restrict__ gate_kind,
                                        const double* __restrict__ gamma, const double* __restrict__ beta,
                                        const uint8_t* __restrict__ xrow, bool density) {
  double t[4] = {1.0, 0.0, 1.0, 0.0};
  if (L.gate >= 0) {
    const int l = gate_layer[L.gate];
    sincos(gamma[l], &t[1], &t[0]);
    sincos(beta[l], &t[3], &t[2]);
  }
  return leaf_entry_trig<V>(L, e, gate_q, gate_in_h, gate_out_kind, gate_kind, t, xrow, density);
}

// Leaf tables of nx bit strings; bit string xi uses angles gamma / beta +
// xi * angle_stride (0: one angle set for all).
template <class V>
__global__ void leaf_build_kernel(const DevLeaf* __restrict__ leaves, const int32_t* __restrict__ gate_q,
                                  const int8_t* __restrict__ gate_layer, const int8_t* __restrict__ gate_in_h,
                                  const int8_t* __restrict__ gate_out_kind, const int8_t* __restrict__ gate_kind,
                                  const double* __restrict__ gamma,
                                  const double* __restrict__ beta, int angle_stride, const uint8_t* __restrict__ x,
                                  int n, uint32_t leaf_elems, int n_leaves, bool density, V* __restrict__ out,
                                  const double* __restrict__ trig) {
  __shared__ double s_t[4];  // trig values of the leaf's layer, once per block
  const DevLeaf L = leaves[blockIdx.x % n_leaves];
  const int xi = blockIdx.x / n_leaves;
  if (L.gate == -2) return;  // pseudo-leaf: written by the prologue kernel
  const int r = L.rank_nc + L.ncut;
  if (threadIdx.x == 0) {
    s_t[0] = 1.0;
    s_t[1] = 0.0;
    s_t[2] = 1.0;
    s_t[3] = 0.0;
    if (L.gate >= 0) {
      const int l = gate_layer[L.gate];
      if (trig) {  // the layer's values, evaluated once per program (fixed angles)
        for (int j = 0; j < 4; ++j) s_t[j] = trig[4 * l + j];
      } else {
        sincos(gamma[(size_t)xi * angle_stride + l], &s_t[1], &s_t[0]);
        sincos(beta[(size_t)xi * angle_stride + l], &s_t[3], &s_t[2]);
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < (1 << r); e += blockDim.x)
    out[(size_t)xi * leaf_elems + L.base + e] = leaf_entry_trig<V>(L, e, gate_q, gate_in_h, gate_out_kind, gate_kind,
                                                                   s_t, x + (size_t)xi * n, density);
}

// ------------------------------------------------------------- lane exec --

// C[m, n] = sum_k A[m + (k << MA)] * B[k + (n << KB)], stored at the bit
// weights w of C's layout.  A stays in registers while B is streamed one
// column (fixed n) at a time.  Operands stride sa / sb elements, C strides sc.
template <int MA, int NB, int KB, class V, class Ops>
__device__ __forceinline__ V lane_merge(const V* __restrict__ A, int sa, const V* __restrict__ B, int sb,
                                        V* __restrict__ C, int sc, const uint16_t* __restrict__ w,
                                        bool store) {
  constexpr int NA = 1 << (MA + KB);
  constexpr int RC = MA + NB;
  V a[NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) a[i] = A[i * sa];
  uint32_t wl[RC > 0 ? RC : 1];
#pragma unroll
  for (int j = 0; j < RC; ++j) wl[j] = w[j];
  V acc = Ops::zero();
#pragma unroll
  for (int n = 0; n < (1 << NB); ++n) {
    V b[1 << KB];
#pragma unroll
    for (int k = 0; k < (1 << KB); ++k) b[k] = B[(k + (n << KB)) * sb];
#pragma unroll
    for (int m = 0; m < (1 << MA); ++m) {
      acc = Ops::mul(a[m], b[0]);
#pragma unroll
      for (int k = 1; k < (1 << KB); ++k) Ops::fma(acc, a[m + (k << MA)], b[k]);
      Ops::finish(acc);
      if (store) {
        const uint32_t o = (uint32_t)(m + (n << MA));
        uint32_t pos = 0;
#pragma unroll
        for (int j = 0; j < RC; ++j)
          if ((o >> j) & 1u) pos += wl[j];
        C[pos * sc] = acc;
      }
    }
  }
  return acc;
}

#define QTN_SHAPE(MA, NB, KB) ((MA) | ((NB) << 3) | ((KB) << 6))
#define QTN_LANE_CASE(MA, NB, KB)                                 \
  case QTN_SHAPE(MA, NB, KB):                                     \
    r = lane_merge<MA, NB, KB, V, Ops>(A, sa, B, sb, C, sc, w, store); \
    break;
// Every (ma, nb, kb) whose three tensors have rank <= kLaneMaxRank (5).
#define QTN_LANE_CASES \
  QTN_LANE_CASE(0, 0, 0) QTN_LANE_CASE(0, 1, 0) QTN_LANE_CASE(0, 2, 0) QTN_LANE_CASE(0, 3, 0) \
  QTN_LANE_CASE(0, 4, 0) QTN_LANE_CASE(0, 5, 0) QTN_LANE_CASE(1, 0, 0) QTN_LANE_CASE(1, 1, 0) \
  QTN_LANE_CASE(1, 2, 0) QTN_LANE_CASE(1, 3, 0) QTN_LANE_CASE(1, 4, 0) QTN_LANE_CASE(2, 0, 0) \
  QTN_LANE_CASE(2, 1, 0) QTN_LANE_CASE(2, 2, 0) QTN_LANE_CASE(2, 3, 0) QTN_LANE_CASE(3, 0, 0) \
  QTN_LANE_CASE(3, 1, 0) QTN_LANE_CASE(3, 2, 0) QTN_LANE_CASE(4, 0, 0) QTN_LANE_CASE(4, 1, 0) \
  QTN_LANE_CASE(5, 0, 0) QTN_LANE_CASE(0, 0, 1) QTN_LANE_CASE(0, 1, 1) QTN_LANE_CASE(0, 2, 1) \
  QTN_LANE_CASE(0, 3, 1) QTN_LANE_CASE(0, 4, 1) QTN_LANE_CASE(1, 0, 1) QTN_LANE_CASE(1, 1, 1) \
  QTN_LANE_CASE(1, 2, 1) QTN_LANE_CASE(1, 3, 1) QTN_LANE_CASE(1, 4, 1) QTN_LANE_CASE(2, 0, 1) \
  QTN_LANE_CASE(2, 1, 1) QTN_LANE_CASE(2, 2, 1) QTN_LANE_CASE(2, 3, 1) QTN_LANE_CASE(3, 0, 1) \
  QTN_LANE_CASE(3, 1, 1) QTN_LANE_CASE(3, 2, 1) QTN_LANE_CASE(4, 0, 1) QTN_LANE_CASE(4, 1, 1) \
  QTN_LANE_CASE(0, 0, 2) QTN_LANE_CASE(0, 1, 2) QTN_LANE_CASE(0, 2, 2) QTN_LANE_CASE(0, 3, 2) \
  QTN_LANE_CASE(1, 0, 2) QTN_LANE_CASE(1, 1, 2) QTN_LANE_CASE(1, 2, 2) QTN_LANE_CASE(1, 3, 2) \
  QTN_LANE_CASE(2, 0, 2) QTN_LANE_CASE(2, 1, 2) QTN_LANE_CASE(2, 2, 2) QTN_LANE_CASE(2, 3, 2) \
  QTN_LANE_CASE(3, 0, 2) QTN_LANE_CASE(3, 1, 2) QTN_LANE_CASE(3, 2, 2) QTN_LANE_CASE(0, 0, 3) \
  QTN_LANE_CASE(0, 1, 3) QTN_LANE_CASE(0, 2, 3) QTN_LANE_CASE(1, 0, 3) QTN_LANE_CASE(1, 1, 3) \
  QTN_LANE_CASE(1, 2, 3) QTN_LANE_CASE(2, 0, 3) QTN_LANE_CASE(2, 1, 3) QTN_LANE_CASE(2, 2, 3) \
  QTN_LANE_CASE(0, 0, 4) QTN_LANE_CASE(0, 1, 4) QTN_LANE_CASE(1, 0, 4) QTN_LANE_CASE(1, 1, 4) \
  QTN_LANE_CASE(0, 0, 5)

template <class V, class Ops = CplxOps<V>>
__global__ void __launch_bounds__(128) lane_exec_kernel(ExecParams P, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x;
  const SmemLayout lay = smem_layout(P.n_steps, P.n_leaves, P.leaf_elems, P.arena_elems, (int)sizeof(V), T, true);
  DevStep* s_steps = reinterpret_cast<DevStep*>(smem);
  DevLeaf* s_leaves = reinterpret_cast<DevLeaf*>(smem + lay.leaves);
  V* s_lt = reinterpret_cast<V*>(smem + lay.table);
  V* s_arena = reinterpret_cast<V*>(smem + lay.arena);
  Partial* s_red = reinterpret_cast<Partial*>(smem + lay.red);
  const int xi = blockIdx.x / P.blocks_per_x;
  const int bx = blockIdx.x % P.blocks_per_x;
  copy_words(s_steps, P.steps, (size_t)P.n_steps * sizeof(DevStep));
  copy_words(s_leaves, P.leaves, (size_t)P.n_leaves * sizeof(DevLeaf));
  copy_words(s_lt, static_cast<const V*>(P.leaf_tables) + (size_t)xi * P.leaf_elems,
             (size_t)P.leaf_elems * sizeof(V));
  __syncthreads();

  V* ar = s_arena + threadIdx.x;
  double sr = 0.0, si = 0.0, cr = 0.0, ci = 0.0;
  const uint64_t S = P.slice_hi - P.slice_lo;
  for (uint64_t i = (uint64_t)bx * T + threadIdx.x; i < S; i += (uint64_t)P.blocks_per_x * T) {
    const uint64_t s = P.slice_lo + i;
    V res = Ops::zero();
    for (int j = 0; j < P.n_steps; ++j) {
      const DevStep& st = s_steps[j];
      const V* A;
      const V* B;
      int sa, sb;
      if (st.flags & STEP_A_LEAF) {
        A = s_lt + leaf_offset(s_leaves[st.a], s);
        sa = 1;
      } else {
        A = ar + (size_t)st.a * T;
        sa = T;
      }
      if (st.flags & STEP_B_LEAF) {
        B = s_lt + leaf_offset(s_leaves[st.b], s);
        sb = 1;
      } else {
        B = ar + (size_t)st.b * T;
        sb = T;
      }
      V* C = ar + (size_t)st.c * T;
      const int sc = T;
      const uint16_t* w = st.w;
      const bool store = !(st.flags & STEP_ROOT);
      V r = Ops::zero();
      switch (QTN_SHAPE(st.ma, st.nb, st.kb)) {
        QTN_LANE_CASES
        default:
          atomicOr(err, 1);
          break;
      }
      if (!store) res = r;
    }
    kahan_add(sr, cr, Ops::re(res));
    kahan_add(si, ci, Ops::im(res));
    if (P.slices) P.slices[(size_t)xi * S + i] = make_double2(Ops::re(res), Ops::im(res));
  }
  s_red[threadIdx.x] = Partial::make(sr, si, cr, ci);
  tree_reduce(s_red, T);
  if (threadIdx.x == 0) P.partials[(size_t)xi * P.blocks_per_x + bx] = s_red[0];
}

// ------------------------------------------------------------ block exec --

// One merge executed by a group of G threads (G = 32: one warp; G = block
// size), thread t of the group: outputs o = t, t + G, ... of the canonical
// C[m, n, b] = sum_k A[m + (k << ma) + (b << (ma+kb))] * B[k + (n << kb) +
// (b << (kb+nb))].  Results are stored at C + pos(o) (bit weights w), or,
// for the root, added to the thread's compensated sum.  The step's fields
// arrive as scalars (registers): read through shared memory, every store of
// C would force them to be read again.
struct StepRegs {
  int ma, nb, kb, rc;
  bool root;
};

template <class V, int K, class Ops>
__device__ __forceinline__ void group_merge_k(const StepRegs sr_, const uint16_t* __restrict__ w,
                                              const V* __restrict__ A, const V* __restrict__ B, V* __restrict__ C,
                                              uint32_t t, uint32_t G, uint32_t pos_t, int log2G, double& sr,
                                              double& cr, double& si, double& ci, double2* slice_out) {
  const int ma = sr_.ma, nb = sr_.nb, kb = sr_.kb, rc = sr_.rc;
  const uint32_t NC = 1u << rc;
  const uint32_t mmask = (1u << ma) - 1u, nmask = (1u << nb) - 1u;
  for (uint32_t o = t; o < NC; o += G) {
    const uint32_t m = o & mmask, n = (o >> ma) & nmask, b = o >> (ma + nb);
    const V* ap = A + m + (b << (ma + kb));
    const V* bp = B + (n << kb) + (b << (kb + nb));
    using F = typename MergeOps<Ops>::type;
    typename F::Acc acc_ = F::mul(ap[0], bp[0]);
    if (K > 0) {
#pragma unroll
      for (int k = 1; k < K; ++k) F::fma(acc_, ap[k << ma], bp[k]);
    } else {
      for (uint32_t k = 1; k < (1u << kb); ++k) F::fma(acc_, ap[k << ma], bp[k]);
    }
    const V acc = F::result(acc_);
    if (sr_.root) {
      kahan_add(sr, cr, Ops::re(acc));
      kahan_add(si, ci, Ops::im(acc));
      if (slice_out && NC == 1) *slice_out = make_double2(Ops::re(acc), Ops::im(acc));
    } else {
      uint32_t pos = pos_t;
      for (uint32_t hi = o >> log2G; hi; hi &= hi - 1u) pos += w[log2G + __ffs(hi) - 1];
      C[pos] = acc;
    }
  }
}

template <class V, class Ops>
__device__ __forceinline__ void group_merge(const StepRegs r, const uint16_t* w, const V* A, const V* B, V* C,
                                            uint32_t t, uint32_t G, int log2G, double& sr, double& cr, double& si,
                                            double& ci, double2* slice_out) {
  if (t >= (1u << r.rc)) return;  // no output of this merge for the thread
  // Store offset of the thread's own low bits, shared by all its outputs.
  uint32_t pos_t = 0;
  if (!r.root)
    for (int bit = 0; bit < log2G && bit < r.rc; ++bit)
      if ((t >> bit) & 1u) pos_t += w[bit];
  switch (r.kb) {
    case 0: group_merge_k<V, 1, Ops>(r, w, A, B, C, t, G, pos_t, log2G, sr, cr, si, ci, slice_out); break;
    case 1: group_merge_k<V, 2, Ops>(r, w, A, B, C, t, G, pos_t, log2G, sr, cr, si, ci, slice_out); break;
    case 2: group_merge_k<V, 4, Ops>(r, w, A, B, C, t, G, pos_t, log2G, sr, cr, si, ci, slice_out); break;
    case 3: group_merge_k<V, 8, Ops>(r, w, A, B, C, t, G, pos_t, log2G, sr, cr, si, ci, slice_out); break;
    case 4: group_merge_k<V, 16, Ops>(r, w, A, B, C, t, G, pos_t, log2G, sr, cr, si, ci, slice_out); break;
    default: group_merge_k<V, 0, Ops>(r, w, A, B, C, t, G, pos_t, log2G, sr, cr, si, ci, slice_out); break;
  }
}

// Scalars of a step, read once.
__device__ __forceinline__ StepRegs step_regs(const DevStep& st) {
  StepRegs r;
  r.ma = st.ma;
  r.nb = st.nb;
  r.kb = st.kb;
  r.rc = st.ma + st.nb + st.bb;
  r.root = st.flags & STEP_ROOT;
  return r;
}

// All merges of one work item (item s selects the leaves' outer sub-blocks),
// by a group of G threads (thread t); G = 32 synchronises with warp barriers.
template <class V, class Ops, bool WARP_SYNC>
__device__ __forceinline__ void run_item(const DevStep* s_steps, int n_steps, const DevLeaf* s_leaves, const V* s_lt,
                                         V* s_arena, uint64_t s, uint32_t t, uint32_t G, int log2G, double& sr,
                                         double& cr, double& si, double& ci, double2* slice_out) {
  for (int j = 0; j < n_steps; ++j) {
    const DevStep& st = s_steps[j];
    // One 32-bit read (ma | nb | kb | bb) decides whether this thread has an
    // output; most merges of an item are small, so most warps skip here.
    const uint32_t hdr = *reinterpret_cast<const uint32_t*>(&st);
    const int rc_h = (int)((hdr & 0xffu) + ((hdr >> 8) & 0xffu) + (hdr >> 24));
    if (t < (1u << rc_h)) {
      const StepRegs r = step_regs(st);
      const uint8_t flags = st.flags;
      const uint32_t ao = st.a, bo = st.b, co = st.c;
      const V* A = (flags & STEP_A_LEAF) ? s_lt + leaf_offset(s_leaves[ao], s) : s_arena + ao;
      const V* B = (flags & STEP_B_LEAF) ? s_lt + leaf_offset(s_leaves[bo], s) : s_arena + bo;
      group_merge<V, Ops>(r, st.w, A, B, s_arena + co, t, G, log2G, sr, cr, si, ci, slice_out);
    }
    if (WARP_SYNC) __syncwarp();
    else __syncthreads();
  }
}

// Work items: a slice (per-slice programs) or one assignment of the outer
// slice classes (batched programs, whose tensors carry the inner classes as
// batch bits: every merge then runs once per distinct value of the inner
// bits it depends on, and the root holds the scalars of all slices of the
// item).  WARP_ITEMS: every warp contracts its own items in its own arena
// (barriers are warp barriers); otherwise the whole block works on one item.
template <class V, bool WARP_ITEMS, class Ops = CplxOps<V>>
__global__ void __launch_bounds__(256) block_exec_kernel(ExecParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x;
  const int groups = WARP_ITEMS ? T / 32 : 1;
  const SmemLayout lay =
      smem_layout(P.n_steps, P.n_leaves, P.leaf_elems, P.arena_elems * groups, (int)sizeof(V), T, false);
  DevStep* s_steps = reinterpret_cast<DevStep*>(smem);
  DevLeaf* s_leaves = reinterpret_cast<DevLeaf*>(smem + lay.leaves);
  V* s_lt = reinterpret_cast<V*>(smem + lay.table);
  Partial* s_red = reinterpret_cast<Partial*>(smem + lay.red);
  const int xi = blockIdx.x / P.blocks_per_x;
  const int bx = blockIdx.x % P.blocks_per_x;
  copy_words(s_steps, P.steps, (size_t)P.n_steps * sizeof(DevStep));
  copy_words(s_leaves, P.leaves, (size_t)P.n_leaves * sizeof(DevLeaf));
  copy_words(s_lt, static_cast<const V*>(P.leaf_tables) + (size_t)xi * P.leaf_elems,
             (size_t)P.leaf_elems * sizeof(V));
  __syncthreads();

  const uint32_t G = WARP_ITEMS ? 32u : (uint32_t)T;
  const int log2G = 31 - __clz((int)G);
  const int grp = WARP_ITEMS ? threadIdx.x / 32 : 0;
  const uint32_t t = threadIdx.x % G;
  V* s_arena = reinterpret_cast<V*>(smem + lay.arena) + (size_t)grp * P.arena_elems;
  double sr = 0.0, si = 0.0, cr = 0.0, ci = 0.0;
  const uint64_t S = P.slice_hi - P.slice_lo;
  const uint64_t stride = (uint64_t)P.blocks_per_x * groups;
  for (uint64_t i = (uint64_t)bx * groups + grp; i < S; i += stride) {
    double2* slice_out = P.slices ? P.slices + (size_t)xi * S + i : nullptr;
    run_item<V, Ops, WARP_ITEMS>(s_steps, P.n_steps, s_leaves, s_lt, s_arena, P.slice_lo + i, t, G, log2G, sr, cr,
                                 si, ci, slice_out);
  }
  s_red[threadIdx.x] = Partial::make(sr, si, cr, ci);
  tree_reduce(s_red, T);
  if (threadIdx.x == 0) P.partials[(size_t)xi * P.blocks_per_x + bx] = s_red[0];
}

// ------------------------------------------------------------ level exec --

// Shared memory of the level executor: steps, per-step output starts, level
// table, leaves, leaf table, then `items` arenas of `stride` elements, which
// the per-thread partials overlay once the last level is done.
struct LevelLayout {
  size_t out_start, nib, levels, leaves, table, arena, red, total;
};
__host__ __device__ inline LevelLayout level_layout(int n_steps, int n_levels, int n_leaves, uint32_t leaf_elems,
                                                    uint32_t stride, int items, int elem_bytes, int threads) {
  LevelLayout L;
  L.out_start = align16((size_t)n_steps * sizeof(DevStep));
  L.nib = L.out_start + align16((size_t)n_steps * 2 * sizeof(uint32_t));
  // Nibble tables of store offsets: 16-byte types only (one output per unit;
  // complex64 units of four compute one offset per four outputs).
  L.levels = L.nib + (elem_bytes == 16 ? align16((size_t)n_steps * kPosNibEntries * sizeof(uint16_t)) : 0);
  L.leaves = L.levels + align16((size_t)n_levels * sizeof(DevLevel));
  L.table = L.leaves + align16((size_t)n_leaves * sizeof(DevLeaf));
  L.arena = L.table + align16((size_t)leaf_elems * elem_bytes);
  L.red = L.arena;
  const size_t arena_bytes = (size_t)stride * items * elem_bytes, red_bytes = (size_t)threads * sizeof(Partial);
  L.total = L.arena + align16(arena_bytes > red_bytes ? arena_bytes : red_bytes);
  return L;
}

struct LevelParams {
  const DevLevel* levels;
  const uint32_t* out_start;
  const uint16_t* pos_nib;
  int n_levels;
  int log2_items;
  uint32_t arena_stride;
};

// A merge's fields, decoded once into registers while a thread stays on it.
struct LStep {
  uint32_t beg, end;  // its units in the level's flat range
  uint32_t a, b, c;
  int ma, nb, kb, ks;
  uint32_t ulog;      // log2 entries per unit
  int groups;         // nibbles of an output index
  uint8_t flags;
  const uint16_t* nib;  // store offsets by nibble (shared memory; 16-byte types)
  const uint16_t* w;    // store bit weights (shared memory)
};

// One unit of a (non-root) merge for one item: outputs o0 .. o0 + u - 1
// (u <= UNIT), C[pos(o)] = sum_k A[..k..] B[..k..] in the merge's canonical
// form.  o0 is a multiple of u, so pos(o0 + r) = pos(o0) + the weights of
// r's low bits.
template <class V, int K, class Ops, int UNIT>
__device__ __forceinline__ void level_unit(const LStep& q, uint32_t o0, uint32_t u, const V* __restrict__ A,
                                           const V* __restrict__ B, V* __restrict__ C) {
  const int ma = q.ma, nb = q.nb, kb = q.kb;
  uint32_t pos0 = 0;
  if (UNIT == 1) {
    for (int g = 0; g < q.groups; ++g) pos0 += q.nib[16 * g + ((o0 >> (4 * g)) & 15u)];
  } else {
    for (uint32_t x = o0; x; x &= x - 1u) pos0 += q.w[__ffs(x) - 1];
  }
  const uint32_t w0 = UNIT > 1 ? q.w[0] : 0u, w1 = UNIT > 2 ? q.w[1] : 0u;
  const uint32_t mmask = (1u << ma) - 1u, nmask = (1u << nb) - 1u;
#pragma unroll
  for (uint32_t r = 0; r < (uint32_t)UNIT; ++r) {
    if (r < u) {
      const uint32_t o = o0 + r;
      const uint32_t m = o & mmask, n = (o >> ma) & nmask, b = o >> (ma + nb);
      const V* ap = A + m + (b << (ma + kb));
      const V* bp = B + (n << kb) + (b << (kb + nb));
      using F = typename MergeOps<Ops>::type;
      typename F::Acc acc_ = F::mul(ap[0], bp[0]);
      if (K > 0) {
#pragma unroll
        for (int k = 1; k < K; ++k) F::fma(acc_, ap[k << ma], bp[k]);
      } else {
        for (uint32_t k = 1; k < (1u << kb); ++k) F::fma(acc_, ap[k << ma], bp[k]);
      }
      C[pos0 + ((r & 1u) ? w0 : 0u) + ((r & 2u) ? w1 : 0u)] = F::result(acc_);
    }
  }
}

// Units per step for the level executor's unit size 2^UL.
__device__ __forceinline__ int root_split(const DevStep& st) {
  return (st.flags & STEP_ROOT) ? (st.kb < kRootSplitLog2 ? st.kb : kRootSplitLog2) : 0;
}

template <int UL>
__device__ __forceinline__ uint32_t level_units(const DevStep& st) {
  const int rc = st.ma + st.nb + st.bb + (UL ? root_split(st) : 0);
  return 1u << (rc > UL ? rc - UL : 0);
}

// The root of one item, its sum over k split into 2^ks parts: entries
// e = (o, part) (part fastest) for e in [e0, e0 + u); each part's partial
// sum over its k range is added to the compensated sums (the root's outputs
// are only summed).
template <class V, class Ops, int UNIT>
__device__ __forceinline__ void level_root_unit(const LStep& q, uint32_t e0, uint32_t u, const V* __restrict__ A,
                                                const V* __restrict__ B, double& sr, double& cr, double& si,
                                                double& ci) {
  const int ma = q.ma, nb = q.nb, kb = q.kb, ks = q.ks;
  const uint32_t kpart = 1u << (kb - ks);
#pragma unroll
  for (uint32_t r = 0; r < (uint32_t)UNIT; ++r) {
    if (r < u) {
      const uint32_t e = e0 + r;
      const uint32_t part = e & ((1u << ks) - 1u), o = e >> ks;
      const uint32_t m = o & ((1u << ma) - 1u), n = (o >> ma) & ((1u << nb) - 1u), b = o >> (ma + nb);
      const uint32_t k0 = part * kpart;
      const V* ap = A + m + (k0 << ma) + (b << (ma + kb));
      const V* bp = B + k0 + (n << kb) + (b << (kb + nb));
      using F = typename MergeOps<Ops>::type;
      typename F::Acc acc_ = F::mul(ap[0], bp[0]);
      for (uint32_t k = 1; k < kpart; ++k) F::fma(acc_, ap[k << ma], bp[k]);
      const V acc = F::result(acc_);
      kahan_add(sr, cr, Ops::re(acc));
      kahan_add(si, ci, Ops::im(acc));
    }
  }
}

// All levels of one group of nI <= 2^log2I consecutive work items (global
// index s0 + item).  For each level the units of all its merges, for all
// those items, form one flat range (item index fastest) that the threads
// stride over; one barrier ends the level.  Item arenas are `stride`
// elements apart (an odd stride, so the items of one warp hit different
// banks).  Units: four outputs per thread for complex64 (amortises a merge's
// decode over cheap arithmetic), one for the 16-byte types (their arithmetic
// dominates, and a level keeps four times more threads busy).
template <class V, class Ops>
__device__ __forceinline__ void level_run(const DevStep* s_steps, const uint32_t* s_out, const uint16_t* s_nib,
                                          const DevLevel* s_levels, int n_levels, const DevLeaf* s_leaves,
                                          const V* s_lt, V* s_arena,
                                          uint32_t stride, uint32_t log2I, uint64_t s0,
                                          uint32_t nI, double& sr, double& cr, double& si, double& ci,
                                          V* g_lt = nullptr) {
  constexpr int UL = sizeof(V) == 16 ? 0 : kLevelUnitLog2;  // log2 outputs per unit
  constexpr int US = UL ? 1 : 0;                            // which unit table
  const uint32_t I = 1u << log2I;
  auto decode = [&](int j, LStep& q) {
    const DevStep& st = s_steps[j];
    q.ma = st.ma;
    q.nb = st.nb;
    q.kb = st.kb;
    q.flags = st.flags;
    q.a = st.a;
    q.b = st.b;
    q.c = (st.flags & STEP_EXPORT) ? s_leaves[st.c].base : st.c;
    q.nib = s_nib + (size_t)j * kPosNibEntries;
    q.w = st.w;
    q.groups = (st.ma + st.nb + st.bb + 3) >> 2;
    q.ks = UL ? root_split(st) : 0;  // split roots in the four-output table only
    const int rc = st.ma + st.nb + st.bb + q.ks;
    q.ulog = rc < UL ? (uint32_t)rc : (uint32_t)UL;
    q.beg = s_out[2 * j + US];
    q.end = q.beg + (1u << (rc - (int)q.ulog));
  };
  for (int l = 0; l < n_levels; ++l) {
    const DevLevel lv = s_levels[l];
    const uint32_t total = lv.units[US] << log2I;
    LStep q;
    q.beg = q.end = 0;
    for (uint32_t f = threadIdx.x; f < total; f += blockDim.x) {
      const uint32_t item = f & (I - 1u), uf = f >> log2I;
      if (uf >= q.end || uf < q.beg) {
        // The level's merge holding unit uf: binary search of the (strictly
        // increasing) unit starts, then one decode.
        int lo = lv.first, hi = lv.first + lv.count - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_out[2 * mid + US] <= uf) lo = mid;
          else hi = mid - 1;
        }
        decode(lo, q);
      }
      if (item >= nI) continue;
      V* arena = s_arena + (size_t)item * stride;
      const V* A = (q.flags & STEP_A_LEAF) ? s_lt + leaf_offset(s_leaves[q.a], s0 + item) : arena + q.a;
      const V* B = (q.flags & STEP_B_LEAF) ? s_lt + leaf_offset(s_leaves[q.b], s0 + item) : arena + q.b;
      const uint32_t u = 1u << q.ulog;
      const uint32_t o0 = (uf - q.beg) << q.ulog;
      if (q.flags & STEP_ROOT) {
        level_root_unit<V, Ops, 1 << UL>(q, o0, u, A, B, sr, cr, si, ci);
        continue;
      }
      // Prologue steps may export their result into the (global) leaf table.
      V* C = (q.flags & STEP_EXPORT) ? g_lt + q.c : arena + q.c;
      switch (q.kb) {
        case 0: level_unit<V, 1, Ops, 1 << UL>(q, o0, u, A, B, C); break;
        case 1: level_unit<V, 2, Ops, 1 << UL>(q, o0, u, A, B, C); break;
        case 2: level_unit<V, 4, Ops, 1 << UL>(q, o0, u, A, B, C); break;
        case 3: level_unit<V, 8, Ops, 1 << UL>(q, o0, u, A, B, C); break;
        default: level_unit<V, 0, Ops, 1 << UL>(q, o0, u, A, B, C); break;
      }
    }
    __syncthreads();  // also orders the last level's arena reads before later reuse of the arena
  }
}

// Level executor: a block takes 2^log2_items consecutive work items at a
// time and runs them level by level (level_run).
template <class V, class Ops = CplxOps<V>>
__global__ void __launch_bounds__(1024) level_exec_kernel(ExecParams P, LevelParams LP) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x;
  const uint32_t log2I = (uint32_t)LP.log2_items;
  const uint32_t I = 1u << log2I;
  const LevelLayout lay = level_layout(P.n_steps, LP.n_levels, P.n_leaves, P.leaf_elems, LP.arena_stride, (int)I,
                                       (int)sizeof(V), T);
  DevStep* s_steps = reinterpret_cast<DevStep*>(smem);
  uint32_t* s_out = reinterpret_cast<uint32_t*>(smem + lay.out_start);
  uint16_t* s_nib = reinterpret_cast<uint16_t*>(smem + lay.nib);
  DevLevel* s_levels = reinterpret_cast<DevLevel*>(smem + lay.levels);
  DevLeaf* s_leaves = reinterpret_cast<DevLeaf*>(smem + lay.leaves);
  V* s_lt = reinterpret_cast<V*>(smem + lay.table);
  V* s_arena = reinterpret_cast<V*>(smem + lay.arena);
  Partial* s_red = reinterpret_cast<Partial*>(smem + lay.red);
  const int xi = blockIdx.x / P.blocks_per_x;
  const int bx = blockIdx.x % P.blocks_per_x;
  copy_words(s_steps, P.steps, (size_t)P.n_steps * sizeof(DevStep));
  copy_words(s_out, LP.out_start, (size_t)P.n_steps * 2 * sizeof(uint32_t));
  if (sizeof(V) == 16) copy_words(s_nib, LP.pos_nib, (size_t)P.n_steps * kPosNibEntries * sizeof(uint16_t));
  copy_words(s_levels, LP.levels, (size_t)LP.n_levels * sizeof(DevLevel));
  copy_words(s_leaves, P.leaves, (size_t)P.n_leaves * sizeof(DevLeaf));
  copy_words(s_lt, static_cast<const V*>(P.leaf_tables) + (size_t)xi * P.leaf_elems,
             (size_t)P.leaf_elems * sizeof(V));
  __syncthreads();

  double sr = 0.0, si = 0.0, cr = 0.0, ci = 0.0;
  const uint64_t S = P.slice_hi - P.slice_lo;
  for (uint64_t i0 = (uint64_t)bx * I; i0 < S; i0 += (uint64_t)P.blocks_per_x * I) {
    const uint32_t nI = (uint32_t)((S - i0) < I ? (S - i0) : I);
    level_run<V, Ops>(s_steps, s_out, s_nib, s_levels, LP.n_levels, s_leaves, s_lt, s_arena, LP.arena_stride,
                      log2I, P.slice_lo + i0, nI, sr, cr, si, ci);
  }
  s_red[threadIdx.x] = Partial::make(sr, si, cr, ci);  // overlays the arenas: every level is done
  tree_reduce(s_red, T);
  if (threadIdx.x == 0) P.partials[(size_t)xi * P.blocks_per_x + bx] = s_red[0];
}

// Hoisted merges of a level-ordered program: one block of up to 1024
// threads per bit string, one barrier per level; exported results go to the
// bit string's leaf table in global memory.
template <class V, class Ops>
__device__ __forceinline__ void prologue_level_body(const DevStep* __restrict__ steps, int n_steps,
                                                    const uint32_t* __restrict__ out_start,
                                                    const uint16_t* __restrict__ pos_nib,
                                                    const DevLevel* __restrict__ levels, int n_levels,
                                                    const DevLeaf* __restrict__ leaves, int n_leaves, V* g_lt,
                                                    uint32_t leaf_elems, uint32_t arena_elems, unsigned char* smem) {
  const LevelLayout lay = level_layout(n_steps, n_levels, n_leaves, leaf_elems, arena_elems | 1u, 1, (int)sizeof(V),
                                       blockDim.x);
  DevStep* s_steps = reinterpret_cast<DevStep*>(smem);
  uint32_t* s_out = reinterpret_cast<uint32_t*>(smem + lay.out_start);
  uint16_t* s_nib = reinterpret_cast<uint16_t*>(smem + lay.nib);
  DevLevel* s_levels = reinterpret_cast<DevLevel*>(smem + lay.levels);
  DevLeaf* s_leaves = reinterpret_cast<DevLeaf*>(smem + lay.leaves);
  V* s_lt = reinterpret_cast<V*>(smem + lay.table);
  V* s_arena = reinterpret_cast<V*>(smem + lay.arena);
  copy_words(s_steps, steps, (size_t)n_steps * sizeof(DevStep));
  copy_words(s_out, out_start, (size_t)n_steps * 2 * sizeof(uint32_t));
  if (sizeof(V) == 16) copy_words(s_nib, pos_nib, (size_t)n_steps * kPosNibEntries * sizeof(uint16_t));
  copy_words(s_levels, levels, (size_t)n_levels * sizeof(DevLevel));
  copy_words(s_leaves, leaves, (size_t)n_leaves * sizeof(DevLeaf));
  copy_words(s_lt, g_lt, (size_t)leaf_elems * sizeof(V));
  __syncthreads();
  double sr = 0, si = 0, cr = 0, ci = 0;  // no root among hoisted merges
  level_run<V, Ops>(s_steps, s_out, s_nib, s_levels, n_levels, s_leaves, s_lt, s_arena, arena_elems | 1u, 0, 0, 1, sr,
                    cr, si, ci, g_lt);
}

template <class V, class Ops = CplxOps<V>>
__global__ void __launch_bounds__(1024) prologue_level_kernel(const DevStep* __restrict__ steps, int n_steps,
                                                              const uint32_t* __restrict__ out_start,
                                                              const uint16_t* __restrict__ pos_nib,
                                                              const DevLevel* __restrict__ levels, int n_levels,
                                                              const DevLeaf* __restrict__ leaves, int n_leaves,
                                                              void* leaf_tables, uint32_t leaf_elems,
                                                              uint32_t arena_elems) {
  extern __shared__ __align__(16) unsigned char smem[];
  V* g_lt = static_cast<V*>(leaf_tables) + (size_t)blockIdx.x * leaf_elems;
  prologue_level_body<V, Ops>(steps, n_steps, out_start, pos_nib, levels, n_levels, leaves, n_leaves, g_lt,
                              leaf_elems, arena_elems, smem);
}

// -------------------------------------------------------------- prologue --

// Hoisted merges (no outer slice class below them): run once per bit string
// (one block each); exported results become pseudo-leaves of the leaf table.
template <class V, class Ops>
__device__ __forceinline__ void prologue_body(const DevStep* __restrict__ steps, int n_steps,
                                              const DevLeaf* __restrict__ leaves, int n_leaves, V* g_lt,
                                              uint32_t leaf_elems, uint32_t arena_elems, unsigned char* smem) {
  const int T = blockDim.x;
  const SmemLayout lay = smem_layout(n_steps, n_leaves, leaf_elems, arena_elems, (int)sizeof(V), T, false);
  DevStep* s_steps = reinterpret_cast<DevStep*>(smem);
  DevLeaf* s_leaves = reinterpret_cast<DevLeaf*>(smem + lay.leaves);
  V* s_lt = reinterpret_cast<V*>(smem + lay.table);
  V* s_arena = reinterpret_cast<V*>(smem + lay.arena);
  copy_words(s_steps, steps, (size_t)n_steps * sizeof(DevStep));
  copy_words(s_leaves, leaves, (size_t)n_leaves * sizeof(DevLeaf));
  copy_words(s_lt, g_lt, (size_t)leaf_elems * sizeof(V));
  __syncthreads();
  const int log2G = 31 - __clz(T);
  double sr = 0, si = 0, cr = 0, ci = 0;
  for (int j = 0; j < n_steps; ++j) {
    const DevStep& st = s_steps[j];
    const StepRegs r = step_regs(st);
    if (threadIdx.x < (1u << r.rc)) {
      const uint8_t flags = st.flags;
      const uint32_t ao = st.a, bo = st.b, co = st.c;
      const V* A = (flags & STEP_A_LEAF) ? s_lt + s_leaves[ao].base : s_arena + ao;
      const V* B = (flags & STEP_B_LEAF) ? s_lt + s_leaves[bo].base : s_arena + bo;
      V* C = (flags & STEP_EXPORT) ? g_lt + s_leaves[co].base : s_arena + co;
      group_merge<V, Ops>(r, st.w, A, B, C, threadIdx.x, T, log2G, sr, cr, si, ci, nullptr);
    }
    __syncthreads();
  }
}

// Hoisted merges (no outer slice class below them): run once per bit string
// (one block each); exported results become pseudo-leaves of the leaf table.
template <class V, class Ops = CplxOps<V>>
__global__ void __launch_bounds__(256) prologue_kernel(const DevStep* __restrict__ steps, int n_steps,
                                                       const DevLeaf* __restrict__ leaves, int n_leaves,
                                                       void* leaf_tables, uint32_t leaf_elems, uint32_t arena_elems) {
  extern __shared__ __align__(16) unsigned char smem[];
  V* g_lt = static_cast<V*>(leaf_tables) + (size_t)blockIdx.x * leaf_elems;
  prologue_body<V, Ops>(steps, n_steps, leaves, n_leaves, g_lt, leaf_elems, arena_elems, smem);
}

// ------------------------------------------------------------ abort check --

// Stop conditions of a persistent launch, checked by one thread per block
// before it takes a chunk (nothing ever waits): a host-mapped cancel word
// set by another host thread, or a time budget (ns of %globaltimer since the
// block started; 0 = none).  The first block that stops records it in
// `status`; every block then stops at its next chunk.
struct AbortCtl {
  const volatile int* cancel;
  unsigned* status;
  uint64_t budget_ns;
};
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool should_stop(const AbortCtl& ac, uint64_t t_start) {
  if (!ac.status) return false;
  if (*reinterpret_cast<volatile unsigned*>(ac.status) != 0u) return true;
  bool stop = ac.cancel && *ac.cancel != 0;
  if (!stop && ac.budget_ns && global_ns() - t_start > ac.budget_ns) stop = true;
  if (stop) atomicExch(ac.status, 1u);
  return stop;
}

// ------------------------------------------------------------- multi-job --

// Many independent (plan, bit string) jobs in one launch sequence: leaf
// tables of all jobs, one prologue block per job, a persistent executor that
// takes chunks (job, item range) from a counter -- in the order of
// descending job cost the host gave them -- and loads a job's program into
// shared memory when its job changes, then one finalising block per job.
__device__ __forceinline__ int job_of_leaf(const JobDesc* jobs, int njobs, uint32_t b) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {  // last job with leaf_start <= b
    const int mid = (lo + hi + 1) / 2;
    if (jobs[mid].leaf_start <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <class V>
__global__ void multi_leaf_kernel(const JobDesc* __restrict__ jobs, int njobs) {
  const int j = job_of_leaf(jobs, njobs, blockIdx.x);
  const JobDesc& J = jobs[j];
  const DevLeaf L = J.leaves[blockIdx.x - J.leaf_start];
  if (L.gate == -2) return;
  const int r = L.rank_nc + L.ncut;
  V* out = static_cast<V*>(J.leaf_table);
  for (int e = threadIdx.x; e < (1 << r); e += blockDim.x)
    out[L.base + e] = leaf_entry<V>(L, e, J.gate_q, J.gate_layer, J.gate_in_h, J.gate_out_kind, J.gate_kind,
                                    J.gamma, J.beta, J.x, J.density != 0);
}

template <class V, class Ops = CplxOps<V>>
__global__ void __launch_bounds__(256) multi_prologue_kernel(const JobDesc* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char smem[];
  const JobDesc& J = jobs[blockIdx.x];
  if (J.n_pro_steps == 0) return;
  prologue_body<V, Ops>(J.pro_steps, J.n_pro_steps, J.leaves, J.n_leaves, static_cast<V*>(J.leaf_table),
                        J.leaf_elems, J.pro_arena_elems, smem);
}

// The same for level programs (level-ordered prologues, 1024 threads).
template <class V, class Ops = CplxOps<V>>
__global__ void __launch_bounds__(1024) multi_prologue_level_kernel(const JobDesc* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char smem[];
  const JobDesc& J = jobs[blockIdx.x];
  if (J.n_pro_steps == 0) return;
  prologue_level_body<V, Ops>(J.pro_steps, J.n_pro_steps, J.pro_out_start, J.pro_pos_nib, J.pro_levels,
                              J.n_pro_levels, J.leaves, J.n_leaves, static_cast<V*>(J.leaf_table), J.leaf_elems,
                              J.pro_arena_elems, smem);
}

template <class V, class Ops = CplxOps<V>>
__global__ void __launch_bounds__(256) multi_exec_kernel(const JobDesc* __restrict__ jobs,
                                                         const ChunkDesc* __restrict__ chunks, uint32_t n_chunks,
                                                         unsigned* __restrict__ counter,
                                                         Partial* __restrict__ chunk_partials, AbortCtl ac) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned s_c;
  __shared__ int s_job;
  const int T = blockDim.x;
  const int log2G = 31 - __clz(T);
  if (threadIdx.x == 0) s_job = -1;
  const uint64_t t_start = threadIdx.x == 0 ? global_ns() : 0;
  for (;;) {
    __syncthreads();  // the previous chunk is done with shared memory
    if (threadIdx.x == 0) s_c = should_stop(ac, t_start) ? n_chunks : atomicAdd(counter, 1u);
    __syncthreads();
    const unsigned c = s_c;
    if (c >= n_chunks) break;
    const ChunkDesc ch = chunks[c];
    const JobDesc& J = jobs[ch.job];
    const SmemLayout lay = smem_layout(J.n_steps, J.n_leaves, J.leaf_elems, J.arena_elems, (int)sizeof(V), T, false);
    DevStep* s_steps = reinterpret_cast<DevStep*>(smem);
    DevLeaf* s_leaves = reinterpret_cast<DevLeaf*>(smem + lay.leaves);
    V* s_lt = reinterpret_cast<V*>(smem + lay.table);
    V* s_arena = reinterpret_cast<V*>(smem + lay.arena);
    Partial* s_red = reinterpret_cast<Partial*>(smem + lay.red);
    if (s_job != (int)ch.job) {
      copy_words(s_steps, J.steps, (size_t)J.n_steps * sizeof(DevStep));
      copy_words(s_leaves, J.leaves, (size_t)J.n_leaves * sizeof(DevLeaf));
      copy_words(s_lt, J.leaf_table, (size_t)J.leaf_elems * sizeof(V));
      __syncthreads();
      if (threadIdx.x == 0) s_job = (int)ch.job;
    }
    double sr = 0.0, si = 0.0, cr = 0.0, ci = 0.0;
    for (uint64_t it = ch.lo; it < ch.hi; ++it)
      run_item<V, Ops, false>(s_steps, J.n_steps, s_leaves, s_lt, s_arena, it, threadIdx.x, T, log2G, sr, cr, si,
                              ci, nullptr);
    s_red[threadIdx.x] = Partial::make(sr, si, cr, ci);
    tree_reduce(s_red, T);
    if (threadIdx.x == 0) chunk_partials[c] = s_red[0];
  }
}

// The multi-job executor on level programs: chunks are (job, item range)
// with the range a multiple of the job's items per block (the last one may
// be short); the job's program, level table and leaf table are loaded into
// shared memory when the job changes.
template <class V, class Ops = CplxOps<V>>
__global__ void __launch_bounds__(1024) multi_level_kernel(const JobDesc* __restrict__ jobs,
                                                           const ChunkDesc* __restrict__ chunks, uint32_t n_chunks,
                                                           unsigned* __restrict__ counter,
                                                           Partial* __restrict__ chunk_partials, AbortCtl ac) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned s_c;
  __shared__ int s_job;
  const int T = blockDim.x;
  if (threadIdx.x == 0) s_job = -1;
  const uint64_t t_start = threadIdx.x == 0 ? global_ns() : 0;
  for (;;) {
    __syncthreads();  // the previous chunk is done with shared memory
    if (threadIdx.x == 0) s_c = should_stop(ac, t_start) ? n_chunks : atomicAdd(counter, 1u);
    __syncthreads();
    const unsigned c = s_c;
    if (c >= n_chunks) break;
    const ChunkDesc ch = chunks[c];
    const JobDesc& J = jobs[ch.job];
    const uint32_t log2I = (uint32_t)J.log2_items;
    const uint32_t I = 1u << log2I;
    const LevelLayout lay = level_layout(J.n_steps, J.n_levels, J.n_leaves, J.leaf_elems, J.arena_stride, (int)I,
                                         (int)sizeof(V), T);
    DevStep* s_steps = reinterpret_cast<DevStep*>(smem);
    uint32_t* s_out = reinterpret_cast<uint32_t*>(smem + lay.out_start);
    uint16_t* s_nib = reinterpret_cast<uint16_t*>(smem + lay.nib);
    DevLevel* s_levels = reinterpret_cast<DevLevel*>(smem + lay.levels);
    DevLeaf* s_leaves = reinterpret_cast<DevLeaf*>(smem + lay.leaves);
    V* s_lt = reinterpret_cast<V*>(smem + lay.table);
    V* s_arena = reinterpret_cast<V*>(smem + lay.arena);
    Partial* s_red = reinterpret_cast<Partial*>(smem + lay.red);
    if (s_job != (int)ch.job) {
      copy_words(s_steps, J.steps, (size_t)J.n_steps * sizeof(DevStep));
      copy_words(s_out, J.out_start, (size_t)J.n_steps * 2 * sizeof(uint32_t));
      if (sizeof(V) == 16) copy_words(s_nib, J.pos_nib, (size_t)J.n_steps * kPosNibEntries * sizeof(uint16_t));
      copy_words(s_levels, J.levels, (size_t)J.n_levels * sizeof(DevLevel));
      copy_words(s_leaves, J.leaves, (size_t)J.n_leaves * sizeof(DevLeaf));
      copy_words(s_lt, J.leaf_table, (size_t)J.leaf_elems * sizeof(V));
      __syncthreads();
      if (threadIdx.x == 0) s_job = (int)ch.job;
    }
    double sr = 0.0, si = 0.0, cr = 0.0, ci = 0.0;
    for (uint64_t i0 = ch.lo; i0 < ch.hi; i0 += I) {
      const uint32_t nI = (uint32_t)((ch.hi - i0) < I ? (ch.hi - i0) : I);
      level_run<V, Ops>(s_steps, s_out, s_nib, s_levels, J.n_levels, s_leaves, s_lt, s_arena, J.arena_stride,
                        log2I, i0, nI, sr, cr, si, ci);
    }
    s_red[threadIdx.x] = Partial::make(sr, si, cr, ci);  // overlays the arenas
    tree_reduce(s_red, T);
    if (threadIdx.x == 0) chunk_partials[c] = s_red[0];
  }
}

__global__ void __launch_bounds__(128) multi_finalize_kernel(const JobDesc* __restrict__ jobs,
                                                             const Partial* __restrict__ chunk_partials,
                                                             double2* __restrict__ out) {
  __shared__ Partial red[128];
  const JobDesc& J = jobs[blockIdx.x];
  double a = 0, b = 0, ca = 0, cb = 0;
  for (uint32_t t = threadIdx.x; t < J.n_chunks; t += blockDim.x) {
    const Partial v = chunk_partials[J.first_chunk + t];
    kahan_add(a, ca, v.re);
    kahan_add(a, ca, -v.cre);
    kahan_add(b, cb, v.im);
    kahan_add(b, cb, -v.cim);
  }
  red[threadIdx.x] = Partial::make(a, b, ca, cb);
  tree_reduce(red, 128);
  if (threadIdx.x == 0) {
    const Partial v = red[0];
    out[blockIdx.x] = make_double2((v.re - v.cre) * J.scale, (v.im - v.cim) * J.scale);
  }
}

// -------------------------------------------------------------- finalize --

// One block per bit string: thread t adds partials t, t + T, ... in order
// (compensated), then the per-thread partials are combined by a fixed
// pairwise tree.  The grouping depends only on the block count, so the result
// is deterministic.
__global__ void __launch_bounds__(128) finalize_kernel(const Partial* __restrict__ partials, int blocks,
                                                       double scale, double2* __restrict__ out,
                                                       Partial* __restrict__ raw) {
  __shared__ Partial red[128];
  const int xi = blockIdx.x;
  double a = 0, b = 0, ca = 0, cb = 0;
  for (int t = threadIdx.x; t < blocks; t += blockDim.x) {
    const Partial v = partials[(size_t)xi * blocks + t];
    kahan_add(a, ca, v.re);
    kahan_add(a, ca, -v.cre);
    kahan_add(b, cb, v.im);
    kahan_add(b, cb, -v.cim);
  }
  red[threadIdx.x] = Partial::make(a, b, ca, cb);
  tree_reduce(red, 128);
  if (threadIdx.x == 0) {
    const Partial v = red[0];
    if (out) out[xi] = make_double2((v.re - v.cre) * scale, (v.im - v.cim) * scale);
    if (raw) raw[xi] = v;
  }
}

int g_num_sms = 0;

template <class Ops>
struct LaneCapable : std::false_type {};
template <class V>
struct LaneCapable<CplxOps<V>> : std::true_type {};

// Every kernel's dynamic shared memory cap is set to the device's opt-in
// maximum, not to one launch's size: a cap is global per kernel, and a
// captured graph of one plan must stay valid after another plan launches the
// same kernel with less shared memory.
int max_optin_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}
template <class K>
cudaError_t allow_max_smem(K kernel) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  // Static and dynamic shared memory together may not exceed the opt-in maximum.
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              max_optin_smem() - (int)fa.sharedSizeBytes);
}

template <class K>
bool shape_for_kernel(K kernel, int threads, size_t smem, int* occ) {
  if (allow_max_smem(kernel) != cudaSuccess) return false;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kernel, threads, smem) == cudaSuccess && *occ >= 1;
}

template <class V, class Ops>
bool exec_shape_typed(const DeviceProgram& prog, int nx, uint64_t slices_per_x, ExecShape* out) {
  const int elem_bytes = (int)sizeof(V);
  int dev = 0;
  cudaGetDevice(&dev);
  if (g_num_sms == 0) {
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  int max_optin = 0;
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  ExecShape sh;
  int occ = 0;
  uint64_t per_block_items = 1;
  if (prog.exec == Executor::Lane) {
    if constexpr (!LaneCapable<Ops>::value) {
      return false;
    } else {
      sh.threads = 128;
      SmemLayout L = smem_layout(prog.n_steps, prog.n_leaves, prog.leaf_elems, prog.arena_elems, elem_bytes,
                                 sh.threads, true);
      if (L.total > (size_t)max_optin) {
        sh.threads = 64;
        L = smem_layout(prog.n_steps, prog.n_leaves, prog.leaf_elems, prog.arena_elems, elem_bytes, sh.threads,
                        true);
      }
      if (L.total > (size_t)max_optin) return false;
      sh.smem = L.total;
      if (!shape_for_kernel(lane_exec_kernel<V, Ops>, sh.threads, sh.smem, &occ)) return false;
      per_block_items = (uint64_t)sh.threads;
    }
  } else if (prog.exec == Executor::Warp) {
    sh.threads = 256;
    SmemLayout L;
    for (;;) {
      L = smem_layout(prog.n_steps, prog.n_leaves, prog.leaf_elems, prog.arena_elems * (sh.threads / 32),
                      elem_bytes, sh.threads, false);
      if (L.total <= (size_t)max_optin || sh.threads == 32) break;
      sh.threads /= 2;
    }
    if (L.total > (size_t)max_optin) return false;
    sh.smem = L.total;
    if (!shape_for_kernel(block_exec_kernel<V, true, Ops>, sh.threads, sh.smem, &occ)) return false;
    per_block_items = (uint64_t)(sh.threads / 32);
  } else if (prog.exec == Executor::Wide) {
    // One partial per item and root block; no shared-memory program.
    if (!prog.wide) return false;
    sh.threads = 256;
    sh.blocks_per_x = (int)std::min<uint64_t>(slices_per_x * (uint64_t)prog.wide->root_blocks, 1ull << 30);
    *out = sh;
    return true;
  } else if (prog.exec == Executor::LevelJit) {
    // Shape fixed when the kernel was generated (jit_level_shape).
    if (!prog.jit_kernel) return false;
    sh.threads = prog.block_threads;
    sh.arena_stride = prog.arena_elems | 1u;
    sh.log2_items = prog.jit_log2_items;
    sh.smem = prog.jit_smem;
    occ = prog.blocks_per_sm > 1 ? prog.blocks_per_sm : 1;
    per_block_items = 1ull << sh.log2_items;
  } else if (prog.exec == Executor::Level) {
    // The most items (power of two, <= 32) whose arenas fit in the block's
    // share of the SM's shared memory (1 KiB per block is the system's).
    sh.threads = prog.block_threads;
    sh.arena_stride = prog.arena_elems | 1u;
    int per_sm = 0;
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const int bps = prog.blocks_per_sm > 1 ? prog.blocks_per_sm : 1;
    const size_t cap = std::min<size_t>((size_t)max_optin, (size_t)per_sm / bps - 1024);
    int lg = 5;
    LevelLayout L;
    for (;; --lg) {
      L = level_layout(prog.n_steps, prog.n_levels, prog.n_leaves, prog.leaf_elems, sh.arena_stride, 1 << lg,
                       elem_bytes, sh.threads);
      if (L.total <= cap || lg == 0) break;
    }
    if (L.total > cap) return false;
    sh.log2_items = lg;
    sh.smem = L.total;
    if (!shape_for_kernel(level_exec_kernel<V, Ops>, sh.threads, sh.smem, &occ)) return false;
    per_block_items = 1ull << lg;
  } else {
    sh.threads = 256;
    SmemLayout L = smem_layout(prog.n_steps, prog.n_leaves, prog.leaf_elems, prog.arena_elems, elem_bytes,
                               sh.threads, false);
    if (L.total > (size_t)max_optin) return false;
    sh.smem = L.total;
    if (!shape_for_kernel(block_exec_kernel<V, false, Ops>, sh.threads, sh.smem, &occ)) return false;
  }
  if (prog.n_pro_steps > 0 && prog.n_pro_levels > 0) {
    const LevelLayout PL = level_layout(prog.n_pro_steps, prog.n_pro_levels, prog.n_leaves, prog.leaf_elems,
                                        prog.pro_arena_elems | 1u, 1, elem_bytes, kLevelPrologueThreads);
    if (PL.total > (size_t)max_optin) return false;
    sh.pro_smem = PL.total;
    if (allow_max_smem(prologue_level_kernel<V, Ops>) != cudaSuccess) return false;
  } else if (prog.n_pro_steps > 0) {
    const SmemLayout PL = smem_layout(prog.n_pro_steps, prog.n_leaves, prog.leaf_elems, prog.pro_arena_elems,
                                      elem_bytes, 256, false);
    if (PL.total > (size_t)max_optin) return false;
    sh.pro_smem = PL.total;
    if (allow_max_smem(prologue_kernel<V, Ops>) != cudaSuccess) return false;
  }
  const uint64_t total_blocks = (uint64_t)g_num_sms * (uint64_t)occ;
  uint64_t per_x = total_blocks / (uint64_t)(nx > 0 ? nx : 1);
  if (per_x < 1) per_x = 1;
  const uint64_t units = (slices_per_x + per_block_items - 1) / per_block_items;
  if (per_x > units) per_x = units;
  if (per_x < 1) per_x = 1;
  sh.blocks_per_x = (int)per_x;
  *out = sh;
  return true;
}

template <class V, class Ops>
cudaError_t launch_typed(const DeviceProgram& prog, const uint8_t* d_x, int nx, uint64_t slice_lo, uint64_t slice_hi,
                         const LaunchBuffers& buf, const ExecShape& shape, double scale, double2* d_out,
                         Partial* d_raw, double2* d_slices, cudaStream_t stream, cudaEvent_t ev0, cudaEvent_t ev1,
                         const double* d_gamma, const double* d_beta) {
  const unsigned lgrid = (unsigned)prog.n_leaves * (unsigned)nx;
  const bool sweep = d_gamma != nullptr;
  leaf_build_kernel<V><<<lgrid, 32, 0, stream>>>(prog.leaves, prog.gate_q, prog.gate_layer, prog.gate_in_h,
                                                 prog.gate_out_kind, prog.gate_kind, sweep ? d_gamma : prog.gamma,
                                                 sweep ? d_beta : prog.beta, sweep ? prog.p : 0, d_x, prog.n,
                                                 prog.leaf_elems, prog.n_leaves, prog.density != 0,
                                                 static_cast<V*>(buf.leaf_tables), sweep ? nullptr : prog.trig);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (prog.exec == Executor::Wide) {
    if (!prog.wide || prog.wide->nx != nx) return cudaErrorInvalidValue;
    if (ev0 && (e = cudaEventRecord(ev0, stream)) != cudaSuccess) return e;
    e = wide_launch(prog.wide, buf.leaf_tables, slice_lo, slice_hi, buf.partials, d_slices, buf.err, stream);
    if (e != cudaSuccess) return e;
    if (ev1 && (e = cudaEventRecord(ev1, stream)) != cudaSuccess) return e;
    finalize_kernel<<<nx, 128, 0, stream>>>(buf.partials, shape.blocks_per_x, scale, d_out, d_raw);
    return cudaGetLastError();
  }
  if (prog.exec == Executor::LevelJit && prog.jit_prologue) {
    e = jit_prologue_launch(prog.jit_prologue, nx, prog.jit_pro_smem, buf.leaf_tables, stream);
    if (e != cudaSuccess) return e;
  } else if (prog.n_pro_steps > 0 && prog.n_pro_levels > 0) {
    prologue_level_kernel<V, Ops><<<nx, kLevelPrologueThreads, shape.pro_smem, stream>>>(
        prog.pro_steps, prog.n_pro_steps, prog.pro_out_start, prog.pro_pos_nib, prog.pro_levels, prog.n_pro_levels,
        prog.leaves,
        prog.n_leaves, buf.leaf_tables, prog.leaf_elems, prog.pro_arena_elems);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  } else if (prog.n_pro_steps > 0) {
    prologue_kernel<V, Ops><<<nx, 256, shape.pro_smem, stream>>>(prog.pro_steps, prog.n_pro_steps, prog.leaves,
                                                                 prog.n_leaves, buf.leaf_tables, prog.leaf_elems,
                                                                 prog.pro_arena_elems);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  ExecParams P;
  P.steps = prog.steps;
  P.leaves = prog.leaves;
  P.leaf_tables = buf.leaf_tables;
  P.partials = buf.partials;
  P.slices = d_slices;
  P.slice_lo = slice_lo;
  P.slice_hi = slice_hi;
  P.leaf_elems = prog.leaf_elems;
  P.arena_elems = prog.arena_elems;
  P.n_steps = prog.n_steps;
  P.n_leaves = prog.n_leaves;
  P.blocks_per_x = shape.blocks_per_x;
  const unsigned grid = (unsigned)shape.blocks_per_x * (unsigned)nx;
  if (ev0) {
    e = cudaEventRecord(ev0, stream);
    if (e != cudaSuccess) return e;
  }
  if (prog.exec == Executor::Lane) {
    if constexpr (LaneCapable<Ops>::value) {
      lane_exec_kernel<V, Ops><<<grid, shape.threads, shape.smem, stream>>>(P, buf.err);
    } else {
      return cudaErrorInvalidValue;
    }
  } else if (prog.exec == Executor::Warp) {
    block_exec_kernel<V, true, Ops><<<grid, shape.threads, shape.smem, stream>>>(P);
  } else if (prog.exec == Executor::LevelJit) {
    JitLevelShape js;
    js.threads = shape.threads;
    js.blocks_per_sm = prog.blocks_per_sm;
    js.log2_items = shape.log2_items;
    js.arena_stride = shape.arena_stride;
    js.smem = shape.smem;
    js.scratch_elems_per_block = prog.jit_scratch_bytes;
    e = jit_level_launch(prog.jit_kernel, js, nx, shape.blocks_per_x, buf.leaf_tables, buf.partials,
                         buf.jit_scratch, slice_lo, slice_hi, stream);
    if (e != cudaSuccess) return e;
  } else if (prog.exec == Executor::Level) {
    const LevelParams LP{prog.levels, prog.out_start, prog.pos_nib, prog.n_levels, shape.log2_items,
                         shape.arena_stride};
    level_exec_kernel<V, Ops><<<grid, shape.threads, shape.smem, stream>>>(P, LP);
  } else {
    block_exec_kernel<V, false, Ops><<<grid, shape.threads, shape.smem, stream>>>(P);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ev1) {
    e = cudaEventRecord(ev1, stream);
    if (e != cudaSuccess) return e;
  }
  finalize_kernel<<<nx, 128, 0, stream>>>(buf.partials, shape.blocks_per_x, scale, d_out, d_raw);
  return cudaGetLastError();
}

template <class V, class Ops>
cudaError_t launch_multi_typed(const JobDesc* d_jobs, int njobs, uint32_t total_leaves, const ChunkDesc* d_chunks,
                               uint32_t n_chunks, unsigned* d_counter, Partial* d_chunk_partials, double2* d_out,
                               size_t exec_smem, size_t pro_smem, bool level, const AbortCtl& ac,
                               cudaStream_t stream) {
  int dev = 0, sms = 0, max_optin = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (exec_smem > (size_t)max_optin || pro_smem > (size_t)max_optin) return cudaErrorInvalidValue;
  cudaError_t e;
  if ((e = allow_max_smem(multi_prologue_kernel<V, Ops>)) != cudaSuccess) return e;
  if ((e = allow_max_smem(multi_prologue_level_kernel<V, Ops>)) != cudaSuccess) return e;
  const int threads = level ? kMultiLevelThreads : 256;
  if (level ? !shape_for_kernel(multi_level_kernel<V, Ops>, threads, exec_smem, &occ)
            : !shape_for_kernel(multi_exec_kernel<V, Ops>, threads, exec_smem, &occ))
    return cudaErrorInvalidConfiguration;
  if ((e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned), stream)) != cudaSuccess) return e;
  multi_leaf_kernel<V><<<total_leaves, 32, 0, stream>>>(d_jobs, njobs);
  if (level)
    multi_prologue_level_kernel<V, Ops><<<njobs, kMultiLevelThreads, pro_smem, stream>>>(d_jobs);
  else
    multi_prologue_kernel<V, Ops><<<njobs, 256, pro_smem, stream>>>(d_jobs);
  const unsigned grid = (unsigned)std::min<uint64_t>((uint64_t)sms * occ, n_chunks);
  if (level)
    multi_level_kernel<V, Ops><<<grid, threads, exec_smem, stream>>>(d_jobs, d_chunks, n_chunks, d_counter,
                                                                     d_chunk_partials, ac);
  else
    multi_exec_kernel<V, Ops><<<grid, threads, exec_smem, stream>>>(d_jobs, d_chunks, n_chunks, d_counter,
                                                                    d_chunk_partials, ac);
  multi_finalize_kernel<<<njobs, 128, 0, stream>>>(d_jobs, d_chunk_partials, d_out);
  return cudaGetLastError();
}

// cos and sin of each layer's gamma and beta, as the leaf kernel evaluates
// them: out[4 l ..] = (cos gamma_l, sin gamma_l, cos beta_l, sin beta_l).
__global__ void trig_table_kernel(const double* __restrict__ gamma, const double* __restrict__ beta, int p,
                                  double* __restrict__ out) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= p) return;
  sincos(gamma[l], &out[4 * l + 1], &out[4 * l]);
  sincos(beta[l], &out[4 * l + 3], &out[4 * l + 2]);
}

// Check of the double-float arithmetic: item i is the complex dot product
// sum_k a[i, k] b[i, k] of K terms (operands rounded to double words), by the
// scalar sequence (CplxOps<dfc>) and by the form the merge loops run
// (MergeOps: packed FP32 pairs where the device has them).
__global__ void arith_check_kernel(const double2* __restrict__ a, const double2* __restrict__ b, int count, int K,
                                   double2* __restrict__ out_scalar, double2* __restrict__ out_merge) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  typedef CplxOps<dfc> S;
  typedef MergeOps<S>::type M;
  const double2* pa = a + (size_t)i * K;
  const double2* pb = b + (size_t)i * K;
  dfc s = S::mul(S::from(pa[0].x, pa[0].y), S::from(pb[0].x, pb[0].y));
  M::Acc m = M::mul(S::from(pa[0].x, pa[0].y), S::from(pb[0].x, pb[0].y));
  for (int k = 1; k < K; ++k) {
    const dfc x = S::from(pa[k].x, pa[k].y), y = S::from(pb[k].x, pb[k].y);
    S::fma(s, x, y);
    M::fma(m, x, y);
  }
  s = S::result(s);
  const dfc r = M::result(m);
  out_scalar[i] = make_double2(S::re(s), S::im(s));
  out_merge[i] = make_double2(S::re(r), S::im(r));
}

}  // namespace

cudaError_t launch_trig_table(const double* d_gamma, const double* d_beta, int p, double* d_out, cudaStream_t stream) {
  if (p <= 0) return cudaSuccess;
  trig_table_kernel<<<(p + 31) / 32, 32, 0, stream>>>(d_gamma, d_beta, p, d_out);
  return cudaGetLastError();
}

cudaError_t launch_arith_check(const double2* d_a, const double2* d_b, int count, int K, double2* d_scalar,
                               double2* d_merge, cudaStream_t stream) {
  if (count <= 0) return cudaSuccess;
  arith_check_kernel<<<(count + 127) / 128, 128, 0, stream>>>(d_a, d_b, count, K, d_scalar, d_merge);
  return cudaGetLastError();
}

int arith_elem_bytes(Arith a) { return (a == Arith::F64 || a == Arith::F32X2) ? 16 : 8; }

#define QTN_ARITH_SWITCH(a, CALL)                                     \
  switch (a) {                                                        \
    case Arith::F64: return CALL(double2, CplxOps<double2>);          \
    case Arith::F32: return CALL(float2, CplxOps<float2>);            \
    case Arith::F32X2: return CALL(dfc, CplxOps<dfc>);                \
    case Arith::TF32: return CALL(float2, RoundOps<Round::TF32>);     \
    case Arith::BF16X3: return CALL(float2, RoundOps<Round::BF16X3>); \
    case Arith::TF32X3: return CALL(float2, RoundOps<Round::TF32X3>); \
    case Arith::BF16X6: return CALL(float2, RoundOps<Round::BF16X6>); \
  }

bool exec_shape(const DeviceProgram& prog, Arith a, int nx, uint64_t slices_per_x, ExecShape* out) {
#define QTN_SHAPE_CALL(V, O) exec_shape_typed<V, O>(prog, nx, slices_per_x, out)
  QTN_ARITH_SWITCH(a, QTN_SHAPE_CALL)
#undef QTN_SHAPE_CALL
  return false;
}

cudaError_t launch_contraction(const DeviceProgram& prog, Arith a, const uint8_t* d_x, int nx, uint64_t slice_lo,
                               uint64_t slice_hi, const LaunchBuffers& buf, const ExecShape& shape, double scale,
                               double2* d_out, Partial* d_raw, double2* d_slices, cudaStream_t stream,
                               cudaEvent_t ev0, cudaEvent_t ev1, const double* d_gamma, const double* d_beta) {
  if (nx <= 0) return cudaSuccess;
  if ((d_gamma == nullptr) != (d_beta == nullptr)) return cudaErrorInvalidValue;
#define QTN_LAUNCH_CALL(V, O)                                                                                   \
  launch_typed<V, O>(prog, d_x, nx, slice_lo, slice_hi, buf, shape, scale, d_out, d_raw, d_slices, stream, ev0, ev1, \
                     d_gamma, d_beta)
  QTN_ARITH_SWITCH(a, QTN_LAUNCH_CALL)
#undef QTN_LAUNCH_CALL
  return cudaErrorInvalidValue;
}

size_t block_smem_bytes(int n_steps, int n_leaves, uint32_t leaf_elems, uint32_t arena_elems, Arith a, int threads) {
  return smem_layout(n_steps, n_leaves, leaf_elems, arena_elems, arith_elem_bytes(a), threads, false).total;
}

size_t level_smem_bytes(int n_steps, int n_levels, int n_leaves, uint32_t leaf_elems, uint32_t arena_stride,
                        int items, Arith a, int threads) {
  return level_layout(n_steps, n_levels, n_leaves, leaf_elems, arena_stride, items, arith_elem_bytes(a), threads)
      .total;
}

cudaError_t launch_multi(Arith a, const JobDesc* d_jobs, int njobs, uint32_t total_leaves, const ChunkDesc* d_chunks,
                         uint32_t n_chunks, unsigned* d_counter, Partial* d_chunk_partials, double2* d_out,
                         size_t exec_smem, size_t pro_smem, bool level, const volatile int* d_cancel,
                         unsigned* d_status, uint64_t budget_ns, cudaStream_t stream) {
  if (njobs <= 0) return cudaSuccess;
  const AbortCtl ac{d_cancel, d_status, budget_ns};
#define QTN_MULTI_CALL(V, O)                                                                                  \
  launch_multi_typed<V, O>(d_jobs, njobs, total_leaves, d_chunks, n_chunks, d_counter, d_chunk_partials, d_out, \
                           exec_smem, pro_smem, level, ac, stream)
  QTN_ARITH_SWITCH(a, QTN_MULTI_CALL)
#undef QTN_MULTI_CALL
  return cudaErrorInvalidValue;
}

}  // namespace qtn
