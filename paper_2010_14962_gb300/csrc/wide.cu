// Wide executor (see wide.hpp): merges of intermediates in global memory,
// one launch per step and group of work items, kernel chosen per step shape.
#include "wide.hpp"

#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <mutex>
#include <sstream>

#include "../../include/qtn.h"
#include "internal.hpp"
#include "wide_tc.hpp"

namespace qtn {
namespace {

std::atomic<int> g_force_kernel{-1};  // -1: autotuned; else a WideKernel for every step that allows it

#include "arith.cuh"
#include "rounding.cuh"

constexpr int kThreads = 256;
constexpr int kPosGroups = (kWideMaxRank + 3) / 4;

// Arguments of one merge launch (by value).  Item g of the launch is global
// item item_lo + g; its bit string and outer-class assignment follow from
// items_per_x (prologue launches: item = bit string, no outer classes).
struct WLeaf {
  uint32_t base;
  uint8_t rank_nc, ncut, cut_bit[kMaxLeafCuts];
};
struct WOperand {
  int leaf;  // 1: leaf table of the item's bit string, 0: the item's arena slot
  uint64_t off;
  WLeaf lf;
};
struct WMergeArgs {
  WOperand A, B;
  int c_export;      // 1: C goes to the bit string's leaf table at c_off
  uint64_t c_off;
  int ma, nb, kb, bb, rc;
  uint8_t wpos[kWideMaxRank];
  void* arena;
  uint64_t arena_stride;  // elements per item slot
  void* leaf_tables;
  uint32_t leaf_elems;
  uint64_t item_lo, n_items, items_per_x, slice_lo;
  int prologue;
};

template <class V>
__device__ __forceinline__ const V* operand_ptr(const WMergeArgs& p, const WOperand& op, uint64_t g, uint64_t xi,
                                                uint64_t s) {
  if (!op.leaf) return static_cast<const V*>(p.arena) + g * p.arena_stride + op.off;
  uint64_t off = op.lf.base;
  for (int j = 0; j < op.lf.ncut; ++j) off += ((s >> op.lf.cut_bit[j]) & 1ull) << (op.lf.rank_nc + j);
  return static_cast<const V*>(p.leaf_tables) + xi * p.leaf_elems + off;
}

__device__ __forceinline__ void item_coords(const WMergeArgs& p, uint64_t g, uint64_t* xi, uint64_t* s) {
  const uint64_t G = p.item_lo + g;
  if (p.prologue) {
    *xi = G;
    *s = 0;
  } else {
    *xi = G / p.items_per_x;
    *s = p.slice_lo + G % p.items_per_x;
  }
}

// Store offsets by nibble of the canonical output index: table[g][v] = the
// weights (1 << wpos) of the set bits of v placed at bits 4g..4g+3.
__device__ __forceinline__ void build_pos_table(const WMergeArgs& p, uint64_t (*t)[16]) {
  for (int i = threadIdx.x; i < kPosGroups * 16; i += blockDim.x) {
    const int g = i >> 4, v = i & 15;
    uint64_t pos = 0;
    for (int b = 0; b < 4; ++b) {
      const int bit = 4 * g + b;
      if (bit < p.rc && ((v >> b) & 1)) pos += 1ull << p.wpos[bit];
    }
    t[g][v] = pos;
  }
  __syncthreads();
}

// SIMT merge: every thread computes U consecutive canonical outputs
// C[m, n, b] = sum_k A[m + (k << ma) + (b << (ma + kb))] * B[k + (n << kb) +
// (b << (kb + nb))] of one item and stores them at their consumer-layout
// positions.  U = 4 needs ma >= 2 (the four share n, b and the B column).
template <class V, class Ops, int K, int U>
__global__ void __launch_bounds__(kThreads) wide_merge_kernel(WMergeArgs p) {
  __shared__ uint64_t s_pos[kPosGroups][16];
  build_pos_table(p, s_pos);
  const int ngroups = (p.rc + 3) >> 2;
  const uint64_t per_item = (1ull << p.rc) / U;
  const uint64_t total = p.n_items * per_item;
  const uint64_t mmask = (1ull << p.ma) - 1, nmask = (1ull << p.nb) - 1;
  const int kcount = 1 << p.kb;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t g = idx / per_item;
    const uint64_t o0 = (idx - g * per_item) * U;
    uint64_t xi, s;
    item_coords(p, g, &xi, &s);
    const V* A = operand_ptr<V>(p, p.A, g, xi, s);
    const V* B = operand_ptr<V>(p, p.B, g, xi, s);
    V* C = p.c_export ? static_cast<V*>(p.leaf_tables) + xi * p.leaf_elems + p.c_off
                      : static_cast<V*>(p.arena) + g * p.arena_stride + p.c_off;
    const uint64_t n = (o0 >> p.ma) & nmask, b = o0 >> (p.ma + p.nb);
    const V* bp = B + (n << p.kb) + (b << (p.kb + p.nb));
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t o = o0 + u;
      const uint64_t m = o & mmask;
      const V* ap = A + m + (b << (p.ma + p.kb));
      using F = typename MergeOps<Ops>::type;
      typename F::Acc acc_ = F::mul(ap[0], bp[0]);
      if (K > 0) {
#pragma unroll
        for (int k = 1; k < K; ++k) F::fma(acc_, ap[(uint64_t)k << p.ma], bp[k]);
      } else {
        for (int k = 1; k < kcount; ++k) F::fma(acc_, ap[(uint64_t)k << p.ma], bp[k]);
      }
      uint64_t pos = 0;
      for (int q = 0; q < ngroups; ++q) pos += s_pos[q][(o >> (4 * q)) & 15];
      C[pos] = F::result(acc_);
    }
  }
}

// Root of every item (rank-0 result): sum_k A[k] B[k], split over R blocks
// per item; each thread adds the products of 4 consecutive k in the working
// arithmetic, then into compensated FP64 sums; one fixed-order block
// reduction; partial (item, r) at partials[xi * (nr * R) + local * R + r].
template <class V, class Ops>
__global__ void __launch_bounds__(kThreads) wide_root_kernel(WMergeArgs p, int R, uint64_t nr,
                                                             Partial* __restrict__ partials) {
  __shared__ Partial s_red[kThreads];
  const uint64_t g = blockIdx.x / R;
  const int r = blockIdx.x % R;
  uint64_t xi, s;
  item_coords(p, g, &xi, &s);
  const V* A = operand_ptr<V>(p, p.A, g, xi, s);
  const V* B = operand_ptr<V>(p, p.B, g, xi, s);
  const uint64_t K = 1ull << p.kb;
  const uint64_t chunk = (K + R - 1) / R;
  const uint64_t lo = chunk * r < K ? chunk * r : K, hi = lo + chunk < K ? lo + chunk : K;
  double sr = 0, si = 0, cr = 0, ci = 0;
  for (uint64_t k0 = lo + 4 * threadIdx.x; k0 < hi; k0 += 4 * blockDim.x) {
    using F = typename MergeOps<Ops>::type;
    typename F::Acc acc_ = F::mul(A[k0], B[k0]);
    for (uint64_t k = k0 + 1; k < k0 + 4 && k < hi; ++k) F::fma(acc_, A[k], B[k]);
    const V acc = F::result(acc_);
    kahan_add(sr, cr, Ops::re(acc));
    kahan_add(si, ci, Ops::im(acc));
  }
  s_red[threadIdx.x] = Partial::make(sr, si, cr, ci);
  tree_reduce(s_red, kThreads);
  if (threadIdx.x == 0) {
    const uint64_t G = p.item_lo + g;
    partials[xi * (nr * R) + (G - xi * nr) * R + r] = s_red[0];
  }
}

// Per-item values (unscaled) from the R root partials of each item.
__global__ void wide_slices_kernel(const Partial* __restrict__ partials, uint64_t total_items, int R,
                                   double2* __restrict__ out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total_items) return;
  double a = 0, b = 0, ca = 0, cb = 0;
  for (int r = 0; r < R; ++r) {
    const Partial v = partials[i * R + r];
    kahan_add(a, ca, v.re);
    kahan_add(a, ca, -v.cre);
    kahan_add(b, cb, v.im);
    kahan_add(b, cb, -v.cim);
  }
  out[i] = make_double2(a - ca, b - cb);
}

// ----------------------------------------------------------------- host --

int g_sms = 0;
int num_sms() {
  if (g_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 1;
  }
  return g_sms;
}

#define QTN_WIDE_ARITH_SWITCH(a, CALL)                                \
  switch (a) {                                                        \
    case Arith::F64: return CALL(double2, CplxOps<double2>);          \
    case Arith::F32: return CALL(float2, CplxOps<float2>);            \
    case Arith::F32X2: return CALL(dfc, CplxOps<dfc>);                \
    case Arith::TF32: return CALL(float2, RoundOps<Round::TF32>);     \
    case Arith::BF16X3: return CALL(float2, RoundOps<Round::BF16X3>); \
    case Arith::TF32X3: return CALL(float2, RoundOps<Round::TF32X3>); \
    case Arith::BF16X6: return CALL(float2, RoundOps<Round::BF16X6>); \
  }

template <class V, class Ops, int U>
cudaError_t launch_simt_typed(const WMergeArgs& p, cudaStream_t stream) {
  const uint64_t total = p.n_items * ((1ull << p.rc) / U);
  const uint64_t want = (total + kThreads - 1) / kThreads;
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)num_sms() * 8));
  switch (p.kb) {
    case 0: wide_merge_kernel<V, Ops, 1, U><<<grid, kThreads, 0, stream>>>(p); break;
    case 1: wide_merge_kernel<V, Ops, 2, U><<<grid, kThreads, 0, stream>>>(p); break;
    case 2: wide_merge_kernel<V, Ops, 4, U><<<grid, kThreads, 0, stream>>>(p); break;
    case 3: wide_merge_kernel<V, Ops, 8, U><<<grid, kThreads, 0, stream>>>(p); break;
    default: wide_merge_kernel<V, Ops, 0, U><<<grid, kThreads, 0, stream>>>(p); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_simt(Arith a, const WMergeArgs& p, int U, cudaStream_t stream) {
#define QTN_SIMT_CALL(V, O) (U == 4 ? launch_simt_typed<V, O, 4>(p, stream) : launch_simt_typed<V, O, 1>(p, stream))
  QTN_WIDE_ARITH_SWITCH(a, QTN_SIMT_CALL)
#undef QTN_SIMT_CALL
  return cudaErrorInvalidValue;
}

cudaError_t launch_root(Arith a, const WMergeArgs& p, int R, uint64_t nr, Partial* partials, cudaStream_t stream) {
  const unsigned grid = (unsigned)(p.n_items * (uint64_t)R);
#define QTN_ROOT_CALL(V, O) \
  (wide_root_kernel<V, O><<<grid, kThreads, 0, stream>>>(p, R, nr, partials), cudaGetLastError())
  QTN_WIDE_ARITH_SWITCH(a, QTN_ROOT_CALL)
#undef QTN_ROOT_CALL
  return cudaErrorInvalidValue;
}

WOperand make_operand(const Program& pg, bool leaf, uint64_t id) {
  WOperand op{};
  op.leaf = leaf ? 1 : 0;
  if (leaf) {
    const DevLeaf& L = pg.leaves[id];
    op.lf.base = L.base;
    op.lf.rank_nc = L.rank_nc;
    op.lf.ncut = L.ncut;
    for (int j = 0; j < kMaxLeafCuts; ++j) op.lf.cut_bit[j] = L.cut_bit[j];
  } else {
    op.off = id;
  }
  return op;
}

WMergeArgs make_args(const WideState& ws, const WideStep& st, bool prologue, void* leaf_tables, uint64_t item_lo,
                     uint64_t n_items, uint64_t items_per_x, uint64_t slice_lo) {
  const Program& pg = *ws.prog;
  WMergeArgs p{};
  p.A = make_operand(pg, st.flags & STEP_A_LEAF, st.a);
  p.B = make_operand(pg, st.flags & STEP_B_LEAF, st.b);
  p.c_export = (st.flags & STEP_EXPORT) ? 1 : 0;
  p.c_off = p.c_export ? pg.leaves[st.c].base : st.c;
  p.ma = st.ma;
  p.nb = st.nb;
  p.kb = st.kb;
  p.bb = st.bb;
  p.rc = st.ma + st.nb + st.bb;
  for (int i = 0; i < kWideMaxRank; ++i) p.wpos[i] = st.wpos[i];
  p.arena = prologue ? ws.d_pro_arena : ws.d_arena;
  p.arena_stride = prologue ? pg.wide_pro_arena_elems : pg.wide_arena_elems;
  p.leaf_tables = leaf_tables;
  p.leaf_elems = pg.leaf_elems;
  p.item_lo = item_lo;
  p.n_items = n_items;
  p.items_per_x = items_per_x;
  p.slice_lo = slice_lo;
  p.prologue = prologue ? 1 : 0;
  return p;
}

cudaError_t launch_step(const WideState& ws, WideKernel k, const WideStep& st, const WMergeArgs& p,
                        int* d_err, cudaStream_t stream) {
  if (k == WideKernel::Tc) {
    WideTcArgs t{};
    auto ref = [](const WOperand& o) {
      WideOperandRef r{};
      r.leaf = o.leaf;
      r.off = o.off;
      r.base = o.lf.base;
      r.rank_nc = o.lf.rank_nc;
      r.ncut = o.lf.ncut;
      for (int j = 0; j < kMaxLeafCuts; ++j) r.cut_bit[j] = o.lf.cut_bit[j];
      return r;
    };
    t.A = ref(p.A);
    t.B = ref(p.B);
    t.c_export = p.c_export;
    t.c_off = p.c_off;
    t.arena = static_cast<const float2*>(p.arena);
    t.arena_stride = p.arena_stride;
    t.leaf_tables = static_cast<const float2*>(p.leaf_tables);
    t.leaf_elems = p.leaf_elems;
    t.item_lo = p.item_lo;
    t.n_items = p.n_items;
    t.items_per_x = p.items_per_x;
    t.slice_lo = p.slice_lo;
    t.prologue = p.prologue;
    t.ma = st.ma;
    t.nb = st.nb;
    t.kb = st.kb;
    t.bb = st.bb;
    for (int i = 0; i < kWideMaxRank; ++i) t.wpos[i] = st.wpos[i];
    t.err = d_err;
    t.ws = ws.d_tc_ws;
    t.ws_floats = ws.tc_ws_floats;
    return wide_tc_launch(t, ws.arith == Arith::TF32X3 ? 3 : 1, stream);
  }
  return launch_simt(ws.arith, p, k == WideKernel::Simt4 ? 4 : 1, stream);
}

size_t elem_bytes(Arith a) { return (size_t)arith_elem_bytes(a); }

std::mutex g_tune_mu;

}  // namespace

int wide_force_mode() { return g_force_kernel.load(); }
bool wide_needs_tuning(const WideState* ws) { return !ws->tuned || ws->force_mode != g_force_kernel.load(); }

const char* wide_kernel_name(WideKernel k) {
  switch (k) {
    case WideKernel::Simt: return "simt";
    case WideKernel::Simt4: return "simt4";
    case WideKernel::Tc: return "tcgen05";
  }
  return "?";
}

std::map<WideShapeKey, WideTuneEntry>& wide_tune_table() {
  static std::map<WideShapeKey, WideTuneEntry> t;
  return t;
}

void wide_tune_load() {
  const char* path = std::getenv("QTN_WIDE_TUNE_CACHE");
  if (!path) return;
  std::ifstream f(path);
  std::string line;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  while (std::getline(f, line)) {
    int ma, nb, kb, bb, ar, best;
    unsigned long long items;
    if (std::sscanf(line.c_str(), "{\"ma\":%d,\"nb\":%d,\"kb\":%d,\"bb\":%d,\"items\":%llu,\"arith\":%d,\"best\":%d",
                    &ma, &nb, &kb, &bb, &items, &ar, &best) == 7)
      wide_tune_table()[WideShapeKey{ma, nb, kb, bb, items, ar}].best = (WideKernel)best;
  }
}

void wide_tune_save() {
  const char* path = std::getenv("QTN_WIDE_TUNE_CACHE");
  if (!path) return;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::ofstream f(path);
  for (const auto& [k, e] : wide_tune_table()) {
    f << "{\"ma\":" << std::get<0>(k) << ",\"nb\":" << std::get<1>(k) << ",\"kb\":" << std::get<2>(k)
      << ",\"bb\":" << std::get<3>(k) << ",\"items\":" << std::get<4>(k) << ",\"arith\":" << std::get<5>(k)
      << ",\"best\":" << (int)e.best << ",\"kernel\":\"" << wide_kernel_name(e.best) << "\",\"ms\":{";
    for (size_t i = 0; i < e.ms.size(); ++i)
      f << (i ? "," : "") << "\"" << wide_kernel_name(e.ms[i].first) << "\":" << e.ms[i].second;
    f << "}}\n";
  }
}

WideState::~WideState() {
  cudaFree(d_arena);
  cudaFree(d_pro_arena);
  cudaFree(d_own_err);
  cudaFree(d_tc_ws);
}

bool wide_tc_eligible(const WideStep& st, Arith a) {
  if (a != Arith::TF32 && a != Arith::TF32X3) return false;
  if (st.flags & STEP_ROOT) return false;
  return wide_tc_shape_ok(st.ma, st.nb, st.kb, st.bb);
}

cudaError_t wide_prepare(WideState* ws, const Program& prog, Arith a, int nx, uint64_t budget_bytes) {
  ws->prog = &prog;
  ws->arith = a;
  ws->nx = nx;
  ws->items_per_x = 1ull << prog.n_outer;
  const uint64_t slot = std::max<uint64_t>(prog.wide_arena_elems, 1) * elem_bytes(a);
  const uint64_t total = (uint64_t)nx * ws->items_per_x;
  ws->group = std::max<uint64_t>(1, std::min<uint64_t>(total, budget_bytes / slot));
  cudaError_t e = cudaMalloc(&ws->d_arena, ws->group * slot);
  if (e != cudaSuccess) return e;
  e = cudaMemset(ws->d_arena, 0, ws->group * slot);
  if (e != cudaSuccess) return e;
  const uint64_t pro = std::max<uint64_t>(prog.wide_pro_arena_elems, 1) * elem_bytes(a) * (uint64_t)nx;
  e = cudaMalloc(&ws->d_pro_arena, pro);
  if (e != cudaSuccess) return e;
  // Split-K partials of the tensor-core merges (TF32 forms only), at most 256 MiB.
  if (a == Arith::TF32 || a == Arith::TF32X3) {
    uint64_t need = 0;
    for (const WideStep& st : prog.wide_steps)
      if (wide_tc_eligible(st, a)) need = std::max(need, wide_tc_workspace_floats(st.ma, st.nb, st.kb, st.bb, ws->group));
    for (const WideStep& st : prog.wide_prologue)
      if (wide_tc_eligible(st, a)) need = std::max(need, wide_tc_workspace_floats(st.ma, st.nb, st.kb, st.bb, nx));
    ws->tc_ws_floats = std::min<uint64_t>(need, 64ull << 20);
    if (ws->tc_ws_floats) {
      e = cudaMalloc(&ws->d_tc_ws, ws->tc_ws_floats * sizeof(float));
      if (e != cudaSuccess) return e;
    }
  }
  e = cudaMalloc(&ws->d_own_err, sizeof(int));
  if (e != cudaSuccess) return e;
  e = cudaMemset(ws->d_own_err, 0, sizeof(int));
  if (e != cudaSuccess) return e;
  // Root reduction: about two blocks per SM over the items of a group.
  uint64_t root_k = 1;
  for (const WideStep& st : prog.wide_steps)
    if (st.flags & STEP_ROOT) root_k = 1ull << st.kb;
  const uint64_t want = std::max<uint64_t>(1, (uint64_t)num_sms() * 2 / std::max<uint64_t>(1, ws->group));
  ws->root_blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>({want, 64, (root_k + 4 * kThreads - 1) / (4 * kThreads)}));
  ws->step_kernel.assign(prog.wide_steps.size(), WideKernel::Simt);
  ws->pro_kernel.assign(prog.wide_prologue.size(), WideKernel::Simt);
  return cudaSuccess;
}

cudaError_t wide_tune(WideState* ws, void* leaf_tables, uint64_t slice_lo, uint64_t slice_hi, cudaStream_t stream,
                      std::string* log) {
  const Program& pg = *ws->prog;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return e;
  std::ostringstream lg;
  // Winners of earlier processes (QTN_WIDE_TUNE_CACHE), read once.
  static std::once_flag loaded;
  std::call_once(loaded, wide_tune_load);
  bool added = false;
  const uint64_t nr = slice_hi - slice_lo;
  const uint64_t n_group = std::min<uint64_t>(ws->group, (uint64_t)ws->nx * nr);
  ws->force_mode = g_force_kernel.load();
  ws->step_ms.assign(pg.wide_steps.size(), {});
  // Each candidate runs on the step's real operands (leaf tables already
  // built on `stream`); running a step out of turn only rewrites its result,
  // which the contraction itself recomputes before anything reads it.
  auto tune_list = [&](const std::vector<WideStep>& steps, std::vector<WideKernel>* out, bool prologue) {
    const uint64_t n_items = prologue ? (uint64_t)ws->nx : n_group;
    for (size_t j = 0; j < steps.size(); ++j) {
      const WideStep& st = steps[j];
      if (st.flags & STEP_ROOT) continue;
      const int rc = st.ma + st.nb + st.bb;
      const WideShapeKey key{st.ma, st.nb, st.kb, st.bb, n_items, (int)ws->arith};
      std::vector<WideKernel> cand{WideKernel::Simt};
      if (st.ma >= 2 && rc >= 2) cand.push_back(WideKernel::Simt4);
      if (wide_tc_eligible(st, ws->arith)) cand.push_back(WideKernel::Tc);
      const int force = ws->force_mode;
      if (force >= 0) {
        if (std::find(cand.begin(), cand.end(), (WideKernel)force) != cand.end()) {
          (*out)[j] = (WideKernel)force;
          continue;
        }
        cand.erase(std::remove(cand.begin(), cand.end(), WideKernel::Tc), cand.end());
      }
      if (force < 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = wide_tune_table().find(key);
        if (it != wide_tune_table().end() &&
            std::find(cand.begin(), cand.end(), it->second.best) != cand.end()) {
          (*out)[j] = it->second.best;
          if (!prologue) ws->step_ms[j] = it->second.ms;
          continue;
        }
      }
      const WMergeArgs p = make_args(*ws, st, prologue, leaf_tables, 0, n_items, prologue ? 1 : nr, slice_lo);
      WideTuneEntry ent{WideKernel::Simt, {}};
      float best = 1e30f;
      for (WideKernel k : cand) {
        float ms_min = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
          cudaEventRecord(e0, stream);
          if (launch_step(*ws, k, st, p, ws->d_own_err, stream) != cudaSuccess) {
            ms_min = 1e30f;
            break;
          }
          cudaEventRecord(e1, stream);
          cudaEventSynchronize(e1);
          float ms = 0;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) ms_min = std::min(ms_min, ms);
        }
        ent.ms.push_back({k, ms_min});
        if (ms_min < best) {
          best = ms_min;
          ent.best = k;
        }
      }
      (*out)[j] = ent.best;
      if (!prologue) ws->step_ms[j] = ent.ms;
      lg << "(" << st.ma << "," << st.nb << "," << st.kb << "," << st.bb << ")x" << n_items << ":"
         << wide_kernel_name(ent.best) << " ";
      if (force < 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        wide_tune_table()[key] = ent;
        added = true;
      }
    }
  };
  tune_list(pg.wide_prologue, &ws->pro_kernel, true);
  tune_list(pg.wide_steps, &ws->step_kernel, false);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ws->tuned = true;
  if (added || ws->force_mode < 0) wide_tune_save();
  if (log) *log = lg.str();
  return cudaSuccess;
}

cudaError_t wide_launch(WideState* ws, void* leaf_tables, uint64_t slice_lo, uint64_t slice_hi, Partial* partials,
                        double2* d_slices, int* d_err, cudaStream_t stream) {
  const Program& pg = *ws->prog;
  cudaError_t e = cudaSuccess;
  if (!d_err) d_err = ws->d_own_err;
  if (!ws->tuned || ws->force_mode != g_force_kernel.load()) {
    // First launch: choose the kernel of every step shape (outside capture;
    // a captured first launch keeps the SIMT kernels).
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cs);
    if (e != cudaSuccess) return e;
    if (cs == cudaStreamCaptureStatusNone) {
      e = wide_tune(ws, leaf_tables, slice_lo, slice_hi, stream, &ws->tune_log);
      if (e != cudaSuccess) return e;
    }
  }
  // Prologue: one item per bit string, results into the leaf tables.
  for (size_t j = 0; j < pg.wide_prologue.size(); ++j) {
    const WideStep& st = pg.wide_prologue[j];
    const WMergeArgs p = make_args(*ws, st, true, leaf_tables, 0, (uint64_t)ws->nx, 1, 0);
    e = launch_step(*ws, ws->pro_kernel[j], st, p, d_err, stream);
    if (e != cudaSuccess) return e;
  }
  const uint64_t nr = slice_hi - slice_lo;
  const uint64_t total = (uint64_t)ws->nx * nr;
  for (uint64_t g0 = 0; g0 < total; g0 += ws->group) {
    const uint64_t n = std::min<uint64_t>(ws->group, total - g0);
    for (size_t j = 0; j < pg.wide_steps.size(); ++j) {
      const WideStep& st = pg.wide_steps[j];
      const WMergeArgs p = make_args(*ws, st, false, leaf_tables, g0, n, nr, slice_lo);
      if (st.flags & STEP_ROOT) {
        if (st.ma + st.nb + st.bb != 0) return cudaErrorInvalidValue;
        e = launch_root(ws->arith, p, ws->root_blocks, nr, partials, stream);
      } else {
        e = launch_step(*ws, ws->step_kernel[j], st, p, d_err, stream);
      }
      if (e != cudaSuccess) return e;
    }
  }
  if (d_slices) {
    wide_slices_kernel<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(partials, total, ws->root_blocks, d_slices);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace qtn

extern "C" qtn_status qtn_wide_set_kernel(const char* name) {
  if (!name) return qtn::internal::set_error(QTN_ERR_INVALID_ARG, "name is NULL");
  int mode = -2;
  if (!std::strcmp(name, "auto")) mode = -1;
  else if (!std::strcmp(name, "simt")) mode = (int)qtn::WideKernel::Simt;
  else if (!std::strcmp(name, "simt4")) mode = (int)qtn::WideKernel::Simt4;
  else if (!std::strcmp(name, "tcgen05")) mode = (int)qtn::WideKernel::Tc;
  if (mode == -2) return qtn::internal::set_error(QTN_ERR_INVALID_ARG, "unknown wide kernel name");
  qtn::g_force_kernel.store(mode);
  return QTN_OK;
}
