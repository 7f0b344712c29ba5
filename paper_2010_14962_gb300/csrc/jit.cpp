// Per-plan specialised level executor: source generation, run-time
// compilation (NVRTC, loaded with dlopen so that the library builds and runs
// without it) and launch.  The generated kernel runs the same merges as
// level_exec_kernel for the same program (canonical C[m, n, b] = sum_k
// A[m, k, b] B[k, n, b], Eq. 1), in the same level order, with the same store
// permutations and arithmetic; the interpretation (merge lookup, field
// decode, leaf sub-block loops, store offset tables) is resolved when the
// source is generated.  It differs in scheduling only: contiguous slice
// ranges per block, the root's sum over k split until every thread has a
// part, root partials summed per thread in the arithmetic's own wide form,
// two outputs per slot where a level has slots to spare (16-byte types), and
// optionally the two-phase schedule (jit.hpp).
#include "jit.hpp"

#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <mutex>
#include <sstream>
#include <vector>

namespace qtn {
namespace {

const char* kArithSource =
#include "arith_src.inc"
    ;

// ------------------------------------------------------------------ NVRTC --

struct Nvrtc {
  bool tried = false, ok = false;
  std::string why;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
};
Nvrtc g_nvrtc;
std::mutex g_nvrtc_mu;

Nvrtc& nvrtc() {
  std::lock_guard<std::mutex> lk(g_nvrtc_mu);
  if (g_nvrtc.tried) return g_nvrtc;
  g_nvrtc.tried = true;
  void* h = nullptr;
  for (const char* name : {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                           "/usr/local/cuda/lib64/libnvrtc.so"}) {
    h = dlopen(name, RTLD_NOW | RTLD_LOCAL);
    if (h) break;
  }
  if (!h) {
    g_nvrtc.why = "libnvrtc not found";
    return g_nvrtc;
  }
  auto sym = [&](const char* s) { return dlsym(h, s); };
  g_nvrtc.create = reinterpret_cast<decltype(&nvrtcCreateProgram)>(sym("nvrtcCreateProgram"));
  g_nvrtc.compile = reinterpret_cast<decltype(&nvrtcCompileProgram)>(sym("nvrtcCompileProgram"));
  g_nvrtc.cubin_size = reinterpret_cast<decltype(&nvrtcGetCUBINSize)>(sym("nvrtcGetCUBINSize"));
  g_nvrtc.cubin = reinterpret_cast<decltype(&nvrtcGetCUBIN)>(sym("nvrtcGetCUBIN"));
  g_nvrtc.log_size = reinterpret_cast<decltype(&nvrtcGetProgramLogSize)>(sym("nvrtcGetProgramLogSize"));
  g_nvrtc.log = reinterpret_cast<decltype(&nvrtcGetProgramLog)>(sym("nvrtcGetProgramLog"));
  g_nvrtc.destroy = reinterpret_cast<decltype(&nvrtcDestroyProgram)>(sym("nvrtcDestroyProgram"));
  g_nvrtc.ok = g_nvrtc.create && g_nvrtc.compile && g_nvrtc.cubin_size && g_nvrtc.cubin && g_nvrtc.log_size &&
               g_nvrtc.log && g_nvrtc.destroy;
  if (!g_nvrtc.ok) g_nvrtc.why = "libnvrtc lacks an entry point";
  return g_nvrtc;
}

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// --------------------------------------------------------------- codegen --

const char* type_name(Arith a) {
  switch (a) {
    case Arith::F64: return "double2";
    case Arith::F32: return "float2";
    case Arith::F32X2: return "dfc";
    default: return nullptr;
  }
}

// sum_i bit(o, i) * w[i] for bits lo..rc-1 of `var`, as runs of bits whose
// weights are consecutive powers of two (each run one shift, mask and add).
std::string pos_expr(const std::string& var, const uint16_t* w, int lo, int rc) {
  std::ostringstream e;
  bool first = true;
  int i = lo;
  while (i < rc) {
    int j = i + 1;
    const bool pow2 = w[i] != 0 && (w[i] & (w[i] - 1)) == 0;
    if (pow2)
      while (j < rc && (uint32_t)w[j] == 2u * w[j - 1]) ++j;
    const uint32_t mask = (1u << (j - i)) - 1u;
    e << (first ? "" : " + ") << "(((" << var << " >> " << i << ") & " << mask << "u) * " << w[i] << "u)";
    first = false;
    i = j;
  }
  return first ? std::string("0u") : e.str();
}

// Pointer to an operand: leaf (sub-block of the item's outer-class values)
// or a tensor of the item's arena.
std::string operand(const Program& pg, bool leaf, uint32_t id) {
  std::ostringstream e;
  if (!leaf) {
    e << "(arena + " << id << "u)";
    return e.str();
  }
  const DevLeaf& L = pg.leaves[id];
  e << "(s_lt + " << L.base << "u";
  for (int j = 0; j < L.ncut; ++j)
    e << " + ((unsigned)((s >> " << (int)L.cut_bit[j] << ") & 1ull) << " << (L.rank_nc + j) << ")";
  e << ")";
  return e.str();
}

// One merge's code for output unit o0 (a multiple of its unit size).
void emit_merge(std::ostringstream& o, const Program& pg, const DevStep& st, uint32_t beg, int ulog, int ks) {
  const int ma = st.ma, nb = st.nb, kb = st.kb, bb = st.bb;
  const int rc = ma + nb + bb;
  const bool root = st.flags & STEP_ROOT;
  const uint32_t u = 1u << ulog;
  o << "      const V* __restrict__ A = " << operand(pg, st.flags & STEP_A_LEAF, st.a) << ";\n";
  o << "      const V* __restrict__ B = " << operand(pg, st.flags & STEP_B_LEAF, st.b) << ";\n";
  o << "      const unsigned e0 = (uf - " << beg << "u) << " << ulog << ";\n";
  if (!root) {
    if (st.flags & STEP_EXPORT)  // hoisted result: a pseudo-leaf of the bit string's global leaf table
      o << "      V* __restrict__ C = g_lt + " << pg.leaves[st.c].base << "u;\n";
    else
      o << "      V* __restrict__ C = arena + " << st.c << "u;\n";
    o << "      const unsigned p0 = " << pos_expr("e0", st.w, ulog, rc) << ";\n";
  }
  const uint32_t kpart = 1u << (kb - ks);
  for (uint32_t r = 0; r < u; ++r) {
    o << "      {\n";
    if (root) {
      o << "        const unsigned e = e0 + " << r << "u;\n";
      o << "        const unsigned oo = e >> " << ks << ", k0 = (e & " << ((1u << ks) - 1u) << "u) * " << kpart
        << "u;\n";
    } else {
      o << "        const unsigned oo = e0 + " << r << "u, k0 = 0u;\n";
    }
    o << "        const unsigned m = oo & " << ((1u << ma) - 1u) << "u, n = (oo >> " << ma << ") & "
      << ((1u << nb) - 1u) << "u, b = oo >> " << (ma + nb) << ";\n";
    o << "        const V* __restrict__ ap = A + m + (k0 << " << ma << ") + (b << " << (ma + kb) << ");\n";
    o << "        const V* __restrict__ bp = B + k0 + (n << " << kb << ") + (b << " << (kb + nb) << ");\n";
    o << "        Ops::Acc acc = Ops::mul(ap[0], bp[0]);\n";
    for (uint32_t k = 1; k < kpart; ++k)
      o << "        Ops::fma(acc, ap[" << (k << ma) << "], bp[" << k << "]);\n";
    if (root) {
      // Root partials: compensated FP64 sums in the FP64 arithmetic; in the
      // FP32-storage arithmetics a double word per thread on the FP32 pipe
      // (TwoSum of the high parts, the errors and low parts collected
      // lazily), converted to FP64 once at the end.
      o << "        root_add(acc);\n";
    } else {
      uint32_t add = 0;
      for (int bit = 0; bit < ulog; ++bit)
        if ((r >> bit) & 1u) add += st.w[bit];
      o << "        C[p0 + " << add << "u] = Ops::result(acc);\n";
    }
    o << "      }\n";
  }
}

// Per-level loop layout for 2^lg items per pass: each merge's first unit in
// the level's flat unit range, its unit size 2^ulog and its k split 2^ks
// (root only: its outputs are summed, not stored, so its sum over k is split
// until the level has a slot for every thread, beyond the four-output
// table's split where that applies).
struct MergeGen {
  int j;
  uint32_t beg;
  int ulog, ks;
};
struct LevelGen {
  std::vector<MergeGen> m;
  uint64_t units = 0;  // slots per item
  uint64_t work = 0;   // largest multiply-add count of one slot
};

LevelGen level_gen_ul(const Program& pg, size_t l, int UL, int lg, int threads);

// Unit size of level l: the arithmetic's (UL), or for the 16-byte types
// (one output per slot) two outputs per slot where that takes no more
// rounds-times-work than one, so that a slot's decode, dispatch and
// addressing serve two outputs.
int level_ul(const Program& pg, size_t l, int UL, int lg, int threads) {
  if (UL) return UL;
  auto cost = [&](const LevelGen& g) { return ((g.units << lg) + threads - 1) / threads * g.work; };
  const LevelGen g0 = level_gen_ul(pg, l, 0, lg, threads), g1 = level_gen_ul(pg, l, 1, lg, threads);
  return (g1.units << lg) >= (uint64_t)threads && cost(g1) <= cost(g0) ? 1 : 0;
}

LevelGen level_gen(const Program& pg, size_t l, int UL, int lg, int threads) {
  return level_gen_ul(pg, l, level_ul(pg, l, UL, lg, threads), lg, threads);
}

LevelGen level_gen_ul(const Program& pg, size_t l, int UL, int lg, int threads) {
  LevelGen g;
  const DevLevel& lv = pg.levels[l];
  for (int j = lv.first; j < lv.first + lv.count; ++j) {
    const DevStep& st = pg.steps[j];
    const int rc0 = st.ma + st.nb + st.bb;
    int ks = 0;
    if (st.flags & STEP_ROOT) {
      ks = UL >= kLevelUnitLog2 ? std::min<int>(st.kb, kRootSplitLog2) : 0;
      auto slots = [&](int k) { return ((uint64_t)1 << (rc0 + k - std::min(rc0 + k, UL))) << lg; };
      while (ks < st.kb && slots(ks) < (uint64_t)threads) ++ks;
    }
    const int rc = rc0 + ks, ulog = std::min(rc, UL);
    g.m.push_back(MergeGen{j, (uint32_t)g.units, ulog, ks});
    g.units += (uint64_t)1 << (rc - ulog);
    g.work = std::max<uint64_t>(g.work, ((uint64_t)1 << ulog) << (st.kb - ks));
  }
  return g;
}

// Estimated time of one pass of level l over 2^lg items, in units of one
// slot multiply-add: rounds of the block over the slots times the longest
// slot, plus one for the barrier.
double level_cost(const Program& pg, size_t l, int UL, int lg, int threads) {
  const LevelGen g = level_gen(pg, l, UL, lg, threads);
  const uint64_t slots = g.units << lg;
  return (double)((slots + threads - 1) / threads) * (double)g.work + 1.0;
}

// Binary dispatch over the merges [lo, hi) of a level by unit index uf.
void emit_dispatch(std::ostringstream& o, const Program& pg, const std::vector<MergeGen>& ms, int lo, int hi) {
  if (hi - lo == 1) {
    const MergeGen& g = ms[lo];
    o << "    {  // merge " << g.j << "\n";
    emit_merge(o, pg, pg.steps[g.j], g.beg, g.ulog, g.ks);
    o << "    }\n";
    return;
  }
  const int mid = (lo + hi) / 2;
  o << "    if (uf < " << ms[mid].beg << "u) {\n";
  emit_dispatch(o, pg, ms, lo, mid);
  o << "    } else {\n";
  emit_dispatch(o, pg, ms, mid, hi);
  o << "    }\n";
}

// One level over 2^lg items of `count` (a variable of the generated code)
// with arenas `stride` elements apart; s0 is the first item's slice.
void emit_level(std::ostringstream& o, const Program& pg, size_t l, int UL, int lg, uint32_t stride,
                const char* count, int threads) {
  const LevelGen g = level_gen(pg, l, UL, lg, threads);
  bool leaf_operand = false;
  for (const MergeGen& m : g.m) leaf_operand |= (pg.steps[m.j].flags & (STEP_A_LEAF | STEP_B_LEAF)) != 0;
  o << "    // level " << l << "\n";
  o << "    for (unsigned f = threadIdx.x; f < " << (g.units << lg) << "u; f += " << threads << "u) {\n";
  o << "      const unsigned item = f & " << ((1u << lg) - 1u) << "u, uf = f >> " << lg << ";\n";
  o << "      if (item >= " << count << ") continue;\n";
  if (leaf_operand) o << "      const unsigned long long s = s0 + item;\n";
  o << "      V* arena = s_arena + item * " << stride << "u;\n";
  emit_dispatch(o, pg, g.m, 0, (int)g.m.size());
  o << "    }\n    __syncthreads();\n";
}

// Tensors made below level `split` and read at or above it (offset, size),
// and the arena extent of the levels below `split`.
using Crossing = JitCrossing;
bool crossings(const Program& pg, size_t split, std::vector<Crossing>* out, uint32_t* extent) {
  std::vector<int> level_of(pg.steps.size());
  for (size_t l = 0; l < pg.levels.size(); ++l)
    for (int j = pg.levels[l].first; j < pg.levels[l].first + pg.levels[l].count; ++j) level_of[j] = (int)l;
  // Last writer of each arena offset, updated at the end of each level (the
  // merges of one level read before any of them writes).
  std::vector<std::pair<uint32_t, int>> last;
  auto writer = [&](uint32_t off) {
    for (auto it = last.rbegin(); it != last.rend(); ++it)
      if (it->first == off) return it->second;
    return -1;
  };
  std::vector<char> crossing(pg.steps.size(), 0);
  uint32_t ext = 0;
  for (size_t l = 0; l < pg.levels.size(); ++l) {
    const DevLevel& lv = pg.levels[l];
    for (int j = lv.first; j < lv.first + lv.count; ++j) {
      const DevStep& st = pg.steps[j];
      const uint32_t ops[2] = {st.a, st.b};
      const bool leaf[2] = {(st.flags & STEP_A_LEAF) != 0, (st.flags & STEP_B_LEAF) != 0};
      for (int t = 0; t < 2; ++t) {
        if (leaf[t]) continue;
        const int w = writer(ops[t]);
        if (w < 0) return false;  // an arena operand nothing wrote
        if (level_of[w] < (int)split && l >= split) crossing[w] = 1;
      }
      if (l < split && !(st.flags & STEP_ROOT))
        ext = std::max<uint32_t>(ext, st.c + (1u << (st.ma + st.nb + st.bb)));
    }
    for (int j = lv.first; j < lv.first + lv.count; ++j)
      if (!(pg.steps[j].flags & STEP_ROOT)) last.emplace_back(pg.steps[j].c, j);
  }
  out->clear();
  uint32_t at = 0;
  for (size_t j = 0; j < pg.steps.size(); ++j)
    if (crossing[j]) {
      const uint32_t z = 1u << (pg.steps[j].ma + pg.steps[j].nb + pg.steps[j].bb);
      out->push_back(Crossing{pg.steps[j].c, z, at});
      at += z;
    }
  *extent = ext;
  return true;
}

}  // namespace

bool jit_crossings(const Program& pg, size_t split, std::vector<JitCrossing>* out, uint32_t* extent) {
  return crossings(pg, split, out, extent);
}

bool jit_available(std::string* why) {
  Nvrtc& n = nvrtc();
  if (!n.ok && why) *why = n.why;
  return n.ok;
}

bool jit_level_shape(const Program& pg, int elem_bytes, int threads, int blocks_per_sm, bool two_phase,
                     JitLevelShape* out) {
  int dev = 0, max_optin = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const int bps = blocks_per_sm > 1 ? blocks_per_sm : 1;
  const size_t cap = std::min<size_t>((size_t)max_optin, (size_t)per_sm / bps - 1024);
  return jit_level_schedule(pg, elem_bytes, threads, bps, cap, two_phase, out);
}

bool jit_level_schedule(const Program& pg, int elem_bytes, int threads, int bps, size_t cap, bool two_phase,
                        JitLevelShape* out) {
  JitLevelShape sh;
  sh.threads = threads;
  sh.blocks_per_sm = bps;
  sh.arena_stride = pg.arena_elems | 1u;
  const size_t table = align16((size_t)pg.leaf_elems * elem_bytes);
  const size_t red = (size_t)threads * 32;  // one Partial per thread, overlaid on the arenas
  auto fits = [&](uint32_t stride, int lg, size_t* total) {
    const size_t arena = (size_t)stride * ((size_t)1 << lg) * elem_bytes;
    *total = table + align16(std::max(arena, red));
    return *total <= cap;
  };
  bool found = false;
  for (int lg = 5; lg >= 0 && !found; --lg)
    if (fits(sh.arena_stride, lg, &sh.smem)) {
      sh.log2_items = lg;
      found = true;
    }
  if (!found) return false;
  // Two-phase schedule: the split level and the item count of the levels
  // below it with the fewest estimated slot-steps per item (the single-phase
  // estimate is kept for comparison).
  const int UL = elem_bytes == 16 ? 0 : kLevelUnitLog2;
  const size_t nl = pg.levels.size();
  std::vector<double> cost_s(nl);
  for (size_t l = 0; l < nl; ++l) cost_s[l] = level_cost(pg, l, UL, sh.log2_items, threads);
  double single = 0;
  for (double c : cost_s) single += c;
  single /= (double)(1 << sh.log2_items);
  sh.est_cost = sh.est_cost_single = single;
  if (!two_phase) {
    *out = sh;
    return true;
  }
  double best = 0;
  double above = single;  // levels >= split, per item
  for (size_t split = 1; split < nl; ++split) {
    above -= cost_s[split - 1] / (double)(1 << sh.log2_items);
    std::vector<Crossing> cr;
    uint32_t ext = 0;
    if (!crossings(pg, split, &cr, &ext)) break;
    uint32_t cross = 0;
    for (const Crossing& c : cr) cross += c.size;
    const uint32_t fstride = ext | 1u;
    for (int lf = sh.log2_items + 1; lf <= 5; ++lf) {
      size_t total = 0;
      if (!fits(fstride, lf, &total) || total > sh.smem) continue;
      double below = 0;
      for (size_t l = 0; l < split; ++l) below += level_cost(pg, l, UL, lf, threads);
      // parking and reloading: two element copies per parked element
      const double est = below / (double)(1 << lf) + above + 2.0 * cross / (double)threads / 4.0;
      if (!sh.split_level || est < best) {
        best = est;
        sh.est_cost = est;
        sh.split_level = (int)split;
        sh.log2_forest = lf;
        sh.forest_stride = fstride;
        sh.cross_elems = cross;
        sh.scratch_elems_per_block = (size_t)cross << lf;
      }
    }
  }
  if (!sh.split_level) return false;
  *out = sh;
  return true;
}

std::string jit_level_source(const Program& pg, Arith a, const JitLevelShape& sh, std::string* err) {
  const char* vt = type_name(a);
  if (!vt) {
    *err = "no specialised executor for this arithmetic";
    return "";
  }
  if (pg.levels.empty()) {
    *err = "not a level program";
    return "";
  }
  for (const DevStep& st : pg.steps)
    if (st.flags & STEP_EXPORT) {
      *err = "item steps export";
      return "";
    }
  const int elem = arith_elem_bytes(a);
  const int UL = elem == 16 ? 0 : kLevelUnitLog2;
  const int T = sh.threads;
  const uint32_t I = 1u << sh.log2_items;
  const size_t table = align16((size_t)pg.leaf_elems * elem);
  const size_t split = (size_t)sh.split_level;
  std::vector<Crossing> cr;
  if (split) {
    uint32_t ext = 0;
    if (!crossings(pg, split, &cr, &ext) || (ext | 1u) != sh.forest_stride) {
      *err = "two-phase schedule does not match the program";
      return "";
    }
  }
  std::ostringstream o;
  o << "// Generated: specialised level executor (" << pg.steps.size() << " merges, " << pg.levels.size()
    << " levels" << (split ? ", two-phase" : "") << ").\n";
  o << "struct __align__(16) Partial {\n  double re, im, cre, cim;\n"
       "  static __device__ __forceinline__ Partial make(double a, double b, double c, double d) {\n"
       "    Partial p; p.re = a; p.im = b; p.cre = c; p.cim = d; return p;\n  }\n};\n";
  o << kArithSource << "\n";
  o << "typedef " << vt << " V;\n";
  if (a == Arith::F64) {
    o << "typedef CplxOps<V> Ops;\n";
    o << "#define root_add(v) do { kahan_add(sr, cr, (v).x); kahan_add(si, ci, (v).y); } while (0)\n";
  } else {
    o << "__device__ __forceinline__ void dw_add(float& ah, float& al, float bh, float bl) {\n"
         "  float t, e;\n  two_sum(ah, bh, t, e);\n  ah = t;\n  al = __fadd_rn(al, __fadd_rn(e, bl));\n}\n";
    if (a == Arith::F32X2)
      // Packed FP32 pairs where the device has them.
      o << "#if __CUDA_ARCH__ >= 1000\ntypedef CplxOpsX2 Ops;\n"
           "#define root_add(v) do { x2 h_, l_; float a_, b_, c_, d_; Ops::sum((v), h_, l_); x2_unpack(h_, a_, b_); "
           "x2_unpack(l_, c_, d_); dw_add(qrh, qrl, a_, c_); dw_add(qih, qil, b_, d_); } while (0)\n"
           "#else\ntypedef CplxOps<V> Ops;\n"
           "#define root_add(v) do { dw_add(qrh, qrl, (v).rh, (v).rl); dw_add(qih, qil, (v).ih, (v).il); } "
           "while (0)\n#endif\n";
    else
      o << "typedef CplxOps<V> Ops;\n"
           "#define root_add(v) do { dw_add(qrh, qrl, (v).x, 0.f); dw_add(qih, qil, (v).y, 0.f); } while (0)\n";
  }
  o << "extern \"C\" __global__ void __launch_bounds__(" << T << ", " << sh.blocks_per_sm
    << ") qtn_level_jit(const V* __restrict__ leaf_tables, Partial* __restrict__ partials, V* __restrict__ scratch,\n"
       "    unsigned long long slice_lo, unsigned long long slice_hi, int blocks_per_x) {\n";
  o << "  extern __shared__ __align__(16) unsigned char smem[];\n";
  o << "  V* s_lt = reinterpret_cast<V*>(smem);\n";
  o << "  V* s_arena = reinterpret_cast<V*>(smem + " << table << ");\n";
  o << "  Partial* s_red = reinterpret_cast<Partial*>(smem + " << table << ");\n";
  o << "  const int xi = blockIdx.x / blocks_per_x, bx = blockIdx.x % blocks_per_x;\n";
  o << "  {\n    const unsigned* src = reinterpret_cast<const unsigned*>(leaf_tables + (size_t)xi * "
    << pg.leaf_elems << "u);\n    unsigned* dst = reinterpret_cast<unsigned*>(s_lt);\n"
    << "    for (unsigned i = threadIdx.x; i < " << (size_t)pg.leaf_elems * elem / 4 << "u; i += " << T
    << "u) dst[i] = src[i];\n  }\n  __syncthreads();\n";
  o << "  double sr = 0.0, si = 0.0, cr = 0.0, ci = 0.0;\n";
  o << "  float qrh = 0.f, qrl = 0.f, qih = 0.f, qil = 0.f;\n";
  // The block's share of the slices: a contiguous range, sizes within one.
  o << "  const unsigned long long S = slice_hi - slice_lo, q = S / (unsigned long long)blocks_per_x,\n"
       "      r = S % (unsigned long long)blocks_per_x;\n"
       "  const unsigned long long ib = (unsigned long long)bx * q + ((unsigned long long)bx < r ? bx : r),\n"
       "      ie = ib + q + ((unsigned long long)bx < r ? 1ull : 0ull);\n";
  if (!split) {
    o << "  for (unsigned long long i0 = ib; i0 < ie; i0 += " << I << "ull) {\n";
    o << "    const unsigned nI = (ie - i0) < " << I << "ull ? (unsigned)(ie - i0) : " << I << "u;\n";
    o << "    const unsigned long long s0 = slice_lo + i0;\n";
    for (size_t l = 0; l < pg.levels.size(); ++l) emit_level(o, pg, l, UL, sh.log2_items, sh.arena_stride, "nI", T);
    o << "  }\n";
  } else {
    const uint32_t F = 1u << sh.log2_forest, X = sh.cross_elems;
    o << "  V* __restrict__ park = scratch + (size_t)blockIdx.x * " << (size_t)F * X << "u;\n";
    o << "  for (unsigned long long c0 = ib; c0 < ie; c0 += " << F << "ull) {\n";
    o << "    const unsigned nF = (ie - c0) < " << F << "ull ? (unsigned)(ie - c0) : " << F << "u;\n";
    o << "    {\n    const unsigned long long s0 = slice_lo + c0;\n";
    for (size_t l = 0; l < split; ++l) emit_level(o, pg, l, UL, sh.log2_forest, sh.forest_stride, "nF", T);
    o << "    }\n";
    o << "    // park the tensors the later levels read\n";
    for (const Crossing& c : cr) {
      int lz = 0;
      while ((1u << lz) < c.size) ++lz;
      o << "    for (unsigned f = threadIdx.x; f < " << ((size_t)c.size << sh.log2_forest) << "u; f += " << T
        << "u) {\n      const unsigned item = f >> " << lz << ", e = f & " << (c.size - 1) << "u;\n"
        << "      if (item < nF) park[item * " << X << "u + " << c.at << "u + e] = s_arena[item * "
        << sh.forest_stride << "u + " << c.off << "u + e];\n    }\n";
    }
    o << "    __syncthreads();\n";
    o << "    for (unsigned p0 = 0; p0 < nF; p0 += " << I << "u) {\n";
    o << "    const unsigned nI = (nF - p0) < " << I << "u ? nF - p0 : " << I << "u;\n";
    o << "    const unsigned long long s0 = slice_lo + c0 + p0;\n";
    for (const Crossing& c : cr) {
      int lz = 0;
      while ((1u << lz) < c.size) ++lz;
      o << "    for (unsigned f = threadIdx.x; f < " << ((size_t)c.size << sh.log2_items) << "u; f += " << T
        << "u) {\n      const unsigned item = f >> " << lz << ", e = f & " << (c.size - 1) << "u;\n"
        << "      if (item < nI) s_arena[item * " << sh.arena_stride << "u + " << c.off << "u + e] = park[(p0 + item) * "
        << X << "u + " << c.at << "u + e];\n    }\n";
    }
    o << "    __syncthreads();\n";
    for (size_t l = split; l < pg.levels.size(); ++l)
      emit_level(o, pg, l, UL, sh.log2_items, sh.arena_stride, "nI", T);
    o << "    }\n  }\n";
  }
  o << "  s_red[threadIdx.x] = Partial::make(sr + ((double)qrh + (double)qrl), si + ((double)qih + (double)qil), cr, ci);\n";
  o << "  tree_reduce(s_red, " << T << ");\n";
  o << "  if (threadIdx.x == 0) partials[(size_t)xi * blocks_per_x + bx] = s_red[0];\n}\n";
  // The hoisted merges (prologue levels, once per bit string: one block of
  // kJitPrologueThreads), also as straight code: their operands are leaves
  // without outer cut bits and the prologue arena; exports go to the global
  // leaf table.
  if (!pg.prologue.empty() && !pg.pro_levels.empty()) {
    Program pp;
    pp.leaves = pg.leaves;
    pp.steps = pg.prologue;
    pp.levels = pg.pro_levels;
    const int PT = kJitPrologueThreads;
    o << "extern \"C\" __global__ void __launch_bounds__(" << PT << ", 1) qtn_prologue_jit(V* __restrict__ leaf_tables) {\n";
    o << "  extern __shared__ __align__(16) unsigned char smem[];\n";
    o << "  V* s_lt = reinterpret_cast<V*>(smem);\n";
    o << "  V* s_arena = reinterpret_cast<V*>(smem + " << table << ");\n";
    o << "  V* __restrict__ g_lt = leaf_tables + (size_t)blockIdx.x * " << pg.leaf_elems << "u;\n";
    o << "  {\n    const unsigned* src = reinterpret_cast<const unsigned*>(g_lt);\n"
      << "    unsigned* dst = reinterpret_cast<unsigned*>(s_lt);\n"
      << "    for (unsigned i = threadIdx.x; i < " << (size_t)pg.leaf_elems * elem / 4 << "u; i += " << PT
      << "u) dst[i] = src[i];\n  }\n  __syncthreads();\n";
    o << "  const unsigned long long s0 = 0ull;\n";
    for (size_t l = 0; l < pp.levels.size(); ++l) emit_level(o, pp, l, UL, 0, 0u, "1u", PT);
    o << "}\n";
  }
  return o.str();
}

bool jit_compile(const std::string& src, size_t smem, const void** kernel, std::string* err, size_t pro_smem,
                 const void** prologue) {
  Nvrtc& n = nvrtc();
  if (!n.ok) {
    *err = n.why;
    return false;
  }
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  const std::string arch = "-arch=sm_" + std::to_string(major * 10 + minor) + (major >= 9 ? "a" : "");
  nvrtcProgram prog;
  if (n.create(&prog, src.c_str(), "qtn_level_jit.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
    *err = "nvrtcCreateProgram failed";
    return false;
  }
  const char* opts[] = {arch.c_str(), "-std=c++17", "-default-device"};
  const nvrtcResult rc = n.compile(prog, 3, opts);
  if (rc != NVRTC_SUCCESS) {
    size_t ls = 0;
    n.log_size(prog, &ls);
    std::string log(ls, '\0');
    n.log(prog, &log[0]);
    *err = "nvrtc: " + log.substr(0, 2000);
    n.destroy(&prog);
    return false;
  }
  size_t cs = 0;
  n.cubin_size(prog, &cs);
  std::vector<char> cubin(cs);
  n.cubin(prog, cubin.data());
  n.destroy(&prog);
  cudaLibrary_t lib;
  cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e != cudaSuccess) {
    *err = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e);
    return false;
  }
  cudaKernel_t k;
  e = cudaLibraryGetKernel(&k, lib, "qtn_level_jit");
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
  if (e != cudaSuccess) {
    *err = std::string("loading the specialised kernel: ") + cudaGetErrorString(e);
    return false;
  }
  *kernel = reinterpret_cast<const void*>(k);  // the library stays loaded for the process
  if (prologue) {
    *prologue = nullptr;
    cudaKernel_t pk;
    if (cudaLibraryGetKernel(&pk, lib, "qtn_prologue_jit") == cudaSuccess) {
      e = cudaFuncSetAttribute(reinterpret_cast<const void*>(pk), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)pro_smem);
      if (e != cudaSuccess) {
        *err = std::string("loading the specialised prologue: ") + cudaGetErrorString(e);
        return false;
      }
      *prologue = reinterpret_cast<const void*>(pk);
    } else {
      cudaGetLastError();
    }
  }
  return true;
}

size_t jit_prologue_smem(const Program& pg, int elem_bytes) {
  return align16((size_t)pg.leaf_elems * elem_bytes) + align16((size_t)(pg.pro_arena_elems | 1u) * elem_bytes);
}

cudaError_t jit_prologue_launch(const void* kernel, int nx, size_t smem, void* leaf_tables, cudaStream_t stream) {
  void* lt = leaf_tables;
  void* args[] = {&lt};
  return cudaLaunchKernel(kernel, dim3((unsigned)nx), dim3((unsigned)kJitPrologueThreads), args, smem, stream);
}

cudaError_t jit_level_launch(const void* kernel, const JitLevelShape& sh, int nx, int blocks_per_x,
                             const void* leaf_tables, Partial* partials, void* scratch, uint64_t slice_lo,
                             uint64_t slice_hi, cudaStream_t stream) {
  if (sh.scratch_elems_per_block && !scratch) return cudaErrorInvalidValue;
  const void* lt = leaf_tables;
  unsigned long long lo = slice_lo, hi = slice_hi;
  int bpx = blocks_per_x;
  void* args[] = {const_cast<void*>(static_cast<const void*>(&lt)), &partials, &scratch, &lo, &hi, &bpx};
  return cudaLaunchKernel(kernel, dim3((unsigned)blocks_per_x * (unsigned)nx), dim3((unsigned)sh.threads), args,
                          sh.smem, stream);
}

}  // namespace qtn
