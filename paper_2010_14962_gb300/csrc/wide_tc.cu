// Tensor-core merge of the wide executor (see wide_tc.hpp).
//
// One CTA of 4 warps per work unit (item, batch index, row tile, column
// tile), persistent over units.  Per unit the complex merge is a real GEMM
// D[row, 2q + c'] = sum_kk X[row, kk] Y[2q + c', kk] with kk = 2k + c:
//   X[row, 2k + c] = (Re, Im) of the "row" operand at (row, k),
//   Y[2q, 2k + c] = (Re y, -Im y), Y[2q + 1, 2k + c] = (Im y, Re y),
// so D[row, 2q] and D[row, 2q + 1] are the real and imaginary part of
// sum_k x(row, k) y(q, k).  Rows are the merge's m (C's own layout) or n
// (the transposed product), whichever side has at least 128 entries.
//
// Pipeline: the threads stage K chunks of 32 real columns into one of two
// shared-memory stages (TF32-rounded, split into high and low parts for the
// three-product form); one thread issues the tcgen05.mma instructions of the
// chunk (M = 128, N = the column tile, K = 8 each) and commits them to the
// stage's mbarrier; a stage is refilled once its commit has arrived.  The
// accumulator lives in tensor memory (one column per real output column);
// the epilogue reads it with tcgen05.ld (warp w: rows 32w..32w+31) and
// stores each complex result at its consumer-layout position.  Every
// mbarrier wait is bounded; a wait that gives up sets the error word and
// the CTA stops after freeing its tensor memory.
#include "wide_tc.hpp"

#include <algorithm>

namespace qtn {
namespace {

constexpr int kRows = 128;      // UMMA M (one row per tensor-memory lane)
constexpr int kChunk = 32;      // real K columns per stage
constexpr int kTcThreads = 256;
constexpr int kStageIlp = 4;     // operand pairs a thread loads before it converts and stores them
constexpr uint32_t kWaitLimit = 1u << 20;

struct TcGeom {
  int rows_is_m;             // 1: rows are m (X = A, Y = B); 0: rows are n (X = B^T, Y = A)
  int ma, nb, kb, bb;
  uint64_t xr, xk, yq, yk;   // element strides: X(row, k), Y(q, k)
  uint64_t xbat, ybat;       // batch-index stride of X and Y
  int nt;                    // real columns per column tile (2 x complex)
  uint64_t row_tiles, col_tiles, base_units, units;
  int kc;                    // real K columns per chunk
  int kchunks;
  int ksplit, cps;           // K splits per output tile, chunks per split
  uint32_t idesc;
  int tmem_cols;
  uint32_t stage_bytes, x_bytes, y_bytes;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (r, kk) in an R-row K-major tile: 8 x 16-byte core
// matrices, cores along the rows 128 bytes apart, along K (R / 8) * 128.
__device__ __forceinline__ uint32_t core_off(int r, int kk, int R) {
  return (uint32_t)((((kk >> 2) * (R >> 3) + (r >> 3)) << 7) + ((r & 7) << 4) + ((kk & 3) << 2));
}

// Shared-memory matrix descriptor: start, leading (K-direction core) and
// stride (row-direction core) byte offsets, fixed field 0b001 at bit 46, no
// swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < kWaitLimit && !done; ++it)
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  return done != 0;
}

__device__ __forceinline__ const float2* operand_base(const WideTcArgs& a, const WideOperandRef& op, uint64_t g,
                                                      uint64_t xi, uint64_t s) {
  if (!op.leaf) return a.arena + g * a.arena_stride + op.off;
  uint64_t off = op.base;
  for (int j = 0; j < op.ncut; ++j) off += ((s >> op.cut_bit[j]) & 1ull) << (op.rank_nc + j);
  return a.leaf_tables + xi * a.leaf_elems + off;
}

// Store offset of the canonical output bits [lo, lo + nbits) of value v.
__device__ __forceinline__ uint64_t pos_bits(const uint8_t* wpos, int lo, int nbits, uint64_t v) {
  uint64_t p = 0;
  for (int i = 0; i < nbits; ++i)
    if ((v >> i) & 1ull) p += 1ull << wpos[lo + i];
  return p;
}

// Writes the 4 real columns kk..kk+3 of one tile row (high part, and the low
// part at +piece_bytes for the split form).
template <int PCS>
__device__ __forceinline__ void put4(unsigned char* base, uint32_t piece_bytes, uint32_t off, float a, float b,
                                     float c, float d) {
  const float ah = tf32_rna(a), bh = tf32_rna(b), ch = tf32_rna(c), dh = tf32_rna(d);
  *reinterpret_cast<float4*>(base + off) = make_float4(ah, bh, ch, dh);
  if (PCS == 2)
    *reinterpret_cast<float4*>(base + piece_bytes + off) =
        make_float4(tf32_rna(a - ah), tf32_rna(b - bh), tf32_rna(c - ch), tf32_rna(d - dh));
}

template <int P>
__global__ void __launch_bounds__(kTcThreads) wide_tc_kernel(WideTcArgs a, TcGeom G) {
  constexpr int PCS = P == 3 ? 2 : 1;  // staged pieces per operand
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t* posR = reinterpret_cast<uint64_t*>(smem + 2 * G.stage_bytes);
  uint64_t* posQ = posR + kRows;
  uint64_t* bar = posQ + kRows;  // two mbarriers
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(G.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const int rlog = G.rows_is_m ? G.ma : G.nb, qlog = G.rows_is_m ? G.nb : G.ma;
  const int rbit = G.rows_is_m ? 0 : G.ma, qbit = G.rows_is_m ? G.ma : 0;
  const int qt = G.nt >> 1;  // complex columns per tile
  const uint32_t lbo_x = (kRows / 8) * 128, lbo_y = (uint32_t)(G.nt / 8) * 128;
  uint32_t chunk_no = 0;
  bool failed = false;
  // Each thread stages the same (row, pair) slots of every chunk: kStageIlp
  // pairs of X (kRows rows x kc/4 pairs) and of Y (nt/2 rows x kc/4 pairs),
  // ordered so that consecutive threads read consecutive elements.
  const int kp = G.kc >> 2;  // complex pairs per row per chunk
  int xr_[kStageIlp], xp[kStageIlp], yq_[kStageIlp], yp[kStageIlp];
  bool xv[kStageIlp], yv[kStageIlp];
#pragma unroll
  for (int u = 0; u < kStageIlp; ++u) {
    const int i = tid + u * kTcThreads;
    xv[u] = i < kRows * kp;
    yv[u] = i < (G.nt >> 1) * kp;
    xr_[u] = G.xr == 1 ? i % kRows : i / kp;
    xp[u] = G.xr == 1 ? i / kRows : i % kp;
    yq_[u] = G.yq == 1 ? i % (G.nt >> 1) : i / kp;
    yp[u] = G.yq == 1 ? i / (G.nt >> 1) : i % kp;
  }
  for (uint64_t unit = blockIdx.x; unit < G.units && !failed; unit += gridDim.x) {
    const int split = (int)(unit % G.ksplit);
    const uint64_t bu = unit / G.ksplit;
    const uint64_t ct = bu % G.col_tiles;
    const uint64_t rt = (bu / G.col_tiles) % G.row_tiles;
    const uint64_t gb = bu / (G.col_tiles * G.row_tiles);
    const uint64_t b = gb & ((1ull << G.bb) - 1), g = gb >> G.bb;
    const uint64_t item = a.item_lo + g;
    const uint64_t xi = a.prologue ? item : item / a.items_per_x;
    const uint64_t sl = a.prologue ? 0 : a.slice_lo + item % a.items_per_x;
    const float2* Ap = operand_base(a, a.A, g, xi, sl);
    const float2* Bp = operand_base(a, a.B, g, xi, sl);
    float2* Cp = const_cast<float2*>(a.c_export ? a.leaf_tables + xi * a.leaf_elems + a.c_off
                                                : a.arena + g * a.arena_stride + a.c_off);
    const float2* Xbase = (G.rows_is_m ? Ap : Bp) + b * G.xbat + rt * kRows * G.xr;
    const float2* Ybase = (G.rows_is_m ? Bp : Ap) + b * G.ybat + ct * qt * G.yq;
    for (int i = tid; i < kRows; i += kTcThreads) posR[i] = pos_bits(a.wpos, rbit, rlog, rt * kRows + i);
    for (int i = tid; i < qt; i += kTcThreads) posQ[i] = pos_bits(a.wpos, qbit, qlog, ct * qt + i);
    const uint64_t posb = pos_bits(a.wpos, G.ma + G.nb, G.bb, b);
    const int c_lo = split * G.cps, c_hi = min(G.kchunks, c_lo + G.cps);
    // Software pipeline: the operands of chunk c + 1 are loaded into
    // registers before chunk c is converted and stored, so their global-load
    // latency overlaps that work, the barrier and the MMA issue.
    float2 cx0[kStageIlp], cx1[kStageIlp], cy0[kStageIlp], cy1[kStageIlp];
    float2 nx0[kStageIlp], nx1[kStageIlp], ny0[kStageIlp], ny1[kStageIlp];
    auto load_chunk = [&](int c, float2* x0, float2* x1, float2* y0, float2* y1) {
      const uint64_t k0 = (uint64_t)c * (G.kc >> 1);  // first complex k of the chunk
#pragma unroll
      for (int u = 0; u < kStageIlp; ++u) {
        if (xv[u]) {
          const uint64_t k = k0 + 2 * xp[u];
          x0[u] = Xbase[xr_[u] * G.xr + k * G.xk];
          x1[u] = Xbase[xr_[u] * G.xr + (k + 1) * G.xk];
        }
        if (yv[u]) {
          const uint64_t k = k0 + 2 * yp[u];
          y0[u] = Ybase[yq_[u] * G.yq + k * G.yk];
          y1[u] = Ybase[yq_[u] * G.yq + (k + 1) * G.yk];
        }
      }
    };
    if (c_lo < c_hi) load_chunk(c_lo, cx0, cx1, cy0, cy1);
    for (int c = c_lo; c < c_hi; ++c, ++chunk_no) {
      const int s = chunk_no & 1;
      if (c + 1 < c_hi) load_chunk(c + 1, nx0, nx1, ny0, ny1);
      if (chunk_no >= 2) {
        const bool ok = bar_wait(&bar[s], ((chunk_no - 2) >> 1) & 1);
        if (__syncthreads_or(!ok)) {
          failed = true;
          break;
        }
      }
      unsigned char* stx = smem + s * G.stage_bytes;
      unsigned char* sty = stx + PCS * G.x_bytes;
#pragma unroll
      for (int u = 0; u < kStageIlp; ++u) {
        if (xv[u]) put4<PCS>(stx, G.x_bytes, core_off(xr_[u], 4 * xp[u], kRows), cx0[u].x, cx0[u].y, cx1[u].x, cx1[u].y);
        if (yv[u]) {
          // Y in block form: rows 2q (Re, -Im) and 2q + 1 (Im, Re).
          put4<PCS>(sty, G.y_bytes, core_off(2 * yq_[u], 4 * yp[u], G.nt), cy0[u].x, -cy0[u].y, cy1[u].x, -cy1[u].y);
          put4<PCS>(sty, G.y_bytes, core_off(2 * yq_[u] + 1, 4 * yp[u], G.nt), cy0[u].y, cy0[u].x, cy1[u].y,
                    cy1[u].x);
        }
      }
#pragma unroll
      for (int u = 0; u < kStageIlp; ++u) {
        cx0[u] = nx0[u];
        cx1[u] = nx1[u];
        cy0[u] = ny0[u];
        cy1[u] = ny1[u];
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t xa = smem_u32(stx), ya = smem_u32(sty);
        // (x piece, y piece) per product: lo*hi, hi*lo, hi*hi (small terms first).
        const int px[3] = {P == 3 ? 1 : 0, 0, 0}, py[3] = {0, P == 3 ? 1 : 0, 0};
        for (int ks = 0; ks < G.kc / 8; ++ks)
          for (int t = (P == 3 ? 0 : 2); t < 3; ++t) {
            const uint64_t ad = sdesc(xa + px[t] * G.x_bytes + ks * 2 * lbo_x, lbo_x, 128);
            const uint64_t bd = sdesc(ya + py[t] * G.y_bytes + ks * 2 * lbo_y, lbo_y, 128);
            const uint32_t acc = (c > c_lo || ks > 0 || t > (P == 3 ? 0 : 2)) ? 1u : 0u;
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(G.idesc), "r"(acc));
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&bar[s])));
      }
    }
    if (failed) break;
    {
      const uint32_t last = chunk_no - 1;
      const bool ok = bar_wait(&bar[last & 1], (last >> 1) & 1);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    // Epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (its
    // rows), columns of half w / 4 (all columns in warps 0-3 when the tile
    // has fewer than 64), 32 real columns at a time.
    const int quarter = warp & 3, half = warp >> 2;
    const int row = quarter * 32 + lane;
    const int c_begin = G.nt >= 64 ? half * (G.nt >> 1) : 0;
    const int c_end = G.nt >= 64 ? c_begin + (G.nt >> 1) : (half == 0 ? G.nt : 0);
    float2* Cbase = Cp + posb + posR[row];
    for (int col0 = c_begin; col0 < c_end; col0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
          "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
            "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
            "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (G.ksplit == 1) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int q = (col0 >> 1) + j;
          if (q < qt) Cbase[posQ[q]] = make_float2(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]));
        }
      } else {
        // Split K: this split's partial rows go to the workspace, unpermuted.
        float* w = a.ws + ((bu * G.ksplit + split) * kRows + row) * (uint64_t)G.nt + col0;
#pragma unroll
        for (int j = 0; j < 32; j += 4)
          if (col0 + j < G.nt)
            *reinterpret_cast<float4*>(w + j) = make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                                                            __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // tensor memory and the position tables are free for the next unit
  }
  if (failed && tid == 0) atomicExch(a.err, 2);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G.tmem_cols));
}

// Sum of the K-split partials of every output (split order, FP64), stored
// at its consumer-layout position.
__global__ void __launch_bounds__(256) wide_tc_splitk_reduce(WideTcArgs a, TcGeom G) {
  const uint64_t qt = (uint64_t)(G.nt >> 1);
  const uint64_t total = G.base_units * kRows * qt;
  const int rlog = G.rows_is_m ? G.ma : G.nb, qlog = G.rows_is_m ? G.nb : G.ma;
  const int rbit = G.rows_is_m ? 0 : G.ma, qbit = G.rows_is_m ? G.ma : 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t q = i % qt, row = (i / qt) % kRows, bu = i / (qt * kRows);
    const uint64_t ct = bu % G.col_tiles;
    const uint64_t rt = (bu / G.col_tiles) % G.row_tiles;
    const uint64_t gb = bu / (G.col_tiles * G.row_tiles);
    const uint64_t b = gb & ((1ull << G.bb) - 1), g = gb >> G.bb;
    double re = 0.0, im = 0.0;
    for (int s = 0; s < G.ksplit; ++s) {
      const float2 v = *reinterpret_cast<const float2*>(a.ws + ((bu * G.ksplit + s) * kRows + row) * (uint64_t)G.nt +
                                                        2 * q);
      re += v.x;
      im += v.y;
    }
    const uint64_t item = a.item_lo + g;
    const uint64_t xi = a.prologue ? item : item / a.items_per_x;
    float2* Cp = const_cast<float2*>(a.c_export ? a.leaf_tables + xi * a.leaf_elems + a.c_off
                                                : a.arena + g * a.arena_stride + a.c_off);
    const uint64_t pos = pos_bits(a.wpos, rbit, rlog, rt * kRows + row) + pos_bits(a.wpos, qbit, qlog, ct * qt + q) +
                         pos_bits(a.wpos, G.ma + G.nb, G.bb, b);
    Cp[pos] = make_float2((float)re, (float)im);
  }
}

int g_tc_max_smem = 0;
// Raises the dynamic shared-memory cap of both kernel variants to the
// device's opt-in maximum (once).
cudaError_t tc_allow_max_smem() {
  if (g_tc_max_smem > 0) return cudaSuccess;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(wide_tc_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(wide_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess) g_tc_max_smem = optin;
  return e;
}

int g_tc_sms = 0;
int tc_sms() {
  if (g_tc_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_tc_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_tc_sms <= 0) g_tc_sms = 1;
  }
  return g_tc_sms;
}

// Launch geometry of a merge; ksplit from the SM count (two CTAs per SM
// wanted, at least two chunks per split) and the workspace capacity.
TcGeom make_geom(int ma, int nb, int kb, int bb, uint64_t n_items, int products, uint64_t ws_floats) {
  TcGeom G{};
  G.rows_is_m = (ma >= 7 && (ma >= nb || nb < 7)) ? 1 : 0;
  G.ma = ma;
  G.nb = nb;
  G.kb = kb;
  G.bb = bb;
  if (G.rows_is_m) {  // X = A (m, k), Y = B (n, k)
    G.xr = 1;
    G.xk = 1ull << ma;
    G.yq = 1ull << kb;
    G.yk = 1;
  } else {  // X = B^T (n, k), Y = A (m, k)
    G.xr = 1ull << kb;
    G.xk = 1;
    G.yq = 1;
    G.yk = 1ull << ma;
  }
  const uint64_t abat = 1ull << (ma + kb), bbat = 1ull << (kb + nb);
  G.xbat = G.rows_is_m ? abat : bbat;
  G.ybat = G.rows_is_m ? bbat : abat;
  const int rlog = G.rows_is_m ? ma : nb, qlog = G.rows_is_m ? nb : ma;
  G.nt = (int)std::min<uint64_t>(256, 2ull << qlog);
  G.row_tiles = 1ull << (rlog - 7);
  G.col_tiles = (2ull << qlog) / (uint64_t)G.nt;
  G.base_units = n_items * (1ull << bb) * G.row_tiles * G.col_tiles;
  G.kc = (int)std::min<uint64_t>(kChunk, 2ull << kb);
  G.kchunks = (int)((2ull << kb) / (uint64_t)G.kc);
  const uint64_t want = 2ull * tc_sms();
  uint64_t ks = 1;
  if (G.base_units < want && G.kchunks >= 4) {
    ks = std::min<uint64_t>((want + G.base_units - 1) / G.base_units, (uint64_t)G.kchunks / 2);
    const uint64_t per = G.base_units * kRows * (uint64_t)G.nt;
    if (per > 0) ks = std::min<uint64_t>(ks, ws_floats / per);
    if (ks < 2) ks = 1;
  }
  G.cps = (int)((G.kchunks + ks - 1) / ks);
  G.ksplit = (int)((G.kchunks + G.cps - 1) / G.cps);
  G.units = G.base_units * G.ksplit;
  G.idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(G.nt >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
  G.tmem_cols = std::max(32, G.nt);
  const int pcs = products == 3 ? 2 : 1;
  G.x_bytes = (uint32_t)kRows * kChunk * 4;
  G.y_bytes = (uint32_t)G.nt * kChunk * 4;
  G.stage_bytes = pcs * (G.x_bytes + G.y_bytes);
  return G;
}

}  // namespace

uint64_t wide_tc_workspace_floats(int ma, int nb, int kb, int bb, uint64_t n_items) {
  if (!wide_tc_shape_ok(ma, nb, kb, bb)) return 0;
  const TcGeom G = make_geom(ma, nb, kb, bb, n_items, 1, ~0ull);
  return G.ksplit > 1 ? G.units * kRows * (uint64_t)G.nt : 0;
}

bool wide_tc_shape_ok(int ma, int nb, int kb, int bb) {
  if (ma + nb + bb > kWideMaxRank || kb < 2 || kb > 24) return false;
  const bool rows_m = ma >= 7, rows_n = nb >= 7;
  if (!rows_m && !rows_n) return false;
  const int other = (rows_m && (ma >= nb || !rows_n)) ? nb : ma;
  return other >= 3;
}

cudaError_t wide_tc_launch(const WideTcArgs& a, int products, cudaStream_t stream) {
  if (!wide_tc_shape_ok(a.ma, a.nb, a.kb, a.bb) || (products != 1 && products != 3) || !a.err)
    return cudaErrorInvalidValue;
  const TcGeom G = make_geom(a.ma, a.nb, a.kb, a.bb, a.n_items, products, a.ws ? a.ws_floats : 0);
  const size_t smem = 2 * (size_t)G.stage_bytes + 2 * kRows * sizeof(uint64_t) + 64;
  // The shared-memory cap is a property of the kernel, not of one launch: it
  // is set to the device's opt-in maximum, so that a captured graph of a
  // larger merge stays launchable after smaller merges have run.
  cudaError_t e = tc_allow_max_smem();
  if (e != cudaSuccess) return e;
  if (smem > (size_t)g_tc_max_smem) return cudaErrorInvalidValue;
  int occ = 0;
  if (products == 3) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, wide_tc_kernel<3>, kTcThreads, smem);
  else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, wide_tc_kernel<1>, kTcThreads, smem);
  if (e != cudaSuccess) return e;
  occ = std::max(1, std::min(occ, 512 / G.tmem_cols));  // tensor memory: 512 columns per SM
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(G.units, (uint64_t)tc_sms() * occ));
  if (products == 3)
    wide_tc_kernel<3><<<grid, kTcThreads, smem, stream>>>(a, G);
  else
    wide_tc_kernel<1><<<grid, kTcThreads, smem, stream>>>(a, G);
  e = cudaGetLastError();
  if (e != cudaSuccess || G.ksplit == 1) return e;
  const uint64_t outs = G.base_units * kRows * (uint64_t)(G.nt >> 1);
  const unsigned rgrid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((outs + 255) / 256, (uint64_t)tc_sms() * 8));
  wide_tc_splitk_reduce<<<rgrid, 256, 0, stream>>>(a, G);
  return cudaGetLastError();
}

}  // namespace qtn
