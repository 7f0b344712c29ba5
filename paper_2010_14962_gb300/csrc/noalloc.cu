// qtn_contract_amplitudes_noalloc: the device-resident amplitude path without
// any device allocation.
//
// Some callers cannot let a library call cudaMalloc: applications whose
// framework has already reserved the device memory in its own caching pool
// (a cudaMalloc from a third party then fails or fragments the pool), code
// running where allocation is forbidden or would stall (latency-critical
// serving loops, host callbacks, plug-ins of runtimes that own the device
// memory).  This entry point serves them: it uses only a fixed scratch array
// defined in this file, which every GPU that loads the library holds (at
// kNoallocScratchBytes) until the process exits.
//
// The array's name is only a host-side stand-in for the device symbol, so the
// host code below asks the runtime for its device address once per device
// (cudaGetSymbolAddress, with that device current) and passes that address to
// the kernels.  The first call on a device does this set-up; make that first
// call before any stream capture.  The array belongs to this file's module:
// the device memory behind it is reserved when that module is loaded on a
// device, which with CUDA's default lazy module loading is this set-up, i.e.
// the first call of this entry point on the device.  A caller whose framework
// later reserves most of the device memory should make that first call before
// the framework's pool takes it.
//
// Every call shares the one array: a call overwrites the previous call's
// contents, so calls that overlap on the GPU (different streams, or host
// threads racing) corrupt each other's results.  Issue them on one stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "internal.hpp"
#include "kernels.cuh"

namespace qtn {
namespace {

constexpr size_t kNoallocScratchBytes = 64ull << 20;  // 64 MiB per device

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_addr_mu;
std::map<int, unsigned char*> g_addr;  // device id -> device address of the array

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the scratch array on the current device.
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_addr_mu);
  auto it = g_addr.find(dev);
  if (it == g_addr.end()) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    it = g_addr.emplace(dev, static_cast<unsigned char*>(p)).first;
  }
  *out = it->second;
  return cudaSuccess;
}

template <class T>
size_t bytes_of(const std::vector<T>& v) {
  return v.size() * sizeof(T);
}

// The executors set the error word when they meet a merge they cannot run;
// this path keeps no state between calls, so a set word turns the call's
// amplitudes into NaN instead of being overwritten by the next call.
__global__ void mark_failed_kernel(const int* __restrict__ err, double* __restrict__ out, int nx) {
  if (*err == 0) return;
  for (int i = threadIdx.x; i < 2 * nx; i += blockDim.x) out[i] = __longlong_as_double(0x7ff8000000000000ll);
}

}  // namespace
}  // namespace qtn

using namespace qtn;

extern "C" qtn_status qtn_contract_amplitudes_noalloc(const qtn_plan_t* plan, const uint8_t* d_x, int nx,
                                                       qtn_precision prec, cudaStream_t stream, double* d_out) {
  internal::PlanView pv;
  if (!internal::plan_view(plan, &pv) || !d_x || !d_out || nx <= 0)
    return internal::set_error(QTN_ERR_INVALID_ARG, "bad argument");
  if (prec != QTN_FP64 && prec != QTN_FP32)
    return internal::set_error(QTN_ERR_UNSUPPORTED, "precision not available on this plan's executor");
  if (pv.wide)
    return internal::set_error(QTN_ERR_UNSUPPORTED, "the plan's per-slice working set does not fit in shared memory");
  std::lock_guard<std::mutex> lk(*pv.mu);
  const Program& pg = *pv.program;
  const Arith arith = prec == QTN_FP64 ? Arith::F64 : Arith::F32;
  const size_t elem = (size_t)arith_elem_bytes(arith);
  const uint64_t S = 1ull << pv.k;

  DeviceProgram dp;
  dp.n = pv.n;
  dp.p = pv.p;
  dp.k = pv.k;
  dp.n_leaves = (int)pg.leaves.size();
  dp.n_steps = (int)pg.steps.size();
  dp.leaf_elems = pg.leaf_elems;
  dp.arena_elems = pg.arena_elems;
  dp.n_pro_steps = (int)pg.prologue.size();
  dp.pro_arena_elems = pg.pro_arena_elems;
  dp.exec = pv.lane ? Executor::Lane : Executor::Block;
  dp.density = pg.density ? 1 : 0;
  ExecShape sh;
  if (!exec_shape(dp, arith, nx, S, &sh))
    return internal::set_error(QTN_ERR_UNSUPPORTED, "the plan's per-slice working set does not fit in shared memory");

  // Scratch layout: program | gate data | angles | leaf tables | partials | error word.
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off += round256(bytes);
    return at;
  };
  const size_t o_leaves = take(bytes_of(pg.leaves));
  const size_t o_steps = take(bytes_of(pg.steps));
  const size_t o_pro = take(bytes_of(pg.prologue));
  const size_t o_gq = take(bytes_of(pg.gate_q));
  const size_t o_gl = take(bytes_of(pg.gate_layer));
  const size_t o_gi = take(bytes_of(pg.gate_in_h));
  const size_t o_go = take(bytes_of(pg.gate_out_kind));
  const size_t o_gk = take(bytes_of(pg.gate_kind));
  const size_t o_ga = take(sizeof(double) * pv.p);
  const size_t o_be = take(sizeof(double) * pv.p);
  const size_t o_lt = take((size_t)nx * pg.leaf_elems * elem);
  const size_t o_pa = take((size_t)nx * sh.blocks_per_x * sizeof(Partial));
  const size_t o_err = take(sizeof(int));
  if (off > kNoallocScratchBytes)
    return internal::set_error(QTN_ERR_INVALID_ARG,
                               "request needs " + std::to_string(off) + " bytes of scratch; the allocation-free path has " +
                                   std::to_string(kNoallocScratchBytes) + " (use fewer bit strings per call)");

  unsigned char* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess)
    return internal::set_error(QTN_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));

  struct Piece {
    size_t at;
    const void* src;
    size_t bytes;
  } pieces[] = {{o_leaves, pg.leaves.data(), bytes_of(pg.leaves)},
                {o_steps, pg.steps.data(), bytes_of(pg.steps)},
                {o_pro, pg.prologue.data(), bytes_of(pg.prologue)},
                {o_gq, pg.gate_q.data(), bytes_of(pg.gate_q)},
                {o_gl, pg.gate_layer.data(), bytes_of(pg.gate_layer)},
                {o_gi, pg.gate_in_h.data(), bytes_of(pg.gate_in_h)},
                {o_go, pg.gate_out_kind.data(), bytes_of(pg.gate_out_kind)},
                {o_gk, pg.gate_kind.data(), bytes_of(pg.gate_kind)},
                {o_ga, pv.gamma, sizeof(double) * pv.p},
                {o_be, pv.beta, sizeof(double) * pv.p}};
  for (const Piece& pc : pieces) {
    if (pc.bytes == 0) continue;
    e = cudaMemcpyAsync(base + pc.at, pc.src, pc.bytes, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess)
      return internal::set_error(QTN_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
  }
  // The array keeps the previous call's contents: the error word must start at 0.
  e = cudaMemsetAsync(base + o_err, 0, sizeof(int), stream);
  if (e != cudaSuccess)
    return internal::set_error(QTN_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));

  dp.leaves = reinterpret_cast<const DevLeaf*>(base + o_leaves);
  dp.steps = reinterpret_cast<const DevStep*>(base + o_steps);
  dp.pro_steps = reinterpret_cast<const DevStep*>(base + o_pro);
  dp.gate_q = reinterpret_cast<const int32_t*>(base + o_gq);
  dp.gate_layer = reinterpret_cast<const int8_t*>(base + o_gl);
  dp.gate_in_h = reinterpret_cast<const int8_t*>(base + o_gi);
  dp.gate_out_kind = reinterpret_cast<const int8_t*>(base + o_go);
  dp.gate_kind = reinterpret_cast<const int8_t*>(base + o_gk);
  dp.gamma = reinterpret_cast<const double*>(base + o_ga);
  dp.beta = reinterpret_cast<const double*>(base + o_be);
  LaunchBuffers buf;
  buf.leaf_tables = base + o_lt;
  buf.partials = reinterpret_cast<Partial*>(base + o_pa);
  buf.err = reinterpret_cast<int*>(base + o_err);
  const double scale = std::pow(2.0, (pg.density ? -1.0 : -0.5) * pv.n);
  e = launch_contraction(dp, arith, d_x, nx, 0, S, buf, sh, scale, reinterpret_cast<double2*>(d_out), nullptr, nullptr,
                         stream);
  if (e != cudaSuccess)
    return internal::set_error(QTN_ERR_CUDA, std::string("launch_contraction: ") + cudaGetErrorString(e));
  mark_failed_kernel<<<1, 256, 0, stream>>>(buf.err, d_out, nx);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return internal::set_error(QTN_ERR_CUDA, std::string("mark_failed_kernel: ") + cudaGetErrorString(e));
  return QTN_OK;
}
