// Arithmetic-pipe peaks of the current GPU, measured: the denominators of the
// roofline fractions of the FP32 and FP64 executors.  Each thread runs
// kChains independent multiply-add chains (enough independent work per warp
// to cover the pipe latency), the grid fills every SM several times over, and
// the kernel is timed with CUDA events; a multiply-add counts as 2 flops.
#include <cuda_runtime.h>

#include <string>

#include "internal.hpp"
#include "kernels.cuh"

namespace qtn {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <class T>
__device__ __forceinline__ T mad(T a, T b, T c);
template <>
__device__ __forceinline__ float mad<float>(float a, float b, float c) {
  return __fmaf_rn(a, b, c);
}
template <>
__device__ __forceinline__ double mad<double>(double a, double b, double c) {
  return __fma_rn(a, b, c);
}

// iters x kChains multiply-adds per thread; b and c are runtime values, so
// nothing folds; the sum of the chains is written only if it equals `never`
// (it does not), which keeps the chains live without memory traffic.
template <class T>
__global__ void __launch_bounds__(kThreads) pipe_peak_kernel(int iters, T b, T c, T never, T* sink) {
  T a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = (T)(threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = mad<T>(a[j], b, c);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == never) sink[blockIdx.x] = s;
}

// Packed FP32 pairs (fma.rn.f32x2, sm_100 and later): each instruction is
// two multiply-adds.  Same chains and grid as above, a pair per chain.
__global__ void __launch_bounds__(kThreads) pipe_peak_x2_kernel(int iters, float b, float c, float never, float* sink) {
  unsigned long long a[kChains], bb, cc;
  asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
  asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    const float lo = (float)(threadIdx.x + j), hi = lo + 0.5f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a[j]) : "f"(lo), "f"(hi));
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[j]) : "l"(bb), "l"(cc));
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[j]));
    s += lo + hi;
  }
  if (s == never) sink[blockIdx.x] = s;
}

template <class T>
void launch_peak(bool packed, int blocks, int iters, T mul, T add, T never, T* sink) {
  pipe_peak_kernel<T><<<blocks, kThreads>>>(iters, mul, add, never, sink);
}
template <>
void launch_peak<float>(bool packed, int blocks, int iters, float mul, float add, float never, float* sink) {
  if (packed)
    pipe_peak_x2_kernel<<<blocks, kThreads>>>(iters, mul, add, never, sink);
  else
    pipe_peak_kernel<float><<<blocks, kThreads>>>(iters, mul, add, never, sink);
}

template <class T>
cudaError_t time_pipe(int iters, int reps, double* tflops, bool packed = false) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = packed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pipe_peak_x2_kernel, kThreads, 0)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pipe_peak_kernel<T>, kThreads, 0);
  if (e != cudaSuccess) return e;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1) * 4;
  T* sink = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaMalloc(&sink, sizeof(T) * blocks);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  // b = 1 - 2^-20 and c = 2^-30 keep every chain finite and normal.
  const T mul = (T)(1.0 - 1.0 / (1 << 20)), add = (T)(1.0 / (1 << 30)), never = (T)-1.0;
  float best = 0.f;
  for (int r = 0; e == cudaSuccess && r < reps + 1; ++r) {  // the first run warms up
    launch_peak<T>(packed, blocks, iters, mul, add, never, sink);
    e = cudaEventRecord(a);
    launch_peak<T>(packed, blocks, iters, mul, add, never, sink);
    if (e == cudaSuccess) e = cudaEventRecord(b);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && r > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return e;
  const double flops = 2.0 * kChains * 4.0 * iters * (double)blocks * kThreads * (packed ? 2.0 : 1.0);
  *tflops = flops / (best / 1e3) / 1e12;
  return cudaSuccess;
}

}  // namespace
}  // namespace qtn

extern "C" qtn_status qtn_pipe_peaks(int reps, double* fp32_tflops, double* fp64_tflops) {
  using qtn::internal::set_error;
  if (!fp32_tflops || !fp64_tflops || reps < 1)
    return set_error(QTN_ERR_INVALID_ARG, "qtn_pipe_peaks: null output or reps < 1");
  double f32 = 0, f64 = 0;
  cudaError_t e = qtn::time_pipe<float>(1 << 14, reps, &f32);
  if (e == cudaSuccess) e = qtn::time_pipe<double>(1 << 9, reps, &f64);
  if (e != cudaSuccess) return set_error(QTN_ERR_CUDA, std::string("qtn_pipe_peaks: ") + cudaGetErrorString(e));
  *fp32_tflops = f32;
  *fp64_tflops = f64;
  return QTN_OK;
}

extern "C" qtn_status qtn_pipe_peak_fp32x2(int reps, double* tflops) {
  using qtn::internal::set_error;
  if (!tflops || reps < 1) return set_error(QTN_ERR_INVALID_ARG, "qtn_pipe_peak_fp32x2: null output or reps < 1");
  int dev = 0, major = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (major < 10) return set_error(QTN_ERR_UNSUPPORTED, "qtn_pipe_peak_fp32x2: no packed FP32 instructions");
  double t = 0;
  cudaError_t e = qtn::time_pipe<float>(1 << 13, reps, &t, true);
  if (e != cudaSuccess) return set_error(QTN_ERR_CUDA, std::string("qtn_pipe_peak_fp32x2: ") + cudaGetErrorString(e));
  *tflops = t;
  return QTN_OK;
}

extern "C" qtn_status qtn_arith_check(const double* a, const double* b, int count, int K, double* out_scalar,
                                      double* out_merge, int* packed) {
  using qtn::internal::set_error;
  if (!a || !b || !out_scalar || !out_merge || count < 0 || K < 1 || count > (1 << 24) || K > 4096)
    return set_error(QTN_ERR_INVALID_ARG, "qtn_arith_check: bad argument");
  int dev = 0, major = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (packed) *packed = major >= 10 ? 1 : 0;
  const size_t in = (size_t)count * K * sizeof(double2), out = (size_t)count * sizeof(double2);
  double2 *d_a = nullptr, *d_b = nullptr, *d_s = nullptr, *d_m = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&d_a, in + 16);
  if (e == cudaSuccess) e = cudaMalloc(&d_b, in + 16);
  if (e == cudaSuccess) e = cudaMalloc(&d_s, out + 16);
  if (e == cudaSuccess) e = cudaMalloc(&d_m, out + 16);
  if (e == cudaSuccess) e = cudaMemcpy(d_a, a, in, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_b, b, in, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = qtn::launch_arith_check(d_a, d_b, count, K, d_s, d_m, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(out_scalar, d_s, out, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(out_merge, d_m, out, cudaMemcpyDeviceToHost);
  cudaFree(d_a);
  cudaFree(d_b);
  cudaFree(d_s);
  cudaFree(d_m);
  if (e != cudaSuccess) return set_error(QTN_ERR_CUDA, std::string("qtn_arith_check: ") + cudaGetErrorString(e));
  return QTN_OK;
}
