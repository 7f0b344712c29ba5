// Tensor-core product numerics emulated on the FP32 pipe.  Included inside
// the kernels' namespace after arith.cuh (needs cuda_bf16.h and stdint).

// Products of operands rounded as the tensor cores see them, accumulated in
// FP32: TF32 (10-bit significand), split BF16 / TF32 in 2 pieces with the
// 3 leading products, split BF16 in 3 pieces with the 6 leading products.
enum class Round { TF32, BF16X3, TF32X3, BF16X6 };

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ float to_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

template <Round R>
struct RoundOps {
  static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
  // acc + x * y for real x, y under the rounding mode.
  static __device__ __forceinline__ float mul_add(float acc, float x, float y) {
    if (R == Round::TF32) return __fmaf_rn(to_tf32(x), to_tf32(y), acc);
    if (R == Round::BF16X3 || R == Round::TF32X3) {
      const float xh = R == Round::BF16X3 ? to_bf16(x) : to_tf32(x);
      const float yh = R == Round::BF16X3 ? to_bf16(y) : to_tf32(y);
      const float xl = R == Round::BF16X3 ? to_bf16(x - xh) : to_tf32(x - xh);
      const float yl = R == Round::BF16X3 ? to_bf16(y - yh) : to_tf32(y - yh);
      acc = __fmaf_rn(xl, yh, acc);
      acc = __fmaf_rn(xh, yl, acc);
      return __fmaf_rn(xh, yh, acc);
    }
    const float x0 = to_bf16(x), x1 = to_bf16(x - x0), x2 = to_bf16(x - x0 - x1);
    const float y0 = to_bf16(y), y1 = to_bf16(y - y0), y2 = to_bf16(y - y0 - y1);
    acc = __fmaf_rn(x0, y2, acc);
    acc = __fmaf_rn(x1, y1, acc);
    acc = __fmaf_rn(x2, y0, acc);
    acc = __fmaf_rn(x0, y1, acc);
    acc = __fmaf_rn(x1, y0, acc);
    return __fmaf_rn(x0, y0, acc);
  }
  static __device__ __forceinline__ void fma(float2& acc, float2 a, float2 b) {
    acc.x = mul_add(acc.x, a.x, b.x);
    acc.x = mul_add(acc.x, -a.y, b.y);
    acc.y = mul_add(acc.y, a.x, b.y);
    acc.y = mul_add(acc.y, a.y, b.x);
  }
  static __device__ __forceinline__ float2 mul(float2 a, float2 b) {
    float2 r = zero();
    fma(r, a, b);
    return r;
  }
  static __device__ __forceinline__ void finish(float2&) {}
  typedef float2 Acc;
  static __device__ __forceinline__ float2 result(float2 v) { return v; }
  static __device__ __forceinline__ double re(float2 v) { return (double)v.x; }
  static __device__ __forceinline__ double im(float2 v) { return (double)v.y; }
};

