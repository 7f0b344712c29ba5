// Complex arithmetic of the contraction kernels and the compensated FP64
// sums of slice results.  Compiled in two ways: included by kernels.cu (inside
// its namespace) and embedded as source text in the kernels the library
// generates per plan at run time (NVRTC), so both run the same arithmetic.
// It therefore includes nothing and uses only built-in CUDA types; a
// `Partial` type with fields re, im, cre, cim and a static make() must be
// declared before it.
template <class V>
struct CplxOps;
template <>
struct CplxOps<float2> {
  using R = float;
  static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ void fma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
  }
  static __device__ __forceinline__ float2 mul(float2 a, float2 b) {
    float2 r = zero();
    fma(r, a, b);
    return r;
  }
  static __device__ __forceinline__ void finish(float2&) {}
  typedef float2 Acc;  // accumulator of a multiply-add chain: the value itself
  static __device__ __forceinline__ float2 result(float2 v) { return v; }
  static __device__ __forceinline__ float2 from(double re, double im) {
    return make_float2((float)re, (float)im);
  }
  static __device__ __forceinline__ double re(float2 v) { return (double)v.x; }
  static __device__ __forceinline__ double im(float2 v) { return (double)v.y; }
};
template <>
struct CplxOps<double2> {
  using R = double;
  static __device__ __forceinline__ double2 zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ void fma(double2& acc, double2 a, double2 b) {
    acc.x = ::fma(a.x, b.x, acc.x);
    acc.x = ::fma(-a.y, b.y, acc.x);
    acc.y = ::fma(a.x, b.y, acc.y);
    acc.y = ::fma(a.y, b.x, acc.y);
  }
  static __device__ __forceinline__ double2 mul(double2 a, double2 b) {
    double2 r = zero();
    fma(r, a, b);
    return r;
  }
  static __device__ __forceinline__ void finish(double2&) {}
  typedef double2 Acc;  // accumulator of a multiply-add chain: the value itself
  static __device__ __forceinline__ double2 result(double2 v) { return v; }
  static __device__ __forceinline__ double2 from(double re, double im) { return make_double2(re, im); }
  static __device__ __forceinline__ double re(double2 v) { return v.x; }
  static __device__ __forceinline__ double im(double2 v) { return v.y; }
};

// ---------------------------------------------------- double-float (FP32X2) --

// A complex number as two double-word floats (value = hi + lo per part).
// Layout: the two high parts first (a packed pair), then the two low parts.
struct __align__(16) dfc {
  float rh, ih, rl, il;
};

// Error-free transform TwoSum (Knuth: s + e = a + b exactly).  The _rn
// intrinsics keep the compiler from contracting them into FMAs, which would
// break exactness.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// Double-word product (xh + xl)(yh + yl) as ph + pl: ph = fl(xh yh), and pl
// = its exact rounding error (FMA) plus the cross terms (the xl yl term is
// below the format's precision).
__device__ __forceinline__ void dw_prod(float xh, float xl, float yh, float yl, float& ph, float& pl) {
  ph = __fmul_rn(xh, yh);
  pl = __fmaf_rn(xh, yh, -ph);
  pl = __fmaf_rn(xh, yl, pl);
  pl = __fmaf_rn(xl, yh, pl);
}
// (ah, al) += x * y with lazy normalisation: ah takes the TwoSum of the
// product's high part, al collects that sum's exact error and the product's
// low part in plain FP32 (a second-order quantity, so its own roundings stay
// below the double-word precision); finish() renormalises once per output
// instead of once per product.
__device__ __forceinline__ void dw_fma_lazy(float& ah, float& al, float xh, float xl, float yh, float yl) {
  float ph, pl, sh, e;
  dw_prod(xh, xl, yh, yl, ph, pl);
  two_sum(ah, ph, sh, e);
  ah = sh;
  al = __fadd_rn(al, __fadd_rn(e, pl));
}

template <>
struct CplxOps<dfc> {
  static __device__ __forceinline__ dfc zero() { return dfc{0.f, 0.f, 0.f, 0.f}; }
  static __device__ __forceinline__ void fma(dfc& acc, dfc a, dfc b) {
    dw_fma_lazy(acc.rh, acc.rl, a.rh, a.rl, b.rh, b.rl);
    dw_fma_lazy(acc.rh, acc.rl, -a.ih, -a.il, b.ih, b.il);
    dw_fma_lazy(acc.ih, acc.il, a.rh, a.rl, b.ih, b.il);
    dw_fma_lazy(acc.ih, acc.il, a.ih, a.il, b.rh, b.rl);
  }
  // a * b: the first product of each part needs no sum.
  static __device__ __forceinline__ dfc mul(dfc a, dfc b) {
    dfc r;
    dw_prod(a.rh, a.rl, b.rh, b.rl, r.rh, r.rl);
    dw_fma_lazy(r.rh, r.rl, -a.ih, -a.il, b.ih, b.il);
    dw_prod(a.rh, a.rl, b.ih, b.il, r.ih, r.il);
    dw_fma_lazy(r.ih, r.il, a.ih, a.il, b.rh, b.rl);
    return r;
  }
  // Renormalise each part to a double word (|lo| <= ulp(hi) / 2).
  static __device__ __forceinline__ void finish(dfc& v) {
    two_sum(v.rh, v.rl, v.rh, v.rl);
    two_sum(v.ih, v.il, v.ih, v.il);
  }
  typedef dfc Acc;
  static __device__ __forceinline__ dfc result(dfc v) {
    finish(v);
    return v;
  }
  static __device__ __forceinline__ dfc from(double re, double im) {
    const float rh = (float)re, ih = (float)im;
    return dfc{rh, ih, (float)(re - (double)rh), (float)(im - (double)ih)};
  }
  static __device__ __forceinline__ double re(dfc v) { return (double)v.rh + (double)v.rl; }
  static __device__ __forceinline__ double im(dfc v) { return (double)v.ih + (double)v.il; }
};

#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
// The same double-float complex multiply-add on packed FP32 pairs (sm_100
// and later: one add/sub/mul/fma .f32x2 instruction computes two lanes, each
// rounded to nearest exactly as the scalar instruction rounds it).  A pair
// lives in a 64-bit register: the first lane in the low word.
typedef unsigned long long x2;
__device__ __forceinline__ x2 x2_pack(float lo, float hi) {
  x2 d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void x2_unpack(x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ x2 x2_swap(x2 v) {
  float lo, hi;
  x2_unpack(v, lo, hi);
  return x2_pack(hi, lo);
}
__device__ __forceinline__ x2 x2_add(x2 a, x2 b) {
  x2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// a - b as the FMA b * (-1) + a (the product is exact, so this is a - b
// rounded once).  The packed subtract instruction is not used: in longer
// sequences built with it the error-free transforms below lost their
// exactness (results differed from the scalar sequence), while this form
// matches the scalar sequence bit for bit.
__device__ __forceinline__ x2 x2_sub(x2 a, x2 b) {
  x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(b), "l"(0xbf800000bf800000ull), "l"(a));
  return d;
}
__device__ __forceinline__ x2 x2_mul(x2 a, x2 b) {
  x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ x2 x2_fma(x2 a, x2 b, x2 c) {
  x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// TwoSum on each lane (s + e = a + b exactly).
__device__ __forceinline__ void two_sum2(x2 a, x2 b, x2& s, x2& e) {
  s = x2_add(a, b);
  const x2 bb = x2_sub(s, a);
  e = x2_add(x2_sub(a, x2_sub(s, bb)), x2_sub(b, bb));
}
// dw_prod on each lane.
__device__ __forceinline__ void dw_prod2(x2 xh, x2 xl, x2 yh, x2 yl, x2& ph, x2& pl) {
  ph = x2_mul(xh, yh);
  pl = x2_fma(xh, yh, x2_fma(ph, 0xbf800000bf800000ull, 0x8000000080000000ull));  // -ph exactly
  pl = x2_fma(xh, yl, pl);
  pl = x2_fma(xl, yh, pl);
}
// dw_fma_lazy on each lane.
__device__ __forceinline__ void dw_fma_lazy2(x2& ah, x2& al, x2 xh, x2 xl, x2 yh, x2 yl) {
  x2 ph, pl, sh, e;
  dw_prod2(xh, xl, yh, yl, ph, pl);
  two_sum2(ah, ph, sh, e);
  ah = sh;
  al = x2_add(al, x2_add(e, pl));
}
// The same with the negated broadcast factor nyh = -yh supplied (built once
// per B element and shared by the outputs that use it): the product is formed
// negated, so its exact error is one FMA and the TwoSum subtracts it, one
// packed operation fewer than dw_fma_lazy2.
__device__ __forceinline__ void dw_fma_lazy2n(x2& ah, x2& al, x2 xh, x2 xl, x2 yh, x2 nyh, x2 yl) {
  const x2 nph = x2_mul(xh, nyh);  // -(xh yh), rounded
  x2 pl = x2_fma(xh, yh, nph);     // its exact rounding error
  pl = x2_fma(xh, yl, pl);
  pl = x2_fma(xl, yh, pl);
  const x2 s = x2_sub(ah, nph);    // TwoSum(ah, -nph)
  const x2 bb = x2_sub(s, ah);
  const x2 e = x2_sub(x2_sub(ah, x2_sub(s, bb)), x2_add(nph, bb));
  ah = s;
  al = x2_add(al, x2_add(e, pl));
}
// The accumulator holds two double-word pairs: (h1, l1) collects the
// products a.r b.r and a.i b.r (lanes: re, im), (h2, l2) collects a.r b.i and
// -a.i b.i (lanes: im, re).  Every product takes the operand A as stored
// (high pair, low pair) and only B is broadcast into pairs; the two
// accumulators are added once per output.
struct DfcX2Acc {
  x2 h1, l1, h2, l2;
};
struct CplxOpsX2 {
  typedef DfcX2Acc Acc;
  static __device__ __forceinline__ Acc mul(dfc a, dfc b) {
    const x2 ah = x2_pack(a.rh, a.ih), al = x2_pack(a.rl, a.il);
    Acc r;
    dw_prod2(ah, al, x2_pack(b.rh, b.rh), x2_pack(b.rl, b.rl), r.h1, r.l1);
    dw_prod2(ah, al, x2_pack(b.ih, -b.ih), x2_pack(b.il, -b.il), r.h2, r.l2);
    return r;
  }
  static __device__ __forceinline__ void fma(Acc& acc, dfc a, dfc b) {
    const x2 ah = x2_pack(a.rh, a.ih), al = x2_pack(a.rl, a.il);
    dw_fma_lazy2n(acc.h1, acc.l1, ah, al, x2_pack(b.rh, b.rh), x2_pack(-b.rh, -b.rh), x2_pack(b.rl, b.rl));
    dw_fma_lazy2n(acc.h2, acc.l2, ah, al, x2_pack(b.ih, -b.ih), x2_pack(-b.ih, b.ih), x2_pack(b.il, -b.il));
  }
  // (re, im) as a high pair and an unnormalised low pair.
  static __device__ __forceinline__ void sum(const Acc& a, x2& h, x2& l) {
    x2 e;
    two_sum2(a.h1, x2_swap(a.h2), h, e);
    l = x2_add(x2_add(a.l1, x2_swap(a.l2)), e);
  }
  static __device__ __forceinline__ dfc result(const Acc& a) {
    x2 h, l, s, e;
    sum(a, h, l);
    two_sum2(h, l, s, e);
    dfc r;
    x2_unpack(s, r.rh, r.ih);
    x2_unpack(e, r.rl, r.il);
    return r;
  }
};
#endif

// The arithmetic the merge loops run for element ops `Ops`: the packed
// double-float form where the device has packed FP32 pairs, else `Ops`
// itself (its accumulator is the value).
template <class Ops>
struct MergeOps {
  typedef Ops type;
};
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
template <>
struct MergeOps<CplxOps<dfc>> {
  typedef CplxOpsX2 type;
};
#endif


__device__ __forceinline__ void kahan_add(double& sum, double& comp, double v) {
  double y = v - comp;
  double t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

// Sum of two compensated partials (value = sum - compensation): the sums are
// added with TwoSum and the rounding error joins the compensations.
__device__ __forceinline__ double two_sum_d(double a, double b, double& err) {
  const double s = a + b;
  const double bb = s - a;
  err = (a - (s - bb)) + (b - bb);
  return s;
}
__device__ __forceinline__ Partial combine(const Partial& x, const Partial& y) {
  double er, ei;
  const double sr = two_sum_d(x.re, y.re, er);
  const double si = two_sum_d(x.im, y.im, ei);
  return Partial::make(sr, si, x.cre + y.cre - er, x.cim + y.cim - ei);
}

// Fixed-order pairwise reduction of `n` partials in shared memory (n a power
// of two, all threads of the block call it); the result is in red[0].
__device__ __forceinline__ void tree_reduce(Partial* red, int n) {
  for (int w = n / 2; w > 0; w >>= 1) {
    __syncthreads();
    for (int t = threadIdx.x; t < w; t += blockDim.x) red[t] = combine(red[t], red[t + w]);
  }
  __syncthreads();
}

