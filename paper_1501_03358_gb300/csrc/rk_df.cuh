// Double-float ("DF") arithmetic for the projection and orthogonalisation
// kernels: a value is an unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2 (about 48 significant bits), and products and sums are
// carried with error-free transformations on the FP32 pipe:
//   TwoProduct(a, b): p = a*b, e = fma(a, b, -p)     (exact: a*b = p + e)
//   TwoSum(a, b):     s = a+b, the rounding error of s recovered with 4 adds
//   FastTwoSum(a, b): the same when |a| >= |b| (2 adds)
// (Dekker 1971; Knuth TAOCP vol. 2; Hida, Li, Bailey 2001 "double-double").
// GB300 runs FP32 FMAs ~58x faster than FP64 FMAs, so one DF multiply-add
// (~15 FP32 operations) costs about a quarter of an FP64 one and the
// streaming kernels become memory-bound instead of FP64-bound.
#pragma once
#include <cuda_runtime.h>

namespace rk {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_from_double(double d) {
  const float h = __double2float_rn(d);
  const float l = __double2float_rn(d - (double)h);
  return {h, l};
}

__device__ __forceinline__ double df_to_double(float2 v) { return (double)v.x + (double)v.y; }
__device__ __forceinline__ double df_to_double(df v) { return (double)v.hi + (double)v.lo; }

__device__ __forceinline__ float2 df_pack(df v) { return make_float2(v.hi, v.lo); }

// Fast2Sum with |a| >= |b| assumed
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

// Accumulator (sh, sl) += (p + e) where p + e is an (unnormalised) pair;
// TwoSum on the leading parts, then renormalise.
__device__ __forceinline__ void df_acc(float& sh, float& sl, float p, float e) {
  const float s = __fadd_rn(sh, p);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  const float t = __fadd_rn(sl, __fadd_rn(err, e));
  const float s2 = __fadd_rn(s, t);
  sl = __fsub_rn(t, __fsub_rn(s2, s));
  sh = s2;
}

// Product of two DF numbers as an unnormalised pair (p, e): the low x low
// term (relative size 2^-48) is dropped.
__device__ __forceinline__ void df_mul_pair(float ah, float al, float bh, float bl, float& p, float& e) {
  p = __fmul_rn(ah, bh);
  float t = __fmaf_rn(ah, bh, -p);
  t = __fmaf_rn(ah, bl, t);
  e = __fmaf_rn(al, bh, t);
}

// s += a * b for DF a, b
__device__ __forceinline__ void df_mac(float& sh, float& sl, float ah, float al, float bh, float bl) {
  float p, e;
  df_mul_pair(ah, al, bh, bl, p, e);
  df_acc(sh, sl, p, e);
}

// On GB300 every FP64<->FP32 conversion issues at the FP64 rate (about 2 per
// clock per SM, like a DFMA), so the kernels below convert O(1) times per
// element at most and keep their inner loops in FP32 operations.

// a + b for DF a, b, normalised
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bb = __fsub_rn(s, a.x);
  float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  const float h = __fadd_rn(s, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

// a * b for DF a, b, normalised
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  float p, e;
  df_mul_pair(a.x, a.y, b.x, b.y, p, e);
  const float h = __fadd_rn(p, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, p)));
}

// Warp sum of DF values (xor tree; every lane gets the result)
__device__ __forceinline__ float2 df_warp_sum(float2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float2 w;
    w.x = __shfl_xor_sync(0xffffffffu, v.x, o);
    w.y = __shfl_xor_sync(0xffffffffu, v.y, o);
    v = df_add(v, w);
  }
  return v;
}

// ---- scalar double-float helpers for the small dense eigenproblem ----

__device__ __forceinline__ float2 df_make(double d) {
  const df v = df_from_double(d);
  return make_float2(v.hi, v.lo);
}

__device__ __forceinline__ float2 df_sub(float2 a, float2 b) { return df_add(a, df_neg(b)); }

// c + a * b, normalised
__device__ __forceinline__ float2 df_fma(float2 a, float2 b, float2 c) {
  float sh = c.x, sl = c.y;
  df_mac(sh, sl, a.x, a.y, b.x, b.y);
  return make_float2(sh, sl);
}

// a / b (three-term long division: q1 + q2 + q3, each from the FP32
// quotient of the current remainder)
__device__ __forceinline__ float2 df_div(float2 a, float2 b) {
  const float q1 = __fdiv_rn(a.x, b.x);
  float2 r = df_fma(make_float2(-q1, 0.f), b, a);
  const float q2 = __fdiv_rn(r.x, b.x);
  r = df_fma(make_float2(-q2, 0.f), b, r);
  const float q3 = __fdiv_rn(r.x, b.x);
  const df s = df_fast_two_sum(q1, q2);
  return df_add(make_float2(s.hi, s.lo), make_float2(q3, 0.f));
}

// sqrt(a) for a >= 0: FP32 root, then one Newton correction in DF
__device__ __forceinline__ float2 df_sqrt(float2 a) {
  if (!(a.x > 0.f)) return make_float2(0.f, 0.f);
  const float s = __fsqrt_rn(a.x);
  const float2 e = df_fma(make_float2(-s, 0.f), make_float2(s, 0.f), a);  // a - s^2
  const float t = __fdiv_rn(e.x, 2.f * s);
  const df r = df_fast_two_sum(s, t);
  return make_float2(r.hi, r.lo);
}

__device__ __forceinline__ float2 df_absv(float2 a) { return a.x < 0.f ? df_neg(a) : a; }

// Faster variants for scalar chains whose operands are scaled near 1 (the
// small eigenproblem): the FP32 seeds come from the approximate reciprocal
// and square root (a few ulp); the double-float remainder steps that follow
// correct any seed error of that size, so the results keep ~2^-46 accuracy.
__device__ __forceinline__ float2 df_div_fast(float2 a, float2 b) {
  const float r = __fdividef(1.f, b.x);
  const float q1 = a.x * r;
  float2 rem = df_fma(make_float2(-q1, 0.f), b, a);
  const float q2 = rem.x * r;
  rem = df_fma(make_float2(-q2, 0.f), b, rem);
  const float q3 = rem.x * r;
  const df s = df_fast_two_sum(q1, q2);
  return df_add(make_float2(s.hi, s.lo), make_float2(q3, 0.f));
}

__device__ __forceinline__ float2 df_sqrt_fast(float2 a) {
  if (!(a.x > 0.f)) return make_float2(0.f, 0.f);
  const float s = a.x * rsqrtf(a.x);
  float2 e = df_fma(make_float2(-s, 0.f), make_float2(s, 0.f), a);  // a - s^2
  const float t = e.x * __fdividef(0.5f, s);
  const df r = df_fast_two_sum(s, t);
  // one more correction: the seed is only a few ulp accurate
  const float2 r2 = make_float2(r.hi, r.lo);
  e = df_sub(a, df_mul(r2, r2));
  return df_add(r2, make_float2(e.x * __fdividef(0.5f, r.hi), 0.f));
}

// Exact FP32 <-> FP64 conversions by IEEE-754 bit manipulation on the integer
// pipe. On GB300 the hardware conversions issue at the FP64 rate (as slowly as
// a DFMA), which makes them a large share of an FP64 kernel that reads and
// writes double-float vectors. Normal numbers take the integer path; zeros,
// subnormals, infinities and NaNs fall back to the hardware conversion.
__device__ __forceinline__ double f32_to_f64_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e - 1u < 254u) {  // normal: widen the exponent bias, shift the mantissa
    const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                    ((unsigned long long)(e + 896u) << 52) |
                                    ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
  }
  return (double)f;
}

// Round to nearest, ties to even (the FP32 value nearest to d).
__device__ __forceinline__ float f64_to_f32_rn(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7ff) - 896;  // FP32 biased exponent
  if (e >= 1 && e <= 254) {
    const unsigned long long m = b & 0xfffffffffffffull;
    unsigned mant = (unsigned)(m >> 29);
    const unsigned rem = (unsigned)(m & 0x1fffffffu);
    const unsigned half = 0x10000000u;
    mant += (rem > half || (rem == half && (mant & 1u))) ? 1u : 0u;
    unsigned ex = (unsigned)e;
    if (mant == 0x800000u) {  // the rounding carried into the exponent
      mant = 0;
      ex += 1;
    }
    if (ex <= 254u) return __uint_as_float((unsigned)((b >> 32) & 0x80000000u) | (ex << 23) | mant);
  }
  return __double2float_rn(d);
}

// double-float <-> FP64 with the exact conversions above (the same values as
// df_to_double / df_from_double)
__device__ __forceinline__ double df_to_double_i(float2 v) {
  return f32_to_f64_exact(v.x) + f32_to_f64_exact(v.y);
}
__device__ __forceinline__ float2 df_from_double_i(double d) {
  const float h = f64_to_f32_rn(d);
  const float l = f64_to_f32_rn(d - f32_to_f64_exact(h));
  return make_float2(h, l);
}

// Lazy accumulation for short dense blocks (the recycle GEMM and Gram): the
// products' leading parts are added to s exactly (TwoSum) and every
// lower-order piece (TwoSum error, product error, cross terms) goes into the
// FP32 companion c; df_renorm folds c back into (s, c) as a normalised pair.
// Renormalising every 8 terms keeps |c| within a few ulp of s, so the error
// stays within a small constant of the renormalising df_mac (11 instead of
// 15 FP32 instructions per multiply-add).
__device__ __forceinline__ void df_mac_lazy(float& s, float& c, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  const float t = __fadd_rn(s, p);
  const float bb = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}
__device__ __forceinline__ void df_renorm(float& s, float& c) {
  const float t = __fadd_rn(s, c);
  c = __fsub_rn(c, __fsub_rn(t, s));
  s = t;
}

}  // namespace rk
