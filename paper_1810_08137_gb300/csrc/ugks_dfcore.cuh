// Scalar double-FP32 numbers: the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, about 48 significand bits, computed on the FP32 pipe (GB300
// executes FP64 at 1/64 of the FP32 rate).  Built from error-free transformations:
//   two_sum       s + e = a + b exactly, s = fl(a + b) (Knuth, TAOCP vol. 2, Sec. 4.2.2)
//   fast_two_sum  the same when |a| >= |b| or a = 0 (Dekker 1971)
//   two_prod      p + e = a b exactly, p = fl(a b), e from one fused multiply-add
// The sums and products round like the "sloppy" double-float operations: relative error a
// few 2^-48 for products and for sums of like-signed terms; a sum of nearly cancelling terms
// is exact in its high parts and carries an absolute error of a few 2^-48 of its operands.
// Every operation uses explicitly rounded intrinsics, so the compiler cannot fuse or reorder
// them.  `df` is the plain pair the DF64 form's kernels use; `dd` wraps it with arithmetic
// operators so that the interface templates (written for a type T) run on it unchanged.
#pragma once

namespace ugks {

struct df {
  float hi, lo;
};

// ---- conversions between FP64 and pairs with the FP32 part on the integer pipe ----
// (a conversion instruction between FP64 and FP32 runs on the 1/64-rate FP64 pipe; the
// interface kernels convert tens of values per face).  IEEE-754 binary64 and binary32 differ
// in exponent bias by 1023 - 127 = 896 and in significand width by 52 - 23 = 29 bits.
// a with its significand cut to FP32 width (toward zero), as FP64 and as FP32; both 0 when |a|
// is below the FP32 normal range (|a| < 2^-126).  |a| >= 2^128 (beyond FP32, infinities,
// NaN) gives an FP32 NaN and cd = a, so that a non-finite input stays non-finite.
__device__ __forceinline__ void f32_cut(double a, double& cd, float& cf) {
  const long long b = __double_as_longlong(a);
  const unsigned hw = (unsigned)((unsigned long long)b >> 32), lw = (unsigned)b;
  const unsigned m = hw & 0x7fffffffu, sg = hw & 0x80000000u;
  const bool normal = m >= 0x38100000u;  // biased FP64 exponent >= 897: FP32 exponent >= 1
  const bool big = m >= 0x47f00000u;     // biased FP64 exponent >= 1151: FP32 exponent >= 255
  const unsigned fb = sg | ((m - 0x38000000u) << 3) | (lw >> 29);
  cf = big ? __uint_as_float(sg | 0x7fc00000u) : (normal ? __uint_as_float(fb) : 0.f);
  cd = big ? a : (normal ? __longlong_as_double(b & ~0x1fffffffLL) : 0.0);
}
// FP64 value of an FP32 number (exact); 0 for zero and FP32 subnormals (flushed, as the
// FP32 arithmetic here flushes them), infinities and NaN kept non-finite
__device__ __forceinline__ double f64_of(float x) {
  const unsigned u = __float_as_uint(x), m = u & 0x7fffffffu, sg = u & 0x80000000u;
  const bool big = m >= 0x7f800000u;
  const unsigned hw = big ? (sg | (m > 0x7f800000u ? 0x7ff80000u : 0x7ff00000u))
                          : (sg | ((m >> 3) + 0x38000000u));
  const unsigned lw = big ? 0u : (m << 29);
  return m >= 0x00800000u ? __hiloint2double((int)hw, (int)lw) : 0.0;
}
// FP64 -> FP32 rounded to nearest (ties to even) on the integer pipe: the binary64
// significand rounded at its bit 29 (round bit 28, sticky bits 0..27), the exponent rebiased
// by 896 (a carry out of the significand increments the exponent, as rounding requires).
// Equal to the conversion instruction for results in the FP32 normal range; below it the
// result is a signed zero, above it (and for infinities) the signed infinity; NaN stays NaN.
__device__ __forceinline__ float f32_rn(double a) {
  const long long b = __double_as_longlong(a);
  const unsigned hw = (unsigned)((unsigned long long)b >> 32), lw = (unsigned)b;
  const unsigned m = hw & 0x7fffffffu, sg = hw & 0x80000000u;
  const unsigned up = ((lw & 0x10000000u) != 0u && (lw & 0x2fffffffu) != 0u) ? 1u : 0u;
  const unsigned rb = (((m - 0x38000000u) << 3) | (lw >> 29)) + up;
  const bool normal = m >= 0x38100000u, fin = m < 0x47f00000u;
  const bool nan = m > 0x7ff00000u || (m == 0x7ff00000u && lw != 0u);
  return __uint_as_float(fin ? (normal ? sg | rb : sg) : (sg | (nan ? 0x7fc00000u : 0x7f800000u)));
}
// FP64 -> normalised pair: the cut high part, the remainder rounded to FP32, renormalised
// (|lo| <= ulp(hi) / 2); |a - (hi + lo)| is a few 2^-48 |a|.  The remainder a - cut(a) is
// +-(the 29 low significand bits) 2^(E - 1075) (E the biased exponent): its FP32 rounding is
// formed without the FP64 pipe, the 29-bit integer rounded to 24 bits by one FMA of its two
// exact FP32 pieces (23 and 6 bits, each read off the bits of 2^23 + n) and then scaled by
// powers of two.  For |a| < 2^-103 (E < 920, where that scale leaves the FP32 normal range) the
// remainder is dropped: such values keep 24 bits (they only arise next to terms of order one).
__device__ __forceinline__ void split_f64(double a, float& hi, float& lo) {
  double cd;
  float cf;
  f32_cut(a, cd, cf);
  const long long b = __double_as_longlong(a);
  const unsigned hw = (unsigned)((unsigned long long)b >> 32), lw = (unsigned)b;
  const unsigned m = hw & 0x7fffffffu, sg = hw & 0x80000000u, E = m >> 20;
  const unsigned ml = lw & 0x1fffffffu;
  const float na = __fsub_rn(__uint_as_float(0x4b000000u | (ml >> 23)), 8388608.f);
  const float nb = __fsub_rn(__uint_as_float(0x4b000000u | (ml & 0x7fffffu)), 8388608.f);
  const float v = __fmaf_rn(na, 8388608.f, nb);  // ml rounded to 24 bits
  const bool scaled = E >= 920u && m < 0x47f00000u;
  const float sc = __uint_as_float(sg | ((scaled ? E - 919u : 1u) << 23));  // +-2^(E - 1046)
  const float r = scaled ? __fmul_rn(__fmul_rn(v, 0x1p-29f), sc) : 0.f;
  const float s = __fadd_rn(cf, r);
  hi = s;
  lo = __fsub_rn(r, __fsub_rn(s, cf));
}

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_of(float a) { return {a, 0.f}; }
// From FP64 (set-up and per-cell constants)
__device__ __forceinline__ df df_of(double a) {
  df r;
  split_f64(a, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ double to_double(df a) { return f64_of(a.hi) + f64_of(a.lo); }

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_mul(df a, df b) {
  const df p = two_prod(a.hi, b.hi);
  const float e = __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.lo, p.lo));
  return fast_two_sum(p.hi, e);
}
__device__ __forceinline__ df df_mul(df a, float b) {
  const df p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
// a b + c
__device__ __forceinline__ df df_fma(df a, df b, df c) {
  const df p = two_prod(a.hi, b.hi);
  const float pl = __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.lo, p.lo));
  const df s = two_sum(c.hi, p.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(c.lo, pl)));
}

// Double-FP32 number with arithmetic operators (the interface templates' T).
struct dd {
  float hi, lo;
  dd() = default;
  __device__ __forceinline__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  // from FP64 (split_f64: one FP64 subtraction and one conversion, the rest on the integer
  // and FP32 pipes)
  __device__ __forceinline__ dd(double a) { split_f64(a, hi, lo); }
  __device__ __forceinline__ explicit dd(int n) : hi((float)n), lo(0.f) {}
};
__device__ __forceinline__ df as_df(dd a) { return {a.hi, a.lo}; }
__device__ __forceinline__ dd as_dd(df a) { return dd(a.hi, a.lo); }
__device__ __forceinline__ dd operator+(dd a, dd b) { return as_dd(df_add(as_df(a), as_df(b))); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return as_dd(df_sub(as_df(a), as_df(b))); }
__device__ __forceinline__ dd operator*(dd a, dd b) { return as_dd(df_mul(as_df(a), as_df(b))); }
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ double to_double(dd a) { return f64_of(a.hi) + f64_of(a.lo); }
__device__ __forceinline__ double to_double(double a) { return a; }
// nearest FP32 (the high part of a normalised pair)
__device__ __forceinline__ float to_float(dd a) { return a.hi; }
__device__ __forceinline__ float to_float(double a) { return (float)a; }

}  // namespace ugks
