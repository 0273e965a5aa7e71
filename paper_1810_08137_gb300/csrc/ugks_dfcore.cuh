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
// From FP64 (set-up and per-cell constants only: FP64 conversions run on the FP64 pipe)
__device__ __forceinline__ df df_of(double a) {
  const float h = __double2float_rn(a);
  return {h, __double2float_rn(a - (double)h)};
}
__device__ __forceinline__ double to_double(df a) { return (double)a.hi + (double)a.lo; }

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
  // from FP64: the nearest FP32 and the FP32 nearest to the remainder (conversions run on
  // the FP64 pipe: inputs and constants only)
  __device__ __forceinline__ dd(double a) : hi((float)a), lo((float)(a - (double)(float)a)) {}
  __device__ __forceinline__ explicit dd(int n) : hi((float)n), lo(0.f) {}
};
__device__ __forceinline__ df as_df(dd a) { return {a.hi, a.lo}; }
__device__ __forceinline__ dd as_dd(df a) { return dd(a.hi, a.lo); }
__device__ __forceinline__ dd operator+(dd a, dd b) { return as_dd(df_add(as_df(a), as_df(b))); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return as_dd(df_sub(as_df(a), as_df(b))); }
__device__ __forceinline__ dd operator*(dd a, dd b) { return as_dd(df_mul(as_df(a), as_df(b))); }
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ double to_double(dd a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double to_double(double a) { return a; }
// nearest FP32 (the high part of a normalised pair)
__device__ __forceinline__ float to_float(dd a) { return a.hi; }
__device__ __forceinline__ float to_float(double a) { return (float)a; }

}  // namespace ugks
