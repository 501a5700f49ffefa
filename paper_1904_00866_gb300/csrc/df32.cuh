// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers (about 48 significant bits), for the few nodes whose FP32
// entropy decision is not certified.  GB300 runs FP64 at a small fraction
// of its FP32 rate, so extended precision is cheaper here as pairs of FP32
// operations than as FP64.
//
// Building blocks (round-to-nearest, no contraction: every operation is an
// explicit *_rn intrinsic, so the compiler neither fuses nor reorders):
//   TwoSum (Moller 1965; Knuth, TAOCP vol. 2): s + e = a + b exactly;
//   FastTwoSum (Dekker 1971): the same in 3 operations when a = 0 or
//     exponent(a) >= exponent(b);
//   TwoProd with a fused multiply-add: p + e = a b exactly.
// The compound operations are the classical double-word sums and products
// (Dekker 1971; Hida, Li & Bailey 2001) with FP32 parts.  With u = 2^-24 and
// |lo| <= u |hi| on the inputs, their absolute errors are below
// 8 u^2 (|a| + |b|) for a sum and 8 u^2 |a b| for a product (generous
// versions of the published bounds, which also cover a FastTwoSum whose
// ordering condition fails after cancellation).
//
// Every helper exists for float and for float2 (two independent lanes in
// packed f32x2 instructions, each lane rounded like the scalar operation).
#pragma once

namespace elbm {

__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma_(float a, float b, float c) {
  return __fmaf_rn(a, b, c);
}
__device__ __forceinline__ float neg_(float a) { return -a; }
__device__ __forceinline__ float2 add_(float2 a, float2 b) {
  return __fadd2_rn(a, b);
}
__device__ __forceinline__ float2 sub_(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);   // a - b, one rounding
}
__device__ __forceinline__ float2 mul_(float2 a, float2 b) {
  return __fmul2_rn(a, b);
}
__device__ __forceinline__ float2 fma_(float2 a, float2 b, float2 c) {
  return __ffma2_rn(a, b, c);
}
__device__ __forceinline__ float2 neg_(float2 a) {
  return make_float2(-a.x, -a.y);
}

template <class T>
struct DF {
  T hi, lo;
};

template <class T>
__device__ __forceinline__ DF<T> two_sum(T a, T b) {
  const T s = add_(a, b);
  const T bb = sub_(s, a);
  return {s, add_(sub_(a, sub_(s, bb)), sub_(b, bb))};
}

template <class T>
__device__ __forceinline__ DF<T> fast_two_sum(T a, T b) {
  const T s = add_(a, b);
  return {s, sub_(b, sub_(s, a))};
}

template <class T>
__device__ __forceinline__ DF<T> two_prod(T a, T b) {
  const T p = mul_(a, b);
  return {p, fma_(a, b, neg_(p))};
}

template <class T>
__device__ __forceinline__ DF<T> df_add(DF<T> a, DF<T> b) {
  const DF<T> s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, add_(s.lo, add_(a.lo, b.lo)));
}

template <class T>
__device__ __forceinline__ DF<T> df_add(DF<T> a, T b) {
  const DF<T> s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, add_(s.lo, a.lo));
}

template <class T>
__device__ __forceinline__ DF<T> df_mul(DF<T> a, DF<T> b) {
  const DF<T> p = two_prod(a.hi, b.hi);
  return fast_two_sum(p.hi, fma_(a.hi, b.lo, fma_(a.lo, b.hi, p.lo)));
}

template <class T>
__device__ __forceinline__ DF<T> df_mul(DF<T> a, T b) {
  const DF<T> p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, fma_(a.lo, b, p.lo));
}

// a / b with b > 0 normal: q1 from the approximate reciprocal (relative
// error below 2^-22), the residual a - q1 b in double-float (TwoProd exact),
// then the correction q2 = residual / b.hi; relative error below 2^-44 for
// |lo| <= u |hi| on both inputs.
__device__ __forceinline__ float rcp_df_(float y) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
  return r;
}
__device__ __forceinline__ float2 rcp_df_(float2 y) {
  return make_float2(rcp_df_(y.x), rcp_df_(y.y));
}
template <class T>
__device__ __forceinline__ DF<T> df_div(DF<T> a, DF<T> b) {
  const T rb = rcp_df_(b.hi);
  const T q1 = mul_(a.hi, rb);
  const DF<T> p = two_prod(q1, b.hi);
  // residual a - q1 b = (a.hi - p.hi) - p.lo + a.lo - q1 b.lo
  const T res = sub_(add_(sub_(sub_(a.hi, p.hi), p.lo), a.lo), mul_(q1, b.lo));
  return fast_two_sum(q1, mul_(res, rb));
}

template <class T>
__device__ __forceinline__ DF<T> df_neg(DF<T> a) {
  return {neg_(a.hi), neg_(a.lo)};
}

// both lanes of a packed double-float from scalar double-floats
__device__ __forceinline__ DF<float2> df_pair(DF<float> a, DF<float> b) {
  return {make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)};
}
__device__ __forceinline__ DF<float2> df_bcast(DF<float> a) {
  return df_pair(a, a);
}

// Double-float constant nearest to a double (hi = fl(v), lo = fl(v - hi)).
__host__ __device__ constexpr float df_hi(double v) { return (float)v; }
__host__ __device__ constexpr float df_lo(double v) {
  return (float)(v - (double)(float)v);
}

}  // namespace elbm
