// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2.  Error-free transformations: the two-sum
// of Knuth (TAOCP vol. 2, §4.2.2), the fast two-sum of Dekker ("A
// floating-point technique for extending the available precision", 1971) for
// |a| >= |b|, and the two-product through a fused multiply-add.  Addition uses
// the accurate variant (both components two-summed); multiplication folds the
// cross terms into the FMA error term.  Complex values are float4
// (x = re.hi, y = re.lo, z = im.hi, w = im.lo).
#pragma once
#include <cuda_runtime.h>

namespace fde {
namespace df {

__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return make_float2(s, e);
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
  const float s = a + b;
  const float e = b - (s - a);
  return make_float2(s, e);
}
__device__ __forceinline__ float2 df_add(float2 x, float2 y) {
  float2 s = two_sum(x.x, y.x);
  const float2 t = two_sum(x.y, y.y);
  s.y += t.x;
  s = fast_two_sum(s.x, s.y);
  s.y += t.y;
  return fast_two_sum(s.x, s.y);
}
// Addition with a normwise bound only: one two-sum on the high parts, the
// low parts added plainly; |error| <= ~4 u^2 (|x| + |y|) (u = 2^-24) instead
// of a bound relative to |x + y|.  Enough where errors are measured against
// the norm of the operands, as in FFT butterflies (about half the operations
// of df_add).
__device__ __forceinline__ float2 df_add_nw(float2 x, float2 y) {
  const float2 s = two_sum(x.x, y.x);
  return fast_two_sum(s.x, s.y + (x.y + y.y));
}
__device__ __forceinline__ float2 df_neg(float2 x) { return make_float2(-x.x, -x.y); }
__device__ __forceinline__ float2 df_mul(float2 x, float2 y) {
  const float p = x.x * y.x;
  float e = fmaf(x.x, y.x, -p);
  e = fmaf(x.x, y.y, e);
  e = fmaf(x.y, y.x, e);
  return fast_two_sum(p, e);
}
// complex double-float: x = re.hi, y = re.lo, z = im.hi, w = im.lo
__device__ __forceinline__ float4 c_mul(float4 a, float4 b) {
  const float2 ar = make_float2(a.x, a.y), ai = make_float2(a.z, a.w);
  const float2 br = make_float2(b.x, b.y), bi = make_float2(b.z, b.w);
  const float2 re = df_add(df_mul(ar, br), df_neg(df_mul(ai, bi)));
  const float2 im = df_add(df_mul(ar, bi), df_mul(ai, br));
  return make_float4(re.x, re.y, im.x, im.y);
}
__device__ __forceinline__ float4 c_add(float4 a, float4 b) {
  const float2 re = df_add(make_float2(a.x, a.y), make_float2(b.x, b.y));
  const float2 im = df_add(make_float2(a.z, a.w), make_float2(b.z, b.w));
  return make_float4(re.x, re.y, im.x, im.y);
}
__device__ __forceinline__ float4 c_sub(float4 a, float4 b) {
  const float2 re = df_add(make_float2(a.x, a.y), make_float2(-b.x, -b.y));
  const float2 im = df_add(make_float2(a.z, a.w), make_float2(-b.z, -b.w));
  return make_float4(re.x, re.y, im.x, im.y);
}
__device__ __forceinline__ float4 c_conj(float4 a) { return make_float4(a.x, a.y, -a.z, -a.w); }
// the same complex operations with the normwise addition (FFT passes)
__device__ __forceinline__ float4 c_mul_nw(float4 a, float4 b) {
  const float2 ar = make_float2(a.x, a.y), ai = make_float2(a.z, a.w);
  const float2 br = make_float2(b.x, b.y), bi = make_float2(b.z, b.w);
  const float2 re = df_add_nw(df_mul(ar, br), df_neg(df_mul(ai, bi)));
  const float2 im = df_add_nw(df_mul(ar, bi), df_mul(ai, br));
  return make_float4(re.x, re.y, im.x, im.y);
}
__device__ __forceinline__ float4 c_add_nw(float4 a, float4 b) {
  const float2 re = df_add_nw(make_float2(a.x, a.y), make_float2(b.x, b.y));
  const float2 im = df_add_nw(make_float2(a.z, a.w), make_float2(b.z, b.w));
  return make_float4(re.x, re.y, im.x, im.y);
}
__device__ __forceinline__ float4 c_sub_nw(float4 a, float4 b) {
  const float2 re = df_add_nw(make_float2(a.x, a.y), make_float2(-b.x, -b.y));
  const float2 im = df_add_nw(make_float2(a.z, a.w), make_float2(-b.z, -b.w));
  return make_float4(re.x, re.y, im.x, im.y);
}
// Cheaper forms for transforms whose error is only needed normwise and that
// feed one another (the passes of an FFT).
//
// df_add_un: df_add_nw without its closing fast two-sum.  hi + lo is the same
// value; lo is no longer at most ulp(hi) / 2, only a few u (|x| + |y|), which
// df_add_un, df_mul and c_mul_fused accept because they use lo linearly.
__device__ __forceinline__ float2 df_add_un(float2 x, float2 y) {
  const float2 s = two_sum(x.x, y.x);
  return make_float2(s.x, s.y + (x.y + y.y));
}
// c_mul_fused: each component a - b of two products with one FP32 error
// accumulator: the exact errors of both high products (FMA), the four cross
// terms and the two-sum of the high products, renormalised once (19 FP32
// operations per component against 25 for two df_mul and a df_add_nw).
// Normwise error a few u^2 |a| |b|; the output is normalised.
__device__ __forceinline__ float4 c_mul_fused(float4 a, float4 b) {
  const float p1 = a.x * b.x, p2 = a.z * b.z;  // re = ar br - ai bi
  float e = fmaf(a.x, b.x, -p1) - fmaf(a.z, b.z, -p2);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  e = fmaf(-a.z, b.w, e);
  e = fmaf(-a.w, b.z, e);
  const float2 s = two_sum(p1, -p2);
  const float2 re = fast_two_sum(s.x, s.y + e);
  const float q1 = a.x * b.z, q2 = a.z * b.x;  // im = ar bi + ai br
  float f = fmaf(a.x, b.z, -q1) + fmaf(a.z, b.x, -q2);
  f = fmaf(a.x, b.w, f);
  f = fmaf(a.y, b.z, f);
  f = fmaf(a.z, b.y, f);
  f = fmaf(a.w, b.x, f);
  const float2 t = two_sum(q1, q2);
  const float2 im = fast_two_sum(t.x, t.y + f);
  return make_float4(re.x, re.y, im.x, im.y);
}
__device__ __forceinline__ float4 c_add_un(float4 a, float4 b) {
  const float2 re = df_add_un(make_float2(a.x, a.y), make_float2(b.x, b.y));
  const float2 im = df_add_un(make_float2(a.z, a.w), make_float2(b.z, b.w));
  return make_float4(re.x, re.y, im.x, im.y);
}
__device__ __forceinline__ float4 c_sub_un(float4 a, float4 b) {
  const float2 re = df_add_un(make_float2(a.x, a.y), make_float2(-b.x, -b.y));
  const float2 im = df_add_un(make_float2(a.z, a.w), make_float2(-b.z, -b.w));
  return make_float4(re.x, re.y, im.x, im.y);
}
__device__ __forceinline__ float2 split_double(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}

}  // namespace df
}  // namespace fde
