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
__device__ __forceinline__ float2 split_double(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}

}  // namespace df
}  // namespace fde
