// Shared-memory FFTs of length P = 2^p <= 8192 for the Toeplitz products of
// the residual, in FP64 (double2), double-float (float4) and FP32 (float2)
// arithmetic.
//
// The forward transform is a decimation in frequency: radix-8 passes from the
// largest stride down, then one radix-2 or radix-4 pass at stride 1 (where
// all outer twiddles are 1).  It takes natural order and leaves the spectrum
// in digit-reversed order; the inverse transform is its exact adjoint (the
// passes in reverse order with conjugated twiddles) and returns natural
// order.  Spectra that are only multiplied pointwise (the weights' spectra
// and the saved transforms of x) stay in the digit-reversed order, so no
// permutation pass is ever needed.
//
// Shared-memory index i is stored at i + i / 8 (one pad element per 8) so
// that the short strides of the last passes hit distinct bank groups.
// The caller provides (P + P / 8) elements; every pass ends with a barrier.
#pragma once
#include "df.cuh"

namespace fde {

// complex arithmetic policies: FP64 (double2) and double-float (float4)
struct ArF64 {
  using C = double2;
  __device__ static C zero() { return make_double2(0.0, 0.0); }
  __device__ static C make(double re, double im) { return make_double2(re, im); }
  __device__ static double re(C a) { return a.x; }
  __device__ static double im(C a) { return a.y; }
  __device__ static C mul(C a, C b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
  __device__ static C add(C a, C b) { return make_double2(a.x + b.x, a.y + b.y); }
  __device__ static C sub(C a, C b) { return make_double2(a.x - b.x, a.y - b.y); }
  __device__ static C conj(C a) { return make_double2(a.x, -a.y); }
  // a e^{-iπ/2} = -i a
  __device__ static C mul_mi(C a) { return make_double2(a.y, -a.x); }
  // a e^{-iπ/4} = (a.x + a.y, a.y - a.x) / √2;  a e^{-3iπ/4} = (a.y - a.x, -(a.x + a.y)) / √2
  __device__ static C mul_w1(C a) {
    const double s = 0.70710678118654752440;
    return make_double2(s * (a.x + a.y), s * (a.y - a.x));
  }
  __device__ static C mul_w3(C a) {
    const double s = 0.70710678118654752440;
    return make_double2(s * (a.y - a.x), -s * (a.x + a.y));
  }
};

struct ArDF {
  using C = float4;  // (re.hi, re.lo, im.hi, im.lo)
  __device__ static C zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ static C make(double re, double im) {
    const float2 r = df::split_double(re), i = df::split_double(im);
    return make_float4(r.x, r.y, i.x, i.y);
  }
  __device__ static double re(C a) { return (double)a.x + (double)a.y; }
  __device__ static double im(C a) { return (double)a.z + (double)a.w; }
  // normwise-accurate double-float operations (df::c_*_nw): an FFT's error is
  // bounded against the norm of its input, not element by element
  __device__ static C mul(C a, C b) { return df::c_mul_nw(a, b); }
  __device__ static C add(C a, C b) { return df::c_add_nw(a, b); }
  __device__ static C sub(C a, C b) { return df::c_sub_nw(a, b); }
  __device__ static C conj(C a) { return df::c_conj(a); }
  __device__ static C mul_mi(C a) { return make_float4(a.z, a.w, -a.x, -a.y); }
  // 1/√2 as a double-float constant
  __device__ static float2 rsqrt2() {
    constexpr double s = 0.70710678118654752440;
    constexpr float hi = (float)s;
    constexpr float lo = (float)(s - (double)hi);
    return make_float2(hi, lo);
  }
  __device__ static C mul_w1(C a) {
    const float2 re = make_float2(a.x, a.y), im = make_float2(a.z, a.w);
    const float2 p = df::df_mul(df::df_add_nw(re, im), rsqrt2());
    const float2 q = df::df_mul(df::df_add_nw(im, df::df_neg(re)), rsqrt2());
    return make_float4(p.x, p.y, q.x, q.y);
  }
  __device__ static C mul_w3(C a) {
    const float2 re = make_float2(a.x, a.y), im = make_float2(a.z, a.w);
    const float2 p = df::df_mul(df::df_add_nw(im, df::df_neg(re)), rsqrt2());
    const float2 q = df::df_mul(df::df_add_nw(re, im), rsqrt2());
    return make_float4(p.x, p.y, -q.x, -q.y);
  }
};

// Double-float with unnormalised additions and fused complex products
// (df::df_add_un, df::c_mul_fused): about a quarter fewer FP32 operations per
// radix-8 butterfly for about 1.4 times the normwise error of ArDF.  For
// transforms of updates, whose error is scaled by the update's norm; exact
// residuals keep ArDF.  Values leave a pass unnormalised (hi + lo exact, lo a
// few u of the operands' norm); every product renormalises.
struct ArDFFast : ArDF {
  __device__ static C mul(C a, C b) { return df::c_mul_fused(a, b); }
  __device__ static C add(C a, C b) { return df::c_add_un(a, b); }
  __device__ static C sub(C a, C b) { return df::c_sub_un(a, b); }
  __device__ static C mul_w1(C a) {
    const float2 re = make_float2(a.x, a.y), im = make_float2(a.z, a.w);
    const float2 p = df::df_mul(df::df_add_un(re, im), rsqrt2());
    const float2 q = df::df_mul(df::df_add_un(im, df::df_neg(re)), rsqrt2());
    return make_float4(p.x, p.y, q.x, q.y);
  }
  __device__ static C mul_w3(C a) {
    const float2 re = make_float2(a.x, a.y), im = make_float2(a.z, a.w);
    const float2 p = df::df_mul(df::df_add_un(im, df::df_neg(re)), rsqrt2());
    const float2 q = df::df_mul(df::df_add_un(re, im), rsqrt2());
    return make_float4(p.x, p.y, -q.x, -q.y);
  }
};

struct ArF32 {
  using C = float2;
  __device__ static C zero() { return make_float2(0.f, 0.f); }
  __device__ static C make(double re, double im) { return make_float2((float)re, (float)im); }
  __device__ static double re(C a) { return (double)a.x; }
  __device__ static double im(C a) { return (double)a.y; }
  __device__ static C mul(C a, C b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
  }
  __device__ static C add(C a, C b) { return make_float2(a.x + b.x, a.y + b.y); }
  __device__ static C sub(C a, C b) { return make_float2(a.x - b.x, a.y - b.y); }
  __device__ static C conj(C a) { return make_float2(a.x, -a.y); }
  __device__ static C mul_mi(C a) { return make_float2(a.y, -a.x); }
  __device__ static C mul_w1(C a) {
    const float s = 0.70710678118654752440f;
    return make_float2(s * (a.x + a.y), s * (a.y - a.x));
  }
  __device__ static C mul_w3(C a) {
    const float s = 0.70710678118654752440f;
    return make_float2(s * (a.y - a.x), -s * (a.x + a.y));
  }
};

__device__ __forceinline__ int fft_pad(int i) { return i + (i >> 3); }
// elements of a padded buffer for a transform of length P
__host__ __device__ constexpr int fft_padded_len(int P) { return P + P / 8; }
// 3-bit reversal: the slot of output k of an 8-point DFT in DIF order
__device__ __forceinline__ int fft_rev3(int k) { return ((k & 1) << 2) | (k & 2) | ((k >> 2) & 1); }

// 4-point DFT in place, natural order in and out: X_k = sum_m a_m e^{-2πi mk/4}
template <class Ar>
__device__ __forceinline__ void fft_dft4(typename Ar::C& a0, typename Ar::C& a1, typename Ar::C& a2,
                                         typename Ar::C& a3) {
  using C = typename Ar::C;
  const C t0 = Ar::add(a0, a2), t1 = Ar::sub(a0, a2), t2 = Ar::add(a1, a3), t3 = Ar::mul_mi(Ar::sub(a1, a3));
  a0 = Ar::add(t0, t2);
  a2 = Ar::sub(t0, t2);
  a1 = Ar::add(t1, t3);
  a3 = Ar::sub(t1, t3);
}

// 8-point DFT in place, natural order in and out (even / odd split into two
// 4-point DFTs and the twiddles e^{-2πik/8}, k = 1, 2, 3)
template <class Ar>
__device__ __forceinline__ void fft_dft8(typename Ar::C (&v)[8]) {
  using C = typename Ar::C;
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  fft_dft4<Ar>(e0, e1, e2, e3);
  fft_dft4<Ar>(o0, o1, o2, o3);
  o1 = Ar::mul_w1(o1);
  o2 = Ar::mul_mi(o2);
  o3 = Ar::mul_w3(o3);
  v[0] = Ar::add(e0, o0);
  v[4] = Ar::sub(e0, o0);
  v[1] = Ar::add(e1, o1);
  v[5] = Ar::sub(e1, o1);
  v[2] = Ar::add(e2, o2);
  v[6] = Ar::sub(e2, o2);
  v[3] = Ar::add(e3, o3);
  v[7] = Ar::sub(e3, o3);
}

// Forward transform (e^{-2πi nk/P}) in place: buf in natural order (padded
// indices) -> digit-reversed spectrum.  tw[k] = e^{-2πik/P}, k < P.
template <class Ar>
__device__ void fft_forward(typename Ar::C* buf, int logP, const typename Ar::C* __restrict__ tw) {
  using C = typename Ar::C;
  const int P = 1 << logP, q = logP / 3, r = logP - 3 * q;
  int ls = logP - 3;  // log2 of the stride of the current radix-8 pass
  for (int pass = 0; pass < q; ++pass, ls -= 3) {
    const int s = 1 << ls;
    for (int b = threadIdx.x; b < (P >> 3); b += blockDim.x) {
      const int g = b >> ls, j = b & (s - 1);
      const int base = (g << (ls + 3)) + j;
      C v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = buf[fft_pad(base + (m << ls))];
      fft_dft8<Ar>(v);
      // output k goes to slot rev3(k) with the twiddle e^{-2πi j k / (8s)} = tw[j k P / (8s)]
      const int tstep = j << (logP - ls - 3);
      buf[fft_pad(base)] = v[0];
#pragma unroll
      for (int k = 1; k < 8; ++k) buf[fft_pad(base + (fft_rev3(k) << ls))] = Ar::mul(v[k], tw[k * tstep]);
    }
    __syncthreads();
  }
  if (r == 1) {
    for (int b = threadIdx.x; b < (P >> 1); b += blockDim.x) {
      const int i0 = fft_pad(2 * b), i1 = fft_pad(2 * b + 1);
      const C a = buf[i0], c = buf[i1];
      buf[i0] = Ar::add(a, c);
      buf[i1] = Ar::sub(a, c);
    }
    __syncthreads();
  } else if (r == 2) {
    for (int b = threadIdx.x; b < (P >> 2); b += blockDim.x) {
      const int i = 4 * b;
      C a0 = buf[fft_pad(i)], a1 = buf[fft_pad(i + 1)], a2 = buf[fft_pad(i + 2)], a3 = buf[fft_pad(i + 3)];
      fft_dft4<Ar>(a0, a1, a2, a3);
      // output k at slot rev2(k): 0, 2, 1, 3
      buf[fft_pad(i)] = a0;
      buf[fft_pad(i + 1)] = a2;
      buf[fft_pad(i + 2)] = a1;
      buf[fft_pad(i + 3)] = a3;
    }
    __syncthreads();
  }
}

// Inverse transform without the 1/P factor (e^{+2πi nk/P}): the adjoint of
// fft_forward, digit-reversed spectrum -> natural order.  Each radix-8 pass
// computes conj(DFT8(conj(y) .* w)) with the forward pass's twiddles w.
template <class Ar>
__device__ void fft_inverse(typename Ar::C* buf, int logP, const typename Ar::C* __restrict__ tw) {
  using C = typename Ar::C;
  const int P = 1 << logP, q = logP / 3, r = logP - 3 * q;
  if (r == 1) {
    for (int b = threadIdx.x; b < (P >> 1); b += blockDim.x) {
      const int i0 = fft_pad(2 * b), i1 = fft_pad(2 * b + 1);
      const C a = buf[i0], c = buf[i1];
      buf[i0] = Ar::add(a, c);
      buf[i1] = Ar::sub(a, c);
    }
    __syncthreads();
  } else if (r == 2) {
    for (int b = threadIdx.x; b < (P >> 2); b += blockDim.x) {
      const int i = 4 * b;
      // slots hold outputs 0, 2, 1, 3; inverse 4-point DFT as conj(DFT4(conj(.)))
      C a0 = Ar::conj(buf[fft_pad(i)]), a2 = Ar::conj(buf[fft_pad(i + 1)]);
      C a1 = Ar::conj(buf[fft_pad(i + 2)]), a3 = Ar::conj(buf[fft_pad(i + 3)]);
      fft_dft4<Ar>(a0, a1, a2, a3);
      buf[fft_pad(i)] = Ar::conj(a0);
      buf[fft_pad(i + 1)] = Ar::conj(a1);
      buf[fft_pad(i + 2)] = Ar::conj(a2);
      buf[fft_pad(i + 3)] = Ar::conj(a3);
    }
    __syncthreads();
  }
  int ls = r;  // stride of the last forward radix-8 pass is 2^r
  for (int pass = 0; pass < q; ++pass, ls += 3) {
    const int s = 1 << ls;
    for (int b = threadIdx.x; b < (P >> 3); b += blockDim.x) {
      const int g = b >> ls, j = b & (s - 1);
      const int base = (g << (ls + 3)) + j;
      const int tstep = j << (logP - ls - 3);
      C v[8];
      v[0] = Ar::conj(buf[fft_pad(base)]);
#pragma unroll
      for (int k = 1; k < 8; ++k) v[k] = Ar::mul(Ar::conj(buf[fft_pad(base + (fft_rev3(k) << ls))]), tw[k * tstep]);
      fft_dft8<Ar>(v);
#pragma unroll
      for (int m = 0; m < 8; ++m) buf[fft_pad(base + (m << ls))] = Ar::conj(v[m]);
    }
    __syncthreads();
  }
}

}  // namespace fde
