// Double-float FFT for the incremental FP64-grade residual (arithmetic in
// df.cuh, transforms in fft_core.cuh).
#include <stdlib.h>

#include "df.cuh"
#include "fft_core.cuh"
#include "fft_df.cuh"

namespace fde {

namespace {

using namespace df;

constexpr int kThreads = 512;

// Block size of the double-float kernel.  At P = 8192 the transform buffer
// and the T part take 200 KB of shared memory, so one CTA runs per SM and the
// block size alone sets the warps that hide the shared-memory and twiddle
// latencies: 1024 threads (at most 64 registers each, spilling a few dozen
// bytes) give 32 warps per SM against 16 for 512 threads (92 registers, no
// spill), 3 % less time per launch at N = 4096.  Shorter transforms keep 512
// threads: their passes have at most 512 butterflies.
inline int df_block_threads(int P) {
  const char* e = getenv("FDE_DF_THREADS");
  const int forced = e ? atoi(e) : 0;
  if (forced == 512 || forced == 1024) return forced;
  return P >= 8192 ? 1024 : 512;
}

// Columns j0 = 2b, j1 = 2b + 1 share one complex transform (x_0 + i x_1):
//   (T x)_i  = -(g * x)[i+1],   (Tᵀx)_i = -(g ⋆ x)[i-1]   (correlation: conj(ĝ))
// Ghat and the saved transform are in the digit-reversed order of fft_forward.
// The update  R(i, j) -= shift x_j(i) - cp(i) (g * x_j)[i+1] - cm(i) (g ⋆ x_j)[i-1]
// (cp, cm = c d_± / P as double-float pairs) is formed in double-float
// arithmetic, the T part kept in shared memory until the Tᵀ part is known, so
// R is read and written once with a few FP64 operations per element.
template <class Ar, int NT>
__global__ void __launch_bounds__(NT) fd_fft_sub_df_kernel(const float* __restrict__ X, long long xs,
                                                                long long xc, int ncols, double* R, long long rs,
                                                                long long rc, const float4* __restrict__ Ghat,
                                                                const float4* __restrict__ tw, int P, int logP,
                                                                const float2* __restrict__ cp,
                                                                const float2* __restrict__ cm, float2 shift, int N,
                                                                float4* __restrict__ scratch, int set) {
  extern __shared__ float4 buf[];
  float4* side = buf + fft_padded_len(P);  // N entries: the T part of both columns
  const int j0 = 2 * blockIdx.x, j1 = j0 + 1;
  const bool has1 = j1 < ncols;
  for (int n = threadIdx.x; n < P; n += blockDim.x) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (n < N) {
      v.x = X[n * xs + j0 * xc];
      if (has1) v.z = X[n * xs + j1 * xc];
    }
    buf[fft_pad(n)] = v;
  }
  __syncthreads();
  fft_forward<Ar>(buf, logP, tw);
  float4* Xh = scratch + (size_t)blockIdx.x * P;
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    const float4 v = buf[fft_pad(k)];
    Xh[k] = v;
    buf[fft_pad(k)] = Ar::mul(v, Ghat[k]);
  }
  __syncthreads();
  fft_inverse<Ar>(buf, logP, tw);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float4 t = buf[fft_pad(i + 1)];
    const float2 c = cp[i];
    const float2 a0 = df_mul(make_float2(t.x, t.y), c), a1 = df_mul(make_float2(t.z, t.w), c);
    side[i] = make_float4(a0.x, a0.y, a1.x, a1.y);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < P; k += blockDim.x) buf[fft_pad(k)] = Ar::mul(Xh[k], c_conj(Ghat[k]));
  __syncthreads();
  fft_inverse<Ar>(buf, logP, tw);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float4 t = buf[fft_pad((i - 1 + P) & (P - 1))];
    const float4 sT = side[i];
    const float2 c = cm[i];
    // u = shift x - (T part + Tᵀ part), then R -= u
    const float2 w0 = df_add_nw(make_float2(sT.x, sT.y), df_mul(make_float2(t.x, t.y), c));
    const float2 u0 = df_add_nw(df_mul(shift, make_float2(X[i * xs + j0 * xc], 0.f)), df_neg(w0));
    double* r0 = R + i * rs + j0 * rc;
    *r0 = set ? (double)u0.x + (double)u0.y : (*r0 - (double)u0.x) - (double)u0.y;
    if (has1) {
      const float2 w1 = df_add_nw(make_float2(sT.z, sT.w), df_mul(make_float2(t.z, t.w), c));
      const float2 u1 = df_add_nw(df_mul(shift, make_float2(X[i * xs + j1 * xc], 0.f)), df_neg(w1));
      double* r1 = R + i * rs + j1 * rc;
      *r1 = set ? (double)u1.x + (double)u1.y : (*r1 - (double)u1.x) - (double)u1.y;
    }
  }
}

// The same update in plain FP32 arithmetic, for the last refinement update of
// a time step: its residual only seeds the next step's predictor, whose
// first sweep recomputes the residual exactly (cp, cm: FP32 parts).
__global__ void __launch_bounds__(kThreads) fd_fft_sub_f32_kernel(const float* __restrict__ X, long long xs,
                                                                 long long xc, int ncols, double* R, long long rs,
                                                                 long long rc, const float2* __restrict__ Ghat,
                                                                 const float2* __restrict__ tw, int P, int logP,
                                                                 const float2* __restrict__ cp,
                                                                 const float2* __restrict__ cm, float shift, int N,
                                                                 float2* __restrict__ scratch, int set) {
  extern __shared__ float2 fbuf[];
  float2* side = fbuf + fft_padded_len(P);  // N entries: the T part of both columns
  const int j0 = 2 * blockIdx.x, j1 = j0 + 1;
  const bool has1 = j1 < ncols;
  for (int n = threadIdx.x; n < P; n += blockDim.x) {
    float2 v = make_float2(0.f, 0.f);
    if (n < N) {
      v.x = X[n * xs + j0 * xc];
      if (has1) v.y = X[n * xs + j1 * xc];
    }
    fbuf[fft_pad(n)] = v;
  }
  __syncthreads();
  fft_forward<ArF32>(fbuf, logP, tw);
  float2* Xh = scratch + (size_t)blockIdx.x * P;
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    const float2 v = fbuf[fft_pad(k)];
    Xh[k] = v;
    fbuf[fft_pad(k)] = ArF32::mul(v, Ghat[k]);
  }
  __syncthreads();
  fft_inverse<ArF32>(fbuf, logP, tw);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float2 t = fbuf[fft_pad(i + 1)];
    const float c = cp[i].x;
    side[i] = make_float2(c * t.x, c * t.y);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < P; k += blockDim.x) fbuf[fft_pad(k)] = ArF32::mul(Xh[k], ArF32::conj(Ghat[k]));
  __syncthreads();
  fft_inverse<ArF32>(fbuf, logP, tw);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float2 t = fbuf[fft_pad((i - 1 + P) & (P - 1))];
    const float2 sT = side[i];
    const float c = cm[i].x;
    const float u0 = fmaf(shift, X[i * xs + j0 * xc], -fmaf(c, t.x, sT.x));
    double* r0 = R + i * rs + j0 * rc;
    *r0 = set ? (double)u0 : *r0 - (double)u0;
    if (has1) {
      const float u1 = fmaf(shift, X[i * xs + j1 * xc], -fmaf(c, t.y, sT.y));
      double* r1 = R + i * rs + j1 * rc;
      *r1 = set ? (double)u1 : *r1 - (double)u1;
    }
  }
}

__global__ void complex_to_f32_kernel(const double2* __restrict__ in, float2* __restrict__ out, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const double2 v = in[k];
    out[k] = make_float2((float)v.x, (float)v.y);
  }
}

__global__ void complex_to_df_kernel(const double2* __restrict__ in, float4* __restrict__ out, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const double2 v = in[k];
    const float2 re = split_double(v.x), im = split_double(v.y);
    out[k] = make_float4(re.x, re.y, im.x, im.y);
  }
}

}  // namespace

fde_status fd_apply_sub_df(const float* X, long long xs, long long xc, int ncols, double* R, long long rs,
                           long long rc, const float4* Ghat, const float4* tw, int P, int logP, const float2* cp,
                           const float2* cm, double shift, int N, float4* scratch, cudaStream_t st, double flops,
                           bool set) {
  if (ncols <= 0 || N <= 0) return FDE_OK;
  if (P > 8192 || P < 2 * N) {
    set_error("fd_apply_sub_df: transform length %d outside [2N, 8192]", P);
    return FDE_ERR_ARG;
  }
  // padded transform buffer + the T part of N rows
  const size_t smem = ((size_t)fft_padded_len(P) + (size_t)N) * sizeof(float4);
  static const cudaError_t attr = [] {
    const int bytes = (int)((fft_padded_len(8192) + 4096) * sizeof(float4));
    const void* fns[] = {(const void*)fd_fft_sub_df_kernel<ArDFFast, 512>,
                         (const void*)fd_fft_sub_df_kernel<ArDFFast, 1024>,
                         (const void*)fd_fft_sub_df_kernel<ArDF, 512>, (const void*)fd_fft_sub_df_kernel<ArDF, 1024>};
    for (const void* f : fns) {
      const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }();
  FDE_CUDA(attr);
  // FDE_DF_THREADS=512 or 1024 overrides the block size chosen by P;
  // FDE_DF_FAST=0 selects the normalised arithmetic of the exact residuals
  const int nt = df_block_threads(P);
  const char* fast_env = getenv("FDE_DF_FAST");
  const bool fast = !(fast_env && fast_env[0] == '0');
  // shift as a double-float pair (host side: FP32 rounding of the value and the remainder)
  const float hi = (float)shift;
  const float2 shift2 = make_float2(hi, (float)(shift - (double)hi));
  ProfScope ps("fft_df", st, flops, 1);
  const unsigned grid = (unsigned)((ncols + 1) / 2);
  const int set_i = set ? 1 : 0;
  if (fast && nt == 1024)
    fd_fft_sub_df_kernel<ArDFFast, 1024><<<grid, 1024, smem, st>>>(X, xs, xc, ncols, R, rs, rc, Ghat, tw, P, logP,
                                                                   cp, cm, shift2, N, scratch, set_i);
  else if (fast)
    fd_fft_sub_df_kernel<ArDFFast, 512><<<grid, 512, smem, st>>>(X, xs, xc, ncols, R, rs, rc, Ghat, tw, P, logP, cp,
                                                                 cm, shift2, N, scratch, set_i);
  else if (nt == 1024)
    fd_fft_sub_df_kernel<ArDF, 1024><<<grid, 1024, smem, st>>>(X, xs, xc, ncols, R, rs, rc, Ghat, tw, P, logP, cp,
                                                               cm, shift2, N, scratch, set_i);
  else
    fd_fft_sub_df_kernel<ArDF, 512><<<grid, 512, smem, st>>>(X, xs, xc, ncols, R, rs, rc, Ghat, tw, P, logP, cp, cm,
                                                             shift2, N, scratch, set_i);
  FDE_LAUNCH("fd_fft_sub_df_kernel");
  return FDE_OK;
}

fde_status fd_apply_sub_f32(const float* X, long long xs, long long xc, int ncols, double* R, long long rs,
                            long long rc, const float2* Ghat, const float2* tw, int P, int logP, const float2* cp,
                            const float2* cm, double shift, int N, float2* scratch, cudaStream_t st, double flops,
                            bool set) {
  if (ncols <= 0 || N <= 0) return FDE_OK;
  if (P > 8192 || P < 2 * N) {
    set_error("fd_apply_sub_f32: transform length %d outside [2N, 8192]", P);
    return FDE_ERR_ARG;
  }
  const size_t smem = ((size_t)fft_padded_len(P) + (size_t)N) * sizeof(float2);
  static const cudaError_t attr =
      cudaFuncSetAttribute(fd_fft_sub_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)((fft_padded_len(8192) + 4096) * sizeof(float2)));
  FDE_CUDA(attr);
  ProfScope ps("fft_f32", st, flops, 1);
  fd_fft_sub_f32_kernel<<<(ncols + 1) / 2, kThreads, smem, st>>>(X, xs, xc, ncols, R, rs, rc, Ghat, tw, P, logP, cp,
                                                                 cm, (float)shift, N, scratch, set ? 1 : 0);
  FDE_LAUNCH("fd_fft_sub_f32_kernel");
  return FDE_OK;
}

fde_status complex_to_f32(const double2* in, float2* out, int n, cudaStream_t st) {
  if (n <= 0) return FDE_OK;
  complex_to_f32_kernel<<<(n + 255) / 256, 256, 0, st>>>(in, out, n);
  FDE_LAUNCH("complex_to_f32_kernel");
  return FDE_OK;
}

fde_status complex_to_df(const double2* in, float4* out, int n, cudaStream_t st) {
  if (n <= 0) return FDE_OK;
  complex_to_df_kernel<<<(n + 255) / 256, 256, 0, st>>>(in, out, n);
  FDE_LAUNCH("complex_to_df_kernel");
  return FDE_OK;
}

}  // namespace fde
