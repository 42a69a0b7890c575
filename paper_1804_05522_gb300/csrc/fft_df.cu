// Double-float FFT for the incremental FP64-grade residual (arithmetic in
// df.cuh).
#include "df.cuh"
#include "fft_df.cuh"

namespace fde {

namespace {

using namespace df;

// in-place radix-2 decimation-in-time FFT on buf (input in bit-reversed
// order), twiddles tw[k] = e^{-2πik/P} (conjugated for the inverse)
__device__ void fft_dit_df(float4* buf, int P, int logP, const float4* __restrict__ tw, bool inverse) {
  for (int s = 1; s <= logP; ++s) {
    const int half = 1 << (s - 1), tstride = P >> s;
    for (int b = threadIdx.x; b < (P >> 1); b += blockDim.x) {
      const int grp = b >> (s - 1), j = b & (half - 1);
      const int i0 = (grp << s) + j, i1 = i0 + half;
      float4 w = tw[j * tstride];
      if (inverse) w = c_conj(w);
      const float4 u = buf[i0];
      const float4 v = (s == 1) ? buf[i1] : c_mul(buf[i1], w);
      buf[i0] = c_add(u, v);
      buf[i1] = c_sub(u, v);
    }
    __syncthreads();
  }
}

// Columns j0 = 2b, j1 = 2b + 1 share one complex transform (x_0 + i x_1):
//   (T x)_i  = -(g * x)[i+1],   (Tᵀx)_i = -(g ⋆ x)[i-1]   (correlation: conj(ĝ))
__global__ void __launch_bounds__(1024) fd_fft_sub_df_kernel(const float* __restrict__ X, long long xs, long long xc,
                                                            int ncols, double* R, long long rs, long long rc,
                                                            const float4* __restrict__ Ghat,
                                                            const float4* __restrict__ tw, int P, int logP,
                                                            const double* __restrict__ dp,
                                                            const double* __restrict__ dm, double c, double shift,
                                                            int N, float4* __restrict__ scratch) {
  extern __shared__ float4 buf[];
  const int j0 = 2 * blockIdx.x, j1 = j0 + 1;
  const bool has1 = j1 < ncols;
  const unsigned sh = 32 - logP;
  for (int n = threadIdx.x; n < P; n += blockDim.x) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (n < N) {
      v.x = X[n * xs + j0 * xc];
      if (has1) v.z = X[n * xs + j1 * xc];
    }
    buf[__brev(n) >> sh] = v;
  }
  __syncthreads();
  fft_dit_df(buf, P, logP, tw, false);
  float4* Xh = scratch + (size_t)blockIdx.x * P;
  for (int k = threadIdx.x; k < P; k += blockDim.x) Xh[k] = buf[k];
  __syncthreads();
  for (int k = threadIdx.x; k < P; k += blockDim.x) buf[__brev(k) >> sh] = c_mul(Xh[k], Ghat[k]);
  __syncthreads();
  fft_dit_df(buf, P, logP, tw, true);
  const double invP = 1.0 / P;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float4 t = buf[i + 1];
    const double conv0 = (double)t.x + (double)t.y, conv1 = (double)t.z + (double)t.w;
    const double x0 = X[i * xs + j0 * xc];
    R[i * rs + j0 * rc] -= shift * x0 - c * dp[i] * conv0 * invP;
    if (has1) {
      const double x1 = X[i * xs + j1 * xc];
      R[i * rs + j1 * rc] -= shift * x1 - c * dp[i] * conv1 * invP;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < P; k += blockDim.x) buf[__brev(k) >> sh] = c_mul(Xh[k], c_conj(Ghat[k]));
  __syncthreads();
  fft_dit_df(buf, P, logP, tw, true);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float4 t = buf[(i - 1 + P) & (P - 1)];
    const double conv0 = (double)t.x + (double)t.y, conv1 = (double)t.z + (double)t.w;
    R[i * rs + j0 * rc] += c * dm[i] * conv0 * invP;
    if (has1) R[i * rs + j1 * rc] += c * dm[i] * conv1 * invP;
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
                           long long rc, const float4* Ghat, const float4* tw, int P, int logP, const double* dp,
                           const double* dm, double c, double shift, int N, float4* scratch, cudaStream_t st,
                           double flops) {
  if (ncols <= 0 || N <= 0) return FDE_OK;
  if (P > 8192 || P < 2 * N) {
    set_error("fd_apply_sub_df: transform length %d outside [2N, 8192]", P);
    return FDE_ERR_ARG;
  }
  const size_t smem = (size_t)P * sizeof(float4);
  static const cudaError_t attr = cudaFuncSetAttribute(
      fd_fft_sub_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(8192 * sizeof(float4)));
  FDE_CUDA(attr);
  ProfScope ps("fft_df", st, flops, 1);
  fd_fft_sub_df_kernel<<<(ncols + 1) / 2, 1024, smem, st>>>(X, xs, xc, ncols, R, rs, rc, Ghat, tw, P, logP, dp, dm,
                                                            c, shift, N, scratch);
  FDE_LAUNCH("fd_fft_sub_df_kernel");
  return FDE_OK;
}

fde_status complex_to_df(const double2* in, float4* out, int n, cudaStream_t st) {
  if (n <= 0) return FDE_OK;
  complex_to_df_kernel<<<(n + 255) / 256, 256, 0, st>>>(in, out, n);
  FDE_LAUNCH("complex_to_df_kernel");
  return FDE_OK;
}

}  // namespace fde
