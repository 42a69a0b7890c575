// Double-float FFT for the incremental FP64-grade residual (arithmetic in
// df.cuh, transforms in fft_core.cuh).
#include "df.cuh"
#include "fft_core.cuh"
#include "fft_df.cuh"

namespace fde {

namespace {

using namespace df;

constexpr int kThreads = 512;

// Columns j0 = 2b, j1 = 2b + 1 share one complex transform (x_0 + i x_1):
//   (T x)_i  = -(g * x)[i+1],   (Tᵀx)_i = -(g ⋆ x)[i-1]   (correlation: conj(ĝ))
// Ghat and the saved transform are in the digit-reversed order of fft_forward.
__global__ void __launch_bounds__(kThreads) fd_fft_sub_df_kernel(const float* __restrict__ X, long long xs,
                                                                long long xc, int ncols, double* R, long long rs,
                                                                long long rc, const float4* __restrict__ Ghat,
                                                                const float4* __restrict__ tw, int P, int logP,
                                                                const double* __restrict__ dp,
                                                                const double* __restrict__ dm, double c, double shift,
                                                                int N, float4* __restrict__ scratch) {
  extern __shared__ float4 buf[];
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
  fft_forward<ArDF>(buf, logP, tw);
  float4* Xh = scratch + (size_t)blockIdx.x * P;
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    const float4 v = buf[fft_pad(k)];
    Xh[k] = v;
    buf[fft_pad(k)] = ArDF::mul(v, Ghat[k]);
  }
  __syncthreads();
  fft_inverse<ArDF>(buf, logP, tw);
  const double invP = 1.0 / P;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float4 t = buf[fft_pad(i + 1)];
    const double conv0 = (double)t.x + (double)t.y, conv1 = (double)t.z + (double)t.w;
    const double x0 = X[i * xs + j0 * xc];
    R[i * rs + j0 * rc] -= shift * x0 - c * dp[i] * conv0 * invP;
    if (has1) {
      const double x1 = X[i * xs + j1 * xc];
      R[i * rs + j1 * rc] -= shift * x1 - c * dp[i] * conv1 * invP;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < P; k += blockDim.x) buf[fft_pad(k)] = ArDF::mul(Xh[k], c_conj(Ghat[k]));
  __syncthreads();
  fft_inverse<ArDF>(buf, logP, tw);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float4 t = buf[fft_pad((i - 1 + P) & (P - 1))];
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
  const size_t smem = (size_t)fft_padded_len(P) * sizeof(float4);
  static const cudaError_t attr = cudaFuncSetAttribute(
      fd_fft_sub_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(fft_padded_len(8192) * sizeof(float4)));
  FDE_CUDA(attr);
  ProfScope ps("fft_df", st, flops, 1);
  fd_fft_sub_df_kernel<<<(ncols + 1) / 2, kThreads, smem, st>>>(X, xs, xc, ncols, R, rs, rc, Ghat, tw, P, logP, dp, dm,
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
