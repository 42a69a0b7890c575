// Block-Toeplitz FFT products with the shifted GL operator for N > 4096.
#include <stdlib.h>

#include "df.cuh"
#include "fft_block.cuh"
#include "fft_core.cuh"

namespace fde {

namespace {

constexpr int B = kFftBlock, P = kFftBlockP, LOGP = kFftBlockLogP;
constexpr int kThreads = 512;

// Hhat[D * P + k]: spectrum of h_D[m] = g[(D-1) B + 1 + m], m < P (blockIdx.x = D),
// in the digit-reversed order of fft_forward
__global__ void __launch_bounds__(kThreads) block_spectra_kernel(const double* __restrict__ g, int N,
                                                                 const double2* __restrict__ tw,
                                                                 double2* __restrict__ Hhat, float4* __restrict__ Hdf) {
  extern __shared__ double2 sbuf[];
  const int D = blockIdx.x;
  for (int m = threadIdx.x; m < P; m += blockDim.x) {
    const long long idx = (long long)(D - 1) * B + 1 + m;
    sbuf[fft_pad(m)] = make_double2((idx >= 0 && idx <= N) ? g[idx] : 0.0, 0.0);
  }
  __syncthreads();
  fft_forward<ArF64>(sbuf, LOGP, tw);
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    const double2 v = sbuf[fft_pad(k)];
    Hhat[(size_t)D * P + k] = v;
    const float2 re = df::split_double(v.x), im = df::split_double(v.y);
    Hdf[(size_t)D * P + k] = make_float4(re.x, re.y, im.x, im.y);
  }
}

// Forward transforms: CTA (pair, J) stores X_J = FFT(x_{j0} + i x_{j1} on block J)
template <class Ar, typename InT>
__global__ void __launch_bounds__(kThreads) block_fwd_kernel(const InT* __restrict__ X, long long xs, long long xc,
                                                             int ncols, int pair0, int nb, int N,
                                                             const typename Ar::C* __restrict__ tw,
                                                             typename Ar::C* __restrict__ scratch) {
  using C = typename Ar::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int pair = pair0 + blockIdx.x, J = blockIdx.y;
  const int j0 = 2 * pair, j1 = j0 + 1;
  const bool has1 = j1 < ncols;
  for (int n = threadIdx.x; n < P; n += blockDim.x) {
    const int i = J * B + n;
    C v = Ar::zero();
    if (n < B && i < N) v = Ar::make((double)X[i * xs + j0 * xc], has1 ? (double)X[i * xs + j1 * xc] : 0.0);
    buf[fft_pad(n)] = v;
  }
  __syncthreads();
  fft_forward<Ar>(buf, LOGP, tw);
  C* out = scratch + ((size_t)blockIdx.x * nb + J) * P;
  for (int k = threadIdx.x; k < P; k += blockDim.x) out[k] = buf[fft_pad(k)];
}

// Products for output block I (CTA (pair, I)): the T part from the sum over
// D of Hhat_D X_{I-D}, the Tᵀ part from conj(Hhat_D) X_{I+D}; then the shift,
// the D_± scalings and the corner terms, written in `mode`.
template <class Ar, typename InT>
__global__ void __launch_bounds__(kThreads) block_inv_kernel(const InT* __restrict__ X, long long xs, long long xc,
                                                             int ncols, int pair0, int nb, int N,
                                                             const double* __restrict__ Cm, double* Y, long long ys,
                                                             long long yc, int mode, const double* __restrict__ g,
                                                             const typename Ar::C* __restrict__ Hhat,
                                                             const typename Ar::C* __restrict__ tw,
                                                             const double* __restrict__ dp,
                                                             const double* __restrict__ dm, double c, double shift,
                                                             const typename Ar::C* __restrict__ scratch) {
  using C = typename Ar::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int pair = pair0 + blockIdx.x, I = blockIdx.y;
  const int j0 = 2 * pair, j1 = j0 + 1;
  const bool has1 = j1 < ncols;
  const C* Xh = scratch + (size_t)blockIdx.x * nb * P;
  const double invP = 1.0 / P;
  // Phase 1 (T part) writes its partial result into Y, phase 2 (Tᵀ part)
  // adds the rest: with a = shift x - c D_+ (T x) and b = c D_- (Tᵀ x),
  //   kApplySet:      Y = a,      then Y -= b   (Y = A x)
  //   kApplyResidual: Y = C - a,  then Y += b   (Y = C - A x)
  //   kApplySub:      Y -= a,     then Y += b   (Y -= A x)
  // ---- T part
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    C acc = Ar::zero();
    for (int D = 0; D <= I; ++D) acc = Ar::add(acc, Ar::mul(Hhat[(size_t)D * P + k], Xh[(size_t)(I - D) * P + k]));
    buf[fft_pad(k)] = acc;
  }
  __syncthreads();
  fft_inverse<Ar>(buf, LOGP, tw);
  const double g0 = g[0];
  for (int il = threadIdx.x; il < B; il += blockDim.x) {
    const int i = I * B + il;
    if (i >= N) break;
    const C t = buf[fft_pad(B + il)];
    double t0 = Ar::re(t) * invP, t1 = Ar::im(t) * invP;  // (g * x)[i + 1] within the blocks
    if (il == B - 1 && i + 1 < N) {                        // g_0 x_{i+1}: first row of the next block
      t0 += g0 * (double)X[(i + 1) * xs + j0 * xc];
      if (has1) t1 += g0 * (double)X[(i + 1) * xs + j1 * xc];
    }
    const double a0 = shift * (double)X[i * xs + j0 * xc] - c * dp[i] * t0;
    double* p0 = Y + i * ys + j0 * yc;
    *p0 = mode == kApplySet ? a0 : mode == kApplyResidual ? Cm[i * ys + j0 * yc] - a0 : *p0 - a0;
    if (has1) {
      const double a1 = shift * (double)X[i * xs + j1 * xc] - c * dp[i] * t1;
      double* p1 = Y + i * ys + j1 * yc;
      *p1 = mode == kApplySet ? a1 : mode == kApplyResidual ? Cm[i * ys + j1 * yc] - a1 : *p1 - a1;
    }
  }
  __syncthreads();
  // ---- Tᵀ part
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    C acc = Ar::zero();
    for (int D = 0; I + D < nb; ++D)
      acc = Ar::add(acc, Ar::mul(Ar::conj(Hhat[(size_t)D * P + k]), Xh[(size_t)(I + D) * P + k]));
    buf[fft_pad(k)] = acc;
  }
  __syncthreads();
  fft_inverse<Ar>(buf, LOGP, tw);
  const double sgn = mode == kApplySet ? -1.0 : 1.0;
  for (int il = threadIdx.x; il < B; il += blockDim.x) {
    const int i = I * B + il;
    if (i >= N) break;
    const C t = buf[fft_pad((il + B) & (P - 1))];
    double t0 = Ar::re(t) * invP, t1 = Ar::im(t) * invP;  // (g ⋆ x)[i - 1] within the blocks
    if (il == 0 && i > 0) {                                // g_0 x_{i-1}: last row of the previous block
      t0 += g0 * (double)X[(i - 1) * xs + j0 * xc];
      if (has1) t1 += g0 * (double)X[(i - 1) * xs + j1 * xc];
    }
    Y[i * ys + j0 * yc] += sgn * c * dm[i] * t0;
    if (has1) Y[i * ys + j1 * yc] += sgn * c * dm[i] * t1;
  }
}

template <class Ar, typename InT>
fde_status launch_block(const InT* X, long long xs, long long xc, int ncols, const double* Cm, double* Y,
                        long long ys, long long yc, int mode, const double* g, const typename Ar::C* Hhat,
                        const typename Ar::C* tw, const double* dp, const double* dm, double c, double shift, int N,
                        typename Ar::C* scratch, int pair_chunk, cudaStream_t st) {
  const size_t smem = (size_t)fft_padded_len(P) * sizeof(typename Ar::C);
  // set once per instantiation (thread-safe initialisation of a local static)
  static const cudaError_t attr = [smem]() {
    cudaError_t e = cudaFuncSetAttribute(block_fwd_kernel<Ar, InT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(block_inv_kernel<Ar, InT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
  }();
  FDE_CUDA(attr);
  const int nb = (N + B - 1) / B, npairs = (ncols + 1) / 2;
  for (int p0 = 0; p0 < npairs; p0 += pair_chunk) {
    const int np = npairs - p0 < pair_chunk ? npairs - p0 : pair_chunk;
    block_fwd_kernel<Ar, InT><<<dim3(np, nb), kThreads, smem, st>>>(X, xs, xc, ncols, p0, nb, N, tw, scratch);
    FDE_LAUNCH("block_fwd_kernel");
    block_inv_kernel<Ar, InT><<<dim3(np, nb), kThreads, smem, st>>>(X, xs, xc, ncols, p0, nb, N, Cm, Y, ys, yc, mode,
                                                                     g, Hhat, tw, dp, dm, c, shift, scratch);
    FDE_LAUNCH("block_inv_kernel");
  }
  return FDE_OK;
}

}  // namespace

fde_status block_spectra(const double* g, int N, const double2* tw, double2* Hhat, float4* Hhat_df, cudaStream_t st) {
  const int nb = (N + B - 1) / B;
  const size_t smem = (size_t)fft_padded_len(P) * sizeof(double2);
  FDE_CUDA(cudaFuncSetAttribute(block_spectra_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  block_spectra_kernel<<<nb, kThreads, smem, st>>>(g, N, tw, Hhat, Hhat_df);
  FDE_LAUNCH("block_spectra_kernel");
  return FDE_OK;
}

double block_apply_flops(int N, int ncols) {
  const double nb = (N + B - 1) / B, npairs = (ncols + 1) / 2;
  // per pair: nb forward + 2 nb inverse FFTs (5 P log2 P) and nb (nb + 1) spectral products (8 P)
  return npairs * (3.0 * nb * 5.0 * P * LOGP + nb * (nb + 1) * 8.0 * P);
}

fde_status block_apply(const void* X, bool x_is_float, long long xs, long long xc, int ncols, const double* Cm,
                       double* Y, long long ys, long long yc, int mode, const double* g, const double2* Hhat,
                       const float4* Hhat_df, const float2* Hhat_f32, const double2* tw, const float4* tw_df,
                       const float2* tw_f32, int prec, const double* dp, const double* dm, double c, double shift,
                       int N, void* scratch, int pair_chunk, cudaStream_t st, double flops) {
  if (ncols <= 0 || N <= 0) return FDE_OK;
  if (pair_chunk <= 0 || mode < kApplySet || mode > kApplySub || (mode == kApplyResidual && !Cm) ||
      prec < kBlockF64 || prec > kBlockF32 || (prec == kBlockF32 && !x_is_float)) {
    set_error("block_apply: bad chunk / mode / precision");
    return FDE_ERR_ARG;
  }
  ProfScope ps(prec == kBlockDF ? "fft_df" : prec == kBlockF32 ? "fft_f32" : "fft_apply", st, flops, 1);
  if (prec == kBlockF32)
    return launch_block<ArF32, float>((const float*)X, xs, xc, ncols, Cm, Y, ys, yc, mode, g, Hhat_f32, tw_f32, dp,
                                      dm, c, shift, N, (float2*)scratch, pair_chunk, st);
  if (prec == kBlockDF) {
    // FP32 input is an update δ: its transforms take the cheaper arithmetic
    // (error scaled by |δ|) unless FDE_DF_FAST=0; FP64 input (exact residuals)
    // keeps the normalised arithmetic
    const char* fast_env = getenv("FDE_DF_FAST");
    if (x_is_float && !(fast_env && fast_env[0] == '0'))
      return launch_block<ArDFFast, float>((const float*)X, xs, xc, ncols, Cm, Y, ys, yc, mode, g, Hhat_df, tw_df, dp,
                                           dm, c, shift, N, (float4*)scratch, pair_chunk, st);
    if (x_is_float)
      return launch_block<ArDF, float>((const float*)X, xs, xc, ncols, Cm, Y, ys, yc, mode, g, Hhat_df, tw_df, dp, dm,
                                       c, shift, N, (float4*)scratch, pair_chunk, st);
    return launch_block<ArDF, double>((const double*)X, xs, xc, ncols, Cm, Y, ys, yc, mode, g, Hhat_df, tw_df, dp, dm,
                                      c, shift, N, (float4*)scratch, pair_chunk, st);
  }
  if (x_is_float)
    return launch_block<ArF64, float>((const float*)X, xs, xc, ncols, Cm, Y, ys, yc, mode, g, Hhat, tw, dp, dm, c,
                                      shift, N, (double2*)scratch, pair_chunk, st);
  return launch_block<ArF64, double>((const double*)X, xs, xc, ncols, Cm, Y, ys, yc, mode, g, Hhat, tw, dp, dm, c,
                                     shift, N, (double2*)scratch, pair_chunk, st);
}

}  // namespace fde
