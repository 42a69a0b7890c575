// Block-Toeplitz FFT products with the shifted GL operator for N > 4096.
#include "df.cuh"
#include "fft_block.cuh"

namespace fde {

namespace {

constexpr int B = kFftBlock, P = kFftBlockP, LOGP = kFftBlockLogP;
constexpr int kThreads = 1024;
constexpr int kPerThread = B / kThreads;  // output rows per thread and block

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
};
struct ArDF {
  using C = float4;
  __device__ static C zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ static C make(double re, double im) {
    const float2 r = df::split_double(re), i = df::split_double(im);
    return make_float4(r.x, r.y, i.x, i.y);
  }
  __device__ static double re(C a) { return (double)a.x + (double)a.y; }
  __device__ static double im(C a) { return (double)a.z + (double)a.w; }
  __device__ static C mul(C a, C b) { return df::c_mul(a, b); }
  __device__ static C add(C a, C b) { return df::c_add(a, b); }
  __device__ static C sub(C a, C b) { return df::c_sub(a, b); }
  __device__ static C conj(C a) { return df::c_conj(a); }
};

// in-place radix-2 decimation-in-time FFT of length P (input in bit-reversed
// order), twiddles tw[k] = e^{-2πik/P}, k < P/2 (conjugated for the inverse)
template <class Ar>
__device__ void fft_dit(typename Ar::C* buf, const typename Ar::C* __restrict__ tw, bool inverse) {
  using C = typename Ar::C;
  for (int s = 1; s <= LOGP; ++s) {
    const int half = 1 << (s - 1), tstride = P >> s;
    for (int b = threadIdx.x; b < (P >> 1); b += blockDim.x) {
      const int grp = b >> (s - 1), j = b & (half - 1);
      const int i0 = (grp << s) + j, i1 = i0 + half;
      C w = tw[j * tstride];
      if (inverse) w = Ar::conj(w);
      const C u = buf[i0];
      const C v = (s == 1) ? buf[i1] : Ar::mul(buf[i1], w);
      buf[i0] = Ar::add(u, v);
      buf[i1] = Ar::sub(u, v);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ unsigned brev_p(int n) { return __brev((unsigned)n) >> (32 - LOGP); }

// Hhat[D * P + k]: spectrum of h_D[m] = g[(D-1) B + 1 + m], m < P (blockIdx.x = D)
__global__ void __launch_bounds__(kThreads) block_spectra_kernel(const double* __restrict__ g, int N,
                                                                 const double2* __restrict__ tw,
                                                                 double2* __restrict__ Hhat, float4* __restrict__ Hdf) {
  extern __shared__ double2 sbuf[];
  const int D = blockIdx.x;
  for (int m = threadIdx.x; m < P; m += blockDim.x) {
    const long long idx = (long long)(D - 1) * B + 1 + m;
    sbuf[brev_p(m)] = make_double2((idx >= 0 && idx <= N) ? g[idx] : 0.0, 0.0);
  }
  __syncthreads();
  fft_dit<ArF64>(sbuf, tw, false);
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    const double2 v = sbuf[k];
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
    buf[brev_p(n)] = v;
  }
  __syncthreads();
  fft_dit<Ar>(buf, tw, false);
  C* out = scratch + ((size_t)blockIdx.x * nb + J) * P;
  for (int k = threadIdx.x; k < P; k += blockDim.x) out[k] = buf[k];
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
  double y0[kPerThread], y1[kPerThread];
  // ---- T part
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    C acc = Ar::zero();
    for (int D = 0; D <= I; ++D) acc = Ar::add(acc, Ar::mul(Hhat[(size_t)D * P + k], Xh[(size_t)(I - D) * P + k]));
    buf[brev_p(k)] = acc;
  }
  __syncthreads();
  fft_dit<Ar>(buf, tw, true);
  const double g0 = g[0];
#pragma unroll
  for (int q = 0; q < kPerThread; ++q) {
    const int il = threadIdx.x + q * kThreads, i = I * B + il;
    y0[q] = 0.0;
    y1[q] = 0.0;
    if (i < N) {
      const C t = buf[B + il];
      double t0 = Ar::re(t) * invP, t1 = Ar::im(t) * invP;  // (g * x)[i + 1] within the blocks
      if (il == B - 1 && i + 1 < N) {                        // g_0 x_{i+1}: first row of the next block
        t0 += g0 * (double)X[(i + 1) * xs + j0 * xc];
        if (has1) t1 += g0 * (double)X[(i + 1) * xs + j1 * xc];
      }
      const double x0 = (double)X[i * xs + j0 * xc], x1 = has1 ? (double)X[i * xs + j1 * xc] : 0.0;
      y0[q] = shift * x0 - c * dp[i] * t0;
      y1[q] = shift * x1 - c * dp[i] * t1;
    }
  }
  __syncthreads();
  // ---- Tᵀ part
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    C acc = Ar::zero();
    for (int D = 0; I + D < nb; ++D)
      acc = Ar::add(acc, Ar::mul(Ar::conj(Hhat[(size_t)D * P + k]), Xh[(size_t)(I + D) * P + k]));
    buf[brev_p(k)] = acc;
  }
  __syncthreads();
  fft_dit<Ar>(buf, tw, true);
#pragma unroll
  for (int q = 0; q < kPerThread; ++q) {
    const int il = threadIdx.x + q * kThreads, i = I * B + il;
    if (i < N) {
      const C t = buf[(il + B) & (P - 1)];
      double t0 = Ar::re(t) * invP, t1 = Ar::im(t) * invP;  // (g ⋆ x)[i - 1] within the blocks
      if (il == 0 && i > 0) {                                // g_0 x_{i-1}: last row of the previous block
        t0 += g0 * (double)X[(i - 1) * xs + j0 * xc];
        if (has1) t1 += g0 * (double)X[(i - 1) * xs + j1 * xc];
      }
      const double a0 = y0[q] - c * dm[i] * t0, a1 = y1[q] - c * dm[i] * t1;
      double* p0 = Y + i * ys + j0 * yc;
      if (mode == kApplySet) {
        *p0 = a0;
      } else if (mode == kApplyResidual) {
        *p0 = Cm[i * ys + j0 * yc] - a0;
      } else {
        *p0 -= a0;
      }
      if (has1) {
        double* p1 = Y + i * ys + j1 * yc;
        if (mode == kApplySet) {
          *p1 = a1;
        } else if (mode == kApplyResidual) {
          *p1 = Cm[i * ys + j1 * yc] - a1;
        } else {
          *p1 -= a1;
        }
      }
    }
  }
}

template <class Ar, typename InT>
fde_status launch_block(const InT* X, long long xs, long long xc, int ncols, const double* Cm, double* Y,
                        long long ys, long long yc, int mode, const double* g, const typename Ar::C* Hhat,
                        const typename Ar::C* tw, const double* dp, const double* dm, double c, double shift, int N,
                        typename Ar::C* scratch, int pair_chunk, cudaStream_t st) {
  const size_t smem = (size_t)P * sizeof(typename Ar::C);
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
  const size_t smem = (size_t)P * sizeof(double2);
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
                       const float4* Hhat_df, const double2* tw, const float4* tw_df, bool df, const double* dp,
                       const double* dm, double c, double shift, int N, void* scratch, int pair_chunk,
                       cudaStream_t st, double flops) {
  if (ncols <= 0 || N <= 0) return FDE_OK;
  if (pair_chunk <= 0 || mode < kApplySet || mode > kApplySub || (mode == kApplyResidual && !Cm)) {
    set_error("block_apply: bad chunk / mode");
    return FDE_ERR_ARG;
  }
  ProfScope ps(df ? "fft_df" : "fft_apply", st, flops, 1);
  if (df) {
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
