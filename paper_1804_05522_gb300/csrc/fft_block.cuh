// Structured operator products for N > 4096: block-Toeplitz FFTs.
#pragma once
#include "common.cuh"

namespace fde {

// Block length of the block-Toeplitz decomposition and its FFT length.
constexpr int kFftBlock = 4096;
constexpr int kFftBlockP = 2 * kFftBlock;
constexpr int kFftBlockLogP = 13;

// Spectra of the nb = ceil(N / kFftBlock) windows of the GL weights,
//   h_D[m] = g[(D-1) B + 1 + m],  m < 2B   (g[k] = 0 outside 0..N),
// one per block distance D = 0..nb-1: Hhat[D * 2B + k], k in the digit-reversed
// order of fft_forward (fft_core.cuh).  FP64 (double2) and the double-float
// split (float4) of the same values.  tw: e^{-2πik/2B}, k < 2B.
fde_status block_spectra(const double* g, int N, const double2* tw, double2* Hhat, float4* Hhat_df, cudaStream_t st);

// Output modes of the operator products below.
enum BlockApplyMode { kApplySet = 0, kApplyResidual = 1, kApplySub = 2 };
// Arithmetic of the block products: FP64, double-float (FP32 pipe, ~48
// bits), or plain FP32.
enum BlockApplyPrec { kBlockF64 = 0, kBlockDF = 1, kBlockF32 = 2 };

// For the columns x_j (x_j(i) = X[i * xs + j * xc], j < ncols) of an N x ncols
// matrix:  y_j = A x_j,  A = shift I + c (D_+ T + D_- Tᵀ),  T = -[g_{i-j+1}]
// (§2.2.1, Eq. (toeplitz_FD)), written as
//   kApplySet:      Y = A X        kApplyResidual: Y = C - A X
//   kApplySub:      Y -= A X       (Y(i, j) = Y[i * ys + j * yc], C likewise)
// Block (I, J) of T depends only on D = I - J; its product with x_J is the
// middle of a circular convolution of length 2B with h_D, so
//   (T x)_I  = -sum_{D >= 0} IFFT(Hhat_D . X_{I-D})[B + i]  (+ one g_0 corner term),
//   (Tᵀx)_I = -sum_{D >= 0} IFFT(conj(Hhat_D) . X_{I+D})[(i + B) mod 2B] (+ corner).
// prec selects the arithmetic (the spectra and twiddles of that precision are
// used: Hhat / tw, Hhat_df / tw_df, Hhat_f32 / tw_f32); the result is
// accumulated in FP64 in every case.
// scratch: min(ceil(ncols/2), pair_chunk) * nb * 2B complex (16 bytes each).
fde_status block_apply(const void* X, bool x_is_float, long long xs, long long xc, int ncols, const double* Cm,
                       double* Y, long long ys, long long yc, int mode, const double* g, const double2* Hhat,
                       const float4* Hhat_df, const float2* Hhat_f32, const double2* tw, const float4* tw_df,
                       const float2* tw_f32, int prec, const double* dp, const double* dm, double c, double shift,
                       int N, void* scratch, int pair_chunk, cudaStream_t st, double flops = 0.0);

// Work of one block_apply call (algorithmic FLOPs) for the instrumentation.
double block_apply_flops(int N, int ncols);

}  // namespace fde
