// Incremental structured residual in double-float arithmetic.
#pragma once
#include "common.cuh"

namespace fde {

// R(i, j) -= (A x_j)(i), i < N, j < ncols, for the columns x_j of a float
// matrix (x_j(i) = X[i * xs + j * xc]; R(i, j) = R[i * rs + j * rc]), with
//   A = shift I + c (D_+ T + D_- Tᵀ),   T = -[g_{i-j+1}]   (§2.2.1, Eq. (toeplitz_FD)),
// given through cp(i), cm(i) = c d_±(i) / P (double-float pairs) and shift.
// The Toeplitz products are evaluated by FFT of length P = 2^logP >= 2N in
// double-float arithmetic (pairs of FP32 numbers, ~48 significant bits) on
// the FP32 pipe; the result is accumulated into R in FP64 (with set: R = A x).  Meant for small
// updates x = δX of an iterative refinement, whose error budget scales with
// ||δX||.  Ghat: spectrum of g_0..g_N in the digit-reversed order of
// fft_forward (fft_core.cuh); tw: twiddles e^{-2πik/P}, k < P; both as
// double-float complex (x = re.hi, y = re.lo, z = im.hi, w = im.lo).
// scratch: ceil(ncols/2) * P float4.
fde_status fd_apply_sub_df(const float* X, long long xs, long long xc, int ncols, double* R, long long rs,
                           long long rc, const float4* Ghat, const float4* tw, int P, int logP, const float2* cp,
                           const float2* cm, double shift, int N, float4* scratch, cudaStream_t st,
                           double flops = 0.0, bool set = false);

// The same update in plain FP32 arithmetic (Ghat, tw as FP32 complex; only
// the FP32 parts of cp, cm are used), accumulated into R in FP64 (or, with
// set, R = A x).  Its error, ~1e-6 ||A|| ||x||, suits a final refinement
// update whose residual is only used to predict the next time step before an
// exact residual replaces it.
fde_status fd_apply_sub_f32(const float* X, long long xs, long long xc, int ncols, double* R, long long rs,
                            long long rc, const float2* Ghat, const float2* tw, int P, int logP, const float2* cp,
                            const float2* cm, double shift, int N, float2* scratch, cudaStream_t st,
                            double flops = 0.0, bool set = false);

// out[k] = double-float split of the complex value in[k]
fde_status complex_to_df(const double2* in, float4* out, int n, cudaStream_t st);
// out[k] = FP32 rounding of the complex value in[k]
fde_status complex_to_f32(const double2* in, float2* out, int n, cudaStream_t st);

}  // namespace fde
