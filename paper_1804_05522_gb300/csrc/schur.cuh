// Leaf real Schur forms and quasi-triangular Sylvester solves.
#pragma once
#include "common.cuh"

namespace fde {

// In place: H (n_i x n_i leaves, ld, stride) -> real Schur form S,
// Q (same layout) -> orthogonal Schur vectors with H_in = Q S Qᵀ.
// Hessenberg reduction by Householder reflectors, then Francis double-shift
// QR with deflation (Golub & Van Loan, Matrix Computations, §7.4-7.5).
// 2x2 diagonal blocks remain only for complex conjugate pairs.
// d_fail[i] = 1 if leaf i hit the iteration cap.
fde_status leaf_schur(double* H, double* Q, int ld, size_t stride, const int* d_n, int count, int* d_fail,
                      cudaStream_t st);

// For every leaf pair (p, q) (p over nleaves_x, q over nleaves_y) solve
//   S_p Y + Y R_qᵀ = C   in place on the (p, q) block of W (ld ldw),
// S_p, R_q upper quasi-triangular (leaf Schur forms).  Bartels–Stewart
// back substitution over 1x1 / 2x2 diagonal blocks.
// flops: algorithmic work for the instrumentation (Σ n1 n2 (n1 + n2)).
template <typename T>
fde_status leaf_trsyl(const T* S, const T* R, int lmax, const int* d_lo_x, const int* d_n_x, int nx,
                      const int* d_lo_y, const int* d_n_y, int ny, T* W, int ldw, cudaStream_t st,
                      double flops = 0.0);

}  // namespace fde
