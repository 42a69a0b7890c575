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

// For every pair (p, q) (p < nx, q < ny) solve
//   S_p Y + Y R_qᵀ = C   in place on rows lo_x[p].. and columns lo_y[q].. of W
// (ld ldw), S_p = S + soff_x[p] (n_x[p] x n_x[p]) and R_q = R + soff_y[q]
// (n_y[q] x n_y[q]), both with leading dimension ld, upper quasi-triangular
// (leaf Schur forms or diagonal blocks of them that split no 2x2 block).
// Bartels–Stewart back substitution over 1x1 / 2x2 diagonal blocks.
// lmax >= every n_x[p], n_y[q] (sizes the launch).
// flops: algorithmic work for the instrumentation (Σ n1 n2 (n1 + n2)).
template <typename T>
fde_status leaf_trsyl(const T* S, const T* R, int ld, int lmax, const int* d_soff_x, const int* d_lo_x,
                      const int* d_n_x, int nx, const int* d_soff_y, const int* d_lo_y, const int* d_n_y, int ny,
                      T* W, int ldw, cudaStream_t st, double flops = 0.0);

// A set of pairs for one launch: (p, q) over nx x (count / nx), as above.
// rest_x[p] / rest_y[q] (device, may be NULL = 0): when the S_p (R_q) above
// is a diagonal block of a larger leaf Schur form, the rows (columns) of that
// leaf after the block.  The solve then first subtracts the coupling with the
// already solved blocks of Y there (block Bartels–Stewart, left-looking):
//   F -= S_p[block, after] Y[after, block] + Y[block, after] R_q[block, after]ᵀ
// (FP32 only).
struct TrsylSet {
  const int *soff_x = nullptr, *lo_x = nullptr, *n_x = nullptr;
  int nx = 1;
  const int *soff_y = nullptr, *lo_y = nullptr, *n_y = nullptr;
  int count = 0;
  const int *rest_x = nullptr, *rest_y = nullptr;
};
// Up to kTrsylMaxSets independent sets of pairs in one launch (blocks of set 0
// first).
constexpr int kTrsylMaxSets = 16;
struct TrsylSets {
  TrsylSet s[kTrsylMaxSets];
  int n = 0;
};
template <typename T>
fde_status leaf_trsyl_sets(const T* S, const T* R, int ld, int lmax, const TrsylSets& sets, T* W, int ldw,
                           cudaStream_t st, double flops = 0.0);

}  // namespace fde
