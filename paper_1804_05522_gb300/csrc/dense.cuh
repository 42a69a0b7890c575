// Batched dense building blocks (SIMT, FP64 and FP32).
#pragma once
#include "common.cuh"

namespace fde {

// One GEMM of a batch: C = alpha op(A) op(B) + beta C, column-major.
// Optional two-level addressing along k (kblk > 0): the k-th column of a
// non-transposed A (and of a transposed B) sits at (k / kblk) * kstr +
// (k % kblk) * ld, i.e. k runs over kblk-wide panels that are kstr apart.
template <typename T>
struct GemmDesc {
  const T* A;
  const T* B;
  T* C;
  int m, n, k, lda, ldb, ldc;
  int kblk = 0;
  long long kstr = 0;
  // k / kblk = (k * kmagic) >> kshift for 0 <= k < 2^31 (set by gemm_batch_upload)
  unsigned long long kmagic = 0;
  int kshift = 0;
  // Packed constant operands for the tensor-core path (gemm_batch_pack): the
  // tiles of op(A) (128 x 32) and op(B) (BN x 32), each pre-split into TF32
  // hi and the remainder lo and stored as the MMA reads them from shared
  // memory (hi tile, then lo tile); tile (row tile r, k tile t) starts at
  // pk + (r * ceil(k / 32) + t) * 2 * rows * 32.
  const T* Apk = nullptr;
  const T* Bpk = nullptr;
};

// A list of GEMMs with the same transposes / scalars, descriptors resident on
// the device so that replays (and CUDA-graph capture) need no host work.
template <typename T>
struct GemmBatch {
  GemmDesc<T>* d_desc = nullptr;
  int batch = 0, max_m = 0, max_n = 0, max_k = 0, max_ldc = 0;
  double flops = 0.0;  // Σ 2 m n k over the batch
  bool ta = false, tb = false;
  // every descriptor's A (resp. B) base is 16-byte aligned and its ld (and
  // kstr) a multiple of 4 elements: 4-wide vector loads are allowed
  bool vec_a = false, vec_b = false;
  bool any_kblk = false;  // some descriptor uses two-level k panels
  bool pk_a = false, pk_b = false;  // every descriptor has Apk (resp. Bpk)
  int pk_bn = 0;                    // tile width B was packed for
  // Operand precision on the tensor cores: kTcDefault follows the library's
  // mode (3xTF32 by default), kTcBF16 rounds both operands to BF16 (one
  // product), kTcBF16x3 splits them into BF16 hi + lo (three products);
  // FP32 accumulation in every case.  Packed tiles are packed for this kind.
  int kind = 0;
  // Repacked operands (gemm_batch_pack with repack): the pack jobs of the
  // operand that changes between runs; gemm_batch_run refreshes its packed
  // tiles from the current values (one pack launch) before each GEMM launch.
  const void* rp_a_jobs = nullptr;
  const void* rp_b_jobs = nullptr;
  int rp_a_n = 0, rp_b_n = 0;
  T alpha = T(1), beta = T(0);
};

template <typename T>
fde_status gemm_batch_upload(DevPool& pool, const std::vector<GemmDesc<T>>& h, bool ta, bool tb, T alpha,
                             T beta, GemmBatch<T>* out, cudaStream_t st);

template <typename T>
fde_status gemm_batch_run(const GemmBatch<T>& b, cudaStream_t st);

// -1: the skinny FP32 kernel by the library's rule (FDE_SKINNY); 0 off; 1 on.
void set_skinny_force(int v);

constexpr int kTcDefault = 0, kTcBF16 = 1, kTcBF16x3 = 2;

// Tensor-core path for FP32 batches (tc_gemm.cu).  Mode from FDE_TC
// (0 = SIMT only, 1 = TF32, 3 = 3xTF32, the default).
fde_status tc_gemm_run(const GemmBatch<float>& b, cudaStream_t st, bool* used);
int tc_mode();
void set_tc_mode(int m);
fde_status tc_error_flag(int* out);                 // expired tensor-core GEMM waits so far
fde_status tc_timeout_counter(unsigned int** ptr);  // device address of that counter
fde_status tc_set_wait_limit(unsigned int iters);   // 0: the default limit
fde_status tc_prepare();
// Tile width (BN) the tensor-core path uses for a batch whose widest problem has n columns.
int tc_bn_for(int max_n);
// Packs the operands of a batch that stay constant for the batch's lifetime
// (A and / or B) for the tensor-core path: allocates the packed tiles from
// `pool`, fills them and stores their addresses in the device descriptors.
// The batch then always runs on the tensor cores when it is eligible, reading
// the packed operands with bulk asynchronous copies; the unpacked operands stay
// valid for the other paths.  Does nothing (and returns FDE_OK) when the
// tensor cores are off or the batch would not run on them, or when the packed
// tiles would take more than *budget bytes (decremented by what is used).
//
// repack_a / repack_b: the operand is not constant; its packed tiles and the
// pack jobs are kept (in `pool`) and gemm_batch_run repacks it from the
// current values before every launch.  Pays off where every tile of that
// operand is read by many tiles of the product (a thin operand against a
// tall or wide one), since the kernel then only issues bulk copies.
fde_status gemm_batch_pack(DevPool& pool, GemmBatch<float>* b, bool pack_a, bool pack_b, size_t* budget,
                           cudaStream_t st, bool repack_a = false, bool repack_b = false);

// In-place inverse of `batch` square matrices (sizes n_i <= nmax, leading
// dimension ld, matrix i at A + i*stride) by Gauss–Jordan elimination with
// partial pivoting on the augmented matrix.  work: batch * nmax * 2*nmax.
// *d_flag is set to 1 if a zero pivot is met (matrix left unchanged then).
template <typename T>
fde_status batched_inverse(T* A, int ld, size_t stride, const int* d_n, int batch, int nmax, T* work,
                           int* d_flag, cudaStream_t st);

// y[i] = (Tout) x[i]   (n elements)
template <typename Tin, typename Tout>
fde_status convert(const Tin* x, Tout* y, size_t n, cudaStream_t st);

// 2D strided copy / convert: Y[i + j*ldy] = (Tout) X[i + j*ldx], m x n
template <typename Tin, typename Tout>
fde_status copy2d(const Tin* X, int ldx, Tout* Y, int ldy, int m, int n, cudaStream_t st);

}  // namespace fde
