// QR + SVD recompression of U Vᵀ (U, V: m x r, m >> r) spread over many CTAs:
// a tall-skinny QR (TSQR: Householder QR of row blocks, then of the stacked
// triangular factors, level by level up a tree, each block in shared memory),
// the SVD of the small core R_U R_Vᵀ, and the products Q_U [W Σ; 0] and
// Q_V [Z; 0] formed down the same tree.  Same result as the one-CTA
// recompression (recompress_jobs) up to rounding; the FP64 work of every level
// runs on as many SMs as it has blocks.
#include <algorithm>
#include <vector>

#include "hodlr_internal.cuh"

namespace fde {
namespace {

constexpr int kTsqrThreads = 256;

// Householder QR of the n x r block A (shared memory, ld n, n >= r): the
// reflectors below the diagonal, beta on it; tau[j] in shared memory.
__device__ void smem_house_qr(double* A, int n, int r, double* tau, double* red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int kq = min(n, r);
  for (int j = 0; j < kq; ++j) {
    double part = 0.0;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) part += A[i + j * n] * A[i + j * n];
    const double sig = block_sum(part, red);
    const double x0 = A[j + j * n];
    double t = 0.0, beta = x0;
    if (sig != 0.0) {
      const double alpha = sqrt(x0 * x0 + sig);
      beta = (x0 <= 0.0) ? alpha : -alpha;
      t = (beta - x0) / beta;
      const double scale = 1.0 / (x0 - beta);
      for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[i + j * n] *= scale;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      tau[j] = t;
      A[j + j * n] = beta;
    }
    __syncthreads();
    if (t != 0.0) {
      for (int c = j + 1 + warp; c < r; c += nw) {
        const double ajc = A[j + c * n];
        double w = 0.0;
        for (int i = j + 1 + lane; i < n; i += 32) w += A[i + j * n] * A[i + c * n];
        w = warp_sum(w);
        w = t * (w + ajc);
        if (lane == 0) A[j + c * n] = ajc - w;
        for (int i = j + 1 + lane; i < n; i += 32) A[i + c * n] -= w * A[i + j * n];
      }
    }
    __syncthreads();
  }
}

// Rows of block b of a level with `rows` rows cut into blocks of `brows`
// (the last block takes the remainder).
__device__ __forceinline__ void block_range(int b, int nb, int brows, int rows, int* lo, int* n) {
  *lo = b * brows;
  *n = (b == nb - 1) ? rows - *lo : brows;
}

struct TsqrSide {
  double* X;      // level input (factor or stacked R's), ld = ldx; reflectors written back in place
  int ldx;
  double* tau;    // nb x r
  double* Rout;   // stacked R's of this level: (nb r) x r, ld nb r
  double* Xin;    // apply: (nb r) x rcap, ld nb r (the level above's output)
  double* Yout;   // apply: rows x rcap, ld ldy (this level's output)
  int ldy;
};
struct TsqrLevel {
  int rows, brows, nb;
  TsqrSide s[2];
};

__global__ void __launch_bounds__(kTsqrThreads) tsqr_qr_kernel(TsqrLevel lv, int r) {
  extern __shared__ double sm[];
  __shared__ double red[32];
  __shared__ double tau[kRecompMax];
  const int b = blockIdx.x;
  const TsqrSide& sd = lv.s[blockIdx.y];
  int lo, n;
  block_range(b, lv.nb, lv.brows, lv.rows, &lo, &n);
  double* A = sm;  // n x r
  for (int e = threadIdx.x; e < n * r; e += blockDim.x) {
    const int i = e % n, c = e / n;
    A[e] = sd.X[(size_t)(lo + i) + (size_t)c * sd.ldx];
  }
  __syncthreads();
  smem_house_qr(A, n, r, tau, red);
  // reflectors back in place, tau, and R into the stacked output
  for (int e = threadIdx.x; e < n * r; e += blockDim.x) {
    const int i = e % n, c = e / n;
    if (i > c) sd.X[(size_t)(lo + i) + (size_t)c * sd.ldx] = A[e];
  }
  const int ldr = lv.nb * r;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, c = e / r;
    sd.Rout[(size_t)(b * r + i) + (size_t)c * ldr] = (i <= c && i < n) ? A[i + c * n] : 0.0;
  }
  for (int j = threadIdx.x; j < r; j += blockDim.x) sd.tau[(size_t)b * r + j] = j < n ? tau[j] : 0.0;
}

// Y_b = Q_b [Xin_b; 0] for every block b of a level (Q_b from the block's
// reflectors and tau), Y: rows x rcap.
__global__ void __launch_bounds__(kTsqrThreads) tsqr_apply_kernel(TsqrLevel lv, int r, int rcap, const int* ncols) {
  extern __shared__ double sm[];
  const int b = blockIdx.x;
  const TsqrSide& sd = lv.s[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  int lo, n;
  block_range(b, lv.nb, lv.brows, lv.rows, &lo, &n);
  const int kq = min(n, r);
  const int nc = min(*ncols, rcap);
  double* Y = sm;  // n x rcap
  const int ldi = lv.nb * r;
  for (int e = threadIdx.x; e < n * rcap; e += blockDim.x) {
    const int i = e % n, c = e / n;
    Y[e] = (i < r) ? sd.Xin[(size_t)(b * r + i) + (size_t)c * ldi] : 0.0;
  }
  __syncthreads();
  const double* V = sd.X + lo;  // reflector j: rows j+1..n-1 of column j, ld ldx
  for (int j = kq - 1; j >= 0; --j) {
    const double t = sd.tau[(size_t)b * r + j];
    if (t != 0.0) {
      for (int c = warp; c < nc; c += nw) {
        const double yjc = Y[j + c * n];
        double w = 0.0;
        for (int i = j + 1 + lane; i < n; i += 32) w += V[i + (size_t)j * sd.ldx] * Y[i + c * n];
        w = warp_sum(w);
        w = t * (w + yjc);
        if (lane == 0) Y[j + c * n] = yjc - w;
        for (int i = j + 1 + lane; i < n; i += 32) Y[i + c * n] -= w * V[i + (size_t)j * sd.ldx];
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * rcap; e += blockDim.x) {
    const int i = e % n, c = e / n;
    sd.Yout[(size_t)(lo + i) + (size_t)c * sd.ldy] = Y[e];
  }
}

// Copies the root's R factors into the workspace layout of the core kernel.
__global__ void tsqr_root_kernel(const double* __restrict__ Ru, const double* __restrict__ Rv, int r,
                                 double* __restrict__ R) {
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    R[e] = Ru[e];
    R[r * r + e] = Rv[e];
  }
}

}  // namespace

// A recompression plan for fixed m, r, rcap and fixed buffers (host side).
struct TsqrPlan {
  int m = 0, r = 0, rcap = 0;
  std::vector<TsqrLevel> levels;
  RecompJob job{};
  const RecompJob* d_job = nullptr;
  RecompWork wk{};
  double* root[2] = {nullptr, nullptr};
};

fde_status tsqr_plan_create(const RecompJob& job, const RecompJob* d_job, int r, int rcap, const RecompWork& wk,
                            DevPool& pool, TsqrPlan** out) {
  if (r > kRecompMax || rcap > r || job.m != job.n || job.m < 128) {
    set_error("tsqr: unsupported shape m = %d, n = %d, r = %d", job.m, job.n, r);
    return FDE_ERR_ARG;
  }
  TsqrPlan* P = new TsqrPlan();
  P->m = job.m;
  P->r = r;
  P->rcap = rcap;
  P->job = job;
  P->d_job = d_job;
  P->wk = wk;
  // level 0 on the factors (blocks of 128 rows: the last one, up to 255 rows,
  // fits shared memory with r <= 96), then on the stacked R's (pairs; the last
  // block up to 3 R's)
  int rows = job.m, brows = 128;
  double* X[2] = {job.Uin, job.Vin};
  int ldx = job.ld;
  double* Yout[2] = {job.Uout, job.Vout};
  int ldy = job.ld;
  while (true) {
    TsqrLevel lv{};
    lv.rows = rows;
    lv.brows = brows;
    lv.nb = std::max(1, rows / brows);
    for (int s = 0; s < 2; ++s) {
      lv.s[s].X = X[s];
      lv.s[s].ldx = ldx;
      fde_status st = pool.alloc(&lv.s[s].tau, (size_t)lv.nb * r);
      if (st == FDE_OK) st = pool.alloc(&lv.s[s].Rout, (size_t)lv.nb * r * r);
      if (st == FDE_OK) st = pool.alloc(&lv.s[s].Xin, (size_t)lv.nb * r * rcap);
      if (st != FDE_OK) {
        delete P;
        return st;
      }
      lv.s[s].Yout = Yout[s];
      lv.s[s].ldy = ldy;
    }
    P->levels.push_back(lv);
    if (lv.nb == 1) break;
    // the next level works on this level's stacked R's; its output feeds this level's Xin
    rows = lv.nb * r;
    brows = 2 * r;
    for (int s = 0; s < 2; ++s) {
      X[s] = lv.s[s].Rout;
      Yout[s] = lv.s[s].Xin;
    }
    ldx = rows;
    ldy = rows;
  }
  for (int s = 0; s < 2; ++s) P->root[s] = P->levels.back().s[s].Rout;
  *out = P;
  return FDE_OK;
}

void tsqr_plan_free(TsqrPlan* P) { delete P; }

size_t tsqr_smem_max(int r) {
  // a block has fewer than 2 brows rows: 255 at the leaves, 3 r above
  const int rows = std::max(255, 3 * r);
  return (size_t)rows * r * sizeof(double);
}

fde_status tsqr_prepare(int rmax) {
  static bool done = false;
  if (done) return FDE_OK;
  const size_t smem = tsqr_smem_max(rmax);
  FDE_CUDA(cudaFuncSetAttribute(tsqr_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  FDE_CUDA(cudaFuncSetAttribute(tsqr_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  done = true;
  return FDE_OK;
}

fde_status tsqr_run(const TsqrPlan* P, double abstol, double reltol, cudaStream_t st) {
  const int r = P->r, rcap = P->rcap;
  // up the tree: QR of every block
  for (const TsqrLevel& lv : P->levels) {
    const int maxn = (lv.nb == 1) ? lv.rows : lv.rows - (lv.nb - 1) * lv.brows;
    const size_t smem = (size_t)std::max(maxn, lv.brows) * r * sizeof(double);
    tsqr_qr_kernel<<<dim3(lv.nb, 2), kTsqrThreads, smem, st>>>(lv, r);
    FDE_LAUNCH("tsqr_qr_kernel");
  }
  // the core: SVD of R_U R_Vᵀ, truncation, the kept factors (r x rcap) in wk.C
  tsqr_root_kernel<<<1, 256, 0, st>>>(P->root[0], P->root[1], r, P->wk.R);
  FDE_LAUNCH("tsqr_root_kernel");
  FDE_TRY(recompress_core(P->d_job, r, rcap, abstol, reltol, P->wk, st));
  // down the tree: the root level's input is the core's output
  for (int k = (int)P->levels.size() - 1; k >= 0; --k) {
    TsqrLevel lv = P->levels[k];
    if (k == (int)P->levels.size() - 1)
      for (int s = 0; s < 2; ++s) lv.s[s].Xin = P->wk.C + (size_t)s * r * rcap;
    const int maxn = (lv.nb == 1) ? lv.rows : lv.rows - (lv.nb - 1) * lv.brows;
    const size_t smem = (size_t)std::max(maxn, lv.brows) * rcap * sizeof(double);
    tsqr_apply_kernel<<<dim3(lv.nb, 2), kTsqrThreads, smem, st>>>(lv, r, rcap, P->wk.rank);
    FDE_LAUNCH("tsqr_apply_kernel");
  }
  return FDE_OK;
}

}  // namespace fde
