// 2D step (§4.2, Eq. (sylv-timestepping)):  A_x X + X A_yᵀ = C.
//
// Inner solver S (FP64 or FP32): divide and conquer over the HODLR trees of
// A_x and A_y (the D&C method the Conclusions name for HODLR right-hand
// sides): the block-diagonal parts are solved recursively down to the leaf
// pairs (Bartels–Stewart with precomputed real Schur forms), and on the way up
// every level adds the low-rank correction δX of
//     A δX + δX Bᵀ = -(A_off X0 + X0 B_offᵀ) = G Hᵀ        (rank <= 2k_x + 2k_y)
// solved by factored ADI (the low-rank Sylvester form AX + XB = UVᵀ of §4.2)
// with shifts from the Zolotarev problem on the spectral intervals of the
// level's diagonal blocks.
// Outer loop: iterative refinement in FP64 against the exact structured
// residual R = C - A_x X - X A_yᵀ (Toeplitz products by FFT).
#include <float.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#include "fft_block.cuh"
#include "fft_core.cuh"
#include "fft_df.cuh"
#include "hodlr_internal.cuh"
#include "schur.cuh"

namespace fde {

// =================================================== spectral bounds / shifts
// Row sums and Gershgorin radii of the diagonal block A[lo:hi, lo:hi].
// A is a nonsingular M-matrix (positive diagonal, non-positive off-diagonal
// entries, strictly diagonally dominant; §2.2.1), so every eigenvalue of a
// principal block has real part >= its smallest row sum, and <= max(a_ii + r_i).
static void node_interval(const std::vector<double>& S, const std::vector<double>& dp, const std::vector<double>& dm,
                          double c, double shift, double alpha, int lo, int hi, double* lam_lo, double* lam_hi) {
  // S[k] = Σ_{m<=k} g_m ; S(-1) = 0
  auto Sk = [&](int k) { return k < 0 ? 0.0 : S[k]; };
  double mn = INFINITY, mx = 0.0;
  for (int i = lo; i < hi; ++i) {
    // Σ_{j=lo}^{hi-1} T[i][j] = -Σ_{k=max(i-hi+2,0)}^{i-lo+1} g_k
    const int kmin = std::max(i - hi + 2, 0), kmax = i - lo + 1;
    const double sT = -(Sk(kmax) - Sk(kmin - 1));
    // Σ_{j=lo}^{hi-1} T[j][i] = -Σ_{k=max(lo-i+1,0)}^{hi-i} g_k
    const int kmin2 = std::max(lo - i + 1, 0), kmax2 = hi - i;
    const double sTt = -(Sk(kmax2) - Sk(kmin2 - 1));
    const double rowsum = shift + c * (dp[i] * sT + dm[i] * sTt);
    const double diag = shift + c * alpha * (dp[i] + dm[i]);
    mn = std::min(mn, rowsum);
    mx = std::max(mx, 2.0 * diag - rowsum);
  }
  *lam_lo = mn;
  *lam_hi = mx;
}

// Jacobi elliptic functions by the arithmetic–geometric mean (descending
// Landen transformation; Abramowitz & Stegun 16.4) and K(m) = π / (2 AGM).
// The parameter comes with its complement m1 = 1 - m, formed by the caller
// without cancellation (m close to 1 is the usual case here).
static void jacobi_dn_K(double u, double m, double m1, double* dn, double* K) {
  double a[64], cc[64];
  a[0] = 1.0;
  double b = sqrt(m1);
  cc[0] = sqrt(m);
  int n = 0;
  while (n < 60 && fabs(cc[n]) > 1e-17 * a[n]) {
    a[n + 1] = 0.5 * (a[n] + b);
    cc[n + 1] = 0.5 * (a[n] - b);
    b = sqrt(a[n] * b);
    ++n;
  }
  *K = M_PI / (2.0 * a[n]);
  double phi = ldexp(1.0, n) * a[n] * u, phi_prev = phi;
  for (int i = n; i > 0; --i) {
    phi_prev = phi;
    phi = 0.5 * (phi + asin(cc[i] * sin(phi) / a[i]));
  }
  *dn = (n == 0) ? 1.0 : cos(phi) / cos(phi_prev - phi);
}

// Shifts for A X + X Bᵀ = G Hᵀ with spec(A) ⊂ [a, b], spec(B) ⊂ [c, d]
// (all > 0): the Zolotarev problem for E = [a, b] and F = [-d, -c] is mapped
// by a Möbius transform onto [k, 1] ∪ [-1, -k], whose optimal zeros are
// dn((2j-1)K'/(2J), k') (Wachspress); alpha_j -> zeros near E, beta_j -> poles near F.
static void zolotarev_shifts(double a, double b, double c, double d, int J, std::vector<double>& al,
                             std::vector<double>& be) {
  // cross ratio m >= 1 and m - 1, formed without cancellation; k is the
  // smaller root of k² - 2(2m - 1)k + 1 = 0, as 1 / (the larger one)
  const double m = (a + d) * (b + c) / ((a + c) * (b + d));
  const double m1 = (b - a) * (d - c) / ((a + c) * (b + d));
  double k = 1.0 / (2.0 * m - 1.0 + 2.0 * sqrt(m * m1));
  k = std::min(std::max(k, 1e-300), 1.0 - 1e-15);
  const double mp = 1.0 - k * k, mp1 = k * k;  // parameter k'² and its complement k²
  double K, dn;
  jacobi_dn_K(0.0, mp, mp1, &dn, &K);
  // Möbius w -> z with k -> a, 1 -> b, -1 -> -d:  z = (A w + B)/(C w + 1)
  // rows: A w + B - z C w = z
  const double W[3] = {k, 1.0, -1.0}, Z[3] = {a, b, -d};
  double M[3][4];
  for (int i = 0; i < 3; ++i) {
    M[i][0] = W[i];
    M[i][1] = 1.0;
    M[i][2] = -Z[i] * W[i];
    M[i][3] = Z[i];
  }
  for (int col = 0; col < 3; ++col) {  // Gauss–Jordan with pivoting
    int pv = col;
    for (int i = col + 1; i < 3; ++i)
      if (fabs(M[i][col]) > fabs(M[pv][col])) pv = i;
    for (int j = 0; j < 4; ++j) std::swap(M[col][j], M[pv][j]);
    for (int i = 0; i < 3; ++i)
      if (i != col) {
        const double f = M[i][col] / M[col][col];
        for (int j = 0; j < 4; ++j) M[i][j] -= f * M[col][j];
      }
  }
  const double A_ = M[0][3] / M[0][0], B_ = M[1][3] / M[1][1], C_ = M[2][3] / M[2][2];
  auto inv = [&](double w) { return (A_ * w + B_) / (C_ * w + 1.0); };
  al.resize(J);
  be.resize(J);
  for (int j = 0; j < J; ++j) {
    double dnj, Kd;
    jacobi_dn_K((2.0 * (j + 1) - 1.0) * K / (2.0 * J), mp, mp1, &dnj, &Kd);
    al[j] = inv(dnj);
    be[j] = inv(-dnj);
  }
}

// max_E |r| / min_F |r| for r(z) = Π (z - alpha_j)/(z - beta_j), on log grids.
static double zolotarev_bound(const std::vector<double>& al, const std::vector<double>& be, double a, double b,
                              double c, double d) {
  const int G = 400;
  double num = 0.0, den = INFINITY;
  for (int i = 0; i < G; ++i) {
    const double z = a * pow(b / a, i / (double)(G - 1));
    const double w = -c * pow(d / c, i / (double)(G - 1));
    double rz = 1.0, rw = 1.0;
    for (size_t j = 0; j < al.size(); ++j) {
      rz *= fabs((z - al[j]) / (z - be[j]));
      rw *= fabs((w - al[j]) / (w - be[j]));
    }
    num = std::max(num, rz);
    den = std::min(den, rw);
  }
  return num / den;
}

// Smallest J <= jmax whose ratio (zolotarev_bound) is <= target, or jmax when
// none is; its shifts in al / be and its ratio in *ratio.
static int select_shifts(double a, double b, double c, double d, double target, int jmax, std::vector<double>& al,
                         std::vector<double>& be, double* ratio) {
  double r = INFINITY;
  int J = 1;
  for (; J <= jmax; ++J) {
    zolotarev_shifts(a, b, c, d, J, al, be);
    r = zolotarev_bound(al, be, a, b, c, d);
    if (r <= target) break;
  }
  if (J > jmax) J = jmax;  // al / be still hold the jmax shifts, r their ratio
  *ratio = r;
  return J;
}

static bool host_readable(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // no device, or a plain host pointer
    return true;
  }
  return at.type != cudaMemoryTypeDevice;
}

// ================================================================ kernels
template <typename T>
__global__ void scale_sub_kernel(T* __restrict__ Z, T* __restrict__ G, size_t n, T cj) {
  // Z <- cj Z ; G <- G - Z
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T z = cj * Z[i];
    Z[i] = z;
    G[i] -= z;
  }
}
template <typename T>
__global__ void axpy_kernel(T* __restrict__ Y, const T* __restrict__ X, size_t n, T a) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    Y[i] += a * X[i];
}
// One fADI step's factor updates for both sides (same element count):
//   Z <- cj Z ; G <- G - Z ; H <- H - cj W
template <typename T>
__global__ void fadi_update_kernel(T* __restrict__ Z, T* __restrict__ G, T* __restrict__ H, const T* __restrict__ W,
                                   size_t n, T cj) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T z = cj * Z[i];
    Z[i] = z;
    G[i] -= z;
    H[i] -= cj * W[i];
  }
}
constexpr int kSumBlocks = 152 * 32;   // the largest grid of grid_for
static int grid_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, kSumBlocks); }

// Deterministic grid-wide sums (the refinement's stop test and its choice of
// residual update read them, so they must not depend on the order in which
// blocks finish).  Each block writes its NV block sums to part[block][v]; the
// last block to arrive (counter *count) adds the partial sums in block order
// — a fixed sequence per thread, then a fixed tree — writes acc[v] and resets
// the counter for the next launch.
template <int NV>
__device__ void grid_sums(double (&v)[NV], double* __restrict__ part, unsigned int* count, double* acc) {
  __shared__ double sh[32];
  __shared__ bool last;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = block_sum(v[i], sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) part[(size_t)blockIdx.x * NV + i] = v[i];
    __threadfence();
    last = atomicAdd(count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double t = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) t += __ldcg(part + (size_t)b * NV + i);
    t = block_sum(t, sh);
    if (threadIdx.x == 0) acc[i] = t;
  }
  if (threadIdx.x == 0) *count = 0u;
}
// X64 += (double) D ; sums of |D|^2 and |X64|^2 into acc[0], acc[1]
template <typename T>
__global__ void refine_update_kernel(double* __restrict__ X, const T* __restrict__ D, size_t n, double* acc,
                                     double* part, unsigned int* count) {
  double s[2] = {0.0, 0.0};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double d = (double)D[i];
    const double x = X[i] + d;
    X[i] = x;
    s[0] += d * d;
    s[1] += x * x;
  }
  grid_sums<2>(s, part, count, acc);
}
// acc[0] = |X|^2
__global__ void sumsq_kernel(const double* __restrict__ X, size_t n, double* acc, double* part, unsigned int* count) {
  double s[1] = {0.0};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s[0] += X[i] * X[i];
  grid_sums<1>(s, part, count, acc);
}
// R <- C - Cprev + R  (residual of the previous solution for the new C)
__global__ void shift_residual_kernel(const double* __restrict__ C, const double* __restrict__ Cp, double* __restrict__ R,
                                      size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    R[i] = C[i] - Cp[i] + R[i];
}
// Linear predictor for a time step from the two previous solutions:
//   X <- 2 X_n - X_{n-1};  R <- C - A(X) = C - 2 (C_n - R_n) + (C_{n-1} - R_{n-1}),
// exact because A X_k = C_k - R_k; the history then moves one step.
__global__ void predict_kernel(const double* __restrict__ C, const double* __restrict__ Cn, double* __restrict__ X,
                               double* __restrict__ R, double* __restrict__ Xp, double* __restrict__ Cp,
                               double* __restrict__ Rp, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double x = X[i], r = R[i], cn = Cn[i];
    X[i] = 2.0 * x - Xp[i];
    R[i] = C[i] - 2.0 * (cn - r) + (Cp[i] - Rp[i]);
    Xp[i] = x;
    Cp[i] = cn;
    Rp[i] = r;
  }
}
// first step of a history: R <- C - Cn + R (as shift_residual) and save (X, Cn, R_n)
__global__ void shift_save_kernel(const double* __restrict__ C, const double* __restrict__ Cn,
                                  const double* __restrict__ X, double* __restrict__ R, double* __restrict__ Xp,
                                  double* __restrict__ Cp, double* __restrict__ Rp, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double r = R[i], cn = Cn[i];
    Xp[i] = X[i];
    Cp[i] = cn;
    Rp[i] = r;
    R[i] = C[i] - cn + r;
  }
}
__global__ void nonfinite_kernel(const double* __restrict__ X, size_t n, int* bad) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(X[i])) atomicExch(bad, 1);
}

// 32x32 tiled transpose of an N x N matrix (ld N):  Y = Xᵀ, or Y -= Xᵀ
template <typename T>
__global__ void transpose_kernel(const T* __restrict__ X, T* __restrict__ Y, int N, int subtract) {
  __shared__ T tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int r = bx + threadIdx.x, c = by + j;
    if (r < N && c < N) tile[j][threadIdx.x] = X[r + (size_t)c * N];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int r = by + threadIdx.x, c = bx + j;
    if (r < N && c < N) {
      const T v = tile[threadIdx.x][j];
      if (subtract)
        Y[r + (size_t)c * N] -= v;
      else
        Y[r + (size_t)c * N] = v;
    }
  }
}

// ------------------------------------------------------------- FFT (FP64)
// Leaves above this many rows are cut into diagonal blocks of about
// kTrsylPart rows (a cut never splits a 2 x 2 block) for the FP32 leaf
// Sylvester solves, solved as a block Bartels–Stewart wavefront: one launch
// per anti-diagonal of the block grid of every leaf pair, each block first
// subtracting its coupling with the blocks solved before it.  A block of at
// most 32 rows is one warp, whose dependency chain per column has no barrier.
constexpr int kTrsylSplit = 64;
constexpr int kTrsylPart = 32;
// ... when there are at least this many leaf pairs: with fewer, the split
// launches leave most SMs idle and the dependent rounds cost more than they
// save (leaf 128 at N = 1024, 64 pairs).
constexpr int kTrsylSplitMinPairs = 512;

// Threads of the residual's FFT kernels (radix-8 passes: P / 8 butterflies).
constexpr int kFftThreads = 512;

// Columns j0 = 2b, j1 = 2b+1 of X (N x ncols): Y = A X (mode 0) or
// Y = C - A X (mode 1), A = s I + c (D_+ T + D_- Tᵀ) applied by FFT:
//   (T x)_i  = -(g * x)[i+1]          (linear convolution, Eq. (toeplitz_FD))
//   (Tᵀx)_i  = -(g ⋆ x)[i-1]          (correlation = conj(ĝ) in frequency)
// Two real columns share one complex transform (x_0 + i x_1).  Ghat and the
// saved transform Xh are in the digit-reversed order of fft_forward;
// cp[i] = c d_+(i) / P and cm[i] = c d_-(i) / P (the inverse transforms are
// not divided by P).
__global__ void __launch_bounds__(kFftThreads) fd_fft_apply_kernel(const double* __restrict__ X, int ncols,
                                                                  const double* __restrict__ Cm,
                                                                  double* __restrict__ Y,
                                                                  const double2* __restrict__ Ghat,
                                                                  const double2* __restrict__ tw, int P, int logP,
                                                                  const double* __restrict__ cp,
                                                                  const double* __restrict__ cm, double shift, int N,
                                                                  double2* __restrict__ scratch, int mode) {
  extern __shared__ double2 buf[];
  const int j0 = 2 * blockIdx.x, j1 = j0 + 1;
  const bool has1 = j1 < ncols;
  const double* x0 = X + (size_t)j0 * N;
  const double* x1 = X + (size_t)j1 * N;
  double2* Xh = scratch + (size_t)blockIdx.x * P;
  for (int n = threadIdx.x; n < P; n += blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    if (n < N) v = make_double2(x0[n], has1 ? x1[n] : 0.0);
    buf[fft_pad(n)] = v;
  }
  __syncthreads();
  fft_forward<ArF64>(buf, logP, tw);
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    const double2 v = buf[fft_pad(k)];
    Xh[k] = v;
    buf[fft_pad(k)] = ArF64::mul(v, Ghat[k]);
  }
  __syncthreads();
  fft_inverse<ArF64>(buf, logP, tw);
  double* y0 = Y + (size_t)j0 * N;
  double* y1 = Y + (size_t)j1 * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double2 tx = buf[fft_pad(i + 1)];
    const double ci = cp[i];
    y0[i] = fma(-ci, tx.x, shift * x0[i]);
    if (has1) y1[i] = fma(-ci, tx.y, shift * x1[i]);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < P; k += blockDim.x) buf[fft_pad(k)] = ArF64::mul(Xh[k], ArF64::conj(Ghat[k]));
  __syncthreads();
  fft_inverse<ArF64>(buf, logP, tw);
  const double* c0 = Cm ? Cm + (size_t)j0 * N : nullptr;
  const double* c1 = Cm ? Cm + (size_t)j1 * N : nullptr;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double2 ttx = buf[fft_pad((i - 1 + P) & (P - 1))];
    const double ci = cm[i];
    double v0 = fma(-ci, ttx.x, y0[i]);
    if (mode == 1) v0 = c0[i] - v0;
    y0[i] = v0;
    if (has1) {
      double v1 = fma(-ci, ttx.y, y1[i]);
      if (mode == 1) v1 = c1[i] - v1;
      y1[i] = v1;
    }
  }
}

// Row coefficients of the FFT products: c d_±(i) / P in FP64 and as
// double-float pairs (the inverse transforms leave a factor P).
__global__ void fft_coef_kernel(const double* __restrict__ dp, const double* __restrict__ dm, double c, double invP,
                                int N, double* cp, double* cm, float2* cp_df, float2* cm_df) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const double a = c * dp[i] * invP, b = c * dm[i] * invP;
    cp[i] = a;
    cm[i] = b;
    cp_df[i] = df::split_double(a);
    cm_df[i] = df::split_double(b);
  }
}

// spectrum of the zero-padded weights g_0..g_N (one transform), in the
// digit-reversed order of fft_forward
__global__ void __launch_bounds__(kFftThreads) ghat_kernel(const double* __restrict__ g, int N,
                                                          const double2* __restrict__ tw, int P, int logP,
                                                          double2* Ghat) {
  extern __shared__ double2 buf[];
  for (int n = threadIdx.x; n < P; n += blockDim.x) buf[fft_pad(n)] = make_double2(n <= N ? g[n] : 0.0, 0.0);
  __syncthreads();
  fft_forward<ArF64>(buf, logP, tw);
  for (int k = threadIdx.x; k < P; k += blockDim.x) Ghat[k] = buf[fft_pad(k)];
}

// Spans of the nodes of one level.
struct NodeSpan {
  int lo, n;
};
// R[lo_p + i][i] = 1 for node p (a block-diagonal identity slab N x smax)
__global__ void slab_diag_kernel(const NodeSpan* __restrict__ nodes, int nn, double* R, int N) {
  const NodeSpan nd = nodes[blockIdx.x];
  for (int i = threadIdx.x; i < nd.n; i += blockDim.x) R[(nd.lo + i) + (size_t)i * N] = 1.0;
  (void)nn;
}
// M_p[(j smax + m) + col (J smax)] = scale * P[lo_p + m][col]  and  R -= cj P
__global__ void rational_step_kernel(const NodeSpan* __restrict__ nodes, const double* __restrict__ P, double* R, int N,
                                     int smax, int J, int j, double scale, double cj, double* M) {
  const NodeSpan nd = nodes[blockIdx.y];
  const size_t ldm = (size_t)J * smax;
  double* Mp = M + (size_t)blockIdx.y * ldm * smax;
  const size_t total = (size_t)nd.n * smax;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(e % nd.n), col = (int)(e / nd.n);
    const size_t gi = (size_t)(nd.lo + m) + (size_t)col * N;
    const double pv = P[gi];
    Mp[(size_t)j * smax + m + (size_t)col * ldm] = scale * pv;
    R[gi] -= cj * pv;
  }
}

// Zero-padding masks for the constant parts of the fADI right-hand sides:
// dst[rows of node, col0 + 0..K) = U masked to child-1 rows, [col0+K, col0+2K) masked to child-2 rows.
template <typename T>
struct MaskJob {
  const T* U;   // level factor, ld N
  T* dst;       // ld N
  int lo, mid, hi, K;
  T scale;
};
template <typename T>
__global__ void mask_copy_kernel(const MaskJob<T>* __restrict__ jobs, int N) {
  const MaskJob<T> jb = jobs[blockIdx.x];
  const int len = jb.hi - jb.lo;
  for (int e = threadIdx.x; e < len * 2 * jb.K; e += blockDim.x) {
    const int r = jb.lo + e % len, cc = e / len;
    const int half = cc / jb.K, kk = cc % jb.K;
    const bool in = (half == 0) ? (r < jb.mid) : (r >= jb.mid);
    jb.dst[r + (size_t)cc * N] = in ? jb.scale * jb.U[r + (size_t)kk * N] : T(0);
  }
}

// =============================================================== solver
template <typename T>
struct LevelSolve {
  int J = 0, Q = 0, ncols = 0;        // shifts, RHS width per pair, N x ncols blocks
  std::vector<double> a, b;           // shifts: (B + a_j I), (A + b_j I)
  T* Gt = nullptr;                    // constant part of G (N x ncols)
  T* Ht = nullptr;                    // constant part of H
  T* G = nullptr;                     // working G, H (N x ncols)
  T* H = nullptr;
  T* Zall = nullptr;                  // J panels of N x ncols
  T* Wall = nullptr;
  std::vector<Plan<T>> plan;          // per shift: both sides' solves, merged launches
  GemmBatch<T> g_rhs_x, g_rhs_y;      // HA (into H) and GB (into G) products with X0
  GemmBatch<T> g_update;              // X += Σ_j Z_j W_jᵀ per pair
  // rational form: Z_j = P_j G_0 with P_j = -c_j (A + b_j)^{-1} Π_{i<j} (I - c_i (A + b_i)^{-1})
  // precomputed per node and stacked over j (rows j*smax + m), same for the B side
  bool rational = false;
  int smax = 0, Kx = 0, Ky = 0;
  T *MA = nullptr, *MB = nullptr;     // 2^l blocks of (J smax) x smax
  T *ZA = nullptr, *WB = nullptr;     // constant parts: MA·GA (J smax x 2Kx), MB·HB (J smax x 2Ky)
  T *Hx = nullptr, *Gy = nullptr;     // X0-dependent RHS factors: N x 2^l 2Kx, N x 2^l 2Ky
  T *ZB = nullptr, *WA = nullptr;     // MA·Gy (J smax x 2^l 2Ky), MB·Hx (J smax x 2^l 2Kx)
  // the two update terms accumulate into the same X tile: separate launches
  GemmBatch<T> r_rhs_h, r_rhs_g, r_apply, r_update, r_update2;
};

template <typename T>
struct Inner {
  cudaGraphExec_t exec = nullptr;     // captured run of the whole inner solve
  size_t graph_kernels = 0;
  T *Cin = nullptr, *W1 = nullptr, *W2 = nullptr, *X = nullptr;
  T *Qx = nullptr, *Sx = nullptr, *Qy = nullptr, *Sy = nullptr;
  GemmBatch<T> g_qxt, g_qy, g_qx, g_qyt;
  // split leaves (sylv_s::trsyl_split): couplings between the diagonal blocks
  //   F12 -= S12 Y22,  F21 -= Y22 R12ᵀ,  F11 -= S12 Y21,  F11 -= Y12 R12ᵀ
  std::vector<LevelSolve<T>> lv;
  std::vector<Fact<T>> facts;         // keeps FP32 demoted factorisations alive
};

// ====================================================== whole-step graphs
// Device-side controller of a refinement loop captured as one CUDA graph per
// time step (FP32 inner solver): the host decisions of sylv_step_impl, taken
// by single-thread kernels from the same accumulators, which set the
// conditional nodes of the graph (a WHILE node over the sweeps, a SWITCH node
// over the residual form of each sweep).
struct StepCtl {
  // configuration (from the host)
  double tol2_update, tol2_relres, incr_tol2;
  int max_sweeps, exact_every, resid_df, f32_last, f32_last_all;
  // incremental-residual chain across steps
  int cyc_streak, cyc_incr, prev_large;
  // the current step
  int in_chain, must_exact, step_incremental, large_first, used_f32, incr_ok, sw, stop;
  double prev_d2;
  // results, accumulated until the host collects them
  int status;             // FDE_OK, FDE_ERR_NUMERIC or FDE_ERR_NOCONV of the first failed step
  int steps, sweeps_total, sweeps_max;
  int kind_count[3];      // residual forms run: exact, double-float, FP32
  double relres_max;
};
enum ResidKind { kResidExact = 0, kResidDF = 1, kResidF32 = 2 };

// Start of a step: a non-finite right-hand side (flag from nonfinite_kernel)
// or an earlier failed step skips the sweeps.
__global__ void ctl_begin_kernel(StepCtl* c, const int* bad, int in_chain, cudaGraphConditionalHandle hloop) {
  if (threadIdx.x != 0) return;
  if (c->status == FDE_OK && *bad) c->status = FDE_ERR_NUMERIC;
  if (c->status != FDE_OK) {
    cudaGraphSetConditional(hloop, 0u);
    return;
  }
  c->in_chain = in_chain;
  if (!in_chain) {
    c->cyc_streak = 0;
    c->cyc_incr = 0;
    c->prev_large = 0;
  }
  const int K = c->exact_every;
  c->must_exact = !in_chain || K <= 2 || !c->resid_df || c->cyc_streak == 1 || c->cyc_incr >= K - 2;
  c->step_incremental = c->large_first = c->used_f32 = 0;
  c->incr_ok = c->resid_df;
  c->sw = 0;
  c->stop = 0;
  c->prev_d2 = -1.0;
  cudaGraphSetConditional(hloop, 1u);
}

// After a sweep's update (acc[0] = ||δ||², acc[1] = ||X||²): the stopping
// test and the form of the residual update (SWITCH value; 3 = none).
__global__ void ctl_solve_kernel(StepCtl* c, const double* acc, cudaGraphConditionalHandle hkind) {
  if (threadIdx.x != 0) return;
  if (c->status != FDE_OK) {
    cudaGraphSetConditional(hkind, 3u);
    return;
  }
  const double a0 = acc[0], a1 = acc[1];
  if (!isfinite(a0) || !isfinite(a1)) {
    c->status = FDE_ERR_NUMERIC;
    cudaGraphSetConditional(hkind, 3u);
    return;
  }
  const double tol2 = c->tol2_update * a1;
  int stop = a0 <= tol2;
  if (!stop && c->prev_d2 > 0.0 && a0 < 0.25 * c->prev_d2) {
    const double rho = sqrt(a0 / c->prev_d2), rest = rho / (1.0 - rho);
    stop = a0 * rest * rest <= tol2;
  }
  if (c->prev_d2 > 0.0 && a0 > 0.01 * c->prev_d2) c->incr_ok = 0;
  c->prev_d2 = a0;
  const int K = c->exact_every;
  int kind = kResidExact;
  if (c->incr_ok) {
    if (c->sw == 0 && c->in_chain && K > 2) {
      const int small = a0 <= c->incr_tol2 * a1;
      if (small && !c->must_exact) c->step_incremental = 1;
      if (!small) c->large_first = 1;
    }
    if (c->sw > 0 || c->step_incremental) {
      const int next_two_exact = K <= 1 || (c->step_incremental && c->cyc_incr + 1 >= K - 2) ||
                                 (c->large_first && c->prev_large && !c->step_incremental);
      kind = (stop && c->f32_last && (next_two_exact || c->f32_last_all)) ? kResidF32 : kResidDF;
      if (kind == kResidF32) c->used_f32 = 1;
    }
  }
  c->stop = stop;
  c->kind_count[kind] += 1;
  cudaGraphSetConditional(hkind, (unsigned)kind);
}

// After the residual (acc[2] = ||R||², acc[4] = ||C||²): the residual stopping
// test, the sweep cap and, at the end of the step, the chain bookkeeping;
// sets the WHILE condition.
__global__ void ctl_resid_kernel(StepCtl* c, const double* acc, cudaGraphConditionalHandle hloop) {
  if (threadIdx.x != 0) return;
  if (c->status != FDE_OK) {
    cudaGraphSetConditional(hloop, 0u);
    return;
  }
  const double a2 = acc[2], a4 = acc[4];
  if (!isfinite(a2)) {
    c->status = FDE_ERR_NUMERIC;
    cudaGraphSetConditional(hloop, 0u);
    return;
  }
  c->sw += 1;
  int stop = c->stop || a2 <= c->tol2_relres * a4;
  if (!stop) {
    const int cap = c->max_sweeps > 1 ? c->max_sweeps : 1;
    if (c->sw >= cap) c->status = FDE_ERR_NOCONV;
    cudaGraphSetConditional(hloop, c->sw >= cap ? 0u : 1u);
    return;
  }
  const int K = c->exact_every;
  c->steps += 1;
  c->sweeps_total += c->sw;
  c->sweeps_max = max(c->sweeps_max, c->sw);
  c->relres_max = fmax(c->relres_max, a4 > 0.0 ? sqrt(a2 / a4) : sqrt(a2));
  if (c->step_incremental) {
    c->cyc_streak = 0;
    c->cyc_incr += 1;
  } else {
    c->cyc_streak = c->cyc_streak < 2 ? c->cyc_streak + 1 : 2;
    if (c->cyc_streak == 2) c->cyc_incr = 0;
  }
  if (c->used_f32 && c->large_first && K > 2) {
    c->cyc_streak = 0;
    c->cyc_incr = K;
  }
  c->prev_large = c->large_first;
  cudaGraphSetConditional(hloop, 0u);
}

}  // namespace fde

using namespace fde;

struct sylv_s {
  cudaStream_t gs = nullptr;          // private stream for graph capture / replay
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  hodlr_s* ax = nullptr;
  hodlr_s* ay = nullptr;
  int prec = 0, N = 0, L = 0, lmax = 0;
  DevPool pool;
  double *Qx = nullptr, *Sx = nullptr, *Qy = nullptr, *Sy = nullptr;  // FP64 leaf Schur forms
  int *d_lo = nullptr, *d_n = nullptr;
  // Leaf Sylvester sub-problems per part (x at [0, nl), y at [nl, 2 nl)):
  // whole leaves, and, when leaves above kTrsylSplit rows are split for the
  // FP32 inner solver, their top and bottom diagonal blocks (the cut moved
  // down by one where it would split a 2 x 2 Schur block).
  struct TrsylPart {
    int *soff = nullptr, *lo = nullptr, *n = nullptr;
    int* rest = nullptr;              // rows of the leaf after the block (blocked leaves)
    int nmax = 0;
  } tp_full;
  bool trsyl_split = false;
  // blocked leaves: tp_part[a] = the block a-th from the bottom of every leaf
  // (n = 0 where a leaf has fewer blocks); one launch per anti-diagonal
  // a + b = d of the (a, b) block grid, with its algorithmic flops
  std::vector<TrsylPart> tp_part;
  std::vector<double> trsyl_step_flops;
  std::vector<Fact<double>> facts64;
  Inner<double> in64;
  Inner<float> in32;
  // residual
  int P = 0, logP = 0;
  double2 *tw = nullptr, *GhX = nullptr, *GhY = nullptr, *fft_scratch = nullptr;
  float4 *tw_df = nullptr, *GhX_df = nullptr, *GhY_df = nullptr;  // double-float copies
  // row coefficients c d_±(i) / P of the FFT products per direction (FP64, double-float)
  double *cpx = nullptr, *cmx = nullptr, *cpy = nullptr, *cmy = nullptr;
  float2 *cpx_df = nullptr, *cmx_df = nullptr, *cpy_df = nullptr, *cmy_df = nullptr;
  bool resid_df = false;              // later sweeps update R in double-float (FP32 inner solver)
  bool resid_f32_last = false;        // the last update of a step in plain FP32 (its residual only predicts)
  bool f32_last_all = false;          // ... in every step, not only before two exact steps
  // Exact FP64 residuals after the first sweep on two consecutive steps of
  // every exact_every, double-float updates in between (see sylv_step_impl);
  // exact_every = 1: after the first sweep of every step.
  int exact_every = 16, cyc_streak = 0, cyc_incr = 0;
  bool prev_large = false;            // the previous step's first update was too large to be incremental
  double incr_tol = 1e-2;             // largest ||δ_0|| / ||X|| for an incremental first update
  float2 *tw_f32 = nullptr, *GhX_f32 = nullptr, *GhY_f32 = nullptr;  // FP32 copies
  // N > 4096: block-Toeplitz FFTs (blocks of kFftBlock) instead of one transform per column
  bool block = false;
  int pair_chunk = 0;
  double2 *HbX = nullptr, *HbY = nullptr;
  float4 *HbX_df = nullptr, *HbY_df = nullptr;
  float2 *HbX_f32 = nullptr, *HbY_f32 = nullptr;
  double *R = nullptr, *Xt = nullptr, *Yt = nullptr, *X64 = nullptr, *C64 = nullptr;
  double* acc = nullptr;              // device accumulators
  double* part = nullptr;             // per-block partial sums of the reductions into acc
  unsigned int* count = nullptr;      // their arrival counter (0 between launches)
  unsigned int* tc_count = nullptr;   // the tensor-core GEMM's expired-wait counter (device)
  unsigned int* tc_base = nullptr;    // its value at the start of the current step (device)
  int* d_bad = nullptr;
  sylv_refine_t refine{};
  std::vector<int> J;
  double trsyl_flops = 0.0, fft_flops = 0.0;
  bool R_valid = false;               // R holds C_last - A(X_last) of the last step
  // time-step predictor: history (X, C, R) of the step before the last one
  bool predict = false;
  int hist = 0;                       // 1 when Xp, Cp, Rp are valid
  double *Xp = nullptr, *Cp = nullptr, *Rp = nullptr;
  bool rational = false;              // fADI levels in precomputed rational form
  // bytes the packed constant GEMM operands of the FP32 inner solver may take
  // (FDE_PACK_GB overrides; 0 turns packing off)
  size_t pack_budget = (size_t)32 << 30;
  // operand kind of the tensor-core level products (fADI applications and
  // low-rank updates): kTcDefault (3xTF32) or BF16 (FDE_BF16_REFINE)
  int level_kind = kTcDefault;
  // whole-step graphs (FP32 inner solver): one executable per variant of the
  // step's first part and per (C, C_prev, X) buffers, the controller state and
  // the streams their sweep bodies are captured on
  struct StepGraph {
    int variant = 0;
    const double *C = nullptr, *Cp = nullptr;
    double* X = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t k_pre = 0, k_body = 0, k_br[3] = {0, 0, 0};
  };
  std::vector<StepGraph> sgraphs;
  bool step_graph = false;            // runner steps run as whole-step graphs
  bool ctl_synced = false;            // the device controller holds the chain state
  StepCtl* ctl = nullptr;
  cudaStream_t gs2 = nullptr, gs3 = nullptr;
  std::vector<size_t> graph_pending;  // whole-step graphs launched since the last collect
  ~sylv_s() {
    for (auto& g : sgraphs)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    if (gs2) cudaStreamDestroy(gs2);
    if (gs3) cudaStreamDestroy(gs3);
    if (in64.exec) cudaGraphExecDestroy(in64.exec);
    if (in32.exec) cudaGraphExecDestroy(in32.exec);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (gs) cudaStreamDestroy(gs);
  }
};

namespace fde {

template <typename T>
static std::vector<T*> level_V(hodlr_s* h);
template <>
std::vector<double*> level_V<double>(hodlr_s* h) {
  return h->V;
}
template <>
std::vector<float*> level_V<float>(hodlr_s* h) {
  return h->V32;
}
template <typename T>
static std::vector<T*> level_U(hodlr_s* h);
template <>
std::vector<double*> level_U<double>(hodlr_s* h) {
  return h->U;
}
template <>
std::vector<float*> level_U<float>(hodlr_s* h) {
  return h->U32;
}

template <typename T>
static fde_status convert_buf(const double* src, T** dst, size_t n, DevPool& pool, cudaStream_t st) {
  FDE_TRY(pool.alloc(dst, n));
  if (sizeof(T) == sizeof(double)) {
    FDE_CUDA(cudaMemcpyAsync((void*)*dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  } else {
    FDE_TRY((convert<double, float>(src, (float*)*dst, n, st)));
  }
  return FDE_OK;
}

// Rational-form fADI level (see LevelSolve): forms, in FP64 with the shifted
// HODLR factorisations, the stacked operators of both sides and the constant
// right-hand-side parts, converts them to T and records the four per-step
// batches (RHS products, operator application, low-rank update).
template <typename T>
static fde_status build_level_rational(sylv_s* S, Inner<T>& in, int l, const std::vector<Fact<double>*>& FA,
                                       const std::vector<Fact<double>*>& FB, const std::vector<double>& a,
                                       const std::vector<double>& b, cudaStream_t st) {
  hodlr_s* ax = S->ax;
  hodlr_s* ay = S->ay;
  const Tree& tr = ax->tree;
  const int N = S->N, nn = 1 << l, J = (int)a.size();
  LevelSolve<T>& ls = in.lv[l];
  DevPool& pool = S->pool;
  DevPool scratch;
  ls.rational = true;
  ls.J = J;
  ls.Kx = ax->K[l];
  ls.Ky = ay->K[l];
  const int Kx = ls.Kx, Ky = ls.Ky;
  int smax = 0;
  std::vector<NodeSpan> nx(nn), ny(nn);
  for (int p = 0; p < nn; ++p) {
    const int id = tr.id(l, p);
    nx[p] = {tr.lo[id], tr.hi[id] - tr.lo[id]};
    ny[p] = {ay->tree.lo[id], ay->tree.hi[id] - ay->tree.lo[id]};
    smax = std::max(smax, std::max(nx[p].n, ny[p].n));
  }
  ls.smax = smax;
  const size_t ldm = (size_t)J * smax;  // leading dimension of stacked blocks
  const size_t mblk = ldm * smax;        // one node's stacked operator
  NodeSpan *dnx, *dny;
  FDE_TRY(scratch.alloc(&dnx, nn));
  FDE_TRY(scratch.alloc(&dny, nn));
  FDE_CUDA(cudaMemcpy(dnx, nx.data(), nn * sizeof(NodeSpan), cudaMemcpyHostToDevice));
  FDE_CUDA(cudaMemcpy(dny, ny.data(), nn * sizeof(NodeSpan), cudaMemcpyHostToDevice));
  double *R, *P, *M64, *zb, *wb;
  FDE_TRY(scratch.alloc(&R, (size_t)N * smax));
  FDE_TRY(scratch.alloc(&P, (size_t)N * smax));
  FDE_TRY(scratch.alloc(&M64, nn * mblk));
  const size_t zel = std::max(solve_scratch_elems(ax, smax, l), solve_scratch_elems(ay, smax, l));
  FDE_TRY(scratch.alloc(&zb, zel));
  FDE_TRY(scratch.alloc(&wb, zel));
  FDE_TRY(pool.alloc(&ls.MA, nn * mblk));
  FDE_TRY(pool.alloc(&ls.MB, nn * mblk));
  for (int side = 0; side < 2; ++side) {
    hodlr_s* h = side == 0 ? ax : ay;
    const NodeSpan* dn = side == 0 ? dnx : dny;
    FDE_CUDA(cudaMemsetAsync(R, 0, (size_t)N * smax * sizeof(double), st));
    FDE_CUDA(cudaMemsetAsync(M64, 0, nn * mblk * sizeof(double), st));
    slab_diag_kernel<<<nn, 256, 0, st>>>(dn, nn, R, N);
    FDE_LAUNCH("slab_diag_kernel");
    for (int j = 0; j < J; ++j) {
      const double cj = a[j] + b[j];
      Plan<double> pl;
      FDE_TRY(build_solve_plan<double>(h, side == 0 ? *FA[j] : *FB[j], h->V, R, N, P, N, smax, l, nullptr, zb, wb,
                                       scratch, &pl, st));
      FDE_TRY(plan_run(pl, st));
      // side A keeps -c_j P_j (the step scale and the sign of G_0 folded in), side B keeps P_j
      dim3 grid((unsigned)std::min<size_t>(((size_t)smax * smax + 255) / 256, 1024), nn);
      rational_step_kernel<<<grid, 256, 0, st>>>(dn, P, R, N, smax, J, j, side == 0 ? -cj : 1.0, cj, M64);
      FDE_LAUNCH("rational_step_kernel");
      FDE_CUDA(cudaStreamSynchronize(st));
    }
    T* dst = side == 0 ? ls.MA : ls.MB;
    if (sizeof(T) == sizeof(double))
      FDE_CUDA(cudaMemcpyAsync((void*)dst, M64, nn * mblk * sizeof(double), cudaMemcpyDeviceToDevice, st));
    else
      FDE_TRY((convert<double, float>(M64, (float*)dst, nn * mblk, st)));
    // constant right-hand-side parts: ZA_p = MA_p [U^x|c1, U^x|c2],  WB_q = MB_q [U^y|c1', U^y|c2']
    const int K = side == 0 ? Kx : Ky;
    double* U2 = P;  // reuse as an N x 2K slab
    std::vector<MaskJob<double>> jobs;
    for (int p = 0; p < nn; ++p) {
      const int id = h->tree.id(l, p);
      const int lo = h->tree.lo[id], hi = h->tree.hi[id], mid = lo + (hi - lo) / 2;
      jobs.push_back({h->U[l], U2, lo, mid, hi, K, 1.0});
    }
    MaskJob<double>* dj;
    FDE_TRY(scratch.alloc(&dj, jobs.size()));
    FDE_CUDA(cudaMemcpy(dj, jobs.data(), jobs.size() * sizeof(MaskJob<double>), cudaMemcpyHostToDevice));
    mask_copy_kernel<double><<<nn, 256, 0, st>>>(dj, N);
    FDE_LAUNCH("mask_copy_kernel");
    double* C64;
    FDE_TRY(scratch.alloc(&C64, nn * ldm * 2 * K));
    std::vector<GemmDesc<double>> dd;
    for (int p = 0; p < nn; ++p)
      dd.push_back({M64 + p * mblk, U2 + (side == 0 ? nx[p].lo : ny[p].lo), C64 + p * ldm * 2 * K, (int)ldm, 2 * K,
                    side == 0 ? nx[p].n : ny[p].n, (int)ldm, N, (int)ldm});
    GemmBatch<double> gbd;
    FDE_TRY(gemm_batch_upload(scratch, dd, false, false, 1.0, 0.0, &gbd, st));
    FDE_TRY(gemm_batch_run(gbd, st));
    T** cdst = side == 0 ? &ls.ZA : &ls.WB;
    FDE_TRY(pool.alloc(cdst, nn * ldm * 2 * K));
    if (sizeof(T) == sizeof(double))
      FDE_CUDA(cudaMemcpyAsync((void*)*cdst, C64, nn * ldm * 2 * K * sizeof(double), cudaMemcpyDeviceToDevice, st));
    else
      FDE_TRY((convert<double, float>(C64, (float*)*cdst, nn * ldm * 2 * K, st)));
    FDE_CUDA(cudaStreamSynchronize(st));
  }
  // per-step buffers and batches
  FDE_TRY(pool.alloc(&ls.Hx, (size_t)N * nn * 2 * Kx));
  FDE_TRY(pool.alloc(&ls.Gy, (size_t)N * nn * 2 * Ky));
  FDE_TRY(pool.alloc(&ls.ZB, nn * ldm * nn * 2 * Ky));
  FDE_TRY(pool.alloc(&ls.WA, nn * ldm * nn * 2 * Kx));
  std::vector<T*> Vx = level_V<T>(ax), Vy = level_V<T>(ay);
  std::vector<GemmDesc<T>> dh, dg, dap, dup, dup2;
  for (int p = 0; p < nn; ++p) {
    const int lo = nx[p].lo, sp = nx[p].n, mid = lo + sp / 2, hi = lo + sp;
    for (int q = 0; q < nn; ++q) {
      const int loy = ny[q].lo, tq = ny[q].n, midy = loy + tq / 2, hiy = loy + tq;
      // Hx[q rows, p block] = [X0[c2_p, q cols]ᵀ V^x[c2_p], X0[c1_p, q cols]ᵀ V^x[c1_p]]
      T* Hb = ls.Hx + loy + (size_t)(p * 2 * Kx) * N;
      dh.push_back({in.X + mid + (size_t)loy * N, Vx[l] + mid, Hb, tq, Kx, hi - mid, N, N, N});
      dh.push_back({in.X + lo + (size_t)loy * N, Vx[l] + lo, Hb + (size_t)Kx * N, tq, Kx, mid - lo, N, N, N});
      // Gy[p rows, q block] = [X0[p rows, c2'_q] V^y[c2'_q], X0[p rows, c1'_q] V^y[c1'_q]]
      T* Gb = ls.Gy + lo + (size_t)(q * 2 * Ky) * N;
      dg.push_back({in.X + lo + (size_t)midy * N, Vy[l] + midy, Gb, sp, Ky, hiy - midy, N, N, N});
      dg.push_back({in.X + lo + (size_t)loy * N, Vy[l] + loy, Gb + (size_t)Ky * N, sp, Ky, midy - loy, N, N, N});
      // X_pq += Σ_j ZA_p,j WA_q,j[p block]ᵀ + ZB_p,j[q block] WB_q,jᵀ   (k = (j, c), two-level)
      GemmDesc<T> u1{ls.ZA + p * ldm * 2 * Kx, ls.WA + q * ldm * nn * 2 * Kx + (size_t)(p * 2 * Kx) * ldm,
                     in.X + lo + (size_t)loy * N, sp, tq, J * 2 * Kx, (int)ldm, (int)ldm, N};
      u1.kblk = 2 * Kx;
      u1.kstr = smax;
      GemmDesc<T> u2{ls.ZB + p * ldm * nn * 2 * Ky + (size_t)(q * 2 * Ky) * ldm, ls.WB + q * ldm * 2 * Ky,
                     in.X + lo + (size_t)loy * N, sp, tq, J * 2 * Ky, (int)ldm, (int)ldm, N};
      u2.kblk = 2 * Ky;
      u2.kstr = smax;
      dup.push_back(u1);
      dup2.push_back(u2);
    }
    // ZB_p = MA_p Gy[p rows] (x node p);  WA_p = MB_p Hx[p rows] (y node p)
    dap.push_back({ls.MA + p * mblk, ls.Gy + lo, ls.ZB + p * ldm * nn * 2 * Ky, (int)ldm, nn * 2 * Ky, sp, (int)ldm,
                   N, (int)ldm});
    dap.push_back({ls.MB + p * mblk, ls.Hx + ny[p].lo, ls.WA + p * ldm * nn * 2 * Kx, (int)ldm, nn * 2 * Kx, ny[p].n,
                   (int)ldm, N, (int)ldm});
  }
  FDE_TRY(gemm_batch_upload(pool, dh, true, false, T(1), T(0), &ls.r_rhs_h, st));
  FDE_TRY(gemm_batch_upload(pool, dg, false, false, T(1), T(0), &ls.r_rhs_g, st));
  FDE_TRY(gemm_batch_upload(pool, dap, false, false, T(1), T(0), &ls.r_apply, st));
  FDE_TRY(gemm_batch_upload(pool, dup, false, true, T(1), T(1), &ls.r_update, st));
  FDE_TRY(gemm_batch_upload(pool, dup2, false, true, T(1), T(1), &ls.r_update2, st));
  if constexpr (sizeof(T) == sizeof(float)) {
    // operand kind of the level products (BF16 for FDE_BF16_REFINE), set
    // before packing: the packed tiles are in that kind's format
    ls.r_apply.kind = ls.r_update.kind = ls.r_update2.kind = S->level_kind;
    // the stacked resolvents and the constant update factors never change:
    // pack them for the tensor cores (operator A of the application, ZA of
    // the first update, WB of the second).  The other operand of each (the
    // thin X0-dependent factors, read by every tile of the tall or wide
    // constant one) is repacked before every launch, so that the kernel only
    // issues bulk copies (FDE_REPACK=0: converted by the loaders instead)
    bool rp = true;
    if (const char* e = getenv("FDE_REPACK"))
      if (!strcmp(e, "0")) rp = false;
    // the right-hand-side factors X0ᵀ V, X0 U: the thin constant factor packed,
    // so that these long-k products run on the tensor cores instead of the
    // skinny FP32 kernel (FDE_PACK_RHS=0 keeps them there)
    bool prhs = true;
    if (const char* e = getenv("FDE_PACK_RHS"))
      if (!strcmp(e, "0")) prhs = false;
    if (prhs) {
      FDE_TRY(gemm_batch_pack(pool, reinterpret_cast<GemmBatch<float>*>(&ls.r_rhs_h), false, true, &S->pack_budget,
                              st));
      FDE_TRY(gemm_batch_pack(pool, reinterpret_cast<GemmBatch<float>*>(&ls.r_rhs_g), false, true, &S->pack_budget,
                              st));
    }
    FDE_TRY(gemm_batch_pack(pool, reinterpret_cast<GemmBatch<float>*>(&ls.r_apply), true, rp, &S->pack_budget,
                            st, false, rp));
    FDE_TRY(gemm_batch_pack(pool, reinterpret_cast<GemmBatch<float>*>(&ls.r_update), true, rp, &S->pack_budget,
                            st, false, rp));
    FDE_TRY(gemm_batch_pack(pool, reinterpret_cast<GemmBatch<float>*>(&ls.r_update2), rp, true,
                            &S->pack_budget, st, rp, false));
  }
  FDE_CUDA(cudaStreamSynchronize(st));
  return FDE_OK;
}

struct RationalSrc {
  std::vector<Fact<double>*> FA, FB;  // FP64 shifted factorisations, level order L-1..0
  std::vector<std::vector<double>> a, b;
};

// Build the inner solver of precision T: leaf transforms, fADI levels, plans.
template <typename T>
static fde_status build_inner(sylv_s* S, Inner<T>& in, const std::vector<Fact<T>*>& FA_all,
                              const std::vector<Fact<T>*>& FB_all, cudaStream_t st,
                              const RationalSrc* rsrc = nullptr) {
  hodlr_s* ax = S->ax;
  hodlr_s* ay = S->ay;
  const Tree& tr = ax->tree;
  const int N = S->N, L = S->L, lmax = S->lmax, nl = tr.nleaves();
  DevPool& pool = S->pool;
  const size_t NN = (size_t)N * N, nleaf_el = (size_t)nl * lmax * lmax;
  FDE_TRY(pool.alloc(&in.Cin, NN));
  FDE_TRY(pool.alloc(&in.W1, NN));
  FDE_TRY(pool.alloc(&in.W2, NN));
  FDE_TRY(pool.alloc(&in.X, NN));
  FDE_TRY(convert_buf<T>(S->Qx, &in.Qx, nleaf_el, pool, st));
  FDE_TRY(convert_buf<T>(S->Sx, &in.Sx, nleaf_el, pool, st));
  FDE_TRY(convert_buf<T>(S->Qy, &in.Qy, nleaf_el, pool, st));
  FDE_TRY(convert_buf<T>(S->Sy, &in.Sy, nleaf_el, pool, st));
  // leaf transforms:  W1 = Qxᵀ C,  W2 = W1 Qy,  (trsyl on W2),  W1 = Qx W2,  X = W1 Qyᵀ
  {
    std::vector<GemmDesc<T>> a, b, c, d;
    for (int p = 0; p < nl; ++p) {
      const int lo = ax->leaf_lo[p], n = ax->leaf_n[p];
      const T* Qp = in.Qx + (size_t)p * lmax * lmax;
      a.push_back({Qp, in.Cin + lo, in.W1 + lo, n, N, n, lmax, N, N});
      c.push_back({Qp, in.W2 + lo, in.W1 + lo, n, N, n, lmax, N, N});
      const int loy = ay->leaf_lo[p], ny = ay->leaf_n[p];
      const T* Qq = in.Qy + (size_t)p * lmax * lmax;
      b.push_back({in.W1 + (size_t)loy * N, Qq, in.W2 + (size_t)loy * N, N, ny, ny, N, lmax, N});
      d.push_back({in.W1 + (size_t)loy * N, Qq, in.X + (size_t)loy * N, N, ny, ny, N, lmax, N});
    }
    FDE_TRY(gemm_batch_upload(pool, a, true, false, T(1), T(0), &in.g_qxt, st));
    FDE_TRY(gemm_batch_upload(pool, b, false, false, T(1), T(0), &in.g_qy, st));
    FDE_TRY(gemm_batch_upload(pool, c, false, false, T(1), T(0), &in.g_qx, st));
    FDE_TRY(gemm_batch_upload(pool, d, false, true, T(1), T(0), &in.g_qyt, st));
    if constexpr (sizeof(T) == sizeof(float)) {
      // the leaf Schur bases are constant operands
      FDE_TRY(gemm_batch_pack(pool, reinterpret_cast<GemmBatch<float>*>(&in.g_qxt), true, false, &S->pack_budget,
                              st));
      FDE_TRY(gemm_batch_pack(pool, reinterpret_cast<GemmBatch<float>*>(&in.g_qx), true, false, &S->pack_budget,
                              st));
      FDE_TRY(gemm_batch_pack(pool, reinterpret_cast<GemmBatch<float>*>(&in.g_qy), false, true, &S->pack_budget,
                              st));
      FDE_TRY(gemm_batch_pack(pool, reinterpret_cast<GemmBatch<float>*>(&in.g_qyt), false, true, &S->pack_budget,
                              st));
    }
  }
  in.lv.resize(L);
  std::vector<T*> Vx = level_V<T>(ax), Vy = level_V<T>(ay), Ux = level_U<T>(ax), Uy = level_U<T>(ay);
  size_t fi = 0;
  if (rsrc) {
    size_t off = 0;
    for (int l = L - 1; l >= 0; --l) {
      const int J = S->J[l];
      std::vector<Fact<double>*> fa(rsrc->FA.begin() + off, rsrc->FA.begin() + off + J);
      std::vector<Fact<double>*> fb(rsrc->FB.begin() + off, rsrc->FB.begin() + off + J);
      FDE_TRY(build_level_rational<T>(S, in, l, fa, fb, rsrc->a[l], rsrc->b[l], st));
      off += J;
    }
    FDE_CUDA(cudaStreamSynchronize(st));
    return FDE_OK;
  }
  for (int l = L - 1; l >= 0; --l) {
    LevelSolve<T>& ls = in.lv[l];
    const int Kx = ax->K[l], Ky = ay->K[l], Qw = 2 * Kx + 2 * Ky, nn = 1 << l;
    ls.J = S->J[l];
    ls.Q = Qw;
    ls.ncols = nn * Qw;
    const size_t blk = (size_t)N * ls.ncols;
    FDE_TRY(pool.alloc(&ls.Gt, blk));
    FDE_TRY(pool.alloc(&ls.Ht, blk));
    FDE_TRY(pool.alloc(&ls.G, blk));
    FDE_TRY(pool.alloc(&ls.H, blk));
    FDE_TRY(pool.alloc(&ls.Zall, blk * ls.J));
    FDE_TRY(pool.alloc(&ls.Wall, blk * ls.J));
    FDE_CUDA(cudaMemsetAsync(ls.Gt, 0, blk * sizeof(T), st));
    FDE_CUDA(cudaMemsetAsync(ls.Ht, 0, blk * sizeof(T), st));
    // constant parts: G[:, qQ + 0..2Kx) = -[U^x|c1, U^x|c2] ; H[:, pQ + 2Kx..Q) = [U^y|c1', U^y|c2']
    {
      std::vector<MaskJob<T>> jobs;
      for (int p = 0; p < nn; ++p) {
        const int idx = tr.id(l, p);
        const int lo = tr.lo[idx], hi = tr.hi[idx], mid = lo + (hi - lo) / 2;
        const int loy = ay->tree.lo[idx], hiy = ay->tree.hi[idx], midy = loy + (hiy - loy) / 2;
        for (int q = 0; q < nn; ++q) {
          jobs.push_back({Ux[l], ls.Gt + (size_t)(q * Qw) * N, lo, mid, hi, Kx, T(-1)});
          jobs.push_back({Uy[l], ls.Ht + (size_t)(q * Qw + 2 * Kx) * N, loy, midy, hiy, Ky, T(1)});
        }
      }
      // note: for the H template, "q" above runs over the x-node index p' of the column block
      MaskJob<T>* dj;
      FDE_TRY(pool.alloc(&dj, jobs.size()));
      FDE_CUDA(cudaMemcpy(dj, jobs.data(), jobs.size() * sizeof(MaskJob<T>), cudaMemcpyHostToDevice));
      mask_copy_kernel<T><<<(int)jobs.size(), 256, 0, st>>>(dj, N);
      FDE_LAUNCH("mask_copy_kernel");
    }
    // X0-dependent parts (GEMMs on the current X):
    //   H[q rows, pQ + 0..Kx)   = X0[c2_p, q cols]ᵀ V^x[c2_p] ; [Kx, 2Kx) = X0[c1_p, q cols]ᵀ V^x[c1_p]
    //   G[p rows, qQ+2Kx..+Ky)  = -X0[p rows, c2'_q] V^y[c2'_q] ; [.. + Ky, Q) = -X0[p rows, c1'_q] V^y[c1'_q]
    {
      std::vector<GemmDesc<T>> dh, dg, du;
      for (int p = 0; p < nn; ++p) {
        const int idx = tr.id(l, p);
        const int lo = tr.lo[idx], hi = tr.hi[idx], mid = lo + (hi - lo) / 2;
        for (int q = 0; q < nn; ++q) {
          const int idy = ay->tree.id(l, q);
          const int loy = ay->tree.lo[idy], hiy = ay->tree.hi[idy], midy = loy + (hiy - loy) / 2;
          const int tq = hiy - loy, sp = hi - lo;
          T* Hb = ls.H + loy + (size_t)(p * Qw) * N;
          dh.push_back({in.X + mid + (size_t)loy * N, Vx[l] + mid, Hb, tq, Kx, hi - mid, N, N, N});
          dh.push_back({in.X + lo + (size_t)loy * N, Vx[l] + lo, Hb + (size_t)Kx * N, tq, Kx, mid - lo, N, N, N});
          T* Gb = ls.G + lo + (size_t)(q * Qw + 2 * Kx) * N;
          dg.push_back({in.X + lo + (size_t)midy * N, Vy[l] + midy, Gb, sp, Ky, hiy - midy, N, N, N});
          dg.push_back({in.X + lo + (size_t)loy * N, Vy[l] + loy, Gb + (size_t)Ky * N, sp, Ky, midy - loy, N, N, N});
          GemmDesc<T> u{ls.Zall + lo + (size_t)(q * Qw) * N, ls.Wall + loy + (size_t)(p * Qw) * N,
                        in.X + lo + (size_t)loy * N, sp, tq, ls.J * Qw, N, N, N};
          u.kblk = Qw;
          u.kstr = (long long)N * ls.ncols;
          du.push_back(u);
        }
      }
      FDE_TRY(gemm_batch_upload(pool, dh, true, false, T(1), T(0), &ls.g_rhs_x, st));
      FDE_TRY(gemm_batch_upload(pool, dg, false, false, T(-1), T(0), &ls.g_rhs_y, st));
      FDE_TRY(gemm_batch_upload(pool, du, false, true, T(1), T(1), &ls.g_update, st));
    }
    // solve plans per shift: Z_j = (A_p + b_j I)^{-1} G,  W_j = (B_q + a_j I)^{-1} H,
    // the two sides merged step by step into shared launches
    T *zbA, *wbA, *zbB, *wbB;
    FDE_TRY(pool.alloc(&zbA, solve_scratch_elems(ax, ls.ncols, l)));
    FDE_TRY(pool.alloc(&wbA, solve_scratch_elems(ax, ls.ncols, l)));
    FDE_TRY(pool.alloc(&zbB, solve_scratch_elems(ay, ls.ncols, l)));
    FDE_TRY(pool.alloc(&wbB, solve_scratch_elems(ay, ls.ncols, l)));
    ls.plan.resize(ls.J);
    for (int j = 0; j < ls.J; ++j) {
      std::vector<std::vector<HostOp<T>>> specs(2);
      FDE_TRY(build_solve_spec<T>(ax, *FA_all[fi + j], Vx, ls.G, N, ls.Zall + (size_t)j * blk, N, ls.ncols, l,
                                  nullptr, zbA, wbA, &specs[0]));
      FDE_TRY(build_solve_spec<T>(ay, *FB_all[fi + j], Vy, ls.H, N, ls.Wall + (size_t)j * blk, N, ls.ncols, l,
                                  nullptr, zbB, wbB, &specs[1]));
      FDE_TRY(upload_specs<T>(specs, pool, &ls.plan[j], st));
    }
    fi += ls.J;
  }
  FDE_CUDA(cudaStreamSynchronize(st));
  return FDE_OK;
}

// X = S(C): in.Cin -> in.X
template <typename T>
static fde_status run_inner(sylv_s* S, Inner<T>& in, cudaStream_t st) {
  hodlr_s* ax = S->ax;
  hodlr_s* ay = S->ay;
  const int N = S->N, nl = ax->tree.nleaves();
  FDE_TRY(gemm_batch_run(in.g_qxt, st));
  FDE_TRY(gemm_batch_run(in.g_qy, st));
  auto trsyl = [&](const sylv_s::TrsylPart& px, const sylv_s::TrsylPart& py, double flops) {
    const int nmax = px.nmax > py.nmax ? px.nmax : py.nmax;
    return leaf_trsyl<T>(in.Sx, in.Sy, S->lmax, nmax, px.soff, px.lo, px.n, nl, py.soff + nl, py.lo + nl, py.n + nl,
                         nl, in.W2, N, st, flops);
  };
  if (sizeof(T) == sizeof(float) && S->trsyl_split) {
    // block Bartels–Stewart over the blocked leaves: anti-diagonal d holds the
    // blocks (a, b) a-th from the bottom of the row leaf and b-th from the
    // right of the column leaf, a + b = d; they need only blocks of smaller d
    const int nb = (int)S->tp_part.size();
    for (int d = 0; d <= 2 * nb - 2; ++d) {
      TrsylSets sets;
      int nmax = 0;
      for (int a = (d - nb + 1 > 0 ? d - nb + 1 : 0); a <= d && a < nb; ++a) {
        const sylv_s::TrsylPart& px = S->tp_part[a];
        const sylv_s::TrsylPart& py = S->tp_part[d - a];
        if (sets.n == kTrsylMaxSets) {
          set_error("sylv: %d leaf blocks per anti-diagonal (at most %d)", nb, kTrsylMaxSets);
          return FDE_ERR_ARG;
        }
        sets.s[sets.n++] = TrsylSet{px.soff, px.lo, px.n, nl, py.soff + nl, py.lo + nl, py.n + nl, nl * nl,
                                    px.rest, py.rest + nl};
        nmax = std::max(nmax, std::max(px.nmax, py.nmax));
      }
      FDE_TRY(leaf_trsyl_sets<T>(in.Sx, in.Sy, S->lmax, nmax, sets, in.W2, N, st, S->trsyl_step_flops[d]));
    }
  } else {
    FDE_TRY(trsyl(S->tp_full, S->tp_full, S->trsyl_flops));
  }
  FDE_TRY(gemm_batch_run(in.g_qx, st));
  FDE_TRY(gemm_batch_run(in.g_qyt, st));
  for (int l = S->L - 1; l >= 0; --l) {
    LevelSolve<T>& ls = in.lv[l];
    if (ls.rational) {
      FDE_TRY(gemm_batch_run(ls.r_rhs_h, st));
      FDE_TRY(gemm_batch_run(ls.r_rhs_g, st));
      FDE_TRY(gemm_batch_run(ls.r_apply, st));
      FDE_TRY(gemm_batch_run(ls.r_update, st));
      FDE_TRY(gemm_batch_run(ls.r_update2, st));
      continue;
    }
    const size_t blk = (size_t)N * ls.ncols;
    FDE_CUDA(cudaMemcpyAsync(ls.G, ls.Gt, blk * sizeof(T), cudaMemcpyDeviceToDevice, st));
    FDE_CUDA(cudaMemcpyAsync(ls.H, ls.Ht, blk * sizeof(T), cudaMemcpyDeviceToDevice, st));
    FDE_TRY(gemm_batch_run(ls.g_rhs_x, st));
    FDE_TRY(gemm_batch_run(ls.g_rhs_y, st));
    for (int j = 0; j < ls.J; ++j) {
      FDE_TRY(plan_run(ls.plan[j], st));
      const T cj = (T)(ls.a[j] + ls.b[j]);
      T* Zj = ls.Zall + (size_t)j * blk;
      T* Wj = ls.Wall + (size_t)j * blk;
      {
        ProfScope ps("fadi_axpy", st, 7.0 * blk * sizeof(T), 0);
        fadi_update_kernel<T><<<grid_for(blk), 256, 0, st>>>(Zj, ls.G, ls.H, Wj, blk, cj);
        FDE_LAUNCH("fadi_update_kernel");
      }
    }
    FDE_TRY(gemm_batch_run(ls.g_update, st));
  }
  (void)ay;
  return FDE_OK;
}

// Capture run_inner into a CUDA graph (on a private stream) so that each
// replay costs one launch; profiling (per-kernel events) uses the eager path.
template <typename T>
static fde_status capture_inner(sylv_s* S, Inner<T>& in);
template <typename T>
static fde_status inner_solve(sylv_s* S, Inner<T>& in, cudaStream_t st);

// R = C - A_x X - X A_yᵀ (FP64, structured)
static fde_status residual(sylv_s* S, const double* C, const double* X, double* R, cudaStream_t st) {
  hodlr_s* ax = S->ax;
  hodlr_s* ay = S->ay;
  const int N = S->N, P = S->P, lp = S->logP;
  if (S->block) {
    // x direction: R = C - A_x X (columns); y direction: R -= X A_yᵀ (rows, read in place)
    FDE_TRY(block_apply(X, false, 1, N, N, C, R, 1, N, kApplyResidual, ax->g, S->HbX, S->HbX_df, S->HbX_f32, S->tw,
                        S->tw_df, S->tw_f32, kBlockF64, ax->dp, ax->dm, ax->c, ax->p.shift, N, S->fft_scratch,
                        S->pair_chunk, st, S->fft_flops));
    FDE_TRY(block_apply(X, false, N, 1, N, nullptr, R, N, 1, kApplySub, ay->g, S->HbY, S->HbY_df, S->HbY_f32, S->tw,
                        S->tw_df, S->tw_f32, kBlockF64, ay->dp, ay->dm, ay->c, ay->p.shift, N, S->fft_scratch,
                        S->pair_chunk, st, S->fft_flops));
    return FDE_OK;
  }
  const int nb = (N + 1) / 2;
  const size_t smem = (size_t)fft_padded_len(P) * sizeof(double2);
  {
    ProfScope ps("fft_apply", st, S->fft_flops, 1);
    fd_fft_apply_kernel<<<nb, kFftThreads, smem, st>>>(X, N, C, R, S->GhX, S->tw, P, lp, S->cpx, S->cmx,
                                                       ax->p.shift, N, S->fft_scratch, 1);
    FDE_LAUNCH("fd_fft_apply_kernel x");
  }
  dim3 tg(ceil_div(N, 32), ceil_div(N, 32)), tb(32, 8);
  {
    ProfScope ps("transpose", st, 16.0 * N * N, 0);
    transpose_kernel<double><<<tg, tb, 0, st>>>(X, S->Xt, N, 0);
    FDE_LAUNCH("transpose_kernel");
  }
  {
    ProfScope ps("fft_apply", st, S->fft_flops, 1);
    fd_fft_apply_kernel<<<nb, kFftThreads, smem, st>>>(S->Xt, N, nullptr, S->Yt, S->GhY, S->tw, P, lp, S->cpy, S->cmy,
                                                       ay->p.shift, N, S->fft_scratch, 0);
    FDE_LAUNCH("fd_fft_apply_kernel y");
  }
  {
    ProfScope ps("transpose", st, 24.0 * N * N, 0);
    transpose_kernel<double><<<tg, tb, 0, st>>>(S->Yt, R, N, 1);
    FDE_LAUNCH("transpose_kernel");
  }
  return FDE_OK;
}

// Reads the accumulators; FDE_ERR_CUDA if a tensor-core GEMM wait of this step
// ran out (the expired-wait counter moved past the value the step started
// from, tc_base, which sylv_step_impl copies on the stream at its start).
static fde_status read_acc(sylv_s* S, double* h, int n, cudaStream_t st) {
  unsigned int tc[2] = {0u, 0u};
  FDE_CUDA(cudaMemcpyAsync(h, S->acc, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  FDE_CUDA(cudaMemcpyAsync(tc, S->tc_base, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  FDE_CUDA(cudaMemcpyAsync(tc + 1, S->tc_count, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  FDE_CUDA(cudaStreamSynchronize(st));
  if (tc[1] != tc[0]) {
    set_error("sylv_step: a bounded wait of the tensor-core GEMM expired (%u)", tc[1] - tc[0]);
    return FDE_ERR_CUDA;
  }
  return FDE_OK;
}

template <typename T>
static fde_status capture_inner(sylv_s* S, Inner<T>& in) {
  if (!S->gs) {
    FDE_CUDA(cudaStreamCreateWithFlags(&S->gs, cudaStreamNonBlocking));
    FDE_CUDA(cudaEventCreateWithFlags(&S->ev_in, cudaEventDisableTiming));
    FDE_CUDA(cudaEventCreateWithFlags(&S->ev_out, cudaEventDisableTiming));
  }
  cudaGraph_t g = nullptr;
  FDE_CUDA(cudaStreamBeginCapture(S->gs, cudaStreamCaptureModeThreadLocal));
  fde_status s = run_inner<T>(S, in, S->gs);
  cudaError_t e = cudaStreamEndCapture(S->gs, &g);
  if (s != FDE_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();  // a failed capture leaves nothing behind
    if (s != FDE_OK) return s;
    FDE_CUDA(e);
  }
  size_t n = 0;
  FDE_CUDA(cudaGraphGetNodes(g, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  if (n) FDE_CUDA(cudaGraphGetNodes(g, nodes.data(), &n));
  size_t kernels = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    FDE_CUDA(cudaGraphNodeGetType(nd, &t));
    if (t == cudaGraphNodeTypeKernel) ++kernels;
  }
  in.graph_kernels = kernels;
  e = cudaGraphInstantiate(&in.exec, g, 0);
  cudaGraphDestroy(g);
  FDE_CUDA(e);
  return FDE_OK;
}

template <typename T>
static fde_status inner_solve(sylv_s* S, Inner<T>& in, cudaStream_t st) {
  if (!in.exec || prof_enabled()) return run_inner<T>(S, in, st);
  FDE_CUDA(cudaEventRecord(S->ev_in, st));
  FDE_CUDA(cudaStreamWaitEvent(S->gs, S->ev_in, 0));
  FDE_CUDA(cudaGraphLaunch(in.exec, S->gs));
  FDE_CUDA(cudaEventRecord(S->ev_out, S->gs));
  FDE_CUDA(cudaStreamWaitEvent(st, S->ev_out, 0));
  count_launches(in.graph_kernels);
  return FDE_OK;
}

// R -= A_x δ + δ A_yᵀ for the FP32 update δ (the inner solution) in
// double-float FFTs.  The x direction reads δ in place; the y direction works
// on δᵀ (coalesced reads and writes) and subtracts the transpose, except in the
// block-Toeplitz form (N > 4096), which reads both directions through strides.
static fde_status residual_update_df(sylv_s* S, const float* d, cudaStream_t st) {
  hodlr_s* ax = S->ax;
  hodlr_s* ay = S->ay;
  const int N = S->N;
  if (S->block) {
    FDE_TRY(block_apply(d, true, 1, N, N, nullptr, S->R, 1, N, kApplySub, ax->g, S->HbX, S->HbX_df, S->HbX_f32,
                        S->tw, S->tw_df, S->tw_f32, kBlockDF, ax->dp, ax->dm, ax->c, ax->p.shift, N, S->fft_scratch,
                        S->pair_chunk, st, S->fft_flops));
    FDE_TRY(block_apply(d, true, N, 1, N, nullptr, S->R, N, 1, kApplySub, ay->g, S->HbY, S->HbY_df, S->HbY_f32,
                        S->tw, S->tw_df, S->tw_f32, kBlockDF, ay->dp, ay->dm, ay->c, ay->p.shift, N, S->fft_scratch,
                        S->pair_chunk, st, S->fft_flops));
    return FDE_OK;
  }
  float4* scr = reinterpret_cast<float4*>(S->fft_scratch);
  FDE_TRY(fd_apply_sub_df(d, 1, N, N, S->R, 1, N, S->GhX_df, S->tw_df, S->P, S->logP, S->cpx_df, S->cmx_df,
                          ax->p.shift, N, scr, st, S->fft_flops));
  // y direction on δᵀ (coalesced): Yt = A_y δᵀ, R -= Ytᵀ
  float* dT = reinterpret_cast<float*>(S->Xt);
  const dim3 tg(ceil_div(N, 32), ceil_div(N, 32)), tb(32, 8);
  transpose_kernel<float><<<tg, tb, 0, st>>>(d, dT, N, 0);
  FDE_LAUNCH("transpose_kernel");
  FDE_TRY(fd_apply_sub_df(dT, 1, N, N, S->Yt, 1, N, S->GhY_df, S->tw_df, S->P, S->logP, S->cpy_df, S->cmy_df,
                          ay->p.shift, N, scr, st, S->fft_flops, /*set=*/true));
  {
    ProfScope ps("transpose", st, 24.0 * N * N, 0);
    transpose_kernel<double><<<tg, tb, 0, st>>>(S->Yt, S->R, N, 1);
    FDE_LAUNCH("transpose_kernel");
  }
  return FDE_OK;
}

// R -= A_x δ + δ A_yᵀ in plain FP32 FFTs: for the last update of a step, whose
// residual only feeds the next step's predictor.
static fde_status residual_update_f32(sylv_s* S, const float* d, cudaStream_t st) {
  hodlr_s* ax = S->ax;
  hodlr_s* ay = S->ay;
  const int N = S->N;
  if (S->block) {
    FDE_TRY(block_apply(d, true, 1, N, N, nullptr, S->R, 1, N, kApplySub, ax->g, S->HbX, S->HbX_df, S->HbX_f32,
                        S->tw, S->tw_df, S->tw_f32, kBlockF32, ax->dp, ax->dm, ax->c, ax->p.shift, N,
                        S->fft_scratch, S->pair_chunk, st, S->fft_flops));
    FDE_TRY(block_apply(d, true, N, 1, N, nullptr, S->R, N, 1, kApplySub, ay->g, S->HbY, S->HbY_df, S->HbY_f32,
                        S->tw, S->tw_df, S->tw_f32, kBlockF32, ay->dp, ay->dm, ay->c, ay->p.shift, N,
                        S->fft_scratch, S->pair_chunk, st, S->fft_flops));
    return FDE_OK;
  }
  float2* scr = reinterpret_cast<float2*>(S->fft_scratch);
  FDE_TRY(fd_apply_sub_f32(d, 1, N, N, S->R, 1, N, S->GhX_f32, S->tw_f32, S->P, S->logP, S->cpx_df, S->cmx_df,
                           ax->p.shift, N, scr, st, S->fft_flops));
  // y direction on δᵀ, so that reads and writes are coalesced: Yt = A_y δᵀ, R -= Ytᵀ
  float* dT = reinterpret_cast<float*>(S->Xt);
  const dim3 tg(ceil_div(N, 32), ceil_div(N, 32)), tb(32, 8);
  transpose_kernel<float><<<tg, tb, 0, st>>>(d, dT, N, 0);
  FDE_LAUNCH("transpose_kernel");
  FDE_TRY(fd_apply_sub_f32(dT, 1, N, N, S->Yt, 1, N, S->GhY_f32, S->tw_f32, S->P, S->logP, S->cpy_df, S->cmy_df,
                           ay->p.shift, N, scr, st, S->fft_flops, /*set=*/true));
  {
    ProfScope ps("transpose", st, 24.0 * N * N, 0);
    transpose_kernel<double><<<tg, tb, 0, st>>>(S->Yt, S->R, N, 1);
    FDE_LAUNCH("transpose_kernel");
  }
  return FDE_OK;
}

// One refinement sweep, in two halves.  sweep_solve: Cin = (T) R, inner
// solve, X64 += X_T; acc[0] = ||δ||², acc[1] = ||X||².  sweep_residual: the
// new residual of X64, acc[2] = ||R||², as
//  - kResidExact: R = C - A(X64) in FP64;
//  - kResidDF:    R -= A(δ) in double-float (FP32 inner solver), whose error
//                 scales with ||δ||, ~1e-3 ||X|| or less after the first sweep;
//  - kResidF32:   R -= A(δ) in FP32, for the last update of a step: that
//                 residual only seeds the next step's predicted residual, and
//                 the next step's first sweep recomputes R exactly.
template <typename T>
static fde_status sweep_solve(sylv_s* S, Inner<T>& in, double* X64, cudaStream_t st) {
  const size_t NN = (size_t)S->N * S->N;
  if (sizeof(T) == sizeof(double)) {
    FDE_CUDA(cudaMemcpyAsync((void*)in.Cin, S->R, NN * sizeof(double), cudaMemcpyDeviceToDevice, st));
  } else {
    FDE_TRY((convert<double, float>(S->R, (float*)in.Cin, NN, st)));
  }
  FDE_TRY(inner_solve<T>(S, in, st));
  FDE_CUDA(cudaMemsetAsync(S->acc, 0, 3 * sizeof(double), st));
  {
    ProfScope ps("refine", st, (16.0 + sizeof(T)) * NN, 0);
    refine_update_kernel<T><<<grid_for(NN), 256, 0, st>>>(X64, in.X, NN, S->acc, S->part, S->count);
    FDE_LAUNCH("refine_update_kernel");
  }
  return FDE_OK;
}

template <typename T>
static fde_status sweep_residual(sylv_s* S, Inner<T>& in, const double* C, double* X64, int kind, cudaStream_t st) {
  const size_t NN = (size_t)S->N * S->N;
  if (sizeof(T) == sizeof(float) && kind == kResidF32)
    FDE_TRY(residual_update_f32(S, reinterpret_cast<const float*>(in.X), st));
  else if (sizeof(T) == sizeof(float) && kind == kResidDF)
    FDE_TRY(residual_update_df(S, reinterpret_cast<const float*>(in.X), st));
  else
    FDE_TRY(residual(S, C, X64, S->R, st));
  sumsq_kernel<<<grid_for(NN), 256, 0, st>>>(S->R, NN, S->acc + 2, S->part, S->count);
  FDE_LAUNCH("sumsq_kernel");
  return FDE_OK;
}

// Iterative refinement (FP64 residual, inner solve in the handle's precision).
// Stops when the error left after the last update is estimated below
// tol_update ||X||_F — ||δX_k||_F itself, or rho ||δX_k||_F / (1 - rho) with
// the observed contraction rho = ||δX_k|| / ||δX_{k-1}|| once rho < 1/2 — or
// when ||R||_F <= tol_relres ||C||_F;
// FDE_ERR_NOCONV if neither holds after max_sweeps.  With fixed_sweeps > 0 it
// runs exactly that many sweeps and never synchronises with the host unless a
// residual is requested.
static fde_status sylv_step_impl(sylv_s* S, const double* C, double* X, cudaStream_t st, double* relres,
                                 int* sweeps, const double* C_prev = nullptr) {
  const size_t NN = (size_t)S->N * S->N;
  const sylv_refine_t& rf = S->refine;
  const bool fixed = rf.fixed_sweeps > 0;
  FDE_CUDA(cudaMemsetAsync(S->acc, 0, 8 * sizeof(double), st));
  FDE_CUDA(cudaMemcpyAsync(S->tc_base, S->tc_count, sizeof(unsigned int), cudaMemcpyDeviceToDevice, st));
  sumsq_kernel<<<grid_for(NN), 256, 0, st>>>(C, NN, S->acc + 4, S->part, S->count);
  FDE_LAUNCH("sumsq_kernel");
  if (!fixed) {
    FDE_CUDA(cudaMemsetAsync(S->d_bad, 0, sizeof(int), st));
    nonfinite_kernel<<<grid_for(NN), 256, 0, st>>>(C, NN, S->d_bad);
    FDE_LAUNCH("nonfinite_kernel");
    int bad = 0;
    FDE_CUDA(cudaMemcpyAsync(&bad, S->d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    FDE_CUDA(cudaStreamSynchronize(st));
    if (bad) {
      set_error("sylv_step: non-finite right-hand side");
      return FDE_ERR_NUMERIC;
    }
  }
  const bool in_chain = C_prev && S->R_valid;  // the starting residual comes from the stored history
  if (in_chain) {
    // X is the solution computed for C_prev and S->R = C_prev - A(X): the new
    // residual follows exactly without applying the operator again.
    if (S->predict && S->hist) {
      predict_kernel<<<grid_for(NN), 256, 0, st>>>(C, C_prev, X, S->R, S->Xp, S->Cp, S->Rp, NN);
      FDE_LAUNCH("predict_kernel");
    } else if (S->predict) {
      shift_save_kernel<<<grid_for(NN), 256, 0, st>>>(C, C_prev, X, S->R, S->Xp, S->Cp, S->Rp, NN);
      FDE_LAUNCH("shift_save_kernel");
    } else {
      shift_residual_kernel<<<grid_for(NN), 256, 0, st>>>(C, C_prev, S->R, NN);
      FDE_LAUNCH("shift_residual_kernel");
    }
    S->hist = S->predict ? 1 : 0;
  } else {
    S->hist = 0;
    FDE_TRY(residual(S, C, X, S->R, st));
  }
  S->R_valid = false;
  // Residual after the first sweep.  Exact FP64 on "refresh" steps; on the
  // others R -= A(δ_0) in double-float when ||δ_0|| <= incr_tol ||X|| (1e-2;
  // the time-step predictor leaves ||δ_0|| at a few 1e-3 ||X|| at N = 4096,
  // dt = 1/100).  The double-float product's error, ~1e-14 ||A|| ||δ_0||
  // normwise, is white noise that A^-1 damps at all but the lowest
  // frequencies.  The predicted residual combines two stored residuals
  // (2 e_n - e_{n-1}), so these errors grow quadratically along a chain of
  // incremental steps: a refresh takes two consecutive exact steps, and a
  // chain lasts at most exact_every - 2 steps.  Any fallback to an exact
  // residual starts a new refresh pair.
  if (!in_chain) {
    S->cyc_streak = 0;
    S->cyc_incr = 0;
    S->prev_large = false;
  }
  const int K = S->exact_every;
  const bool must_exact = !in_chain || fixed || K <= 2 || S->prec == FDE_FP64 || !S->resid_df ||
                          S->cyc_streak == 1 || S->cyc_incr >= K - 2;
  bool step_incremental = false;
  // set when ||δ_0|| was too large for an incremental first update: such a
  // step recomputes its residual exactly anyway, and when the previous step's
  // was too large as well (a regime where the next ones will be exact too) it
  // may take the FP32 last update and make the next two steps exact
  bool large_first = false, used_f32 = false;
  const int nsw = fixed ? rf.fixed_sweeps : rf.max_sweeps;
  int done = 0;
  bool converged = fixed;
  double a[8];
  double prev_d2 = -1.0;
  bool incr_ok = S->resid_df;
  for (int sw = 0; sw < nsw; ++sw) {
    if (S->prec == FDE_FP64)
      FDE_TRY(sweep_solve<double>(S, S->in64, X, st));
    else
      FDE_TRY(sweep_solve<float>(S, S->in32, X, st));
    ++done;
    // decide on the update first: the last update of a step may take the cheap residual
    bool stop = fixed && sw == nsw - 1;
    if (!fixed) {
      FDE_TRY(read_acc(S, a, 8, st));
      if (!std::isfinite(a[0]) || !std::isfinite(a[1])) {
        set_error("sylv_step: non-finite iterate after sweep %d", done);
        return FDE_ERR_NUMERIC;
      }
      const double tol2 = rf.tol_update * rf.tol_update * a[1];
      stop = a[0] <= tol2;
      if (!stop && prev_d2 > 0.0 && a[0] < 0.25 * prev_d2) {
        // the sweeps contract the error by rho ~ ||δ_k|| / ||δ_{k-1}|| < 1/2:
        // what the next sweeps would still add is about rho ||δ_k|| / (1 - rho)
        const double rho = sqrt(a[0] / prev_d2);
        const double rest = rho / (1.0 - rho);
        stop = a[0] * rest * rest <= tol2;
      }
      // incremental residuals only while the sweeps contract well (rho < 0.1)
      if (prev_d2 > 0.0 && a[0] > 0.01 * prev_d2) incr_ok = false;
      prev_d2 = a[0];
    }
    int kind = kResidExact;
    if (S->prec != FDE_FP64 && incr_ok) {
      if (sw == 0 && !fixed && in_chain && K > 2) {
        const bool small = a[0] <= S->incr_tol * S->incr_tol * a[1];
        if (small && !must_exact) step_incremental = true;
        if (!small) large_first = true;
      }
      if (sw > 0 || step_incremental) {
        // the last update of a step may be FP32 when the next two steps are
        // sure to recompute their residual exactly: the last step of a chain,
        // or a step with a large first update (which then forces them)
        const bool next_two_exact =
            K <= 1 || (step_incremental && S->cyc_incr + 1 >= K - 2) ||
            (large_first && S->prev_large && !step_incremental);
        kind = (stop && S->resid_f32_last && (next_two_exact || S->f32_last_all)) ? kResidF32 : kResidDF;
        if (kind == kResidF32) used_f32 = true;
      }
    }
    if (S->prec == FDE_FP64)
      FDE_TRY(sweep_residual<double>(S, S->in64, C, X, kind, st));
    else
      FDE_TRY(sweep_residual<float>(S, S->in32, C, X, kind, st));
    if (fixed) continue;
    if (!stop) {
      FDE_TRY(read_acc(S, a, 8, st));
      if (!std::isfinite(a[2])) {
        set_error("sylv_step: non-finite residual after sweep %d", done);
        return FDE_ERR_NUMERIC;
      }
      stop = a[2] <= rf.tol_relres * rf.tol_relres * a[4];
    }
    if (stop) {
      converged = true;
      break;
    }
  }
  if (sweeps) *sweeps = done;
  if (relres) {
    FDE_TRY(read_acc(S, a, 8, st));
    *relres = (a[4] > 0.0) ? sqrt(a[2] / a[4]) : sqrt(a[2]);
  }
  if (!converged) {
    set_error("sylv_step: no convergence after %d refinement sweeps", done);
    return FDE_ERR_NOCONV;
  }
  S->R_valid = done > 0;
  if (!S->R_valid) S->hist = 0;
  if (step_incremental) {
    S->cyc_streak = 0;
    ++S->cyc_incr;
  } else {
    S->cyc_streak = S->cyc_streak < 2 ? S->cyc_streak + 1 : 2;
    if (S->cyc_streak == 2) S->cyc_incr = 0;
  }
  if (used_f32 && large_first && K > 2) {
    // the FP32 residual may only feed exact steps: the next two
    S->cyc_streak = 0;
    S->cyc_incr = K;
  }
  S->prev_large = large_first;
  S->ctl_synced = false;
  return FDE_OK;
}

// ---------------------------------------------------- whole-step graphs
// Kernel nodes of a graph (top level only: conditional bodies are counted
// separately).
static fde_status count_kernel_nodes(cudaGraph_t g, size_t* n) {
  size_t cnt = 0;
  FDE_CUDA(cudaGraphGetNodes(g, nullptr, &cnt));
  std::vector<cudaGraphNode_t> nodes(cnt);
  if (cnt) FDE_CUDA(cudaGraphGetNodes(g, nodes.data(), &cnt));
  *n = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    FDE_CUDA(cudaGraphNodeGetType(nd, &t));
    if (t == cudaGraphNodeTypeKernel) ++*n;
  }
  return FDE_OK;
}

// Appends a conditional node (handle h, `size` bodies) to the graph being
// captured on `st`, after the stream's current dependencies, and makes it the
// stream's only dependency.  *bodies: the node's body graphs.
static fde_status add_conditional(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                                  unsigned size, cudaGraph_t** bodies) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  FDE_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) {
    set_error("sylv: stream not capturing");
    return FDE_ERR_CUDA;
  }
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = size;
  cudaGraphNode_t node;
  FDE_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
  FDE_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  *bodies = p.conditional.phGraph_out;
  return FDE_OK;
}

static fde_status capture_graph_of(cudaStream_t st, cudaGraph_t* g) {
  cudaStreamCaptureStatus cs;
  FDE_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, g, nullptr, nullptr, nullptr));
  return FDE_OK;
}

// One refinement sweep of the FP32 inner solver as a graph body (captured on
// gs2): Cin = (float) R, inner solve, X += δ with its norms, the controller's
// decision, a SWITCH over the residual forms (bodies captured on gs3), ||R||²,
// the controller's stopping test (which sets the enclosing WHILE node).
static fde_status capture_sweep_body(sylv_s* S, cudaGraph_t body, const double* C, double* X,
                                     cudaGraphConditionalHandle hloop, sylv_s::StepGraph* sg) {
  Inner<float>& in = S->in32;
  const size_t NN = (size_t)S->N * S->N;
  cudaStream_t s2 = S->gs2, s3 = S->gs3;
  FDE_CUDA(cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  fde_status st = FDE_OK;
  cudaGraph_t* br = nullptr;
  cudaGraphConditionalHandle hkind = 0;
  do {
    if ((st = convert<double, float>(S->R, in.Cin, NN, s2)) != FDE_OK) break;
    if ((st = run_inner<float>(S, in, s2)) != FDE_OK) break;
    refine_update_kernel<float><<<grid_for(NN), 256, 0, s2>>>(X, in.X, NN, S->acc, S->part, S->count);
    if (cudaGetLastError() != cudaSuccess) { st = FDE_ERR_CUDA; break; }
    cudaGraph_t bg = nullptr;
    if ((st = capture_graph_of(s2, &bg)) != FDE_OK) break;
    if (cudaGraphConditionalHandleCreate(&hkind, bg, 0, 0) != cudaSuccess) { st = FDE_ERR_CUDA; break; }
    ctl_solve_kernel<<<1, 32, 0, s2>>>(S->ctl, S->acc, hkind);
    if ((st = add_conditional(s2, hkind, cudaGraphCondTypeSwitch, 3, &br)) != FDE_OK) break;
    for (int k = 0; k < 3 && st == FDE_OK; ++k) {
      if (cudaStreamBeginCaptureToGraph(s3, br[k], nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
          cudaSuccess) {
        st = FDE_ERR_CUDA;
        break;
      }
      if (k == kResidExact)
        st = residual(S, C, X, S->R, s3);
      else if (k == kResidDF)
        st = residual_update_df(S, in.X, s3);
      else
        st = residual_update_f32(S, in.X, s3);
      cudaGraph_t g3 = nullptr;
      const cudaError_t e3 = cudaStreamEndCapture(s3, &g3);
      if (st == FDE_OK && e3 != cudaSuccess) st = FDE_ERR_CUDA;
      if (st == FDE_OK) st = count_kernel_nodes(br[k], &sg->k_br[k]);
    }
    if (st != FDE_OK) break;
    sumsq_kernel<<<grid_for(NN), 256, 0, s2>>>(S->R, NN, S->acc + 2, S->part, S->count);
    ctl_resid_kernel<<<1, 32, 0, s2>>>(S->ctl, S->acc, hloop);
    if (cudaGetLastError() != cudaSuccess) st = FDE_ERR_CUDA;
  } while (false);
  cudaGraph_t g2 = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s2, &g2);
  if (st != FDE_OK) {
    cudaGetLastError();
    return st;
  }
  FDE_CUDA(e);
  return count_kernel_nodes(body, &sg->k_body);
}

// Captures a whole time step on S->gs: the first part (variant 0: exact
// residual of the initial guess; 1: linear predictor; 2: residual shift with a
// new history; 3: residual shift), then the sweeps in a WHILE node.
static fde_status capture_step(sylv_s* S, sylv_s::StepGraph* sg) {
  const size_t NN = (size_t)S->N * S->N;
  const double* C = sg->C;
  const double* Cp = sg->Cp;
  double* X = sg->X;
  cudaStream_t s = S->gs;
  FDE_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  fde_status st = FDE_OK;
  do {
    cudaMemsetAsync(S->d_bad, 0, sizeof(int), s);
    nonfinite_kernel<<<grid_for(NN), 256, 0, s>>>(C, NN, S->d_bad);
    sumsq_kernel<<<grid_for(NN), 256, 0, s>>>(C, NN, S->acc + 4, S->part, S->count);
    if (sg->variant == 0) {
      if ((st = residual(S, C, X, S->R, s)) != FDE_OK) break;
    } else if (sg->variant == 1) {
      predict_kernel<<<grid_for(NN), 256, 0, s>>>(C, Cp, X, S->R, S->Xp, S->Cp, S->Rp, NN);
      } else if (sg->variant == 2) {
      shift_save_kernel<<<grid_for(NN), 256, 0, s>>>(C, Cp, X, S->R, S->Xp, S->Cp, S->Rp, NN);
      } else {
      shift_residual_kernel<<<grid_for(NN), 256, 0, s>>>(C, Cp, S->R, NN);
      }
    cudaGraph_t g = nullptr;
    if ((st = capture_graph_of(s, &g)) != FDE_OK) break;
    cudaGraphConditionalHandle hloop = 0;
    if (cudaGraphConditionalHandleCreate(&hloop, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
      st = FDE_ERR_CUDA;
      break;
    }
    ctl_begin_kernel<<<1, 32, 0, s>>>(S->ctl, S->d_bad, sg->variant == 0 ? 0 : 1, hloop);
    if (cudaGetLastError() != cudaSuccess) {
      st = FDE_ERR_CUDA;
      break;
    }
    cudaGraph_t* body = nullptr;
    if ((st = add_conditional(s, hloop, cudaGraphCondTypeWhile, 1, &body)) != FDE_OK) break;
    st = capture_sweep_body(S, body[0], C, X, hloop, sg);
  } while (false);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &g);
  if (st != FDE_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (st != FDE_OK) return st;
    FDE_CUDA(e);
  }
  st = count_kernel_nodes(g, &sg->k_pre);
  if (st == FDE_OK) {
    const cudaError_t ei = cudaGraphInstantiate(&sg->exec, g, 0);
    if (ei != cudaSuccess) {
      set_error("sylv: whole-step graph instantiation failed: %s", cudaGetErrorString(ei));
      st = FDE_ERR_CUDA;
    }
  }
  cudaGraphDestroy(g);
  return st;
}

static fde_status ctl_upload(sylv_s* S, cudaStream_t st) {
  StepCtl h{};
  const sylv_refine_t& rf = S->refine;
  h.tol2_update = rf.tol_update * rf.tol_update;
  h.tol2_relres = rf.tol_relres * rf.tol_relres;
  h.incr_tol2 = S->incr_tol * S->incr_tol;
  h.max_sweeps = rf.max_sweeps;
  h.exact_every = S->exact_every;
  h.resid_df = S->resid_df ? 1 : 0;
  h.f32_last = S->resid_f32_last ? 1 : 0;
  h.f32_last_all = S->f32_last_all ? 1 : 0;
  h.cyc_streak = S->cyc_streak;
  h.cyc_incr = S->cyc_incr;
  h.prev_large = S->prev_large ? 1 : 0;
  h.status = FDE_OK;
  FDE_CUDA(cudaMemcpyAsync(S->ctl, &h, sizeof(h), cudaMemcpyHostToDevice, st));
  FDE_CUDA(cudaStreamSynchronize(st));
  return FDE_OK;
}

// One time step as one graph launch (no host synchronisation); results and
// errors are read by sylv_graph_collect.
static fde_status step_graph_impl(sylv_s* S, const double* C, double* X, cudaStream_t st, const double* C_prev) {
  if (!S->ctl_synced) {
    FDE_TRY(ctl_upload(S, st));
    FDE_CUDA(cudaMemcpyAsync(S->tc_base, S->tc_count, sizeof(unsigned int), cudaMemcpyDeviceToDevice, st));
    S->ctl_synced = true;
  }
  const bool in_chain = C_prev && S->R_valid;
  const int variant = !in_chain ? 0 : (S->predict && S->hist) ? 1 : S->predict ? 2 : 3;
  sylv_s::StepGraph* sg = nullptr;
  for (auto& g : S->sgraphs)
    if (g.variant == variant && g.C == C && g.Cp == (in_chain ? C_prev : nullptr) && g.X == X) sg = &g;
  if (!sg) {
    if (!S->gs) {
      FDE_CUDA(cudaStreamCreateWithFlags(&S->gs, cudaStreamNonBlocking));
      FDE_CUDA(cudaEventCreateWithFlags(&S->ev_in, cudaEventDisableTiming));
      FDE_CUDA(cudaEventCreateWithFlags(&S->ev_out, cudaEventDisableTiming));
    }
    if (!S->gs2) FDE_CUDA(cudaStreamCreateWithFlags(&S->gs2, cudaStreamNonBlocking));
    if (!S->gs3) FDE_CUDA(cudaStreamCreateWithFlags(&S->gs3, cudaStreamNonBlocking));
    sylv_s::StepGraph g;
    g.variant = variant;
    g.C = C;
    g.Cp = in_chain ? C_prev : nullptr;
    g.X = X;
    count_suspend(true);  // a capture launches nothing: its kernels are counted per replay
    const fde_status cs = capture_step(S, &g);
    count_suspend(false);
    FDE_TRY(cs);
    S->sgraphs.push_back(g);
    sg = &S->sgraphs.back();
  }
  FDE_CUDA(cudaEventRecord(S->ev_in, st));
  FDE_CUDA(cudaStreamWaitEvent(S->gs, S->ev_in, 0));
  FDE_CUDA(cudaGraphLaunch(sg->exec, S->gs));
  FDE_CUDA(cudaEventRecord(S->ev_out, S->gs));
  FDE_CUDA(cudaStreamWaitEvent(st, S->ev_out, 0));
  S->graph_pending.push_back(sg - S->sgraphs.data());
  S->hist = (in_chain && S->predict) ? 1 : 0;
  S->R_valid = true;
  return FDE_OK;
}

static fde_status graph_collect_impl(sylv_s* S, cudaStream_t st, int* steps, int* sweeps_total, int* sweeps_max,
                                     double* relres_max) {
  *steps = *sweeps_total = *sweeps_max = 0;
  *relres_max = 0.0;
  if (!S->ctl_synced) return FDE_OK;
  StepCtl h{};
  unsigned int tc[2] = {0u, 0u};
  FDE_CUDA(cudaMemcpyAsync(&h, S->ctl, sizeof(h), cudaMemcpyDeviceToHost, st));
  FDE_CUDA(cudaMemcpyAsync(tc, S->tc_base, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  FDE_CUDA(cudaMemcpyAsync(tc + 1, S->tc_count, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  FDE_CUDA(cudaStreamSynchronize(st));
  // kernels these graph launches ran: first parts, sweep bodies and residual branches
  unsigned long long k = 0;
  for (size_t i : S->graph_pending) k += S->sgraphs[i].k_pre;
  if (!S->graph_pending.empty()) {
    const sylv_s::StepGraph& g = S->sgraphs[S->graph_pending.back()];
    k += (unsigned long long)h.sweeps_total * g.k_body;
    for (int i = 0; i < 3; ++i) k += (unsigned long long)h.kind_count[i] * g.k_br[i];
  }
  count_launches(k);
  S->graph_pending.clear();
  *steps = h.steps;
  *sweeps_total = h.sweeps_total;
  *sweeps_max = h.sweeps_max;
  *relres_max = h.relres_max;
  S->cyc_streak = h.cyc_streak;
  S->cyc_incr = h.cyc_incr;
  S->prev_large = h.prev_large != 0;
  S->ctl_synced = false;  // the next graph step re-uploads (clears the results)
  if (tc[1] != tc[0]) {
    S->R_valid = false;
    set_error("sylv_step: a bounded wait of the tensor-core GEMM expired (%u)", tc[1] - tc[0]);
    return FDE_ERR_CUDA;
  }
  if (h.status != FDE_OK) {
    S->R_valid = false;
    set_error(h.status == FDE_ERR_NUMERIC ? "sylv_step: non-finite data in a whole-step graph"
                                          : "sylv_step: no convergence within the sweep cap in a whole-step graph");
    return (fde_status)h.status;
  }
  return FDE_OK;
}

static fde_status create_impl(hodlr_s* ax, hodlr_s* ay, int prec, cudaStream_t st, sylv_s* S) {
  S->ax = ax;
  S->ay = ay;
  S->prec = prec;
  const int N = ax->tree.N, L = ax->tree.L;
  S->N = N;
  S->L = L;
  S->lmax = ax->lmax;
  DevPool& pool = S->pool;
  const int nl = ax->tree.nleaves();
  const size_t nleaf_el = (size_t)nl * S->lmax * S->lmax;
  FDE_TRY(tc_prepare());
  // ---- leaf Schur forms (K8)
  FDE_TRY(pool.alloc(&S->Sx, nleaf_el));
  FDE_TRY(pool.alloc(&S->Qx, nleaf_el));
  FDE_TRY(pool.alloc(&S->Sy, nleaf_el));
  FDE_TRY(pool.alloc(&S->Qy, nleaf_el));
  FDE_CUDA(cudaMemcpyAsync(S->Sx, ax->D, nleaf_el * sizeof(double), cudaMemcpyDeviceToDevice, st));
  FDE_CUDA(cudaMemcpyAsync(S->Sy, ay->D, nleaf_el * sizeof(double), cudaMemcpyDeviceToDevice, st));
  FDE_TRY(pool.alloc(&S->d_lo, 2 * nl));
  FDE_TRY(pool.alloc(&S->d_n, 2 * nl));
  {
    std::vector<int> lo(2 * nl), n(2 * nl);
    for (int p = 0; p < nl; ++p) {
      lo[p] = ax->leaf_lo[p];
      n[p] = ax->leaf_n[p];
      lo[nl + p] = ay->leaf_lo[p];
      n[nl + p] = ay->leaf_n[p];
    }
    FDE_CUDA(cudaMemcpy(S->d_lo, lo.data(), 2 * nl * sizeof(int), cudaMemcpyHostToDevice));
    FDE_CUDA(cudaMemcpy(S->d_n, n.data(), 2 * nl * sizeof(int), cudaMemcpyHostToDevice));
  }
  int* d_fail;
  FDE_TRY(pool.alloc(&d_fail, 2 * nl));
  FDE_CUDA(cudaMemsetAsync(d_fail, 0, 2 * nl * sizeof(int), st));
  FDE_TRY(leaf_schur(S->Sx, S->Qx, S->lmax, (size_t)S->lmax * S->lmax, S->d_n, nl, d_fail, st));
  FDE_TRY(leaf_schur(S->Sy, S->Qy, S->lmax, (size_t)S->lmax * S->lmax, S->d_n + nl, nl, d_fail + nl, st));
  {
    std::vector<int> f(2 * nl);
    FDE_CUDA(cudaMemcpyAsync(f.data(), d_fail, 2 * nl * sizeof(int), cudaMemcpyDeviceToHost, st));
    FDE_CUDA(cudaStreamSynchronize(st));
    for (int v : f)
      if (v) {
        set_error("sylv_create: leaf Schur iteration did not converge");
        return FDE_ERR_NOCONV;
      }
  }
  // ---- leaf Sylvester sub-problems (whole leaves; blocked leaves for the FP32 inner solver)
  if (const char* pg = getenv("FDE_PACK_GB")) S->pack_budget = (size_t)(atof(pg) * (double)(1ull << 30));
  S->trsyl_split = prec != FDE_FP64 && S->lmax > kTrsylSplit && (long long)nl * nl >= kTrsylSplitMinPairs;
  int part = kTrsylPart;
  if (const char* ts = getenv("FDE_TRSYL_SPLIT")) {  // "1": block every leaf (tests), "0": never
    if (!strcmp(ts, "1")) S->trsyl_split = prec != FDE_FP64 && S->lmax >= 2;
    if (!strcmp(ts, "0")) S->trsyl_split = false;
  }
  if (const char* tp = getenv("FDE_TRSYL_PART")) {  // block rows (tests, experiments)
    const int v = atoi(tp);
    if (v >= 2) part = v;
  }
  {
    const int lm = S->lmax;
    std::vector<int> soff(2 * nl), lo(2 * nl), n(2 * nl);
    // blocked leaves: cuts[side][p] = block boundaries of leaf p, bottom block last
    std::vector<std::vector<int>> cuts(2 * nl);
    int nb = 0;
    for (int side = 0; side < 2; ++side) {
      hodlr_s* h_ = side == 0 ? ax : ay;
      const double* Sd = side == 0 ? S->Sx : S->Sy;
      for (int p = 0; p < nl; ++p) {
        const int i = side * nl + p, np = h_->leaf_n[p];
        soff[i] = p * lm * lm;
        lo[i] = h_->leaf_lo[p];
        n[i] = np;
        S->tp_full.nmax = std::max(S->tp_full.nmax, np);
        if (!S->trsyl_split) continue;
        // q blocks of about np / q <= part - 1 rows, so that a cut inside a
        // 2 x 2 block, moved down by one, still leaves every block at most
        // `part` rows (one warp per block for part = 32: a launch takes the
        // warps of its largest block)
        const int q = np > part ? (np + part - 2) / (part - 1) : (np >= 2 ? 2 : 1);
        std::vector<double> sub(np > 0 ? np : 1, 0.0);  // sub[r] = S_p(r, r - 1)
        if (np > 1)
          FDE_CUDA(cudaMemcpy2D(&sub[1], sizeof(double), Sd + (size_t)p * lm * lm + 1, (size_t)(lm + 1) * sizeof(double),
                                sizeof(double), np - 1, cudaMemcpyDeviceToHost));
        std::vector<int>& c = cuts[i];
        c.push_back(0);
        for (int k = 1; k < q; ++k) {
          int cut = (int)(((long long)np * k) / q);
          if (cut > 0 && cut < np && sub[cut] != 0.0) ++cut;
          if (cut > c.back() && cut < np) c.push_back(cut);
        }
        c.push_back(np);
        nb = std::max(nb, (int)c.size() - 1);
      }
    }
    auto upload_arr = [&](int** d, const std::vector<int>& a) -> fde_status {
      FDE_TRY(pool.alloc(d, a.size()));
      FDE_CUDA(cudaMemcpy(*d, a.data(), a.size() * sizeof(int), cudaMemcpyHostToDevice));
      return FDE_OK;
    };
    FDE_TRY(upload_arr(&S->tp_full.soff, soff));
    FDE_TRY(upload_arr(&S->tp_full.lo, lo));
    FDE_TRY(upload_arr(&S->tp_full.n, n));
    if (S->trsyl_split) {
      if (2 * nb - 1 > 0 && nb > kTrsylMaxSets) {
        set_error("sylv_create: %d leaf blocks per leaf (at most %d)", nb, kTrsylMaxSets);
        return FDE_ERR_ARG;
      }
      // part a (from the bottom) of every leaf, x entries then y entries
      std::vector<std::vector<int>> bsoff(nb), blo(nb), bn(nb), brest(nb);
      S->tp_part.assign(nb, sylv_s::TrsylPart{});
      for (int a = 0; a < nb; ++a) {
        bsoff[a].assign(2 * nl, 0);
        blo[a].assign(2 * nl, 0);
        bn[a].assign(2 * nl, 0);
        brest[a].assign(2 * nl, 0);
        for (int i = 0; i < 2 * nl; ++i) {
          const std::vector<int>& c = cuts[i];
          const int nblk = (int)c.size() - 1;
          if (a >= nblk) continue;
          const int k = nblk - 1 - a, r0 = c[k], r1 = c[k + 1];
          bsoff[a][i] = soff[i] + r0 * (lm + 1);
          blo[a][i] = lo[i] + r0;
          bn[a][i] = r1 - r0;
          brest[a][i] = n[i] - r1;
          S->tp_part[a].nmax = std::max(S->tp_part[a].nmax, r1 - r0);
        }
        FDE_TRY(upload_arr(&S->tp_part[a].soff, bsoff[a]));
        FDE_TRY(upload_arr(&S->tp_part[a].lo, blo[a]));
        FDE_TRY(upload_arr(&S->tp_part[a].n, bn[a]));
        FDE_TRY(upload_arr(&S->tp_part[a].rest, brest[a]));
      }
      // algorithmic flops per anti-diagonal: the block solves n1 n2 (n1 + n2)
      // and their couplings 2 n1 n2 (rest_x + rest_y)
      S->trsyl_step_flops.assign(2 * nb - 1, 0.0);
      for (int a = 0; a < nb; ++a)
        for (int b2 = 0; b2 < nb; ++b2)
          for (int p = 0; p < nl; ++p)
            for (int q = 0; q < nl; ++q) {
              const double n1 = bn[a][p], n2 = bn[b2][nl + q];
              if (n1 <= 0 || n2 <= 0) continue;
              S->trsyl_step_flops[a + b2] +=
                  n1 * n2 * (n1 + n2) + 2.0 * n1 * n2 * (brest[a][p] + brest[b2][nl + q]);
            }
    }
  }
  // ---- shifts per level (host: spectral intervals of the level's blocks)
  std::vector<double> gx(N + 2), gy(N + 2), dpx(N), dmx(N), dpy(N), dmy(N);
  FDE_CUDA(cudaMemcpy(gx.data(), ax->g, (N + 2) * sizeof(double), cudaMemcpyDeviceToHost));
  FDE_CUDA(cudaMemcpy(gy.data(), ay->g, (N + 2) * sizeof(double), cudaMemcpyDeviceToHost));
  FDE_CUDA(cudaMemcpy(dpx.data(), ax->dp, N * sizeof(double), cudaMemcpyDeviceToHost));
  FDE_CUDA(cudaMemcpy(dmx.data(), ax->dm, N * sizeof(double), cudaMemcpyDeviceToHost));
  FDE_CUDA(cudaMemcpy(dpy.data(), ay->dp, N * sizeof(double), cudaMemcpyDeviceToHost));
  FDE_CUDA(cudaMemcpy(dmy.data(), ay->dm, N * sizeof(double), cudaMemcpyDeviceToHost));
  std::vector<double> Sxs(N + 2), Sys(N + 2);
  {
    long double ax_ = 0, ay_ = 0;
    for (int k = 0; k < N + 2; ++k) {
      ax_ += gx[k];
      ay_ += gy[k];
      Sxs[k] = (double)ax_;
      Sys[k] = (double)ay_;
    }
  }
  // fADI accuracy per level: the FP64 inner solver is used unrefined-grade;
  // the FP32 one only preconditions the FP64 refinement (FDE_FADI_TOL overrides)
  double target = (prec == FDE_FP64) ? 1e-13 : 1e-5;
  if (prec != FDE_FP64)
    if (const char* e = getenv("FDE_FADI_TOL")) {
      const double v = atof(e);
      if (v > 0.0 && v < 1.0) target = v;
    }
  S->J.assign(L, 0);
  std::vector<std::vector<double>> A_(L), B_(L);
  for (int l = 0; l < L; ++l) {
    double a = INFINITY, b = 0.0, c = INFINITY, d = 0.0;
    for (int p = 0; p < (1 << l); ++p) {
      const int id = ax->tree.id(l, p);
      double lo_, hi_;
      node_interval(Sxs, dpx, dmx, ax->c, ax->p.shift, ax->p.alpha, ax->tree.lo[id], ax->tree.hi[id], &lo_, &hi_);
      a = std::min(a, lo_);
      b = std::max(b, hi_);
      node_interval(Sys, dpy, dmy, ay->c, ay->p.shift, ay->p.alpha, ay->tree.lo[id], ay->tree.hi[id], &lo_, &hi_);
      c = std::min(c, lo_);
      d = std::max(d, hi_);
    }
    std::vector<double> al, be;
    double ratio;
    const int J = select_shifts(a, b, c, d, target, 64, al, be, &ratio);
    S->J[l] = J;
    A_[l] = al;
    B_[l] = be;
  }
  // ---- shifted factorisations: A_x + b_j I and A_y + a_j I (b_j = -beta_j).
  // FP64 inner solver: per-step shifted HODLR solves (fewest flops, kept).
  // FP32 inner solver: rational form (factorisations only needed at setup).
  bool rational = (prec == FDE_FP32_REFINE);
  if (const char* fm = getenv("FDE_FADI")) {
    if (!strcmp(fm, "hodlr")) rational = false;
    if (!strcmp(fm, "rational")) rational = true;
  }
  S->rational = rational;
  DevPool setup_pool;
  DevPool& fpool = rational ? setup_pool : S->pool;
  S->facts64.reserve(2 * 64 * L);
  std::vector<Fact<double>*> FA64, FB64;
  for (int l = L - 1; l >= 0; --l) {
    for (int j = 0; j < S->J[l]; ++j) {
      S->facts64.emplace_back();
      FDE_TRY(hodlr_factorize(ax, -B_[l][j], l, &S->facts64.back(), st, &fpool));
    }
    for (int j = 0; j < S->J[l]; ++j) {
      S->facts64.emplace_back();
      FDE_TRY(hodlr_factorize(ay, A_[l][j], l, &S->facts64.back(), st, &fpool));
    }
  }
  {
    size_t idx = 0;
    for (int l = L - 1; l >= 0; --l) {
      for (int j = 0; j < S->J[l]; ++j) FA64.push_back(&S->facts64[idx++]);
      for (int j = 0; j < S->J[l]; ++j) FB64.push_back(&S->facts64[idx++]);
    }
  }
  // ---- inner solver(s)
  auto set_shifts = [&](auto& in) {
    for (int l = 0; l < L; ++l) {
      in.lv[l].a = A_[l];
      in.lv[l].b.resize(S->J[l]);
      for (int j = 0; j < S->J[l]; ++j) in.lv[l].b[j] = -B_[l][j];
    }
  };
  RationalSrc rs;
  if (rational) {
    rs.FA = FA64;
    rs.FB = FB64;
    rs.a.resize(L);
    rs.b.resize(L);
    for (int l = 0; l < L; ++l) {
      rs.a[l] = A_[l];
      rs.b[l].resize(S->J[l]);
      for (int j = 0; j < S->J[l]; ++j) rs.b[l][j] = -B_[l][j];
    }
  }
  if (prec == FDE_FP64) {
    if (rational)
      FDE_TRY(build_inner<double>(S, S->in64, {}, {}, st, &rs));
    else
      FDE_TRY(build_inner<double>(S, S->in64, FA64, FB64, st));
    set_shifts(S->in64);
    FDE_CUDA(cudaStreamSynchronize(st));
    FDE_TRY(capture_inner<double>(S, S->in64));
  } else {
    FDE_TRY(hodlr_make_fp32(ax, st));
    FDE_TRY(hodlr_make_fp32(ay, st));
    if (rational) {
      FDE_TRY(build_inner<float>(S, S->in32, {}, {}, st, &rs));
    } else {
      S->in32.facts.resize(FA64.size() + FB64.size());
      std::vector<Fact<float>*> FA32, FB32;
      for (size_t i = 0; i < FA64.size(); ++i) {
        FDE_TRY(fact_demote(ax, *FA64[i], &S->in32.facts[i], S->pool, st));
        FA32.push_back(&S->in32.facts[i]);
      }
      for (size_t i = 0; i < FB64.size(); ++i) {
        FDE_TRY(fact_demote(ay, *FB64[i], &S->in32.facts[FA64.size() + i], S->pool, st));
        FB32.push_back(&S->in32.facts[FA64.size() + i]);
      }
      FDE_TRY(build_inner<float>(S, S->in32, FA32, FB32, st));
    }
    set_shifts(S->in32);
    FDE_CUDA(cudaStreamSynchronize(st));
    FDE_TRY(capture_inner<float>(S, S->in32));
  }
  if (rational) {
    S->facts64.clear();  // their memory lives in setup_pool, released on return
  }
  // ---- residual (FFT)
  S->block = N > kFftBlock;
  S->logP = 1;
  while ((1 << S->logP) < 2 * N) ++S->logP;
  if (S->block) S->logP = kFftBlockLogP;
  S->P = 1 << S->logP;
  {
    // the whole circle: the radix-8 passes index up to 7P/8
    std::vector<double2> tw(S->P);
    for (int k = 0; k < S->P; ++k) {
      const double ang = -2.0 * M_PI * (double)k / (double)S->P;
      tw[k] = make_double2(cos(ang), sin(ang));
    }
    FDE_TRY(pool.alloc(&S->tw, S->P));
    FDE_CUDA(cudaMemcpy(S->tw, tw.data(), tw.size() * sizeof(double2), cudaMemcpyHostToDevice));
  }
  if (prec != FDE_FP64) {
    // FDE_RESID: "fp64" = every residual exact; "df" = incremental updates in
    // double-float only; default ("f32tail"): also the last update of a step
    // in FP32 when the next two steps recompute their residual exactly;
    // "f32last": the last update of every step in FP32, also inside a chain.
    // Its error, ~1e-7 of A applied to the last update, then enters the
    // chain's predicted residuals until the next refresh: at N = 4096 the
    // states stay as close to a dense FP64 Bartels–Stewart loop (1.6e-10 after
    // 20 steps), but the exact residuals, and the error bound summed from
    // them, grow (20 steps, refresh every 16: 2.9e-9 -> 1.3e-8), so it is not
    // the default.
    const char* rm = getenv("FDE_RESID");
    S->resid_df = !(rm && strcmp(rm, "fp64") == 0);
    S->resid_f32_last = S->resid_df && !(rm && strcmp(rm, "df") == 0);
    S->f32_last_all = S->resid_f32_last && rm && strcmp(rm, "f32last") == 0;
    if (const char* it = getenv("FDE_INCR_TOL")) {
      const double v = atof(it);
      if (v > 0.0 && v < 1.0) S->incr_tol = v;
    }
    if (const char* ee = getenv("FDE_EXACT_EVERY")) {
      const int v = atoi(ee);
      if (v >= 1) S->exact_every = v;
    }
    FDE_TRY(pool.alloc(&S->tw_df, S->P));
    FDE_TRY(complex_to_df(S->tw, S->tw_df, S->P, st));
    FDE_TRY(pool.alloc(&S->tw_f32, S->P));
    FDE_TRY(complex_to_f32(S->tw, S->tw_f32, S->P, st));
  }
  {
    FDE_TRY(pool.alloc(&S->cpx, N));
    FDE_TRY(pool.alloc(&S->cmx, N));
    FDE_TRY(pool.alloc(&S->cpy, N));
    FDE_TRY(pool.alloc(&S->cmy, N));
    FDE_TRY(pool.alloc(&S->cpx_df, N));
    FDE_TRY(pool.alloc(&S->cmx_df, N));
    FDE_TRY(pool.alloc(&S->cpy_df, N));
    FDE_TRY(pool.alloc(&S->cmy_df, N));
    const double invP = 1.0 / S->P;
    fft_coef_kernel<<<grid_for(N), 256, 0, st>>>(ax->dp, ax->dm, ax->c, invP, N, S->cpx, S->cmx, S->cpx_df,
                                                 S->cmx_df);
    FDE_LAUNCH("fft_coef_kernel");
    fft_coef_kernel<<<grid_for(N), 256, 0, st>>>(ay->dp, ay->dm, ay->c, invP, N, S->cpy, S->cmy, S->cpy_df,
                                                 S->cmy_df);
    FDE_LAUNCH("fft_coef_kernel");
  }
  const size_t NN = (size_t)N * N;
  if (S->block) {
    const int nb = (N + kFftBlock - 1) / kFftBlock, npairs = (N + 1) / 2;
    S->pair_chunk = npairs < 2048 ? npairs : 2048;
    FDE_TRY(pool.alloc(&S->HbX, (size_t)nb * S->P));
    FDE_TRY(pool.alloc(&S->HbY, (size_t)nb * S->P));
    FDE_TRY(pool.alloc(&S->HbX_df, (size_t)nb * S->P));
    FDE_TRY(pool.alloc(&S->HbY_df, (size_t)nb * S->P));
    FDE_TRY(block_spectra(ax->g, N, S->tw, S->HbX, S->HbX_df, st));
    FDE_TRY(block_spectra(ay->g, N, S->tw, S->HbY, S->HbY_df, st));
    FDE_TRY(pool.alloc(&S->HbX_f32, (size_t)nb * S->P));
    FDE_TRY(pool.alloc(&S->HbY_f32, (size_t)nb * S->P));
    FDE_TRY(complex_to_f32(S->HbX, S->HbX_f32, nb * S->P, st));
    FDE_TRY(complex_to_f32(S->HbY, S->HbY_f32, nb * S->P, st));
    FDE_TRY(pool.alloc(&S->fft_scratch, (size_t)S->pair_chunk * nb * S->P));
    FDE_TRY(pool.alloc(&S->R, NN));
    S->fft_flops = block_apply_flops(N, N);
  } else {
    FDE_TRY(pool.alloc(&S->GhX, S->P));
    FDE_TRY(pool.alloc(&S->GhY, S->P));
    const size_t smem = (size_t)fft_padded_len(S->P) * sizeof(double2);
    // the attribute is per kernel, shared by every handle: always allow the largest transform
    const int smax = fft_padded_len(8192) * (int)sizeof(double2);
    FDE_CUDA(cudaFuncSetAttribute(fd_fft_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
    FDE_CUDA(cudaFuncSetAttribute(ghat_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
    ghat_kernel<<<1, kFftThreads, smem, st>>>(ax->g, N, S->tw, S->P, S->logP, S->GhX);
    FDE_LAUNCH("ghat_kernel");
    ghat_kernel<<<1, kFftThreads, smem, st>>>(ay->g, N, S->tw, S->P, S->logP, S->GhY);
    FDE_LAUNCH("ghat_kernel");
    if (prec != FDE_FP64) {
      FDE_TRY(pool.alloc(&S->GhX_df, S->P));
      FDE_TRY(pool.alloc(&S->GhY_df, S->P));
      FDE_TRY(complex_to_df(S->GhX, S->GhX_df, S->P, st));
      FDE_TRY(complex_to_df(S->GhY, S->GhY_df, S->P, st));
      FDE_TRY(pool.alloc(&S->GhX_f32, S->P));
      FDE_TRY(pool.alloc(&S->GhY_f32, S->P));
      FDE_TRY(complex_to_f32(S->GhX, S->GhX_f32, S->P, st));
      FDE_TRY(complex_to_f32(S->GhY, S->GhY_f32, S->P, st));
    }
    FDE_TRY(pool.alloc(&S->fft_scratch, (size_t)((N + 1) / 2) * S->P));
    FDE_TRY(pool.alloc(&S->R, NN));
    FDE_TRY(pool.alloc(&S->Xt, NN));
    FDE_TRY(pool.alloc(&S->Yt, NN));
    // per residual direction: (N+1)/2 column pairs x (3 complex FFTs of 5 P log2 P + 2 pointwise products)
    S->fft_flops = (double)((N + 1) / 2) * (3.0 * 5.0 * S->P * S->logP + 12.0 * S->P);
  }
  FDE_TRY(pool.alloc(&S->acc, 8));
  FDE_TRY(pool.alloc(&S->part, 2 * (size_t)kSumBlocks));
  FDE_TRY(pool.alloc(&S->count, 1));
  FDE_CUDA(cudaMemsetAsync(S->count, 0, sizeof(unsigned int), st));
  if (prec != FDE_FP64) {
    // time loops run every step of the FP32 inner solver as one graph launch
    // (FDE_STEP_GRAPH=0: eager steps with a host decision after every sweep)
    const char* sg = getenv("FDE_STEP_GRAPH");
    S->step_graph = !(sg && strcmp(sg, "0") == 0);
    FDE_TRY(pool.alloc(&S->ctl, 1));
  }
  FDE_TRY(tc_timeout_counter(&S->tc_count));
  FDE_TRY(pool.alloc(&S->tc_base, 1));
  FDE_CUDA(cudaMemcpyAsync(S->tc_base, S->tc_count, sizeof(unsigned int), cudaMemcpyDeviceToDevice, st));
  FDE_TRY(pool.alloc(&S->d_bad, 1));
  {
    // time-step predictor (used by time loops that pass the previous right-hand side)
    const char* pe = getenv("FDE_PREDICT");
    S->predict = !(pe && strcmp(pe, "0") == 0);
    if (S->predict) {
      FDE_TRY(pool.alloc(&S->Xp, NN));
      FDE_TRY(pool.alloc(&S->Cp, NN));
      FDE_TRY(pool.alloc(&S->Rp, NN));
    }
  }
  // algorithmic work for the instrumentation
  for (int p = 0; p < nl; ++p)
    for (int q = 0; q < nl; ++q) {
      const double n1 = ax->leaf_n[p], n2 = ay->leaf_n[q];
      S->trsyl_flops += n1 * n2 * (n1 + n2);
    }
  S->refine.max_sweeps = 12;
  S->refine.tol_update = (prec == FDE_FP64) ? 1e-13 : 1e-11;
  S->refine.tol_relres = 1e-14;
  S->refine.fixed_sweeps = 0;
  FDE_CUDA(cudaStreamSynchronize(st));
  return FDE_OK;
}

}  // namespace fde

// ===================================================================== ABI
extern "C" fde_status sylv_create(hodlr_t Ax, hodlr_t Ay, int prec, void* stream, sylv_t* out) {
  FDE_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  FDE_ARG(Ax != nullptr && Ay != nullptr, "NULL operator");
  FDE_ARG(prec == FDE_FP64 || prec == FDE_FP32_REFINE || prec == FDE_BF16_REFINE, "unknown precision");
  FDE_ARG(Ax->tree.N == Ay->tree.N && Ax->tree.leaf == Ay->tree.leaf, "A_x and A_y must share N and leaf");
  FDE_ARG(Ax->tree.L >= 1, "N must exceed the leaf size");
  FDE_ARG(Ax->p.shift == 0.5 && Ay->p.shift == 0.5, "A_x and A_y must be built with shift 1/2");
  sylv_s* S = new sylv_s();
  // BF16: the FP32 inner solver with BF16 operands in the level products,
  // split into BF16 hi + lo (three products); FDE_BF16_SPLIT=0 rounds them to
  // BF16 (one product: a coarser inner solve, more refinement sweeps)
  if (prec == FDE_BF16_REFINE) {
    S->level_kind = kTcBF16x3;
    if (const char* e = getenv("FDE_BF16_SPLIT"))
      if (!strcmp(e, "0")) S->level_kind = kTcBF16;
    prec = FDE_FP32_REFINE;
  }
  fde_status s = create_impl(Ax, Ay, prec, (cudaStream_t)stream, S);
  if (s != FDE_OK) {
    delete S;
    return s;
  }
  *out = S;
  return FDE_OK;
}

extern "C" fde_status sylv_get_refine(sylv_t s, sylv_refine_t* r) {
  FDE_ARG(s != nullptr && r != nullptr, "NULL argument");
  *r = s->refine;
  return FDE_OK;
}
extern "C" fde_status sylv_set_refine(sylv_t s, const sylv_refine_t* r) {
  FDE_ARG(s != nullptr && r != nullptr, "NULL argument");
  FDE_ARG(r->max_sweeps >= 1 && r->max_sweeps <= 100, "max_sweeps must be in [1, 100]");
  FDE_ARG(r->fixed_sweeps >= 0 && r->fixed_sweeps <= 100, "fixed_sweeps must be in [0, 100]");
  FDE_ARG(r->tol_update >= 0.0 && r->tol_relres >= 0.0, "tolerances must be >= 0");
  s->refine = *r;
  return FDE_OK;
}

static fde_status with_contig(sylv_t s, const double* C, double* X, int ld, cudaStream_t st,
                              fde_status (*fn)(sylv_t, const double*, double*, cudaStream_t, void*), void* ctx) {
  const int N = s->N;
  if (ld == N) return fn(s, C, X, st, ctx);
  if (!s->X64) {
    FDE_TRY(s->pool.alloc(&s->X64, (size_t)N * N));
    FDE_TRY(s->pool.alloc(&s->C64, (size_t)N * N));
  }
  FDE_TRY((copy2d<double, double>(C, ld, s->C64, N, N, N, st)));
  FDE_TRY((copy2d<double, double>(X, ld, s->X64, N, N, N, st)));
  FDE_TRY(fn(s, s->C64, s->X64, st, ctx));
  FDE_TRY((copy2d<double, double>(s->X64, N, X, ld, N, N, st)));
  return FDE_OK;
}

struct StepCtx {
  double* relres;
  int* sweeps;
  fde_status status;
};
static fde_status step_fn(sylv_t s, const double* C, double* X, cudaStream_t st, void* ctx) {
  StepCtx* c = (StepCtx*)ctx;
  return sylv_step_impl(s, C, X, st, c->relres, c->sweeps);
}

extern "C" fde_status sylv_step(sylv_t s, const double* d_C, double* d_X, int ld, void* stream, double* relres_out,
                                int* sweeps_out) {
  FDE_ARG(s != nullptr, "handle is NULL");
  FDE_ARG(d_C != nullptr && d_X != nullptr && d_C != d_X, "bad C / X");
  FDE_ARG(ld >= s->N, "ld < N");
  StepCtx ctx{relres_out, sweeps_out, FDE_OK};
  return with_contig(s, d_C, d_X, ld, (cudaStream_t)stream, step_fn, &ctx);
}

static fde_status inner_fn(sylv_t s, const double* C, double* X, cudaStream_t st, void*) {
  const size_t NN = (size_t)s->N * s->N;
  if (s->prec == FDE_FP64) {
    FDE_CUDA(cudaMemcpyAsync(s->in64.Cin, C, NN * sizeof(double), cudaMemcpyDeviceToDevice, st));
    FDE_TRY(inner_solve<double>(s, s->in64, st));
    FDE_CUDA(cudaMemcpyAsync(X, s->in64.X, NN * sizeof(double), cudaMemcpyDeviceToDevice, st));
  } else {
    FDE_TRY((convert<double, float>(C, s->in32.Cin, NN, st)));
    FDE_TRY(inner_solve<float>(s, s->in32, st));
    FDE_TRY((convert<float, double>(s->in32.X, X, NN, st)));
  }
  return FDE_OK;
}

extern "C" fde_status sylv_inner_solve(sylv_t s, const double* d_C, double* d_X, int ld, void* stream) {
  FDE_ARG(s != nullptr, "handle is NULL");
  FDE_ARG(d_C != nullptr && d_X != nullptr && d_C != d_X, "bad C / X");
  FDE_ARG(ld >= s->N, "ld < N");
  return with_contig(s, d_C, d_X, ld, (cudaStream_t)stream, inner_fn, nullptr);
}

extern "C" fde_status sylv_residual(sylv_t s, const double* d_C, const double* d_X, double* d_R, int ld,
                                    void* stream) {
  FDE_ARG(s != nullptr, "handle is NULL");
  FDE_ARG(d_C != nullptr && d_X != nullptr && d_R != nullptr, "NULL buffer");
  FDE_ARG(ld == s->N, "sylv_residual requires ld == N");
  return residual(s, d_C, d_X, d_R, (cudaStream_t)stream);
}

// Work model of one inner solve (§3.4 D&C with §3.3 fADI on every level),
// from the counted leaf sizes n_i, level ranks K_l and shift counts J_l:
//  - leaf Bartels–Stewart: the four orthogonal transforms, 4 n_i n_j (n_i + n_j)
//    per leaf pair (the quasi-triangular solve itself is not a GEMM);
//  - per level l and node pair (s_x, s_y): the X0-dependent right-hand-side
//    factors X0ᵀ V_A and X0 U_B, 2 K_x s_x s_y + 2 K_y s_x s_y; J_l shifted
//    HODLR solves of 2K_y columns of size s_x and 2K_x columns of size s_y,
//    each 2 n s + 4 K s log2(s / n) (leaf LU solves, then one rank-K product
//    pair per level below); the update X += Z Wᵀ of rank 2 J_l (K_x + K_y),
//    2 s_x s_y J_l · 2 (K_x + K_y).
// impl: Σ 2 m n k of the batched GEMMs the implementation launches per inner
// solve (the rational fADI form applies dense stacked resolvents).
static double hodlr_solve_flops(double s, double n, double K) {
  const double lv = s > n ? std::log2(s / n) : 0.0;
  return 2.0 * n * s + 4.0 * K * s * lv;
}

template <typename T>
static double impl_gemm_flops(const sylv_s* S, const Inner<T>& in) {
  double f = in.g_qxt.flops + in.g_qy.flops + in.g_qx.flops + in.g_qyt.flops;
  for (int l = 0; l < S->L; ++l) {
    const LevelSolve<T>& ls = in.lv[l];
    f += ls.g_rhs_x.flops + ls.g_rhs_y.flops + ls.g_update.flops;
    f += ls.r_rhs_h.flops + ls.r_rhs_g.flops + ls.r_apply.flops + ls.r_update.flops + ls.r_update2.flops;
  }
  return f;
}

extern "C" fde_status sylv_flop_model(sylv_t s, double* method_flops, double* impl_flops) {
  FDE_ARG(s != nullptr && method_flops != nullptr && impl_flops != nullptr, "NULL argument");
  const Tree& tx = s->ax->tree;
  const Tree& ty = s->ay->tree;
  const int nl = tx.nleaves();
  const double n = (double)tx.maxleaf;
  double m = 0.0;
  for (int i = 0; i < nl; ++i)
    for (int j = 0; j < nl; ++j) {
      const double a = tx.hi[tx.id(s->L, i)] - tx.lo[tx.id(s->L, i)];
      const double b = ty.hi[ty.id(s->L, j)] - ty.lo[ty.id(s->L, j)];
      m += 4.0 * a * b * (a + b);
    }
  for (int l = 0; l < s->L; ++l) {
    const double Kx = s->ax->K[l], Ky = s->ay->K[l];
    const double J = (l < (int)s->J.size()) ? s->J[l] : 0.0;
    for (int p = 0; p < (1 << l); ++p)
      for (int q = 0; q < (1 << l); ++q) {
        const double sx = tx.hi[tx.id(l, p)] - tx.lo[tx.id(l, p)];
        const double sy = ty.hi[ty.id(l, q)] - ty.lo[ty.id(l, q)];
        m += 2.0 * (Kx + Ky) * sx * sy;
        m += J * (2.0 * Ky * hodlr_solve_flops(sx, n, Kx) + 2.0 * Kx * hodlr_solve_flops(sy, n, Ky));
        m += 2.0 * sx * sy * J * 2.0 * (Kx + Ky);
      }
  }
  *method_flops = m;
  *impl_flops = (s->prec == FDE_FP32_REFINE) ? impl_gemm_flops(s, s->in32) : impl_gemm_flops(s, s->in64);
  return FDE_OK;
}

extern "C" void sylv_free(sylv_t s) { delete s; }

// Host-only views of the shift selection sylv_create performs (no device work).
extern "C" fde_status fde_fadi_shifts(double a, double b, double c, double d, double target, int jmax, int* J,
                                      double* h_alpha, double* h_beta, double* ratio) {
  FDE_ARG(J != nullptr && h_alpha != nullptr && h_beta != nullptr && ratio != nullptr, "NULL output");
  FDE_ARG(a > 0.0 && b > a && std::isfinite(b), "need 0 < a < b < inf");
  FDE_ARG(c > 0.0 && d > c && std::isfinite(d), "need 0 < c < d < inf");
  FDE_ARG(target > 0.0 && target < 1.0, "target must be in (0, 1)");
  FDE_ARG(jmax >= 1 && jmax <= 64, "jmax must be in [1, 64]");
  std::vector<double> al, be;
  *J = fde::select_shifts(a, b, c, d, target, jmax, al, be, ratio);
  for (int j = 0; j < *J; ++j) {
    h_alpha[j] = al[j];
    h_beta[j] = be[j];
  }
  return FDE_OK;
}

extern "C" fde_status fde_block_interval(const fde_op_params* p, int lo, int hi, double* lam_lo, double* lam_hi) {
  FDE_ARG(p != nullptr && lam_lo != nullptr && lam_hi != nullptr, "NULL argument");
  FDE_ARG(p->N >= 2 && p->N <= (1 << 20), "N must be in [2, 2^20]");
  FDE_ARG(p->alpha > 1.0 && p->alpha <= 2.0, "alpha must lie in (1, 2]");
  FDE_ARG(p->h > 0.0 && std::isfinite(p->h) && p->dt > 0.0 && std::isfinite(p->dt), "h, dt must be > 0");
  FDE_ARG(p->shift > 0.0 && std::isfinite(p->shift), "shift must be > 0");
  FDE_ARG(p->d_plus != nullptr && p->d_minus != nullptr, "d_plus / d_minus are NULL");
  FDE_ARG(0 <= lo && lo < hi && hi <= p->N, "need 0 <= lo < hi <= N");
  FDE_ARG(fde::host_readable(p->d_plus) && fde::host_readable(p->d_minus), "d_plus / d_minus must be host pointers");
  const int N = p->N;
  // g_0..g_{N+1} by the recurrence of Eq. (Grun) and their partial sums, as
  // sylv_create has them from the operator
  std::vector<double> S(N + 2), dp(p->d_plus, p->d_plus + N), dm(p->d_minus, p->d_minus + N);
  double gk = 1.0;
  long double acc = 1.0L;
  S[0] = 1.0;
  for (int k = 1; k < N + 2; ++k) {
    gk = gk * (1.0 - (p->alpha + 1.0) / k);
    acc += gk;
    S[k] = (double)acc;
  }
  const double cc = p->dt * pow(p->h, -p->alpha);
  fde::node_interval(S, dp, dm, cc, p->shift, p->alpha, lo, hi, lam_lo, lam_hi);
  return FDE_OK;
}

// Exposed for the time loop (fde_run.cu)
namespace fde {
fde_status sylv_step_internal(sylv_s* s, const double* C, double* X, cudaStream_t st, double* relres, int* sweeps,
                              const double* C_prev) {
  return sylv_step_impl(s, C, X, st, relres, sweeps, C_prev);
}
// Profiling brackets every launch with events, which a graph cannot hold:
// profiled steps run eagerly.
bool sylv_graph_steps(sylv_s* s) { return s->step_graph && !prof_enabled(); }
fde_status sylv_step_graph(sylv_s* s, const double* C, double* X, cudaStream_t st, const double* C_prev) {
  return step_graph_impl(s, C, X, st, C_prev);
}
fde_status sylv_graph_collect(sylv_s* s, cudaStream_t st, int* steps, int* sweeps_total, int* sweeps_max,
                              double* relres_max) {
  return graph_collect_impl(s, st, steps, sweeps_total, sweeps_max, relres_max);
}
int sylv_N(sylv_s* s) { return s->N; }
}  // namespace fde
