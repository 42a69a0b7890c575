// Leaf real Schur decomposition (Francis double-shift QR) and the
// quasi-triangular leaf Sylvester solve of the divide-and-conquer base case.
#include <float.h>
#include <math.h>

#include "schur.cuh"

namespace fde {

// Householder vector for a short vector x (len 2 or 3): P = I - beta v vᵀ,
// v[0] = 1, P x = ±||x|| e_1.  Computed redundantly by every thread.
__device__ __forceinline__ void house_small(const double* x, int len, double* v, double* beta) {
  double sig = 0.0;
  for (int i = 1; i < len; ++i) sig += x[i] * x[i];
  v[0] = 1.0;
  if (sig == 0.0) {
    for (int i = 1; i < len; ++i) v[i] = 0.0;
    *beta = 0.0;
    return;
  }
  const double mu = sqrt(x[0] * x[0] + sig);
  const double v0 = (x[0] <= 0.0) ? x[0] - mu : -sig / (x[0] + mu);
  *beta = 2.0 * v0 * v0 / (sig + v0 * v0);
  for (int i = 1; i < len; ++i) v[i] = x[i] / v0;
}

// rows r0..r0+len-1, columns c0..n-1:  H <- P H
__device__ __forceinline__ void refl_left(double* H, int ld, int n, int r0, int len, int c0, const double* v,
                                          double beta) {
  for (int c = c0 + threadIdx.x; c < n; c += blockDim.x) {
    double w = 0.0;
    for (int i = 0; i < len; ++i) w += v[i] * H[(r0 + i) + (size_t)c * ld];
    w *= beta;
    for (int i = 0; i < len; ++i) H[(r0 + i) + (size_t)c * ld] -= w * v[i];
  }
}
// rows 0..r1, columns c0..c0+len-1:  H <- H P
__device__ __forceinline__ void refl_right(double* H, int ld, int r1, int c0, int len, const double* v,
                                           double beta) {
  for (int r = threadIdx.x; r <= r1; r += blockDim.x) {
    double w = 0.0;
    for (int i = 0; i < len; ++i) w += H[r + (size_t)(c0 + i) * ld] * v[i];
    w *= beta;
    for (int i = 0; i < len; ++i) H[r + (size_t)(c0 + i) * ld] -= w * v[i];
  }
}

__global__ void __launch_bounds__(256) schur_kernel(double* Hall, double* Qall, int ld, size_t stride,
                                                   const int* __restrict__ dn, int* fail) {
  double* H = Hall + (size_t)blockIdx.x * stride;
  double* Q = Qall + (size_t)blockIdx.x * stride;
  const int n = dn[blockIdx.x];
  extern __shared__ double vbuf[];  // n
  __shared__ double red[32];
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) Q[(e % n) + (size_t)(e / n) * ld] = (e % n == e / n);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  // ---- Hessenberg reduction (Householder), accumulating Q
  for (int k = 0; k + 2 < n; ++k) {
    double part = 0.0;
    for (int i = k + 2 + threadIdx.x; i < n; i += blockDim.x) part += H[i + (size_t)k * ld] * H[i + (size_t)k * ld];
    const double sig = block_sum(part, red);
    const double x0 = H[(k + 1) + (size_t)k * ld];
    double beta = 0.0, v0 = 1.0;
    if (sig != 0.0) {
      const double mu = sqrt(x0 * x0 + sig);
      v0 = (x0 <= 0.0) ? x0 - mu : -sig / (x0 + mu);
      beta = 2.0 * v0 * v0 / (sig + v0 * v0);
    }
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x)
      vbuf[i] = (i == k + 1) ? 1.0 : H[i + (size_t)k * ld] / v0;
    __syncthreads();
    if (beta != 0.0) {
      // left: rows k+1..n-1, columns k..n-1 (one warp per column)
      for (int c = k + warp; c < n; c += nw) {
        double w = 0.0;
        for (int i = k + 1 + lane; i < n; i += 32) w += vbuf[i] * H[i + (size_t)c * ld];
        w = warp_sum(w) * beta;
        for (int i = k + 1 + lane; i < n; i += 32) H[i + (size_t)c * ld] -= w * vbuf[i];
      }
      __syncthreads();
      // right: rows 0..n-1, columns k+1..n-1 (one warp per row), same for Q
      for (int r = warp; r < 2 * n; r += nw) {
        double* M = (r < n) ? H : Q;
        const int rr = (r < n) ? r : r - n;
        double w = 0.0;
        for (int c = k + 1 + lane; c < n; c += 32) w += M[rr + (size_t)c * ld] * vbuf[c];
        w = warp_sum(w) * beta;
        for (int c = k + 1 + lane; c < n; c += 32) M[rr + (size_t)c * ld] -= w * vbuf[c];
      }
    }
    __syncthreads();
    for (int i = k + 2 + threadIdx.x; i < n; i += blockDim.x) H[i + (size_t)k * ld] = 0.0;
    __syncthreads();
  }
  // ---- Francis double-shift QR on the unreduced windows
  int p = n - 1, its = 0, total = 0;
  const int cap = 40 * n + 100;
  bool failed = false;
  while (p > 0) {
    // deflation search
    int l = p;
    while (l > 0) {
      double tst = fabs(H[(l - 1) + (size_t)(l - 1) * ld]) + fabs(H[l + (size_t)l * ld]);
      if (tst == 0.0) tst = 1e-300;
      if (fabs(H[l + (size_t)(l - 1) * ld]) <= DBL_EPSILON * tst) break;
      --l;
    }
    __syncthreads();
    if (l > 0 && threadIdx.x == 0) H[l + (size_t)(l - 1) * ld] = 0.0;
    __syncthreads();
    if (l == p) {
      --p;
      its = 0;
      continue;
    }
    if (l == p - 1) {
      // 2x2 block: split it if its eigenvalues are real
      const double a = H[(p - 1) + (size_t)(p - 1) * ld], b = H[(p - 1) + (size_t)p * ld];
      const double c = H[p + (size_t)(p - 1) * ld], d = H[p + (size_t)p * ld];
      const double hd = 0.5 * (a - d);
      const double disc = hd * hd + b * c;
      if (c != 0.0 && disc >= 0.0) {
        const double lam = 0.5 * (a + d) + (hd >= 0.0 ? 1.0 : -1.0) * sqrt(disc);
        double v1 = lam - d, v2 = c;       // from the second row
        double u1 = b, u2 = lam - a;       // from the first row
        if (u1 * u1 + u2 * u2 > v1 * v1 + v2 * v2) {
          v1 = u1;
          v2 = u2;
        }
        const double nv = sqrt(v1 * v1 + v2 * v2);
        const double cs = v1 / nv, sn = v2 / nv;
        __syncthreads();
        // left Gᵀ on rows p-1, p, columns p-1..n-1
        for (int cc = p - 1 + threadIdx.x; cc < n; cc += blockDim.x) {
          const double r1 = H[(p - 1) + (size_t)cc * ld], r2 = H[p + (size_t)cc * ld];
          H[(p - 1) + (size_t)cc * ld] = cs * r1 + sn * r2;
          H[p + (size_t)cc * ld] = -sn * r1 + cs * r2;
        }
        __syncthreads();
        // right G on columns p-1, p: rows 0..p of H, all rows of Q
        for (int r = threadIdx.x; r < 2 * n; r += blockDim.x) {
          double* M = (r < n) ? H : Q;
          const int rr = (r < n) ? r : r - n;
          if (r < n && rr > p) continue;
          const double c1 = M[rr + (size_t)(p - 1) * ld], c2 = M[rr + (size_t)p * ld];
          M[rr + (size_t)(p - 1) * ld] = cs * c1 + sn * c2;
          M[rr + (size_t)p * ld] = -sn * c1 + cs * c2;
        }
        __syncthreads();
        if (threadIdx.x == 0) H[p + (size_t)(p - 1) * ld] = 0.0;
        __syncthreads();
      }
      p -= 2;
      its = 0;
      continue;
    }
    if (++total > cap) {
      failed = true;
      break;
    }
    ++its;
    // shifts: eigenvalues of the trailing 2x2 (exceptional shift every 10 its)
    double s, t;
    if (its % 10 == 0) {
      const double ex = fabs(H[p + (size_t)(p - 1) * ld]) + fabs(H[(p - 1) + (size_t)(p - 2) * ld]);
      const double h11 = 0.75 * ex + H[p + (size_t)p * ld], h12 = -0.4375 * ex, h21 = ex, h22 = h11;
      s = h11 + h22;
      t = h11 * h22 - h12 * h21;
    } else {
      const double a = H[(p - 1) + (size_t)(p - 1) * ld], b = H[(p - 1) + (size_t)p * ld];
      const double c = H[p + (size_t)(p - 1) * ld], d = H[p + (size_t)p * ld];
      s = a + d;
      t = a * d - b * c;
    }
    double x = H[l + (size_t)l * ld] * H[l + (size_t)l * ld] + H[l + (size_t)(l + 1) * ld] * H[(l + 1) + (size_t)l * ld] -
               s * H[l + (size_t)l * ld] + t;
    double y = H[(l + 1) + (size_t)l * ld] * (H[l + (size_t)l * ld] + H[(l + 1) + (size_t)(l + 1) * ld] - s);
    double z = H[(l + 1) + (size_t)l * ld] * H[(l + 2) + (size_t)(l + 1) * ld];
    for (int k = l; k <= p - 2; ++k) {
      double xv[3] = {x, y, z}, v[3], beta;
      house_small(xv, 3, v, &beta);
      __syncthreads();
      if (beta != 0.0) {
        refl_left(H, ld, n, k, 3, max(l, k - 1), v, beta);
        __syncthreads();
        refl_right(H, ld, min(k + 3, p), k, 3, v, beta);
        refl_right(Q, ld, n - 1, k, 3, v, beta);
      }
      __syncthreads();
      x = H[(k + 1) + (size_t)k * ld];
      y = H[(k + 2) + (size_t)k * ld];
      if (k < p - 2) z = H[(k + 3) + (size_t)k * ld];
    }
    {
      double xv[2] = {x, y}, v[2], beta;
      house_small(xv, 2, v, &beta);
      __syncthreads();
      if (beta != 0.0) {
        refl_left(H, ld, n, p - 1, 2, p - 2, v, beta);
        __syncthreads();
        refl_right(H, ld, p, p - 1, 2, v, beta);
        refl_right(Q, ld, n - 1, p - 1, 2, v, beta);
      }
      __syncthreads();
    }
  }
  __syncthreads();
  // clean everything below the first subdiagonal
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    if (i > j + 1) H[i + (size_t)j * ld] = 0.0;
  }
  if (failed && threadIdx.x == 0) fail[blockIdx.x] = 1;
}

fde_status leaf_schur(double* H, double* Q, int ld, size_t stride, const int* d_n, int count, int* d_fail,
                      cudaStream_t st) {
  if (count == 0) return FDE_OK;
  ProfScope ps("schur", st);
  schur_kernel<<<count, 256, ld * sizeof(double), st>>>(H, Q, ld, stride, d_n, d_fail);
  FDE_LAUNCH("schur_kernel");
  return FDE_OK;
}

// ------------------------------------------------ quasi-triangular Sylvester
//
// For every leaf pair (p, q):  S Y + Y Rᵀ = F  in place of F, S = S_p (n1 x n1)
// and R = R_q (n2 x n2) upper quasi-triangular (real Schur forms: 2 x 2
// diagonal blocks for complex-conjugate pairs).  Bartels–Stewart order:
// columns of Y from the last to the first (Rᵀ is lower quasi-triangular),
// rows of each column from the last to the first (S upper quasi-triangular).
//
// One CTA per pair.  The rows are cut, from the bottom, into blocks of at most
// 32 rows that never split a 2 x 2 block of S; warp w owns block w (lane =
// row).  The columns are taken in groups of one, or two for a 2 x 2 block of
// R, from the right.  Warp w solves group g at barrier step g + w (a wavefront
// over the row blocks), so the rows below its block are final for that group
// when it starts: their values come from a ring of shared-memory columns, and
// the S coupling with them is a dot product per lane.  Inside the block the
// back substitution runs over the row groups bottom-up with shuffles only:
// the owner lane of a row group solves its small system (1, 2 or 4 unknowns,
// closed form from inverses each lane prepared before the chain) and
// broadcasts the solution, every lane removes its coupling.
//
// Each lane keeps, for its row, the right-hand sides of a window of 32
// consecutive columns in registers (yb[31] = the current group's last
// column).  Columns are further cut, from the right, into blocks of at most
// 32 that never split a 2 x 2 block of R: at the start of a block the window
// is reloaded from F minus the coupling with all columns solved before the
// block (read back from Y, written by this lane); after each group its
// coupling is subtracted from the rest of the window, which then shifts.
constexpr int kMaxRowWarps = 9;   // leaves up to 256 rows: blocks of >= 31 rows

// FP32: 128 registers.  A 96-register build (no spills, seven 3-warp CTAs per
// SM instead of five) was 19 % slower on the 1024-pair launches: the SM's
// issue slots, not the resident chains, bound the solve.
// Blocks of at most this many rows stage their R block in shared memory.
constexpr int kTrsylStageR = 64;

// Shared-memory elements in front of the diagonal blocks: the ring of solved
// columns, or the 32 x kStg staging tile of the coupling prologue (larger).
constexpr int kStg = 36;  // row stride of the staging tile: 16-byte aligned rows
__host__ __device__ inline int trsyl_ring_elems(int warps, int lmax) {
  const int ring = (warps + 1) * 2 * lmax;
  return ring > 32 * kStg ? ring : 32 * kStg;
}

// Left-looking block coupling (FP32): F -= S[block, after] Y[after, block]
// + Y[block, after] R[block, after]ᵀ for the rx rows and ry columns of the
// leaf after this block (Y there already solved).  Lane = row of the block
// (warp w: rows rlo..rlo+nr), 32 columns of F per pass in registers; the
// 32-row chunks of Y (S term) and 32-column chunks of R (R term) are staged
// in shared memory and read as broadcasts.  Every global load is issued in
// batches (16 per thread for a staging pass, 32 per lane for the lane's own
// S row or Y row chunk) ahead of its use, so each chunk waits on memory a
// few times instead of once per element.
template <typename T>
__device__ __forceinline__ void trsyl_stage(T* stg, const T* __restrict__ src, size_t s_minor, size_t s_major,
                                            int lim_minor, int lim_major) {
  // stg[major * kStg + minor] = src[minor * s_minor + major * s_major] inside
  // the limits, 0 outside; consecutive threads take consecutive minor indices
  for (int e0 = threadIdx.x; e0 < 32 * 32; e0 += 16 * blockDim.x) {
    T v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = e0 + u * (int)blockDim.x, mi = e & 31, ma = e >> 5;
      v[u] = (e < 32 * 32 && mi < lim_minor && ma < lim_major) ? src[mi * s_minor + ma * s_major] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      if (e < 32 * 32) stg[(e >> 5) * kStg + (e & 31)] = v[u];
    }
  }
}

template <typename T>
__device__ __forceinline__ void trsyl_couple(const T* __restrict__ S, const T* __restrict__ R, int ld,
                                             T* __restrict__ Y, int ldw, int n1, int n2, int rx, int ry, int rlo,
                                             int nr, T* stg) {
  const int lane = threadIdx.x & 31;
  const bool act = lane < nr;
  const int i = rlo + lane;
  for (int c0 = 0; c0 < n2; c0 += 32) {
    T acc[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] = T(0);
    const int nc = n2 - c0 < 32 ? n2 - c0 : 32;
    for (int t0 = 0; t0 < rx; t0 += 32) {
      const int tn = rx - t0 < 32 ? rx - t0 : 32;
      T sv[32];  // S(i, n1 + t0 + r)
#pragma unroll
      for (int r = 0; r < 32; ++r) sv[r] = (act && r < tn) ? S[i + (size_t)(n1 + t0 + r) * ld] : T(0);
      __syncthreads();
      // stg[r][c] = Y(n1 + t0 + r, c0 + c): minor = row r of Y (contiguous)
      trsyl_stage<T>(stg, Y + (n1 + t0) + (size_t)c0 * ldw, 1, (size_t)ldw, tn, nc);
      __syncthreads();
      // stg[c][r .. r + 3] as one 16-byte broadcast read
#pragma unroll
      for (int r = 0; r < 32; r += 4) {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const float4 v = *reinterpret_cast<const float4*>(stg + c * kStg + r);
          acc[c] += sv[r] * v.x;
          acc[c] += sv[r + 1] * v.y;
          acc[c] += sv[r + 2] * v.z;
          acc[c] += sv[r + 3] * v.w;
        }
      }
    }
    for (int t0 = 0; t0 < ry; t0 += 32) {
      const int tn = ry - t0 < 32 ? ry - t0 : 32;
      T yv[32];  // Y(i, n2 + t0 + r)
#pragma unroll
      for (int r = 0; r < 32; ++r) yv[r] = (act && r < tn) ? Y[i + (size_t)(n2 + t0 + r) * ldw] : T(0);
      __syncthreads();
      // stg[r][c] = R(c0 + c, n2 + t0 + r): minor = row c of R (contiguous)
      trsyl_stage<T>(stg, R + c0 + (size_t)(n2 + t0) * ld, 1, (size_t)ld, nc, tn);
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        const float4* row = reinterpret_cast<const float4*>(stg + r * kStg);
#pragma unroll
        for (int c = 0; c < 32; c += 4) {
          const float4 v = row[c >> 2];
          acc[c] += yv[r] * v.x;
          acc[c + 1] += yv[r] * v.y;
          acc[c + 2] += yv[r] * v.z;
          acc[c + 3] += yv[r] * v.w;
        }
      }
    }
    if (act) {
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c < nc) Y[i + (size_t)(c0 + c) * ldw] -= acc[c];
    }
  }
  __syncthreads();
}

// RSM: the R block (n2 x n2, ld lmax) is staged in shared memory at the start
// (blocks of blocked leaves), so the per-column reads of R on the dependency
// chain do not wait on L2.
template <typename T, bool RSM>
__global__ void __launch_bounds__(kMaxRowWarps * 32) __maxnreg__(sizeof(T) == 4 ? 128 : 168)
    trsyl_kernel(const T* __restrict__ Sall, const T* __restrict__ Rall, int ld, int lmax,
                 const __grid_constant__ TrsylSets sets, T* __restrict__ W, int ldw, int use_panel, int panel_elems) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the CTAs walk the sets in order: blocks [0, count_0) solve set 0, ...
  int b = (int)blockIdx.x, si = 0;
  while (si + 1 < sets.n && b >= sets.s[si].count) {
    b -= sets.s[si].count;
    ++si;
  }
  const TrsylSet& ps = sets.s[si];
  const int* __restrict__ soff_x = ps.soff_x;
  const int* __restrict__ lo_x = ps.lo_x;
  const int* __restrict__ n_x = ps.n_x;
  const int* __restrict__ soff_y = ps.soff_y;
  const int* __restrict__ lo_y = ps.lo_y;
  const int* __restrict__ n_y = ps.n_y;
  const int nx = ps.nx;
  const int p = b % nx, q = b / nx;
  const int n1 = n_x[p], n2 = n_y[q];
  if (n1 <= 0 || n2 <= 0) return;
  T* Y = W + lo_x[p] + (size_t)lo_y[q] * ldw;
  const T* S = Sall + soff_x[p];  // leading dimension ld
  const T* R = Rall + soff_y[q];
  // ring of solved columns: one slot per launched warp + 1 (a slot is reread
  // by the warps above for nwarps - 1 steps after it is written)
  const int ring = (int)(blockDim.x >> 5) + 1;
  T* ycol = reinterpret_cast<T*>(smem_raw);                  // ring x [col k | col k-1] x lmax
  T* sdiag = ycol + trsyl_ring_elems((int)(blockDim.x >> 5), lmax);  // per warp: its diagonal S block, 32 x 33
  T* panel = sdiag + (size_t)(blockDim.x >> 5) * 32 * 33;    // S panels (use_panel), see below
  int* cg_top = reinterpret_cast<int*>(panel + (use_panel ? panel_elems : 0));
  int* cg_info = cg_top + lmax;                              // bit 0: two columns; bit 1: block start
  int* cg_cblo = cg_info + lmax;                             // first column of the group's column block
  T* Rsm = reinterpret_cast<T*>(((uintptr_t)(cg_cblo + lmax) + 15) & ~(uintptr_t)15);  // RSM: R block, ld lmax
  __shared__ int rb_lo[kMaxRowWarps], rb_n[kMaxRowWarps], poff[kMaxRowWarps];
  __shared__ int s_ncg, s_nrb;
#define SS(i, j) S[(i) + (size_t)(j)*ld]
#define RR(i, j) R[(i) + (size_t)(j)*ld]
#define RV(i, j) (RSM ? Rsm[(i) + (j)*lmax] : __ldg(R + (i) + (size_t)(j)*ld))
  if constexpr (RSM) {
    // loads in batches of 16 per thread, then the stores
    const int tot = n2 * n2;
    for (int e0 = threadIdx.x; e0 < tot; e0 += 16 * blockDim.x) {
      T v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int e = e0 + u * (int)blockDim.x;
        v[u] = e < tot ? R[(e % n2) + (size_t)(e / n2) * ld] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int e = e0 + u * (int)blockDim.x;
        if (e < tot) Rsm[(e % n2) + (e / n2) * lmax] = v[u];
      }
    }
  }
  if (threadIdx.x == 0) {
    int w = 0;
    for (int hi = n1; hi > 0 && w < kMaxRowWarps; ++w) {
      int lo = hi - 32 > 0 ? hi - 32 : 0;
      if (lo > 0 && SS(lo, lo - 1) != T(0)) ++lo;  // keep the 2 x 2 block (lo-1, lo) together
      rb_lo[w] = lo;
      rb_n[w] = hi - lo;
      hi = lo;
    }
    s_nrb = w;
    // panel of warp w: S(block rows, columns rhi..n1-1), column-major, ld 33
    int off = 0;
    for (int v = 0; v < w; ++v) {
      poff[v] = off;
      off += 33 * (n1 - (rb_lo[v] + rb_n[v]));
    }
  }
  // the column tables come from the second warp's first thread, or from
  // thread 0 as well when the CTA is a single warp (leaves of <= 31 rows)
  if (threadIdx.x == (blockDim.x > 32 ? 32u : 0u)) {
    int g = 0, cb_lo = n2;
    for (int k = n2 - 1; k >= 0;) {
      int info = 0;
      if (k < cb_lo) {  // a new column block [cb_lo, k + 1)
        int lo = k + 1 - 32 > 0 ? k + 1 - 32 : 0;
        if (lo > 0 && RR(lo, lo - 1) != T(0)) ++lo;
        cb_lo = lo;
        info |= 2;
      }
      const int gs = (k > 0 && RR(k, k - 1) != T(0)) ? 2 : 1;
      cg_top[g] = k;
      cg_info[g] = info | (gs == 2 ? 1 : 0);
      cg_cblo[g] = cb_lo;
      ++g;
      k -= gs;
    }
    s_ncg = g;
  }
  __syncthreads();
  const int ncg = s_ncg, nrb = s_nrb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if constexpr (sizeof(T) == sizeof(float)) {
    const int rx = ps.rest_x ? ps.rest_x[p] : 0, ry = ps.rest_y ? ps.rest_y[q] : 0;
    if (rx > 0 || ry > 0)  // the staging tile overlays the (not yet used) ring
      trsyl_couple<T>(S, R, ld, Y, ldw, n1, n2, rx, ry, warp < nrb ? rb_lo[warp] : 0, warp < nrb ? rb_n[warp] : 0,
                      ycol);
  }
  {
    // every warp's diagonal block (the back-substitution chain reads a column
    // per row), without the lane's own 1 x 1 or 2 x 2 diagonal block: the
    // chain then leaves a solved row's right-hand side as it is, and the row
    // solves its own unknown from it after the chain
    const int w_ = threadIdx.x >> 5, l_ = threadIdx.x & 31;
    const int vlo = w_ < s_nrb ? rb_lo[w_] : 0, vn = w_ < s_nrb ? rb_n[w_] : 0;
    T* sv = sdiag + (size_t)w_ * 32 * 33 + l_;
    const bool pr_lo = l_ < vn && l_ > 0 && SS(vlo + l_, vlo + l_ - 1) != T(0);       // pair (l_-1, l_)
    const bool pr_hi = l_ + 1 < vn && SS(vlo + l_ + 1, vlo + l_) != T(0);            // pair (l_, l_+1)
    for (int t = 0; t < 32; ++t) {
      const bool own = t == l_ || (t == l_ - 1 && pr_lo) || (t == l_ + 1 && pr_hi);
      sv[t * 33] = (l_ < vn && t < vn && !own) ? SS(vlo + l_, vlo + t) : T(0);
    }
  }
  if (use_panel) {
    // the S coupling of every column group rereads these entries: stage them
    for (int v = 0; v < nrb; ++v) {
      const int vlo = rb_lo[v], vn = rb_n[v], vhi = vlo + vn, cols = n1 - vhi;
      T* pv = panel + poff[v];
      for (int e = threadIdx.x; e < 32 * cols; e += blockDim.x) {
        const int r = e & 31, c = e >> 5;
        pv[c * 33 + r] = r < vn ? SS(vlo + r, vhi + c) : T(0);
      }
    }
  }
  __syncthreads();
  const bool wact = warp < nrb;
  const int rlo = wact ? rb_lo[warp] : 0, nr = wact ? rb_n[warp] : 0, rhi = rlo + nr;
  const bool active = lane < nr;
  const int i = rlo + lane;
  // this lane's row of the diagonal block of S (sd[t * 33] = S(i, rlo + t),
  // filled before the first barrier below), and its 2 x 2 block if any
  T* sd = sdiag + (size_t)warp * 32 * 33 + lane;
  const T sii = active ? SS(i, i) : T(1);
  const bool bottom = active && lane > 0 && SS(i, i - 1) != T(0);
  const unsigned pair_mask = __ballot_sync(0xffffffffu, bottom);  // bit r: rows (r-1, r) form a 2 x 2 block
  T s00 = T(0), s01 = T(0), s10 = T(0), s11 = T(0);  // the 2 x 2 block of S (bottom lanes)
  if (bottom) {
    s00 = SS(i - 1, i - 1);
    s01 = SS(i - 1, i);
    s10 = SS(i, i - 1);
    s11 = sii;
  }
  T yb[32];
#pragma unroll
  for (int t = 0; t < 32; ++t) yb[t] = T(0);
  const int nsteps = ncg + (int)(blockDim.x >> 5) - 1;
  for (int m = 0; m < nsteps; ++m) {
    const int g = m - warp;
    if (wact && g >= 0 && g < ncg) {
      const int k = cg_top[g], info = cg_info[g], cb_lo = cg_cblo[g];
      const bool two = (info & 1) != 0;
      if (info & 2) {
        // block start: window columns k-31..k = F minus the coupling with the
        // columns l > k solved before (Y(i, l), written by this lane)
#pragma unroll
        for (int t = 0; t < 32; ++t) {
          const int col = k - 31 + t;
          yb[t] = (active && col >= cb_lo) ? Y[i + (size_t)col * ldw] : T(0);
        }
#pragma unroll 4
        for (int l = k + 1; l < n2; ++l) {
          const T yl = active ? Y[i + (size_t)l * ldw] : T(0);
#pragma unroll
          for (int t = 0; t < 32; ++t) {
            const int col = k - 31 + t;
            if (col >= cb_lo) yb[t] -= RV(col, l) * yl;
          }
        }
      }
      const int slot = g % ring;
      T* yk = ycol + (size_t)slot * 2 * lmax;  // column k, then column k-1
      T fb = yb[31], fa = two ? yb[30] : T(0);  // fb: column k, fa: column k-1
      // coupling with the rows below this block (final, from the ring)
      if (active) {
        if (use_panel) {
          const T* pw = panel + poff[warp] + lane;
          T b0 = T(0), b1 = T(0), a0 = T(0), a1 = T(0);
          int j = rhi;
          for (; j + 1 < n1; j += 2) {
            const T s0 = pw[(j - rhi) * 33], s1 = pw[(j + 1 - rhi) * 33];
            b0 += s0 * yk[j];
            b1 += s1 * yk[j + 1];
            if (two) {
              a0 += s0 * yk[lmax + j];
              a1 += s1 * yk[lmax + j + 1];
            }
          }
          if (j < n1) {
            const T s0 = pw[(j - rhi) * 33];
            b0 += s0 * yk[j];
            if (two) a0 += s0 * yk[lmax + j];
          }
          fb -= b0 + b1;
          fa -= a0 + a1;
        } else {
          for (int j = rhi; j < n1; ++j) {
            const T sij = __ldg(S + i + (size_t)j * ld);
            fb -= sij * yk[j];
            if (two) fa -= sij * yk[lmax + j];
          }
        }
      }
      T ya_fin = T(0), yb_fin = T(0);
      if (!two) {
        const T mu = RV(k, k);
        T inv = T(1) / (sii + mu), p00 = T(0), p01 = T(0), p10 = T(0), p11 = T(0);
        if (bottom) {  // inverse of (S_2x2 + mu I)
          const T d = (s00 + mu) * (s11 + mu) - s01 * s10;
          p00 = (s11 + mu) / d;
          p01 = -s01 / d;
          p10 = -s10 / d;
          p11 = (s00 + mu) / d;
        }
        // rows bottom-up, unrolled (a block has at most 32 rows): the owner
        // lane's solution is broadcast, every row removes its coupling (the
        // owner's own diagonal block is zero in sd, so its fb stays final)
#pragma unroll
        for (int rr = 31; rr >= 0; --rr) {
          if (rr < nr) {
            if (rr > 0 && ((pair_mask >> rr) & 1u)) {
              const T ftop = __shfl_sync(0xffffffffu, fb, rr - 1);
              const T y0 = __shfl_sync(0xffffffffu, p00 * ftop + p01 * fb, rr);
              const T y1 = __shfl_sync(0xffffffffu, p10 * ftop + p11 * fb, rr);
              fb -= sd[(rr - 1) * 33] * y0 + sd[rr * 33] * y1;
            } else if (!(rr + 1 < nr && ((pair_mask >> (rr + 1)) & 1u))) {
              const T y = __shfl_sync(0xffffffffu, fb * inv, rr);
              fb -= sd[rr * 33] * y;
            }
          }
        }
        // this row's unknown from its final right-hand side (2 x 2 blocks:
        // solved by the bottom lane, the top one's value shifted up)
        const T fdn = __shfl_up_sync(0xffffffffu, fb, 1);
        const T ytop = p00 * fdn + p01 * fb, ybot = p10 * fdn + p11 * fb;
        const T ytop_below = __shfl_down_sync(0xffffffffu, ytop, 1);
        const bool is_top = lane + 1 < nr && ((pair_mask >> (lane + 1)) & 1u);
        yb_fin = bottom ? ybot : (is_top ? ytop_below : fb * inv);
      } else {
        // R block [[a, b], [c, d]] couples columns k-1 (unknown 1) and k (unknown 2)
        const T a = RV(k - 1, k - 1), b = RV(k - 1, k);
        const T c = RV(k, k - 1), d = RV(k, k);
        // 1 x 1 row: [[s+a, b], [c, s+d]]^{-1}
        const T det1 = (sii + a) * (sii + d) - b * c;
        const T e00 = (sii + d) / det1, e01 = -b / det1, e10 = -c / det1, e11 = (sii + a) / det1;
        // 2 x 2 row block S2: the blocks of I(x)S2 + R(x)I commute, so the
        // inverse needs only Δ = (S2 + aI)(S2 + dI) - bc I
        T q00 = T(0), q01 = T(0), q10 = T(0), q11 = T(0);
        if (bottom) {
          const T tr = s00 + s11 + a + d, cst = a * d - b * c;
          const T D00 = s00 * s00 + s01 * s10 + (a + d) * s00 + cst, D01 = s01 * tr;
          const T D10 = s10 * tr, D11 = s10 * s01 + s11 * s11 + (a + d) * s11 + cst;
          const T dd = D00 * D11 - D01 * D10;
          q00 = D11 / dd;
          q01 = -D01 / dd;
          q10 = -D10 / dd;
          q11 = D00 / dd;
        }
        for (int rr = nr - 1; rr >= 0;) {
          if (rr > 0 && ((pair_mask >> rr) & 1u)) {
            const T st = sd[(rr - 1) * 33], sb = sd[rr * 33];
            const T fat = __shfl_sync(0xffffffffu, fa, rr - 1), fbt = __shfl_sync(0xffffffffu, fb, rr - 1);
            T u0 = T(0), u1 = T(0), v0 = T(0), v1 = T(0);  // column k-1 (top, bottom), column k
            if (lane == rr) {
              const T g1t = (s00 + d) * fat + s01 * fa - b * fbt, g1b = s10 * fat + (s11 + d) * fa - b * fb;
              const T g2t = (s00 + a) * fbt + s01 * fb - c * fat, g2b = s10 * fbt + (s11 + a) * fb - c * fa;
              u0 = q00 * g1t + q01 * g1b;
              u1 = q10 * g1t + q11 * g1b;
              v0 = q00 * g2t + q01 * g2b;
              v1 = q10 * g2t + q11 * g2b;
            }
            u0 = __shfl_sync(0xffffffffu, u0, rr);
            u1 = __shfl_sync(0xffffffffu, u1, rr);
            v0 = __shfl_sync(0xffffffffu, v0, rr);
            v1 = __shfl_sync(0xffffffffu, v1, rr);
            if (lane == rr - 1) {
              ya_fin = u0;
              yb_fin = v0;
            }
            if (lane == rr) {
              ya_fin = u1;
              yb_fin = v1;
            }
            fa -= st * u0 + sb * u1;
            fb -= st * v0 + sb * v1;
            rr -= 2;
          } else {
            const T sb = sd[rr * 33];
            T u = T(0), v = T(0);
            if (lane == rr) {
              u = e00 * fa + e01 * fb;
              v = e10 * fa + e11 * fb;
            }
            u = __shfl_sync(0xffffffffu, u, rr);
            v = __shfl_sync(0xffffffffu, v, rr);
            if (lane == rr) {
              ya_fin = u;
              yb_fin = v;
            }
            fa -= sb * u;
            fb -= sb * v;
            rr -= 1;
          }
        }
      }
      if (active) {
        Y[i + (size_t)k * ldw] = yb_fin;
        yk[i] = yb_fin;
        if (two) {
          Y[i + (size_t)(k - 1) * ldw] = ya_fin;
          yk[lmax + i] = ya_fin;
        }
      }
      // remove the group's coupling from the rest of the window, then shift it
#pragma unroll
      for (int t = 0; t < 31; ++t) {
        const int col = k - 31 + t;
        if (col >= cb_lo && (t < 30 || !two)) {
          T v = RV(col, k) * yb_fin;
          if (two) v += RV(col, k - 1) * ya_fin;
          yb[t] -= v;
        }
      }
      if (two) {
#pragma unroll
        for (int t = 31; t >= 2; --t) yb[t] = yb[t - 2];
        yb[1] = T(0);
        yb[0] = T(0);
      } else {
#pragma unroll
        for (int t = 31; t >= 1; --t) yb[t] = yb[t - 1];
        yb[0] = T(0);
      }
    }
    __syncthreads();
  }
#undef SS
#undef RR
#undef RV
}

// Blocks of at most 32 x 32 (FP32): an anti-diagonal wavefront over the
// block's entries instead of a column-by-column back substitution.  Lane =
// row i.  Rows are grouped into units (1 row, or the 2 rows of a 2 x 2 block
// of S) and columns into units from the right (1 column, or the 2 of a 2 x 2
// block of R); the unit of row i solves column unit u at step base_i + u,
// base_i = the number of row units below it.  At that step every entry it
// needs is solved: the rows below in the same columns (earlier steps of the
// lanes below) and its own row to the right (its earlier steps).  So each
// step is one pull: rhs = F(i, c) - Σ_{k below} S(i, k) Y(k, c)
// - Σ_{l right} Y(i, l) R(c, l), independent loads and products, then the
// unit's 1, 2 or 4-unknown solve.  Y (holding F until solved) and R sit in
// shared memory, row i of S in registers.
__global__ void __launch_bounds__(32, 16) trsyl_wave_kernel(const float* __restrict__ Sall, const float* __restrict__ Rall,
                                                        int ld, const __grid_constant__ TrsylSets sets,
                                                        float* __restrict__ W, int ldw) {
  __shared__ float Ys[32][33];    // Ys[i][c]: F(i, c), then Y(i, c)
  __shared__ float Rs[32][33];    // Rs[c][l] = R(c, l)
  __shared__ __align__(16) float stg[32 * kStg];  // staging tile of the coupling prologue
  __shared__ int cu_c0[32], cu_w[32];  // column unit u (from the right): first column, width
  __shared__ int s_ncu, s_nru;
  int b = (int)blockIdx.x, si = 0;
  while (si + 1 < sets.n && b >= sets.s[si].count) {
    b -= sets.s[si].count;
    ++si;
  }
  const TrsylSet& ps = sets.s[si];
  const int p = b % ps.nx, q = b / ps.nx;
  const int n1 = ps.n_x[p], n2 = ps.n_y[q];
  if (n1 <= 0 || n2 <= 0) return;
  float* Y = W + ps.lo_x[p] + (size_t)ps.lo_y[q] * ldw;
  const float* S = Sall + ps.soff_x[p];
  const float* R = Rall + ps.soff_y[q];
  const int lane = threadIdx.x;
  {
    const int rx = ps.rest_x ? ps.rest_x[p] : 0, ry = ps.rest_y ? ps.rest_y[q] : 0;
    if (rx > 0 || ry > 0) trsyl_couple<float>(S, R, ld, Y, ldw, n1, n2, rx, ry, 0, n1, stg);
  }
  // F (after the coupling) and R into shared memory, zeros outside the block
  // (every entry the steps read is finite); coalesced along rows
  for (int c = 0; c < 32; ++c) {
    Ys[lane][c] = (lane < n1 && c < n2) ? Y[lane + (size_t)c * ldw] : 0.f;
    Rs[lane][c] = (lane < n2 && c < n2) ? R[lane + (size_t)c * ld] : 0.f;
  }
  // this lane's row of S beyond its own row unit, and its unit's 2 x 2 block
  const bool act = lane < n1;
  const bool bottom = act && lane > 0 && S[lane + (size_t)(lane - 1) * ld] != 0.f;
  const bool top = lane + 1 < n1 && S[(lane + 1) + (size_t)lane * ld] != 0.f;
  const int own_hi = top ? lane + 1 : lane;  // last row of this lane's unit
  float srow[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) srow[k] = (act && k > own_hi && k < n1) ? S[lane + (size_t)k * ld] : 0.f;
  const float sii = act ? S[lane + (size_t)lane * ld] : 1.f;
  float s00 = 0.f, s01 = 0.f, s10 = 0.f, s11 = 0.f;  // the unit's 2 x 2 block (both lanes)
  if (bottom) {
    s00 = S[(lane - 1) + (size_t)(lane - 1) * ld];
    s01 = S[(lane - 1) + (size_t)lane * ld];
    s10 = S[lane + (size_t)(lane - 1) * ld];
    s11 = sii;
  } else if (top) {
    s00 = sii;
    s01 = S[lane + (size_t)(lane + 1) * ld];
    s10 = S[(lane + 1) + (size_t)lane * ld];
    s11 = S[(lane + 1) + (size_t)(lane + 1) * ld];
  }
  // row units below each row (ballot over the unit starts), column units
  const unsigned unit_start = __ballot_sync(0xffffffffu, act && !bottom);  // a unit's top row
  const int base = __popc(unit_start & ~((2u << own_hi) - 1u));              // units strictly below
  if (lane == 0) {
    int u = 0;
    for (int c = n2 - 1; c >= 0; ++u) {
      const bool pair = c > 0 && R[c + (size_t)(c - 1) * ld] != 0.f;
      cu_c0[u] = pair ? c - 1 : c;
      cu_w[u] = pair ? 2 : 1;
      c -= pair ? 2 : 1;
    }
    s_ncu = u;
    s_nru = __popc(unit_start);
  }
  __syncwarp();
  const int ncu = s_ncu, nsteps = s_nru + ncu - 1;
  for (int t = 0; t < nsteps; ++t) {
    const int u = t - base;
    const bool go = act && u >= 0 && u < ncu;
    const int c0 = go ? cu_c0[u] : 0, cw = go ? cu_w[u] : 1;
    float r0 = go ? Ys[lane][c0] : 0.f, r1 = (go && cw == 2) ? Ys[lane][c0 + 1] : 0.f;
    // rows below the unit in the unit's columns (solved at earlier steps)
    float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
#pragma unroll
    for (int k = 0; k < 32; k += 2) {
      a0 += srow[k] * Ys[k][c0];
      a1 += srow[k + 1] * Ys[k + 1][c0];
      if (cw == 2) {
        b0 += srow[k] * Ys[k][c0 + 1];
        b1 += srow[k + 1] * Ys[k + 1][c0 + 1];
      }
    }
    r0 -= a0 + a1;
    r1 -= b0 + b1;
    // this row right of the unit (solved at earlier steps of this lane)
    const int l0 = c0 + cw;
    a0 = a1 = b0 = b1 = 0.f;
#pragma unroll
    for (int l = 0; l < 32; l += 2) {
      const bool v0 = l >= l0 && l < n2, v1 = l + 1 >= l0 && l + 1 < n2;
      const float y0 = v0 ? Ys[lane][l] : 0.f, y1 = v1 ? Ys[lane][l + 1] : 0.f;
      a0 += y0 * Rs[c0][l];
      a1 += y1 * Rs[c0][l + 1];
      if (cw == 2) {
        b0 += y0 * Rs[c0 + 1][l];
        b1 += y1 * Rs[c0 + 1][l + 1];
      }
    }
    r0 -= a0 + a1;
    r1 -= b0 + b1;
    // the unit's solve; pairs of rows exchange their right-hand sides
    const bool prow = bottom || top;
    const int partner = bottom ? lane - 1 : lane + 1;
    const float pr0 = __shfl_sync(0xffffffffu, r0, prow ? partner : lane);
    const float pr1 = __shfl_sync(0xffffffffu, r1, prow ? partner : lane);
    if (go) {
      const float ra = Rs[c0][c0];
      float y0, y1 = 0.f;
      if (!prow && cw == 1) {
        y0 = r0 / (sii + ra);
      } else if (!prow) {
        // [[s + a, b], [c, s + d]] (y(i, c0), y(i, c0 + 1))ᵀ = (r0, r1)ᵀ
        const float bb = Rs[c0][c0 + 1], cc = Rs[c0 + 1][c0], dd = Rs[c0 + 1][c0 + 1];
        const float det = (sii + ra) * (sii + dd) - bb * cc;
        y0 = ((sii + dd) * r0 - bb * r1) / det;
        y1 = ((sii + ra) * r1 - cc * r0) / det;
      } else {
        // top / bottom right-hand sides of the unit
        const float ft0 = bottom ? pr0 : r0, fb0 = bottom ? r0 : pr0;
        if (cw == 1) {
          const float d = (s00 + ra) * (s11 + ra) - s01 * s10;
          const float yt = ((s11 + ra) * ft0 - s01 * fb0) / d;
          const float yb = ((s00 + ra) * fb0 - s10 * ft0) / d;
          y0 = bottom ? yb : yt;
        } else {
          const float ft1 = bottom ? pr1 : r1, fb1 = bottom ? r1 : pr1;
          const float a = ra, bq = Rs[c0][c0 + 1], cq = Rs[c0 + 1][c0], dq = Rs[c0 + 1][c0 + 1];
          // the blocks of I (x) S2 + R2 (x) I commute: Δ = (S2 + aI)(S2 + dI) - bc I
          const float tr = s00 + s11 + a + dq, cst = a * dq - bq * cq;
          const float D00 = s00 * s00 + s01 * s10 + (a + dq) * s00 + cst, D01 = s01 * tr;
          const float D10 = s10 * tr, D11 = s10 * s01 + s11 * s11 + (a + dq) * s11 + cst;
          const float dd = D00 * D11 - D01 * D10;
          const float q00 = D11 / dd, q01 = -D01 / dd, q10 = -D10 / dd, q11 = D00 / dd;
          const float g1t = (s00 + dq) * ft0 + s01 * fb0 - bq * ft1, g1b = s10 * ft0 + (s11 + dq) * fb0 - bq * fb1;
          const float g2t = (s00 + a) * ft1 + s01 * fb1 - cq * ft0, g2b = s10 * ft1 + (s11 + a) * fb1 - cq * fb0;
          const float u0 = q00 * g1t + q01 * g1b, u1 = q10 * g1t + q11 * g1b;  // column c0: top, bottom
          const float v0 = q00 * g2t + q01 * g2b, v1 = q10 * g2t + q11 * g2b;  // column c0 + 1
          y0 = bottom ? u1 : u0;
          y1 = bottom ? v1 : v0;
        }
      }
      Ys[lane][c0] = y0;
      if (cw == 2) Ys[lane][c0 + 1] = y1;
    }
    __syncwarp();
  }
  if (act)
    for (int c = 0; c < n2; ++c) Y[lane + (size_t)c * ldw] = Ys[lane][c];
}

template <typename T>
fde_status leaf_trsyl(const T* S, const T* R, int ld, int lmax, const int* d_soff_x, const int* d_lo_x,
                      const int* d_n_x, int nx, const int* d_soff_y, const int* d_lo_y, const int* d_n_y, int ny,
                      T* W, int ldw, cudaStream_t st, double flops) {
  TrsylSets sets;
  sets.s[0] = TrsylSet{d_soff_x, d_lo_x, d_n_x, nx, d_soff_y, d_lo_y, d_n_y, nx * ny};
  sets.n = 1;
  return leaf_trsyl_sets<T>(S, R, ld, lmax, sets, W, ldw, st, flops);
}

// FDE_TRSYL_WAVE=0 keeps blocks of at most 32 x 32 on trsyl_kernel.
static bool trsyl_wave_enabled() {
  static const bool on = [] {
    const char* e = getenv("FDE_TRSYL_WAVE");
    return !(e && e[0] == '0');
  }();
  return on;
}

template <typename T>
fde_status leaf_trsyl_sets(const T* S, const T* R, int ld, int lmax, const TrsylSets& sets, T* W, int ldw,
                           cudaStream_t st, double flops) {
  if (lmax > 32 * kMaxRowWarps - kMaxRowWarps || lmax > ld) {
    set_error("leaf_trsyl: problem size %d above %d (or above ld %d)", lmax, 32 * kMaxRowWarps - kMaxRowWarps, ld);
    return FDE_ERR_ARG;
  }
  if (sets.n < 1 || sets.n > kTrsylMaxSets) {
    set_error("leaf_trsyl: %d sets (1..%d)", sets.n, kTrsylMaxSets);
    return FDE_ERR_ARG;
  }
  if (sizeof(T) != sizeof(float))
    for (int k = 0; k < sets.n; ++k)
      if (sets.s[k].rest_x || sets.s[k].rest_y) {
        set_error("leaf_trsyl: block coupling is FP32 only");
        return FDE_ERR_ARG;
      }
  // blocks of at most 32 rows need one warp; longer ones are cut into blocks
  // of 31 or 32 rows (a cut never splits a 2 x 2 block)
  int warps = lmax <= 32 ? 1 : (lmax + 30) / 31;
  if (warps > kMaxRowWarps) warps = kMaxRowWarps;
  // largest panel total: warp w has at most 32 w rows below its block
  int panel_elems = 0;
  for (int w = 0; w < warps; ++w) panel_elems += 33 * (32 * w < lmax ? 32 * w : lmax);
  const size_t base = ((size_t)trsyl_ring_elems(warps, lmax) + (size_t)warps * 32 * 33) * sizeof(T) +
                      3 * (size_t)lmax * sizeof(int);
  const size_t with_panel = base + (size_t)panel_elems * sizeof(T);
  const size_t limit = 224 * 1024;
  const int use_panel = with_panel <= limit ? 1 : 0;
  const size_t smem = use_panel ? with_panel : base;
  // small blocks: R staged in shared memory (16 bytes of alignment slack)
  const bool rsm = lmax <= kTrsylStageR;
  const size_t smem_launch = smem + (rsm ? 16 + (size_t)lmax * lmax * sizeof(T) : 0);
  static const cudaError_t attr0 =
      cudaFuncSetAttribute(trsyl_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit);
  static const cudaError_t attr1 = cudaFuncSetAttribute(trsyl_kernel<T, true>,
                                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit);
  FDE_CUDA(attr0);
  FDE_CUDA(attr1);
  if (smem_launch > limit) {
    set_error("leaf_trsyl: %zu bytes of shared memory above %zu", smem_launch, limit);
    return FDE_ERR_ARG;
  }
  ProfScope ps(sizeof(T) == 4 ? "trsyl32" : "trsyl64", st, flops, 1);
  long long blocks = 0;
  for (int k = 0; k < sets.n; ++k) blocks += sets.s[k].count;
  if (blocks == 0) return FDE_OK;
  if constexpr (sizeof(T) == sizeof(float)) {
    if (lmax <= 32 && trsyl_wave_enabled()) {
      trsyl_wave_kernel<<<(unsigned)blocks, 32, 0, st>>>(S, R, ld, sets, W, ldw);
      FDE_LAUNCH("trsyl_wave_kernel");
      return FDE_OK;
    }
  }
  if (rsm)
    trsyl_kernel<T, true><<<(unsigned)blocks, warps * 32, smem_launch, st>>>(S, R, ld, lmax, sets, W, ldw, use_panel,
                                                                             panel_elems);
  else
    trsyl_kernel<T, false><<<(unsigned)blocks, warps * 32, smem_launch, st>>>(S, R, ld, lmax, sets, W, ldw,
                                                                              use_panel, panel_elems);
  FDE_LAUNCH("trsyl_kernel");
  return FDE_OK;
}

template fde_status leaf_trsyl_sets<double>(const double*, const double*, int, int, const TrsylSets&, double*, int,
                                            cudaStream_t, double);
template fde_status leaf_trsyl_sets<float>(const float*, const float*, int, int, const TrsylSets&, float*, int,
                                           cudaStream_t, double);
template fde_status leaf_trsyl<double>(const double*, const double*, int, int, const int*, const int*, const int*,
                                       int, const int*, const int*, const int*, int, double*, int, cudaStream_t, double);
template fde_status leaf_trsyl<float>(const float*, const float*, int, int, const int*, const int*, const int*, int,
                                      const int*, const int*, const int*, int, float*, int, cudaStream_t, double);

}  // namespace fde
