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
// Small dense solve M y = b (size m <= 4) by Gaussian elimination with
// partial pivoting.
template <typename T>
__device__ void small_solve(T M[4][4], T b[4], int m) {
  for (int k = 0; k < m; ++k) {
    int pv = k;
    for (int i = k + 1; i < m; ++i)
      if (fabs((double)M[i][k]) > fabs((double)M[pv][k])) pv = i;
    if (pv != k) {
      for (int j = 0; j < m; ++j) {
        T t = M[k][j];
        M[k][j] = M[pv][j];
        M[pv][j] = t;
      }
      T t = b[k];
      b[k] = b[pv];
      b[pv] = t;
    }
    for (int i = k + 1; i < m; ++i) {
      const T f = M[i][k] / M[k][k];
      for (int j = k; j < m; ++j) M[i][j] -= f * M[k][j];
      b[i] -= f * b[k];
    }
  }
  for (int k = m - 1; k >= 0; --k) {
    T s = b[k];
    for (int j = k + 1; j < m; ++j) s -= M[k][j] * b[j];
    b[k] = s / M[k][k];
  }
}

// One CTA per leaf pair, solving  S Y + Y Rᵀ = C  (S, R upper quasi-triangular)
// by back substitution over the diagonal blocks (1x1 / 2x2) of both factors.
// Column groups (R's diagonal blocks, last first) are handled in waves of up
// to kWarps groups, one warp per group.  Inside a wave the warps advance as a
// wavefront: warp g solves row group ρ (S's blocks, bottom first) at step
// ρ + g, so every coupling it needs — rows below in its own columns and the
// same rows in the later columns of the wave — was finalised at earlier steps.
// A small coupled system (I ⊗ S_bb + R_bb ⊗ I) vec Y_b = vec B_b of size <= 4
// is solved per (row group, column group).  Before a wave, its columns get
// the contribution of all columns solved in earlier waves (a GEMM-like update).
constexpr int kWarps = 32;

template <typename T>
__global__ void __launch_bounds__(kWarps * 32) trsyl_kernel(const T* __restrict__ Sall, const T* __restrict__ Rall,
                                                           int lmax, const int* __restrict__ lo_x,
                                                           const int* __restrict__ n_x, int nx,
                                                           const int* __restrict__ lo_y,
                                                           const int* __restrict__ n_y, T* W, int ldw, int mode) {
  // mode 0: everything in global memory; 1: Y in shared; 2: Y, S, R in shared.
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = blockIdx.x % nx, q = blockIdx.x / nx;
  const int n1 = n_x[p], n2 = n_y[q];
  T* Yg = W + lo_x[p] + (size_t)lo_y[q] * ldw;
  int* rg0 = (int*)smem_raw;  // start row of row group ρ (bottom first)
  int* rgs = rg0 + lmax;      // its size
  int* cg0 = rgs + lmax;      // start column of column group γ (last first)
  int* cgs = cg0 + lmax;
  __shared__ int s_nrg, s_ncg;
  const T* S = Sall + (size_t)p * lmax * lmax;
  const T* R = Rall + (size_t)q * lmax * lmax;
  int lds = lmax, ldr = lmax;
  T* Y = Yg;
  int ldy = ldw;
  T* dyn = (T*)(cgs + lmax);
  if (mode >= 1) {
    // odd leading dimensions keep the strided (row-wise) accesses conflict free
    Y = dyn;
    ldy = n1 | 1;
    for (int e = threadIdx.x; e < n1 * n2; e += blockDim.x)
      Y[e % n1 + (e / n1) * ldy] = Yg[e % n1 + (size_t)(e / n1) * ldw];
    dyn += (size_t)ldy * n2;
  }
  if (mode == 2) {
    T* Ss = dyn;
    const int ls = n1 | 1;
    for (int e = threadIdx.x; e < n1 * n1; e += blockDim.x) Ss[e % n1 + (e / n1) * ls] = S[e % n1 + (size_t)(e / n1) * lmax];
    dyn += (size_t)ls * n1;
    T* Rs = dyn;
    const int lr = n2 | 1;
    for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) Rs[e % n2 + (e / n2) * lr] = R[e % n2 + (size_t)(e / n2) * lmax];
    S = Ss;
    R = Rs;
    lds = ls;
    ldr = lr;
  }
  __syncthreads();
#define SS(i, j) S[(i) + (size_t)(j)*lds]
#define RR(i, j) R[(i) + (size_t)(j)*ldr]
#define YY(i, j) Y[(i) + (size_t)(j)*ldy]
  if (threadIdx.x == 0) {
    int c = 0;
    for (int i1 = n1 - 1; i1 >= 0;) {
      const int ib = (i1 > 0 && SS(i1, i1 - 1) != T(0)) ? 2 : 1;
      rg0[c] = i1 - ib + 1;
      rgs[c] = ib;
      ++c;
      i1 -= ib;
    }
    s_nrg = c;
  } else if (threadIdx.x == 32) {
    int c = 0;
    for (int k1 = n2 - 1; k1 >= 0;) {
      const int kb = (k1 > 0 && RR(k1, k1 - 1) != T(0)) ? 2 : 1;
      cg0[c] = k1 - kb + 1;
      cgs[c] = kb;
      ++c;
      k1 -= kb;
    }
    s_ncg = c;
  }
  __syncthreads();
  const int nrg = s_nrg, ncg = s_ncg;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int wb = 0; wb < ncg; wb += kWarps) {
    const int we = min(ncg, wb + kWarps);
    // columns of this wave: [cfirst, clast]; columns already solved: > clast
    const int clast = cg0[wb] + cgs[wb] - 1;
    const int cfirst = cg0[we - 1];
    if (clast + 1 < n2) {
      const int wcols = clast - cfirst + 1;
      for (int e = threadIdx.x; e < n1 * wcols; e += blockDim.x) {
        const int i = e % n1, k = cfirst + e / n1;
        T acc = T(0);
        for (int l = clast + 1; l < n2; ++l) acc += RR(k, l) * YY(i, l);
        YY(i, k) -= acc;
      }
    }
    __syncthreads();
    const int nsteps = nrg + (we - wb) - 1;
    for (int t = 0; t < nsteps; ++t) {
      const int g = warp, gam = wb + g, rho = t - g;
      if (gam < we && rho >= 0 && rho < nrg && rgs[rho] == 1 && cgs[gam] == 1) {
        // 1x1 blocks (real eigenvalues on both sides): the common case
        const int i0 = rg0[rho], k0 = cg0[gam];
        T acc = T(0);
        for (int l = k0 + 1 + lane; l <= clast; l += 32) acc += RR(k0, l) * YY(i0, l);
        acc = warp_sum(acc);
        const T y = (YY(i0, k0) - acc) / (SS(i0, i0) + RR(k0, k0));
        __syncwarp();
        if (lane == 0) YY(i0, k0) = y;
        for (int i = lane; i < i0; i += 32) YY(i, k0) -= SS(i, i0) * y;
      } else if (gam < we && rho >= 0 && rho < nrg) {
        // 2x2 blocks (complex pairs) on one or both sides: a system of size
        // ib*kb <= 4, laid out with stride 2 (unknown ia + 2 kb) and padded with
        // identity rows, solved in registers by unrolled Gaussian elimination
        const int i0 = rg0[rho], ib = rgs[rho];
        const int k0 = cg0[gam], kb = cgs[gam];
        const int k1 = k0 + kb - 1;
        T c[2][2] = {{T(0), T(0)}, {T(0), T(0)}};
        for (int l = k1 + 1 + lane; l <= clast; l += 32) {
          const T y0 = YY(i0, l), y1 = (ib == 2) ? YY(i0 + 1, l) : T(0);
          const T r0 = RR(k0, l), r1 = (kb == 2) ? RR(k0 + 1, l) : T(0);
          c[0][0] += r0 * y0;
          c[0][1] += r1 * y0;
          c[1][0] += r0 * y1;
          c[1][1] += r1 * y1;
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int bb = 0; bb < 2; ++bb) c[a][bb] = warp_sum(c[a][bb]);
        T yv[2][2] = {{T(0), T(0)}, {T(0), T(0)}};
        if (lane == 0) {
          T M[4][4], rhs[4];
#pragma unroll
          for (int kb_ = 0; kb_ < 2; ++kb_)
#pragma unroll
            for (int ia = 0; ia < 2; ++ia) {
              const int u = ia + 2 * kb_;
              const bool used = ia < ib && kb_ < kb;
              rhs[u] = used ? YY(i0 + ia, k0 + kb_) - c[ia][kb_] : T(0);
#pragma unroll
              for (int kc = 0; kc < 2; ++kc)
#pragma unroll
                for (int ic = 0; ic < 2; ++ic) {
                  const int v = ic + 2 * kc;
                  T m = T(0);
                  if (used && ic < ib && kc < kb)
                    m = (kb_ == kc ? SS(i0 + ia, i0 + ic) : T(0)) + (ia == ic ? RR(k0 + kb_, k0 + kc) : T(0));
                  else if (!used && u == v)
                    m = T(1);
                  M[u][v] = m;
                }
            }
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            int pv = k;
            T best = fabs(M[k][k]);
#pragma unroll
            for (int i = k + 1; i < 4; ++i)
              if (fabs(M[i][k]) > best) {
                best = fabs(M[i][k]);
                pv = i;
              }
#pragma unroll
            for (int i = k + 1; i < 4; ++i)
              if (i == pv) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                  const T t = M[k][j];
                  M[k][j] = M[i][j];
                  M[i][j] = t;
                }
                const T t = rhs[k];
                rhs[k] = rhs[i];
                rhs[i] = t;
              }
#pragma unroll
            for (int i = k + 1; i < 4; ++i) {
              const T f = M[i][k] / M[k][k];
#pragma unroll
              for (int j = k; j < 4; ++j) M[i][j] -= f * M[k][j];
              rhs[i] -= f * rhs[k];
            }
          }
#pragma unroll
          for (int k = 3; k >= 0; --k) {
            T sacc = rhs[k];
#pragma unroll
            for (int j = k + 1; j < 4; ++j) sacc -= M[k][j] * rhs[j];
            rhs[k] = sacc / M[k][k];
          }
#pragma unroll
          for (int kb_ = 0; kb_ < 2; ++kb_)
#pragma unroll
            for (int ia = 0; ia < 2; ++ia) yv[ia][kb_] = rhs[ia + 2 * kb_];
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int bb = 0; bb < 2; ++bb) yv[a][bb] = __shfl_sync(0xffffffffu, yv[a][bb], 0);
        __syncwarp();
        if (lane == 0) {
#pragma unroll
          for (int ia = 0; ia < 2; ++ia)
#pragma unroll
            for (int kb_ = 0; kb_ < 2; ++kb_)
              if (ia < ib && kb_ < kb) YY(i0 + ia, k0 + kb_) = yv[ia][kb_];
        }
        // rows above the block, same columns: Y[i][k] -= S[i][i0..] y
        for (int i = lane; i < i0; i += 32) {
          const T s0 = SS(i, i0), s1 = (ib == 2) ? SS(i, i0 + 1) : T(0);
          YY(i, k0) -= s0 * yv[0][0] + s1 * yv[1][0];
          if (kb == 2) YY(i, k0 + 1) -= s0 * yv[0][1] + s1 * yv[1][1];
        }
      }
      __syncthreads();
    }
  }
  if (mode >= 1) {
    for (int e = threadIdx.x; e < n1 * n2; e += blockDim.x)
      Yg[e % n1 + (size_t)(e / n1) * ldw] = Y[e % n1 + (e / n1) * ldy];
  }
#undef SS
#undef RR
#undef YY
}

template <typename T>
fde_status leaf_trsyl(const T* S, const T* R, int lmax, const int* d_lo_x, const int* d_n_x, int nx,
                      const int* d_lo_y, const int* d_n_y, int ny, T* W, int ldw, cudaStream_t st, double flops) {
  const size_t tables = 4 * (size_t)lmax * sizeof(int);
  const size_t mat = (size_t)(lmax | 1) * lmax * sizeof(T);  // one padded lmax x lmax block
  const size_t limit = 220 * 1024;
  const int mode = (tables + 3 * mat <= limit) ? 2 : (tables + mat <= limit) ? 1 : 0;
  const size_t smem = tables + (mode == 2 ? 3 * mat : mode == 1 ? mat : 0);
  static bool attr_set[2] = {false, false};
  if (!attr_set[sizeof(T) == 8]) {
    FDE_CUDA(cudaFuncSetAttribute(trsyl_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit));
    attr_set[sizeof(T) == 8] = true;
  }
  ProfScope ps(sizeof(T) == 4 ? "trsyl32" : "trsyl64", st, flops, 1);
  trsyl_kernel<T><<<nx * ny, kWarps * 32, smem, st>>>(S, R, lmax, d_lo_x, d_n_x, nx, d_lo_y, d_n_y, W, ldw, mode);
  FDE_LAUNCH("trsyl_kernel");
  return FDE_OK;
}

template fde_status leaf_trsyl<double>(const double*, const double*, int, const int*, const int*, int, const int*,
                                       const int*, int, double*, int, cudaStream_t, double);
template fde_status leaf_trsyl<float>(const float*, const float*, int, const int*, const int*, int, const int*,
                                      const int*, int, float*, int, cudaStream_t, double);

}  // namespace fde
