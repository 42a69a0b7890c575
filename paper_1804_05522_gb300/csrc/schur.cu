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

// One CTA per leaf pair.  Columns of Y are solved from the last block to the
// first (Rᵀ is lower quasi-triangular); inside a column block the rows are
// solved bottom-up over the 1x1 / 2x2 blocks of S (the small coupled system
// for a (row block, column block) is (I ⊗ S_bb + R_bb ⊗ I) vec Y_b = vec B_b).
template <typename T>
__global__ void __launch_bounds__(256) trsyl_kernel(const T* __restrict__ Sall, const T* __restrict__ Rall, int lmax,
                                                   const int* __restrict__ lo_x, const int* __restrict__ n_x, int nx,
                                                   const int* __restrict__ lo_y, const int* __restrict__ n_y, T* W,
                                                   int ldw) {
  const int p = blockIdx.x % nx, q = blockIdx.x / nx;
  const T* S = Sall + (size_t)p * lmax * lmax;
  const T* R = Rall + (size_t)q * lmax * lmax;
  const int n1 = n_x[p], n2 = n_y[q];
  T* Y = W + lo_x[p] + (size_t)lo_y[q] * ldw;
#define SS(i, j) S[(i) + (size_t)(j)*lmax]
#define RR(i, j) R[(i) + (size_t)(j)*lmax]
#define YY(i, j) Y[(i) + (size_t)(j)*ldw]
  int k1 = n2 - 1;
  while (k1 >= 0) {
    const int kb = (k1 > 0 && RR(k1, k1 - 1) != T(0)) ? 2 : 1;
    const int k0 = k1 - kb + 1;
    // right-hand side: Y[:, k] -= Σ_{l > k1} R[k][l] Y[:, l]
    for (int i = threadIdx.x; i < n1; i += blockDim.x)
      for (int k = k0; k <= k1; ++k) {
        T acc = T(0);
        for (int l = k1 + 1; l < n2; ++l) acc += RR(k, l) * YY(i, l);
        YY(i, k) -= acc;
      }
    __syncthreads();
    int i1 = n1 - 1;
    while (i1 >= 0) {
      const int ib = (i1 > 0 && SS(i1, i1 - 1) != T(0)) ? 2 : 1;
      const int i0 = i1 - ib + 1;
      if (threadIdx.x == 0) {
        T M[4][4], b[4];
        const int m = ib * kb;
        for (int ka = 0; ka < kb; ++ka)
          for (int ia = 0; ia < ib; ++ia) {
            const int a = ia + ib * ka;
            b[a] = YY(i0 + ia, k0 + ka);
            for (int kc = 0; kc < kb; ++kc)
              for (int ic = 0; ic < ib; ++ic) {
                const int c = ic + ib * kc;
                M[a][c] = (ka == kc ? SS(i0 + ia, i0 + ic) : T(0)) + (ia == ic ? RR(k0 + ka, k0 + kc) : T(0));
              }
          }
        small_solve(M, b, m);
        for (int ka = 0; ka < kb; ++ka)
          for (int ia = 0; ia < ib; ++ia) YY(i0 + ia, k0 + ka) = b[ia + ib * ka];
      }
      __syncthreads();
      for (int i = threadIdx.x; i < i0; i += blockDim.x)
        for (int k = k0; k <= k1; ++k) {
          T acc = SS(i, i0) * YY(i0, k);
          if (ib == 2) acc += SS(i, i1) * YY(i1, k);
          YY(i, k) -= acc;
        }
      __syncthreads();
      i1 = i0 - 1;
    }
    k1 = k0 - 1;
  }
#undef SS
#undef RR
#undef YY
}

template <typename T>
fde_status leaf_trsyl(const T* S, const T* R, int lmax, const int* d_lo_x, const int* d_n_x, int nx,
                      const int* d_lo_y, const int* d_n_y, int ny, T* W, int ldw, cudaStream_t st) {
  trsyl_kernel<T><<<nx * ny, 256, 0, st>>>(S, R, lmax, d_lo_x, d_n_x, nx, d_lo_y, d_n_y, W, ldw);
  FDE_LAUNCH("trsyl_kernel");
  return FDE_OK;
}

template fde_status leaf_trsyl<double>(const double*, const double*, int, const int*, const int*, int, const int*,
                                       const int*, int, double*, int, cudaStream_t);
template fde_status leaf_trsyl<float>(const float*, const float*, int, const int*, const int*, int, const int*,
                                      const int*, int, float*, int, cudaStream_t);

}  // namespace fde
