// HODLR construction (§3.4), factorisation and solve (§3.5) for the shifted
// Grünwald–Letnikov operator A = s I + c (D_+ T + D_- Tᵀ), Eq. (system_FD).
#include <math.h>
#include <stdarg.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>

#include "hodlr_internal.cuh"

namespace fde {

// ------------------------------------------------------------ error state
static thread_local char g_err[1024] = "no error";
void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
fde_status cuda_status(cudaError_t e, const char* what, const char* file, int line) {
  set_error("CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
  if (e == cudaErrorMemoryAllocation) return FDE_ERR_NOMEM;
  return FDE_ERR_CUDA;
}
double now_seconds() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// ------------------------------------------------------- K1: GL weights
// g_0 = 1, g_k = g_{k-1} (1 - (α+1)/k)  (Eq. (Grun) via the recurrence of
// §3.4.2), one correctly rounded divide, subtract, multiply per step, in that
// order and never contracted, so that the sequence is reproducible bit for bit.
__global__ void gl_weights_kernel(double alpha, int K, double* g) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double a1 = __dadd_rn(alpha, 1.0);
  double prev = 1.0;
  g[0] = 1.0;
  for (int k = 1; k <= K; ++k) {
    const double q = __ddiv_rn(a1, (double)k);
    const double f = __dsub_rn(1.0, q);
    prev = __dmul_rn(prev, f);
    g[k] = prev;
  }
}

// --------------------------------------------- dense-on-the-fly matvec
// y = A x (trans = 0) or y = Aᵀ x (trans = 1), A = s I + c (D_+ T + D_- Tᵀ),
// T[i][j] = -g[i-j+1] (j <= i+1).  One warp per output entry.  FP64.
__global__ void fd_matvec_kernel(const double* __restrict__ g, const double* __restrict__ dp,
                                 const double* __restrict__ dm, double c, double shift, int N,
                                 const double* __restrict__ x, double* __restrict__ y, int trans) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= N) return;
  const int i = warp;
  double s1 = 0.0, s2 = 0.0;
  if (!trans) {
    // Σ_{j <= i+1} g[i-j+1] x_j   and   Σ_{j >= i-1} g[j-i+1] x_j
    const int jmax = min(i + 1, N - 1);
    for (int j = lane; j <= jmax; j += 32) s1 += g[i - j + 1] * x[j];
    for (int j = max(i - 1, 0) + lane; j < N; j += 32) s2 += g[j - i + 1] * x[j];
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (lane == 0) y[i] = shift * x[i] - c * (dp[i] * s1 + dm[i] * s2);
  } else {
    // (Aᵀx)_j = s x_j - c (Σ_{i >= j-1} g[i-j+1] d+_i x_i + Σ_{i <= j+1} g[j-i+1] d-_i x_i)
    const int j = i;
    for (int r = max(j - 1, 0) + lane; r < N; r += 32) s1 += g[r - j + 1] * dp[r] * x[r];
    const int rmax = min(j + 1, N - 1);
    for (int r = lane; r <= rmax; r += 32) s2 += g[j - r + 1] * dm[r] * x[r];
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (lane == 0) y[j] = shift * x[j] - c * (s1 + s2);
  }
}

__global__ void norm2_kernel(const double* __restrict__ x, int n, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i] * x[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *out = sqrt(s);
}
__global__ void scale_inv_kernel(double* x, int n, const double* s) {
  const double inv = (*s > 0.0) ? 1.0 / *s : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] *= inv;
}
__global__ void fill_kernel(double* x, int n, double v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = v;
}
__global__ void finite_check_kernel(const double* __restrict__ x, int n, int* bad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (!isfinite(x[i]) || x[i] < 0.0) atomicExch(bad, 1);
}

// ------------------------------------------------------- K2: ACA on T21
// ACA with partial pivoting on T21 = [-g_{N1+i-j+1}] (N2 x N1), the block
// that contains every lower off-diagonal block of T by restriction (§3.4.2).
// Operation order is fixed, so that any FP64 implementation of the same
// sequence reproduces the pivots exactly: residual
// entries by sequential mul-then-sub, pivots by first argmax of |.| over
// unused indices, stop when (Σu²)(Σv²) <= tol² with both sums sequential.
struct ArgMax {
  double v;
  int i;
};
__device__ __forceinline__ ArgMax argmax_merge(ArgMax a, ArgMax b) {
  if (b.v > a.v || (b.v == a.v && b.i < a.i)) return b;
  return a;
}
__device__ ArgMax block_argmax(ArgMax a, double* sv, int* si) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ArgMax b;
    b.v = __shfl_xor_sync(0xffffffffu, a.v, o);
    b.i = __shfl_xor_sync(0xffffffffu, a.i, o);
    a = argmax_merge(a, b);
  }
  __syncthreads();
  if (lane == 0) {
    sv[wid] = a.v;
    si[wid] = a.i;
  }
  __syncthreads();
  if (wid == 0) {
    ArgMax b = (lane < nw) ? ArgMax{sv[lane], si[lane]} : ArgMax{-2.0, 0x7fffffff};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ArgMax c;
      c.v = __shfl_xor_sync(0xffffffffu, b.v, o);
      c.i = __shfl_xor_sync(0xffffffffu, b.i, o);
      b = argmax_merge(b, c);
    }
    if (lane == 0) {
      sv[0] = b.v;
      si[0] = b.i;
    }
  }
  __syncthreads();
  ArgMax r{sv[0], si[0]};
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(1024) aca_kernel(const double* __restrict__ g, int N1, int N2, double tol,
                                                   int maxrank, double* U, double* V, int* rows, int* cols,
                                                   int* out, unsigned char* used_r, unsigned char* used_c) {
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int s_istar, s_done, s_conv, s_k;
  __shared__ double s_su, s_sv;
  for (int i = threadIdx.x; i < N2; i += blockDim.x) used_r[i] = 0;
  for (int j = threadIdx.x; j < N1; j += blockDim.x) used_c[j] = 0;
  if (threadIdx.x == 0) {
    s_istar = 0;
    s_done = 0;
    s_conv = 0;
    s_k = 0;
  }
  __syncthreads();
  const double tol2 = __dmul_rn(tol, tol);
  int guard = 0;
  while (!s_done && s_k < maxrank && guard < N1 + N2 + maxrank + 2) {
    ++guard;
    const int k = s_k, is = s_istar;
    double* vk = V + (size_t)k * N1;
    double* uk = U + (size_t)k * N2;
    // residual row i*
    ArgMax best{-1.0, 0x7fffffff};
    for (int j = threadIdx.x; j < N1; j += blockDim.x) {
      double r = -g[N1 + is - j + 1];
      for (int l = 0; l < k; ++l) r = __dsub_rn(r, __dmul_rn(U[is + (size_t)l * N2], V[j + (size_t)l * N1]));
      vk[j] = r;
      if (!used_c[j]) best = argmax_merge(best, ArgMax{fabs(r), j});
    }
    __syncthreads();
    if (threadIdx.x == 0) used_r[is] = 1;
    best = block_argmax(best, sv, si);
    if (!(best.v > 0.0)) {
      // zero residual row (or no unused column): move to the lowest unused row
      ArgMax fr{-1.0, 0x7fffffff};
      for (int i = threadIdx.x; i < N2; i += blockDim.x)
        if (!used_r[i]) fr = argmax_merge(fr, ArgMax{0.0, i});
      fr = block_argmax(fr, sv, si);
      if (threadIdx.x == 0) {
        if (fr.v < 0.0 || best.v < 0.0) {
          s_done = 1;
          s_conv = 1;
        } else {
          s_istar = fr.i;
        }
      }
      __syncthreads();
      continue;
    }
    const int js = best.i;
    const double piv = vk[js];
    __syncthreads();
    for (int j = threadIdx.x; j < N1; j += blockDim.x) vk[j] = __ddiv_rn(vk[j], piv);
    // residual column j*
    for (int i = threadIdx.x; i < N2; i += blockDim.x) {
      double c = -g[N1 + i - js + 1];
      for (int l = 0; l < k; ++l) c = __dsub_rn(c, __dmul_rn(U[i + (size_t)l * N2], V[js + (size_t)l * N1]));
      uk[i] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      used_c[js] = 1;
      rows[k] = is;
      cols[k] = js;
      double s = 0.0;
      for (int i = 0; i < N2; ++i) s = __dadd_rn(s, __dmul_rn(uk[i], uk[i]));
      s_su = s;
    } else if (threadIdx.x == 32) {
      double s = 0.0;
      for (int j = 0; j < N1; ++j) s = __dadd_rn(s, __dmul_rn(vk[j], vk[j]));
      s_sv = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_k = k + 1;
    if (__dmul_rn(s_su, s_sv) <= tol2) {
      if (threadIdx.x == 0) {
        s_done = 1;
        s_conv = 1;
      }
      __syncthreads();
      break;
    }
    ArgMax nb{-1.0, 0x7fffffff};
    for (int i = threadIdx.x; i < N2; i += blockDim.x)
      if (!used_r[i]) nb = argmax_merge(nb, ArgMax{fabs(uk[i]), i});
    nb = block_argmax(nb, sv, si);
    if (threadIdx.x == 0) {
      if (nb.v < 0.0) {
        s_done = 1;
        s_conv = 1;
      } else {
        s_istar = nb.i;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s_k;
    out[1] = s_conv;
  }
}

// ------------------------------------------------ K4: block factors
// For every internal node (lo, mid, hi), t = mid - lo, s = hi - mid:
//  upper block A[lo:mid, mid:hi] = c D_-[rows] V0[N1-t:N1] U0[0:s]ᵀ - c d_+[mid-1] e_{t-1} e_0ᵀ
//  lower block A[mid:hi, lo:mid] = c D_+[rows] U0[0:s] V0[N1-t:N1]ᵀ - c d_-[mid]   e_0 e_{t-1}ᵀ
// (restriction of T21, §3.4.2; the corner is the single entry -g_0 of the
// rank-one upper blocks of T, proof of Lemma lem:fd-qsrank).  Written into
// the level arrays Uin_l (rows lo..mid: upper U, rows mid..hi: lower U) and
// Vin_l (rows mid..hi: upper V, rows lo..mid: lower V), r = kaca + 1 columns.
struct NodeRef {
  int lo, mid, hi;
  double* Uin;
  double* Vin;
};
__global__ void block_factors_kernel(const NodeRef* __restrict__ nodes, const double* __restrict__ U0,
                                     const double* __restrict__ V0, const double* __restrict__ dp,
                                     const double* __restrict__ dm, double c, int N, int N1, int N2, int kaca) {
  const NodeRef nd = nodes[blockIdx.x];
  const int t = nd.mid - nd.lo, r = kaca + 1;
  const int len = nd.hi - nd.lo;
  for (int e = threadIdx.x; e < len * r; e += blockDim.x) {
    const int row = nd.lo + e % len, l = e / len;
    double u, v;
    if (row < nd.mid) {
      const int i = row - nd.lo;  // upper U row i; lower V row i
      if (l < kaca) {
        u = c * dm[row] * V0[(N1 - t + i) + (size_t)l * N1];
        v = V0[(N1 - t + i) + (size_t)l * N1];
      } else {
        u = (i == t - 1) ? -c * dp[nd.mid - 1] : 0.0;
        v = (i == t - 1) ? 1.0 : 0.0;
      }
    } else {
      const int i = row - nd.mid;  // lower U row i; upper V row i
      if (l < kaca) {
        u = c * dp[row] * U0[i + (size_t)l * N2];
        v = U0[i + (size_t)l * N2];
      } else {
        u = (i == 0) ? -c * dm[nd.mid] : 0.0;
        v = (i == 0) ? 1.0 : 0.0;
      }
    }
    nd.Uin[row + (size_t)l * N] = u;
    nd.Vin[row + (size_t)l * N] = v;
  }
}

// ------------------------------------------- K3: QR + SVD recompression

// Householder QR of A (m x r, lda), reflectors below the diagonal, tau[j];
// R (r x r, ld r) gets the upper trapezoid (rows >= min(m,r) zero).
__device__ void house_qr(double* A, int lda, int m, int r, double* tau, double* R, double* red) {
  const int kq = min(m, r);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = 0; j < kq; ++j) {
    double part = 0.0;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) {
      const double v = A[i + (size_t)j * lda];
      part += v * v;
    }
    const double sig = block_sum(part, red);
    const double x0 = A[j + (size_t)j * lda];
    double t = 0.0, beta = x0;
    if (sig != 0.0) {
      const double alpha = sqrt(x0 * x0 + sig);
      beta = (x0 <= 0.0) ? alpha : -alpha;
      t = (beta - x0) / beta;
      const double scale = 1.0 / (x0 - beta);
      for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) A[i + (size_t)j * lda] *= scale;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      tau[j] = t;
      A[j + (size_t)j * lda] = beta;
    }
    __syncthreads();
    if (t != 0.0) {
      for (int cc = j + 1 + warp; cc < r; cc += nw) {
        const double yj = A[j + (size_t)cc * lda];
        double w = 0.0;
        for (int i = j + 1 + lane; i < m; i += 32) w += A[i + (size_t)j * lda] * A[i + (size_t)cc * lda];
        w = warp_sum(w);
        w = t * (w + yj);
        if (lane == 0) A[j + (size_t)cc * lda] = yj - w;
        for (int i = j + 1 + lane; i < m; i += 32) A[i + (size_t)cc * lda] -= w * A[i + (size_t)j * lda];
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, cc = e / r;
    R[i + cc * r] = (i <= cc && i < kq) ? A[i + (size_t)cc * lda] : 0.0;
  }
  __syncthreads();
}

// Y <- Q Y with Q = H_0 ... H_{kq-1} stored by house_qr (Y: m x nc, ldy).
__device__ void house_apply(const double* A, int lda, int m, int kq, const double* tau, double* Y, int ldy,
                            int nc) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = kq - 1; j >= 0; --j) {
    const double t = tau[j];
    if (t != 0.0) {
      for (int cc = warp; cc < nc; cc += nw) {
        const double yj = Y[j + (size_t)cc * ldy];
        double w = 0.0;
        for (int i = j + 1 + lane; i < m; i += 32) w += A[i + (size_t)j * lda] * Y[i + (size_t)cc * ldy];
        w = warp_sum(w);
        w = t * (w + yj);
        if (lane == 0) Y[j + (size_t)cc * ldy] = yj - w;
        for (int i = j + 1 + lane; i < m; i += 32) Y[i + (size_t)cc * ldy] -= w * A[i + (size_t)j * lda];
      }
    }
    __syncthreads();
  }
}

// One-sided (Hestenes) Jacobi SVD of M (rows x cols, ld ldm), Z accumulates
// the right rotations (cols x cols, ld ldz); columns of M end up W Σ.
// A pair is rotated while |γ| > ortho_tol sqrt(αβ); pairs with a column of
// squared norm <= floor2 (negligible against the matrix) are left alone.
__device__ void jacobi_svd(double* M, int ldm, int rows, int cols, double* Z, int ldz, int* s_rot,
                           double ortho_tol = 1e-15, double floor2 = 0.0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int e = threadIdx.x; e < cols * cols; e += blockDim.x) Z[(e % cols) + (e / cols) * ldz] = (e % cols == e / cols);
  __syncthreads();
  const int np = (cols + 1) & ~1;
  if (np < 2) return;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (threadIdx.x == 0) *s_rot = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      for (int pr = warp; pr < np / 2; pr += nw) {
        int a, b;
        if (pr == 0) {
          a = 0;
          b = 1 + (round % (np - 1));
        } else {
          a = 1 + ((round + pr) % (np - 1));
          b = 1 + ((round - pr + (np - 1)) % (np - 1));
        }
        if (a > b) {
          int tt = a;
          a = b;
          b = tt;
        }
        if (b >= cols) continue;  // phantom column
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < rows; i += 32) {
          const double x = M[i + a * ldm], y = M[i + b * ldm];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga != 0.0 && fabs(ga) > ortho_tol * sqrt(al * be) && al > floor2 && be > floor2) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
          for (int i = lane; i < rows; i += 32) {
            const double x = M[i + a * ldm], y = M[i + b * ldm];
            M[i + a * ldm] = cs * x - sn * y;
            M[i + b * ldm] = sn * x + cs * y;
          }
          for (int i = lane; i < cols; i += 32) {
            const double x = Z[i + a * ldz], y = Z[i + b * ldz];
            Z[i + a * ldz] = cs * x - sn * y;
            Z[i + b * ldz] = sn * x + cs * y;
          }
          if (lane == 0) *s_rot = 1;
        }
      }
      __syncthreads();
    }
    if (*s_rot == 0) break;
    __syncthreads();
  }
}

size_t recompress_smem(int r);

// One CTA per job.  U Vᵀ (U: m x r, V: n x r, in place) -> U' V'ᵀ, rank r'
// = #{σ > abstol}; U' = Q_U W Σ, V' = Q_V Z (§4.1 recompression).  Outputs
// have rcap columns, zero beyond r'.
__global__ void __launch_bounds__(512) recompress_kernel(const RecompJob* __restrict__ jobs, int r, int rcap,
                                                         double abstol, double reltol) {
  extern __shared__ double smem[];
  const RecompJob jb = jobs[blockIdx.x];
  double* Ru = smem;          // r x r (later Z)
  double* Rv = Ru + r * r;    // r x r
  double* M = Rv + r * r;     // r x r
  double* tau_u = M + r * r;  // r
  double* tau_v = tau_u + r;  // r
  double* sig = tau_v + r;    // r
  int* perm = (int*)(sig + r);
  __shared__ double red[32];
  __shared__ int s_rot, s_rank;
  const int m = jb.m, n = jb.n, ld = jb.ld;
  house_qr(jb.Uin, ld, m, r, tau_u, Ru, red);
  house_qr(jb.Vin, ld, n, r, tau_v, Rv, red);
  const int qm = min(m, r), qn = min(n, r);
  for (int e = threadIdx.x; e < qm * qn; e += blockDim.x) {
    const int i = e % qm, j = e / qm;
    double s = 0.0;
    for (int k = 0; k < r; ++k) s += Ru[i + k * r] * Rv[j + k * r];
    M[i + j * r] = s;
  }
  __syncthreads();
  double* Z = Ru;
  jacobi_svd(M, r, qm, qn, Z, r, &s_rot);
  __syncthreads();
  for (int j = threadIdx.x; j < qn; j += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < qm; ++i) s += M[i + j * r] * M[i + j * r];
    sig[j] = sqrt(s);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < qn; j += blockDim.x) {
    int rk = 0;
    for (int q = 0; q < qn; ++q)
      if (sig[q] > sig[j] || (sig[q] == sig[j] && q < j)) ++rk;
    perm[rk] = j;
  }
  if (threadIdx.x == 0) {
    // drop σ <= max(abstol, reltol σ_max)
    double smax = 0.0;
    for (int j = 0; j < qn; ++j) smax = fmax(smax, sig[j]);
    const double thr = fmax(abstol, reltol * smax);
    int cnt = 0;
    for (int j = 0; j < qn; ++j)
      if (sig[j] > thr) ++cnt;
    s_rank = min(cnt, rcap);
    if (jb.rank_full) atomicMax(jb.rank_full, cnt);
  }
  __syncthreads();
  const int rr = s_rank;
  for (int e = threadIdx.x; e < m * rcap; e += blockDim.x) {
    const int i = e % m, cc = e / m;
    jb.Uout[i + (size_t)cc * ld] = (cc < rr && i < qm) ? M[i + perm[cc] * r] : 0.0;
  }
  for (int e = threadIdx.x; e < n * rcap; e += blockDim.x) {
    const int i = e % n, cc = e / n;
    jb.Vout[i + (size_t)cc * ld] = (cc < rr && i < qn) ? Z[i + perm[cc] * r] : 0.0;
  }
  __syncthreads();
  house_apply(jb.Uin, ld, m, qm, tau_u, jb.Uout, ld, rr);
  house_apply(jb.Vin, ld, n, qn, tau_v, jb.Vout, ld, rr);
  if (threadIdx.x == 0) *jb.rank_out = rr;
}

// The same recompression in three launches, so that the two factors' QR and
// their final products run in separate CTAs (one per factor and job): the
// FP64 pipe of one SM is the limit of a single-CTA QR of a tall factor.
// Workspace per job (RecompWork): tau and R of both factors, the small
// factors of the kept part of the core's SVD, the core's rank.
__global__ void __launch_bounds__(512) recomp_qr_kernel(const RecompJob* __restrict__ jobs, int r,
                                                         RecompWork wk) {
  extern __shared__ double smem[];
  __shared__ double red[32];
  const int j = blockIdx.x >> 1, side = blockIdx.x & 1;
  const RecompJob jb = jobs[j];
  double* R = smem;  // r x r
  double* tau = wk.tau + ((size_t)j * 2 + side) * r;
  house_qr(side ? jb.Vin : jb.Uin, jb.ld, side ? jb.n : jb.m, r, tau, R, red);
  double* Rout = wk.R + ((size_t)j * 2 + side) * r * r;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) Rout[e] = R[e];
}

__global__ void __launch_bounds__(512) recomp_core_kernel(const RecompJob* __restrict__ jobs, int r, int rcap,
                                                           double abstol, double reltol, RecompWork wk) {
  extern __shared__ double smem[];
  const int j = blockIdx.x;
  const RecompJob jb = jobs[j];
  double* M = smem;           // r x r
  double* Z = M + r * r;      // r x r
  double* sig = Z + r * r;    // r
  int* perm = (int*)(sig + r);
  __shared__ int s_rot, s_rank;
  const double* Ru = wk.R + (size_t)j * 2 * r * r;
  const double* Rv = Ru + (size_t)r * r;
  const int qm = min(jb.m, r), qn = min(jb.n, r);
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, c = e / r;
    double s = 0.0;
    if (i < qm && c < qn)
      for (int k = 0; k < r; ++k) s += Ru[i + k * r] * Rv[c + k * r];
    M[e] = s;
  }
  __syncthreads();
  {
    // orthogonality to the rounding level of an r-column FP64 rotation
    // sequence, and no rotations among columns below 1e-15 ||M||_F (their
    // singular values are far below any truncation threshold): without these
    // the sweeps run to their cap on the rank-deficient cores of padded factors
    __shared__ double red[32];
    double part = 0.0;
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) part += M[e] * M[e];
    const double fro2 = block_sum(part, red);
    jacobi_svd(M, r, qm, qn, Z, r, &s_rot, 4.0 * r * 1.1102230246251565e-16, 1e-30 * fro2);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < qn; c += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < qm; ++i) s += M[i + c * r] * M[i + c * r];
    sig[c] = sqrt(s);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < qn; c += blockDim.x) {
    int rk = 0;
    for (int q = 0; q < qn; ++q)
      if (sig[q] > sig[c] || (sig[q] == sig[c] && q < c)) ++rk;
    perm[rk] = c;
  }
  if (threadIdx.x == 0) {
    double smax = 0.0;
    for (int c = 0; c < qn; ++c) smax = fmax(smax, sig[c]);
    const double thr = fmax(abstol, reltol * smax);
    int cnt = 0;
    for (int c = 0; c < qn; ++c)
      if (sig[c] > thr) ++cnt;
    s_rank = min(cnt, rcap);
    *jb.rank_out = s_rank;
    if (jb.rank_full) atomicMax(jb.rank_full, cnt);
    wk.rank[j] = s_rank;
  }
  __syncthreads();
  const int rr = s_rank;
  double* Cu = wk.C + (size_t)j * 2 * r * rcap;  // r x rcap: W Σ (kept columns)
  double* Cv = Cu + (size_t)r * rcap;           // r x rcap: Z
  for (int e = threadIdx.x; e < r * rcap; e += blockDim.x) {
    const int i = e % r, c = e / r;
    Cu[e] = (c < rr && i < qm) ? M[i + perm[c] * r] : 0.0;
    Cv[e] = (c < rr && i < qn) ? Z[i + perm[c] * r] : 0.0;
  }
}

__global__ void __launch_bounds__(512) recomp_apply_kernel(const RecompJob* __restrict__ jobs, int r, int rcap,
                                                            RecompWork wk) {
  const int j = blockIdx.x >> 1, side = blockIdx.x & 1;
  const RecompJob jb = jobs[j];
  const int m = side ? jb.n : jb.m, q = min(m, r);
  const double* C = wk.C + ((size_t)j * 2 + side) * r * rcap;
  double* out = side ? jb.Vout : jb.Uout;
  for (int e = threadIdx.x; e < m * rcap; e += blockDim.x) {
    const int i = e % m, c = e / m;
    out[i + (size_t)c * jb.ld] = (i < q) ? C[i + (size_t)c * r] : 0.0;
  }
  __syncthreads();
  house_apply(side ? jb.Vin : jb.Uin, jb.ld, m, q, wk.tau + ((size_t)j * 2 + side) * r, out, jb.ld, wk.rank[j]);
}

// --------------------------------------------------------- leaves (dense)
__global__ void leaves_kernel(const double* __restrict__ g, const double* __restrict__ dp,
                              const double* __restrict__ dm, double c, double shift, const int* __restrict__ leaf_lo,
                              const int* __restrict__ leaf_n, int lmax, double* D) {
  const int p = blockIdx.x, lo = leaf_lo[p], n = leaf_n[p];
  double* Dp = D + (size_t)p * lmax * lmax;
  for (int e = threadIdx.x; e < lmax * lmax; e += blockDim.x) {
    const int i = e % lmax, j = e / lmax;
    double v = 0.0;
    if (i < n && j < n) {
      const int a = lo + i, b = lo + j;
      const double tij = (a - b + 1 >= 0) ? -g[a - b + 1] : 0.0;  // T[a][b]
      const double tji = (b - a + 1 >= 0) ? -g[b - a + 1] : 0.0;  // T[b][a] = Tᵀ[a][b]
      v = c * (dp[a] * tij + dm[a] * tji);
      if (i == j) v += shift;
    } else if (i == j) {
      v = 1.0;  // padding: identity keeps padded blocks invertible
    }
    Dp[i + (size_t)j * lmax] = v;
  }
}

// Dst = Src + sigma I over all leaves (same layout)
template <typename T>
__global__ void leaves_shift_kernel(const T* __restrict__ S, T* __restrict__ Dst, int lmax, size_t total, T sigma) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t w = e % ((size_t)lmax * lmax);
    const int i = (int)(w % lmax), j = (int)(w / lmax);
    Dst[e] = S[e] + ((i == j) ? sigma : T(0));
  }
}

__global__ void set_identity_blocks_kernel(double* K, int n, int count) {
  const size_t total = (size_t)count * n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t w = e % ((size_t)n * n);
    K[e] = ((w % n) == (w / n)) ? 1.0 : 0.0;
  }
}

// ------------------------------------------------------------ to dense
struct LevelPtrs {
  const double* U[24];
  const double* V[24];
  int K[24];
};
__global__ void to_dense_kernel(LevelPtrs lp, const double* __restrict__ D, int lmax, int N, int L,
                                const int* __restrict__ tlo, const int* __restrict__ thi, double* A, int lda) {
  const size_t total = (size_t)N * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % N), j = (int)(e / N);
    int node = 0, l = 0;
    double val = 0.0;
    bool done = false;
    while (l < L) {
      const int lo = tlo[node], hi = thi[node], mid = lo + (hi - lo) / 2;
      const int ci = i >= mid, cj = j >= mid;
      if (ci != cj) {
        double s = 0.0;
        for (int k = 0; k < lp.K[l]; ++k) s += lp.U[l][i + (size_t)k * N] * lp.V[l][j + (size_t)k * N];
        val = s;
        done = true;
        break;
      }
      node = 2 * node + 1 + ci;  // level-order ids: children of node id x are 2x+1, 2x+2
      ++l;
    }
    if (!done) {
      const int p = node - ((1 << L) - 1);
      const int lo = tlo[node];
      val = D[(size_t)p * lmax * lmax + (i - lo) + (size_t)(j - lo) * lmax];
    }
    A[i + (size_t)j * lda] = val;
  }
}

// ------------------------------------------------------------- plans
template <typename T>
fde_status plan_run(const Plan<T>& p, cudaStream_t st) {
  for (const auto& op : p.ops) {
    if (op.kind == 0) {
      FDE_TRY(gemm_batch_run(op.g, st));
    } else {
      FDE_TRY((copy2d<T, T>(op.src, op.ld_src, op.dst, op.ld_dst, op.m, op.n, st)));
    }
  }
  return FDE_OK;
}

size_t solve_scratch_elems(const hodlr_s* h, int ncols, int lvl0) {
  size_t mx = 1;
  for (int l = lvl0; l < h->tree.L; ++l) {
    size_t s = (size_t)(1 << l) * 2 * h->K[l] * ncols;
    mx = std::max(mx, s);
  }
  return mx;
}

template <typename T>
fde_status build_solve_spec(const hodlr_s* h, const Fact<T>& F, const std::vector<T*>& V, const T* X, int ldx, T* Y,
                            int ldy, int ncols, int lvl0, T* tmp, T* zbuf, T* wbuf, std::vector<HostOp<T>>* ops) {
  const Tree& tr = h->tree;
  const int N = tr.N, L = tr.L, lmax = h->lmax;
  if (lvl0 < F.lmin) {
    set_error("build_solve_plan: level %d below factorised level %d", lvl0, F.lmin);
    return FDE_ERR_ARG;
  }
  const bool inplace = (X == Y);
  T* W = inplace ? tmp : Y;
  const int ldw = inplace ? N : ldy;
  ops->clear();
  {
    HostOp<T> op;
    for (int p = 0; p < tr.nleaves(); ++p) {
      const int id = tr.id(L, p), lo = tr.lo[id], n = tr.hi[id] - lo;
      op.d.push_back({F.Dinv + (size_t)p * lmax * lmax, X + lo, W + lo, n, ncols, n, lmax, ldx, ldw});
    }
    ops->push_back(op);
  }
  for (int l = L - 1; l >= lvl0; --l) {
    const int K = h->K[l], K2 = 2 * K;
    HostOp<T> oz, ow, ou;
    oz.ta = true;
    ou.alpha = T(-1);
    ou.beta = T(1);
    for (int p = 0; p < (1 << l); ++p) {
      const int id = tr.id(l, p), lo = tr.lo[id], hi = tr.hi[id], mid = lo + (hi - lo) / 2;
      const int t = mid - lo, s = hi - mid;
      T* zp = zbuf + (size_t)p * K2 * ncols;
      T* wp = wbuf + (size_t)p * K2 * ncols;
      oz.d.push_back({V[l] + mid, W + mid, zp, K, ncols, s, N, ldw, K2});
      oz.d.push_back({V[l] + lo, W + lo, zp + K, K, ncols, t, N, ldw, K2});
      ow.d.push_back({F.Kinv[l] + (size_t)p * K2 * K2, zp, wp, K2, ncols, K2, K2, K2, K2});
      ou.d.push_back({F.Ut[l] + lo, wp, W + lo, t, ncols, K, N, K2, ldw});
      ou.d.push_back({F.Ut[l] + mid, wp + K, W + mid, s, ncols, K, N, K2, ldw});
    }
    ops->push_back(oz);
    ops->push_back(ow);
    ops->push_back(ou);
  }
  if (inplace) {
    HostOp<T> cp;
    cp.kind = 1;
    cp.src = tmp;
    cp.ld_src = N;
    cp.dst = Y;
    cp.ld_dst = ldy;
    cp.m = N;
    cp.n = ncols;
    ops->push_back(cp);
  }
  return FDE_OK;
}

template <typename T>
fde_status upload_specs(const std::vector<std::vector<HostOp<T>>>& specs, DevPool& pool, Plan<T>* out,
                        cudaStream_t st) {
  out->ops.clear();
  size_t nsteps = 0;
  for (const auto& s : specs) nsteps = std::max(nsteps, s.size());
  for (size_t i = 0; i < nsteps; ++i) {
    HostOp<T> m;
    bool first = true;
    for (const auto& s : specs) {
      if (i >= s.size()) continue;
      const HostOp<T>& o = s[i];
      if (o.kind == 1) {  // copies are never merged
        PlanOp<T> cp;
        cp.kind = 1;
        cp.src = o.src;
        cp.dst = o.dst;
        cp.ld_src = o.ld_src;
        cp.ld_dst = o.ld_dst;
        cp.m = o.m;
        cp.n = o.n;
        out->ops.push_back(cp);
        continue;
      }
      if (first) {
        m = o;
        first = false;
      } else {
        if (o.ta != m.ta || o.tb != m.tb || o.alpha != m.alpha || o.beta != m.beta) {
          set_error("upload_specs: incompatible steps");
          return FDE_ERR_ARG;
        }
        m.d.insert(m.d.end(), o.d.begin(), o.d.end());
      }
    }
    if (!first) {
      PlanOp<T> op;
      FDE_TRY(gemm_batch_upload(pool, m.d, m.ta, m.tb, m.alpha, m.beta, &op.g, st));
      out->ops.push_back(op);
    }
  }
  return FDE_OK;
}

template <typename T>
fde_status build_solve_plan(const hodlr_s* h, const Fact<T>& F, const std::vector<T*>& V, const T* X, int ldx,
                            T* Y, int ldy, int ncols, int lvl0, T* tmp, T* zbuf, T* wbuf, DevPool& pool,
                            Plan<T>* out, cudaStream_t st) {
  std::vector<std::vector<HostOp<T>>> specs(1);
  FDE_TRY(build_solve_spec<T>(h, F, V, X, ldx, Y, ldy, ncols, lvl0, tmp, zbuf, wbuf, &specs[0]));
  return upload_specs<T>(specs, pool, out, st);
}

#define INST_SPEC(T)                                                                                        \
  template fde_status build_solve_spec<T>(const hodlr_s*, const Fact<T>&, const std::vector<T*>&, const T*, int, \
                                          T*, int, int, int, T*, T*, T*, std::vector<HostOp<T>>*);           \
  template fde_status upload_specs<T>(const std::vector<std::vector<HostOp<T>>>&, DevPool&, Plan<T>*,        \
                                      cudaStream_t);
INST_SPEC(double)
INST_SPEC(float)
#undef INST_SPEC

template fde_status plan_run<double>(const Plan<double>&, cudaStream_t);
template fde_status plan_run<float>(const Plan<float>&, cudaStream_t);
template fde_status build_solve_plan<double>(const hodlr_s*, const Fact<double>&, const std::vector<double*>&,
                                             const double*, int, double*, int, int, int, double*, double*, double*,
                                             DevPool&, Plan<double>*, cudaStream_t);
template fde_status build_solve_plan<float>(const hodlr_s*, const Fact<float>&, const std::vector<float*>&,
                                            const float*, int, float*, int, int, int, float*, float*, float*,
                                            DevPool&, Plan<float>*, cudaStream_t);

// ------------------------------------------------------ factorisation
fde_status hodlr_factorize(hodlr_s* h, double sigma, int lmin, Fact<double>* F, cudaStream_t st, DevPool* ext) {
  const Tree& tr = h->tree;
  const int N = tr.N, L = tr.L, lmax = h->lmax, nl = tr.nleaves();
  DevPool& pool = ext ? *ext : h->pool;
  DevPool scratch;
  F->sigma = sigma;
  F->lmin = lmin;
  F->Ut.assign(L, nullptr);
  F->Kinv.assign(L, nullptr);
  int* d_flag;
  FDE_TRY(scratch.alloc(&d_flag, 1));
  FDE_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), st));
  FDE_TRY(pool.alloc(&F->Dinv, (size_t)nl * lmax * lmax));
  {
    size_t total = (size_t)nl * lmax * lmax;
    leaves_shift_kernel<double><<<std::min<size_t>((total + 255) / 256, 4096), 256, 0, st>>>(h->D, F->Dinv, lmax,
                                                                                         total, sigma);
    FDE_LAUNCH("leaves_shift_kernel");
    int kmax2 = 0;
    for (int l = 0; l < L; ++l) kmax2 = std::max(kmax2, 2 * h->K[l]);
    int wn = std::max(lmax, kmax2);
    double* work;
    FDE_TRY(scratch.alloc(&work, (size_t)std::max(nl, 1 << std::max(L - 1, 0)) * wn * 2 * wn));
    FDE_TRY(batched_inverse<double>(F->Dinv, lmax, (size_t)lmax * lmax, h->d_leaf_n, nl, lmax, work, d_flag, st));
    // capacitance matrices, bottom-up
    size_t zel = 1;
    for (int l = lmin; l < L; ++l) zel = std::max(zel, solve_scratch_elems(h, h->K[l], l + 1));
    double *tmp, *zb, *wb;
    int kmaxall = 1;
    for (int l = 0; l < L; ++l) kmaxall = std::max(kmaxall, h->K[l]);
    FDE_TRY(scratch.alloc(&tmp, (size_t)N * kmaxall));
    FDE_TRY(scratch.alloc(&zb, zel));
    FDE_TRY(scratch.alloc(&wb, zel));
    int* d_n2;
    FDE_TRY(scratch.alloc(&d_n2, (size_t)(1 << std::max(L - 1, 0))));
    for (int l = L - 1; l >= lmin; --l) {
      const int K = h->K[l], K2 = 2 * K, nn = 1 << l;
      FDE_TRY(pool.alloc(&F->Ut[l], (size_t)N * K));
      FDE_TRY((copy2d<double, double>(h->U[l], N, F->Ut[l], N, N, K, st)));
      Plan<double> pl;
      FDE_TRY(build_solve_plan<double>(h, *F, h->V, F->Ut[l], N, F->Ut[l], N, K, l + 1, tmp, zb, wb, scratch,
                                       &pl, st));
      FDE_TRY(plan_run(pl, st));
      FDE_TRY(pool.alloc(&F->Kinv[l], (size_t)nn * K2 * K2));
      set_identity_blocks_kernel<<<std::min(4096, ceil_div((long)nn * K2 * K2, 256)), 256, 0, st>>>(F->Kinv[l], K2,
                                                                                                    nn);
      FDE_LAUNCH("set_identity_blocks_kernel");
      std::vector<GemmDesc<double>> dk;
      for (int p = 0; p < nn; ++p) {
        const int id = tr.id(l, p), lo = tr.lo[id], hi = tr.hi[id], mid = lo + (hi - lo) / 2;
        double* Kp = F->Kinv[l] + (size_t)p * K2 * K2;
        // K[0:K, K:2K] = V12ᵀ Ut2 (child-2 rows), K[K:2K, 0:K] = V21ᵀ Ut1 (child-1 rows)
        dk.push_back({h->V[l] + mid, F->Ut[l] + mid, Kp + (size_t)K * K2, K, K, hi - mid, N, N, K2});
        dk.push_back({h->V[l] + lo, F->Ut[l] + lo, Kp + K, K, K, mid - lo, N, N, K2});
      }
      GemmBatch<double> gk;
      FDE_TRY(gemm_batch_upload(scratch, dk, true, false, 1.0, 1.0, &gk, st));
      FDE_TRY(gemm_batch_run(gk, st));
      std::vector<int> sizes(nn, K2);
      FDE_CUDA(cudaMemcpyAsync(d_n2, sizes.data(), nn * sizeof(int), cudaMemcpyHostToDevice, st));
      FDE_TRY(batched_inverse<double>(F->Kinv[l], K2, (size_t)K2 * K2, d_n2, nn, K2, work, d_flag, st));
      FDE_CUDA(cudaStreamSynchronize(st));
    }
  }
  int flag = 0;
  FDE_CUDA(cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  FDE_CUDA(cudaStreamSynchronize(st));
  if (flag) {
    set_error("hodlr_factorize: singular leaf or capacitance matrix (sigma=%g)", sigma);
    return FDE_ERR_NUMERIC;
  }
  return FDE_OK;
}

fde_status fd_apply_dense(hodlr_s* h, const double* x, double* y, int trans, cudaStream_t st) {
  const int N = h->tree.N;
  fd_matvec_kernel<<<ceil_div((long)N * 32, 256), 256, 0, st>>>(h->g, h->dp, h->dm, h->c, h->p.shift, N, x, y, trans);
  FDE_LAUNCH("fd_matvec_kernel");
  return FDE_OK;
}

fde_status fact_demote(hodlr_s* h, const Fact<double>& F, Fact<float>* G, DevPool& pool, cudaStream_t st) {
  const Tree& tr = h->tree;
  const int N = tr.N, L = tr.L, lmax = h->lmax, nl = tr.nleaves();
  G->sigma = F.sigma;
  G->lmin = F.lmin;
  G->Ut.assign(L, nullptr);
  G->Kinv.assign(L, nullptr);
  FDE_TRY(pool.alloc(&G->Dinv, (size_t)nl * lmax * lmax));
  FDE_TRY((convert<double, float>(F.Dinv, G->Dinv, (size_t)nl * lmax * lmax, st)));
  for (int l = F.lmin; l < L; ++l) {
    const size_t nu = (size_t)N * h->K[l], nk = (size_t)(1 << l) * 4 * h->K[l] * h->K[l];
    FDE_TRY(pool.alloc(&G->Ut[l], nu));
    FDE_TRY((convert<double, float>(F.Ut[l], G->Ut[l], nu, st)));
    FDE_TRY(pool.alloc(&G->Kinv[l], nk));
    FDE_TRY((convert<double, float>(F.Kinv[l], G->Kinv[l], nk, st)));
  }
  return FDE_OK;
}

fde_status hodlr_make_fp32(hodlr_s* h, cudaStream_t st) {
  if (h->D32) return FDE_OK;
  const int N = h->tree.N, L = h->tree.L;
  h->U32.assign(L, nullptr);
  h->V32.assign(L, nullptr);
  for (int l = 0; l < L; ++l) {
    FDE_TRY(h->pool.alloc(&h->U32[l], (size_t)N * h->K[l]));
    FDE_TRY(h->pool.alloc(&h->V32[l], (size_t)N * h->K[l]));
    FDE_TRY((copy2d<double, float>(h->U[l], N, h->U32[l], N, N, h->K[l], st)));
    FDE_TRY((copy2d<double, float>(h->V[l], N, h->V32[l], N, N, h->K[l], st)));
  }
  const size_t nd = (size_t)h->tree.nleaves() * h->lmax * h->lmax;
  FDE_TRY(h->pool.alloc(&h->D32, nd));
  FDE_TRY((convert<double, float>(h->D, h->D32, nd, st)));
  return FDE_OK;
}

}  // namespace fde

using namespace fde;

hodlr_s::~hodlr_s() {
  delete f0;
  delete solve_plan;
}

// ===================================================================== ABI
static fde_status upload_coeff(const double* src, double* dst, int N, cudaStream_t st) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, src);
  if (e != cudaSuccess) cudaGetLastError();
  const bool dev = (e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged));
  FDE_CUDA(cudaMemcpyAsync(dst, src, (size_t)N * sizeof(double),
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  if (!dev) FDE_CUDA(cudaStreamSynchronize(st));
  return FDE_OK;
}

static fde_status build_impl(const fde_op_params* p, cudaStream_t st, hodlr_s* h) {
  const int N = p->N;
  h->p = *p;
  h->p.d_plus = h->p.d_minus = nullptr;
  h->c = p->dt * pow(p->h, -p->alpha);
  Tree& tr = h->tree;
  tr.build(N, p->leaf);
  const int L = tr.L;
  DevPool& pool = h->pool;
  DevPool scratch;
  FDE_TRY(pool.alloc(&h->g, (size_t)N + 2));
  FDE_TRY(pool.alloc(&h->dp, (size_t)N));
  FDE_TRY(pool.alloc(&h->dm, (size_t)N));
  FDE_TRY(upload_coeff(p->d_plus, h->dp, N, st));
  FDE_TRY(upload_coeff(p->d_minus, h->dm, N, st));
  int* d_flag;
  FDE_TRY(scratch.alloc(&d_flag, 4));
  FDE_CUDA(cudaMemsetAsync(d_flag, 0, 4 * sizeof(int), st));
  finite_check_kernel<<<64, 256, 0, st>>>(h->dp, N, d_flag);
  FDE_LAUNCH("finite_check_kernel");
  finite_check_kernel<<<64, 256, 0, st>>>(h->dm, N, d_flag);
  FDE_LAUNCH("finite_check_kernel");
  gl_weights_kernel<<<1, 32, 0, st>>>(p->alpha, N + 1, h->g);
  FDE_LAUNCH("gl_weights_kernel");
  // ||A||_2 by 30 power steps on AᵀA from the normalised ones vector
  double *v, *w, *nrm;
  FDE_TRY(scratch.alloc(&v, N));
  FDE_TRY(scratch.alloc(&w, N));
  FDE_TRY(scratch.alloc(&nrm, 1));
  fill_kernel<<<64, 256, 0, st>>>(v, N, 1.0 / sqrt((double)N));
  const int mvb = ceil_div((long)N * 32, 256);
  for (int it = 0; it < 30; ++it) {
    fd_matvec_kernel<<<mvb, 256, 0, st>>>(h->g, h->dp, h->dm, h->c, p->shift, N, v, w, 0);
    FDE_LAUNCH("fd_matvec_kernel");
    fd_matvec_kernel<<<mvb, 256, 0, st>>>(h->g, h->dp, h->dm, h->c, p->shift, N, w, v, 1);
    FDE_LAUNCH("fd_matvec_kernel");
    norm2_kernel<<<1, 1024, 0, st>>>(v, N, nrm);
    FDE_LAUNCH("norm2_kernel");
    scale_inv_kernel<<<64, 256, 0, st>>>(v, N, nrm);
    FDE_LAUNCH("scale_inv_kernel");
  }
  int hflag[4];
  double hn;
  FDE_CUDA(cudaMemcpyAsync(hflag, d_flag, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
  FDE_CUDA(cudaMemcpyAsync(&hn, nrm, sizeof(double), cudaMemcpyDeviceToHost, st));
  FDE_CUDA(cudaStreamSynchronize(st));
  if (hflag[0]) {
    set_error("hodlr_build: d_plus / d_minus must be finite and non-negative");
    return FDE_ERR_NUMERIC;
  }
  h->norm2 = sqrt(hn);
  if (!(h->norm2 > 0.0) || !isfinite(h->norm2)) {
    set_error("hodlr_build: bad norm estimate %g", h->norm2);
    return FDE_ERR_NUMERIC;
  }
  // truncation budget: half to the ACA of T21 (scaled by c max d_±), half to
  // the per-block recompression, so each block error is <= ε||A||_2 (§3.4.1)
  double maxd = 0.0;
  {
    std::vector<double> hd(N);
    FDE_CUDA(cudaMemcpy(hd.data(), h->dp, N * sizeof(double), cudaMemcpyDeviceToHost));
    for (double x : hd) maxd = std::max(maxd, x);
    FDE_CUDA(cudaMemcpy(hd.data(), h->dm, N * sizeof(double), cudaMemcpyDeviceToHost));
    for (double x : hd) maxd = std::max(maxd, x);
  }
  h->blk_tol = 0.5 * p->tol * h->norm2;
  h->aca_tol = (maxd > 0.0 && h->c > 0.0) ? 0.01 * h->blk_tol / (h->c * maxd) : 0.0;
  if (L == 0) {
    h->kaca = 0;
    h->aca_conv = 1;
  } else {
    const int N1 = N / 2, N2 = N - N1;
    const int maxrank = std::min(std::min(N1, N2), 90);
    FDE_TRY(pool.alloc(&h->U0, (size_t)N2 * maxrank));
    FDE_TRY(pool.alloc(&h->V0, (size_t)N1 * maxrank));
    int *d_rows, *d_cols, *d_out;
    unsigned char *ur, *uc;
    FDE_TRY(scratch.alloc(&d_rows, maxrank));
    FDE_TRY(scratch.alloc(&d_cols, maxrank));
    FDE_TRY(scratch.alloc(&d_out, 2));
    FDE_TRY(scratch.alloc(&ur, N2));
    FDE_TRY(scratch.alloc(&uc, N1));
    aca_kernel<<<1, 1024, 0, st>>>(h->g, N1, N2, h->aca_tol, maxrank, h->U0, h->V0, d_rows, d_cols, d_out, ur, uc);
    FDE_LAUNCH("aca_kernel");
    int out2[2];
    FDE_CUDA(cudaMemcpyAsync(out2, d_out, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    FDE_CUDA(cudaStreamSynchronize(st));
    h->kaca = out2[0];
    h->aca_conv = out2[1];
    h->aca_rows.resize(h->kaca);
    h->aca_cols.resize(h->kaca);
    if (h->kaca > 0) {
      FDE_CUDA(cudaMemcpy(h->aca_rows.data(), d_rows, h->kaca * sizeof(int), cudaMemcpyDeviceToHost));
      FDE_CUDA(cudaMemcpy(h->aca_cols.data(), d_cols, h->kaca * sizeof(int), cudaMemcpyDeviceToHost));
    }
    if (!h->aca_conv && h->kaca < std::min(N1, N2)) {
      set_error("hodlr_build: ACA did not reach tolerance %g within rank %d", h->aca_tol, maxrank);
      return FDE_ERR_NOCONV;
    }
  }
  // level arrays: recompression inputs (scratch) and outputs (kept)
  const int r = h->kaca + 1;
  h->rcap = r;
  h->U.assign(L, nullptr);
  h->V.assign(L, nullptr);
  h->K.assign(L, 1);
  h->rank12.assign(tr.lo.size(), 0);
  h->rank21.assign(tr.lo.size(), 0);
  if (L > 0) {
    std::vector<double*> Uin(L), Vin(L);
    std::vector<NodeRef> nodes;
    std::vector<RecompJob> jobs;
    int* d_ranks;
    const int njobs = 2 * ((1 << L) - 1);
    FDE_TRY(scratch.alloc(&d_ranks, njobs));
    for (int l = 0; l < L; ++l) {
      FDE_TRY(scratch.alloc(&Uin[l], (size_t)N * r));
      FDE_TRY(scratch.alloc(&Vin[l], (size_t)N * r));
      FDE_TRY(pool.alloc(&h->U[l], (size_t)N * r));
      FDE_TRY(pool.alloc(&h->V[l], (size_t)N * r));
      for (int q = 0; q < (1 << l); ++q) {
        const int id = tr.id(l, q), lo = tr.lo[id], hi = tr.hi[id], mid = lo + (hi - lo) / 2;
        nodes.push_back({lo, mid, hi, Uin[l], Vin[l]});
        const int j0 = (int)jobs.size();
        // upper block A12: U rows lo..mid, V rows mid..hi
        jobs.push_back({Uin[l] + lo, Vin[l] + mid, h->U[l] + lo, h->V[l] + mid, mid - lo, hi - mid, N, d_ranks + j0});
        // lower block A21: U rows mid..hi, V rows lo..mid
        jobs.push_back({Uin[l] + mid, Vin[l] + lo, h->U[l] + mid, h->V[l] + lo, hi - mid, mid - lo, N, d_ranks + j0 + 1});
      }
    }
    NodeRef* d_nodes;
    RecompJob* d_jobs;
    FDE_TRY(scratch.alloc(&d_nodes, nodes.size()));
    FDE_TRY(scratch.alloc(&d_jobs, jobs.size()));
    FDE_CUDA(cudaMemcpy(d_nodes, nodes.data(), nodes.size() * sizeof(NodeRef), cudaMemcpyHostToDevice));
    FDE_CUDA(cudaMemcpy(d_jobs, jobs.data(), jobs.size() * sizeof(RecompJob), cudaMemcpyHostToDevice));
    const int N1 = N / 2, N2 = N - N1;
    block_factors_kernel<<<(int)nodes.size(), 256, 0, st>>>(d_nodes, h->U0, h->V0, h->dp, h->dm, h->c, N, N1, N2,
                                                            h->kaca);
    FDE_LAUNCH("block_factors_kernel");
    const size_t smem = recompress_smem(r);
    // per-kernel attribute shared by all handles and threads: only ever raised
    FDE_TRY(recompress_prepare(r));
    ProfScope ps("recompress", st);
    recompress_kernel<<<(int)jobs.size(), 512, smem, st>>>(d_jobs, r, r, h->blk_tol, 0.0);
    FDE_LAUNCH("recompress_kernel");
    std::vector<int> ranks(njobs);
    FDE_CUDA(cudaMemcpyAsync(ranks.data(), d_ranks, njobs * sizeof(int), cudaMemcpyDeviceToHost, st));
    FDE_CUDA(cudaStreamSynchronize(st));
    int j = 0;
    for (int l = 0; l < L; ++l) {
      int K = 1;
      for (int q = 0; q < (1 << l); ++q) {
        const int id = tr.id(l, q);
        h->rank12[id] = ranks[j++];
        h->rank21[id] = ranks[j++];
        K = std::max(K, std::max(h->rank12[id], h->rank21[id]));
      }
      h->K[l] = K;
    }
  }
  // leaves
  const int nl = tr.nleaves();
  h->leaf_n.resize(nl);
  h->leaf_lo.resize(nl);
  h->lmax = tr.maxleaf;
  for (int q = 0; q < nl; ++q) {
    const int id = tr.id(L, q);
    h->leaf_lo[q] = tr.lo[id];
    h->leaf_n[q] = tr.hi[id] - tr.lo[id];
  }
  int* d_leaf_lo;
  FDE_TRY(pool.alloc(&h->d_leaf_n, nl));
  FDE_TRY(scratch.alloc(&d_leaf_lo, nl));
  FDE_CUDA(cudaMemcpy(h->d_leaf_n, h->leaf_n.data(), nl * sizeof(int), cudaMemcpyHostToDevice));
  FDE_CUDA(cudaMemcpy(d_leaf_lo, h->leaf_lo.data(), nl * sizeof(int), cudaMemcpyHostToDevice));
  FDE_TRY(pool.alloc(&h->D, (size_t)nl * h->lmax * h->lmax));
  leaves_kernel<<<nl, 256, 0, st>>>(h->g, h->dp, h->dm, h->c, p->shift, d_leaf_lo, h->d_leaf_n, h->lmax, h->D);
  FDE_LAUNCH("leaves_kernel");
  FDE_CUDA(cudaStreamSynchronize(st));
  return FDE_OK;
}

namespace fde {
size_t recompress_smem(int r) { return (3 * (size_t)r * r + 3 * r) * sizeof(double) + r * sizeof(int); }

fde_status recompress_prepare(int rmax) {
  static std::mutex mu;
  static size_t set_to = 0;
  const size_t smem = recompress_smem(rmax);
  std::lock_guard<std::mutex> lk(mu);
  if (smem > set_to) {
    FDE_CUDA(cudaFuncSetAttribute(recompress_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FDE_CUDA(cudaFuncSetAttribute(recomp_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FDE_CUDA(cudaFuncSetAttribute(recomp_core_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    set_to = smem;
  }
  return FDE_OK;
}

fde_status recompress_split(const RecompJob* d_jobs, int njobs, int r, int rcap, double abstol, double reltol,
                            const RecompWork& wk, cudaStream_t st) {
  if (r > kRecompMax || rcap > r) {
    set_error("recompression of rank %d above %d", r, kRecompMax);
    return FDE_ERR_ARG;
  }
  recomp_qr_kernel<<<2 * njobs, 512, (size_t)r * r * sizeof(double), st>>>(d_jobs, r, wk);
  FDE_LAUNCH("recomp_qr_kernel");
  recomp_core_kernel<<<njobs, 512, (2 * (size_t)r * r + r) * sizeof(double) + r * sizeof(int), st>>>(
      d_jobs, r, rcap, abstol, reltol, wk);
  FDE_LAUNCH("recomp_core_kernel");
  recomp_apply_kernel<<<2 * njobs, 512, 0, st>>>(d_jobs, r, rcap, wk);
  FDE_LAUNCH("recomp_apply_kernel");
  return FDE_OK;
}

fde_status recompress_core(const RecompJob* d_job, int r, int rcap, double abstol, double reltol,
                           const RecompWork& wk, cudaStream_t st) {
  recomp_core_kernel<<<1, 512, (2 * (size_t)r * r + r) * sizeof(double) + r * sizeof(int), st>>>(
      d_job, r, rcap, abstol, reltol, wk);
  FDE_LAUNCH("recomp_core_kernel");
  return FDE_OK;
}

fde_status recompress_jobs(const RecompJob* d_jobs, int njobs, int r, int rcap, double abstol, double reltol,
                           cudaStream_t st) {
  if (r > kRecompMax || rcap > r) {
    set_error("recompression of rank %d above %d", r, kRecompMax);
    return FDE_ERR_ARG;
  }
  recompress_kernel<<<njobs, 512, recompress_smem(r), st>>>(d_jobs, r, rcap, abstol, reltol);
  FDE_LAUNCH("recompress_kernel");
  return FDE_OK;
}
}  // namespace fde

static fde_status check_op(const fde_op_params* p) {
  FDE_ARG(p != nullptr, "params is NULL");
  FDE_ARG(p->N >= 2, "N must be >= 2");
  FDE_ARG(p->N <= (1 << 20), "N too large");
  FDE_ARG(p->alpha > 1.0 && p->alpha <= 2.0, "alpha must lie in (1, 2]");
  FDE_ARG(p->h > 0.0 && isfinite(p->h), "h must be > 0");
  FDE_ARG(p->dt > 0.0 && isfinite(p->dt), "dt must be > 0");
  FDE_ARG(p->shift > 0.0 && isfinite(p->shift), "shift must be > 0");
  FDE_ARG(p->leaf >= 8 && p->leaf <= 256, "leaf must be in [8, 256]");
  FDE_ARG(p->tol > 0.0 && p->tol < 1.0, "tol must be in (0, 1)");
  FDE_ARG(p->d_plus != nullptr && p->d_minus != nullptr, "d_plus / d_minus are NULL");
  return FDE_OK;
}

extern "C" fde_status hodlr_build(const fde_op_params* p, void* stream, hodlr_t* out) {
  FDE_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  FDE_TRY(check_op(p));
  hodlr_s* h = new hodlr_s();
  fde_status s = build_impl(p, (cudaStream_t)stream, h);
  if (s != FDE_OK) {
    delete h;
    return s;
  }
  *out = h;
  return FDE_OK;
}

extern "C" fde_status hodlr_factor(hodlr_t h, void* stream) {
  FDE_ARG(h != nullptr, "handle is NULL");
  if (h->f0) return FDE_OK;
  Fact<double>* F = new Fact<double>();
  fde_status s = hodlr_factorize(h, 0.0, 0, F, (cudaStream_t)stream);
  if (s != FDE_OK) {
    delete F;
    return s;
  }
  h->f0 = F;
  return FDE_OK;
}

extern "C" fde_status hodlr_solve(hodlr_t h, const double* d_b, double* d_x, int nrhs, int ldb, void* stream) {
  FDE_ARG(h != nullptr, "handle is NULL");
  FDE_ARG(h->f0 != nullptr, "hodlr_factor has not been called");
  FDE_ARG(d_b != nullptr && d_x != nullptr, "NULL vector");
  FDE_ARG(nrhs >= 1 && ldb >= h->tree.N, "bad nrhs / ldb");
  cudaStream_t st = (cudaStream_t)stream;
  const int N = h->tree.N;
  if (d_x != d_b) FDE_TRY((copy2d<double, double>(d_b, ldb, d_x, ldb, N, nrhs, st)));
  if (!h->solve_plan || h->solve_plan_x != d_x || h->solve_plan_ncols != nrhs || h->solve_plan_ld != ldb) {
    // (re)build the cached plan for this output buffer
    delete h->solve_plan;
    h->solve_plan = new Plan<double>();
    double *zb, *wb;
    const size_t zel = solve_scratch_elems(h, nrhs, 0);
    FDE_TRY(h->pool.alloc(&h->solve_tmp, (size_t)N * nrhs));
    FDE_TRY(h->pool.alloc(&zb, zel));
    FDE_TRY(h->pool.alloc(&wb, zel));
    FDE_TRY(build_solve_plan<double>(h, *h->f0, h->V, d_x, ldb, d_x, ldb, nrhs, 0, h->solve_tmp, zb, wb,
                                     h->pool, h->solve_plan, st));
    h->solve_plan_x = d_x;
    h->solve_plan_ncols = nrhs;
    h->solve_plan_ld = ldb;
  }
  FDE_TRY(plan_run(*h->solve_plan, st));
  return FDE_OK;
}

extern "C" fde_status hodlr_matvec(hodlr_t h, const double* d_x, double* d_y, int nrhs, int ldx, void* stream) {
  FDE_ARG(h != nullptr, "handle is NULL");
  FDE_ARG(d_x != nullptr && d_y != nullptr && d_x != d_y, "bad vectors");
  FDE_ARG(nrhs >= 1 && ldx >= h->tree.N, "bad nrhs / ldx");
  cudaStream_t st = (cudaStream_t)stream;
  const Tree& tr = h->tree;
  const int N = tr.N, L = tr.L, lmax = h->lmax;
  DevPool scratch;
  std::vector<GemmDesc<double>> dl;
  for (int q = 0; q < tr.nleaves(); ++q) {
    const int id = tr.id(L, q), lo = tr.lo[id], n = tr.hi[id] - lo;
    dl.push_back({h->D + (size_t)q * lmax * lmax, d_x + lo, d_y + lo, n, nrhs, n, lmax, ldx, ldx});
  }
  GemmBatch<double> gl;
  FDE_TRY(gemm_batch_upload(scratch, dl, false, false, 1.0, 0.0, &gl, st));
  FDE_TRY(gemm_batch_run(gl, st));
  for (int l = 0; l < L; ++l) {
    const int K = h->K[l], K2 = 2 * K;
    double* z;
    FDE_TRY(scratch.alloc(&z, (size_t)(1 << l) * K2 * nrhs));
    std::vector<GemmDesc<double>> dz, du;
    for (int q = 0; q < (1 << l); ++q) {
      const int id = tr.id(l, q), lo = tr.lo[id], hi = tr.hi[id], mid = lo + (hi - lo) / 2;
      double* zp = z + (size_t)q * K2 * nrhs;
      dz.push_back({h->V[l] + mid, d_x + mid, zp, K, nrhs, hi - mid, N, ldx, K2});
      dz.push_back({h->V[l] + lo, d_x + lo, zp + K, K, nrhs, mid - lo, N, ldx, K2});
      du.push_back({h->U[l] + lo, zp, d_y + lo, mid - lo, nrhs, K, N, K2, ldx});
      du.push_back({h->U[l] + mid, zp + K, d_y + mid, hi - mid, nrhs, K, N, K2, ldx});
    }
    GemmBatch<double> gz, gu;
    FDE_TRY(gemm_batch_upload(scratch, dz, true, false, 1.0, 0.0, &gz, st));
    FDE_TRY(gemm_batch_upload(scratch, du, false, false, 1.0, 1.0, &gu, st));
    FDE_TRY(gemm_batch_run(gz, st));
    FDE_TRY(gemm_batch_run(gu, st));
  }
  FDE_CUDA(cudaStreamSynchronize(st));
  return FDE_OK;
}

extern "C" fde_status hodlr_get_info(hodlr_t h, hodlr_info_t* info) {
  FDE_ARG(h != nullptr && info != nullptr, "NULL argument");
  info->N = h->tree.N;
  info->leaf = h->tree.leaf;
  info->levels = h->tree.L;
  info->nleaves = h->tree.nleaves();
  int km = 0;
  for (int k : h->K) km = std::max(km, k);
  info->kmax = km;
  info->aca_rank = h->kaca;
  info->aca_converged = h->aca_conv;
  info->norm2 = h->norm2;
  info->c = h->c;
  info->aca_tol = h->aca_tol;
  return FDE_OK;
}

extern "C" fde_status hodlr_to_dense(hodlr_t h, double* d_A, int ld, void* stream) {
  FDE_ARG(h != nullptr && d_A != nullptr, "NULL argument");
  FDE_ARG(ld >= h->tree.N, "ld < N");
  FDE_ARG(h->tree.L <= 24, "tree too deep");
  cudaStream_t st = (cudaStream_t)stream;
  LevelPtrs lp;
  for (int l = 0; l < h->tree.L; ++l) {
    lp.U[l] = h->U[l];
    lp.V[l] = h->V[l];
    lp.K[l] = h->K[l];
  }
  DevPool scratch;
  int *tlo, *thi;
  FDE_TRY(scratch.alloc(&tlo, h->tree.lo.size()));
  FDE_TRY(scratch.alloc(&thi, h->tree.hi.size()));
  FDE_CUDA(cudaMemcpy(tlo, h->tree.lo.data(), h->tree.lo.size() * sizeof(int), cudaMemcpyHostToDevice));
  FDE_CUDA(cudaMemcpy(thi, h->tree.hi.data(), h->tree.hi.size() * sizeof(int), cudaMemcpyHostToDevice));
  to_dense_kernel<<<1024, 256, 0, st>>>(lp, h->D, h->lmax, h->tree.N, h->tree.L, tlo, thi, d_A, ld);
  FDE_LAUNCH("to_dense_kernel");
  FDE_CUDA(cudaStreamSynchronize(st));
  return FDE_OK;
}

extern "C" fde_status hodlr_get_weights(hodlr_t h, double* h_g) {
  FDE_ARG(h != nullptr && h_g != nullptr, "NULL argument");
  FDE_CUDA(cudaMemcpy(h_g, h->g, ((size_t)h->tree.N + 2) * sizeof(double), cudaMemcpyDeviceToHost));
  return FDE_OK;
}

extern "C" fde_status hodlr_get_aca_pivots(hodlr_t h, int* h_rows, int* h_cols, int cap, int* h_k) {
  FDE_ARG(h != nullptr && h_k != nullptr, "NULL argument");
  *h_k = h->kaca;
  const int n = std::min(cap, h->kaca);
  for (int i = 0; i < n; ++i) {
    if (h_rows) h_rows[i] = h->aca_rows[i];
    if (h_cols) h_cols[i] = h->aca_cols[i];
  }
  return FDE_OK;
}

extern "C" fde_status hodlr_get_tree(hodlr_t h, int* h_lo, int* h_hi, int cap) {
  FDE_ARG(h != nullptr && h_lo != nullptr && h_hi != nullptr, "NULL argument");
  FDE_ARG(cap >= (int)h->tree.lo.size(), "capacity too small");
  for (size_t i = 0; i < h->tree.lo.size(); ++i) {
    h_lo[i] = h->tree.lo[i];
    h_hi[i] = h->tree.hi[i];
  }
  return FDE_OK;
}

extern "C" void hodlr_free(hodlr_t h) { delete h; }

extern "C" fde_status fde_tree_layout(int N, int leaf, int* h_lo, int* h_hi, int cap, int* levels) {
  FDE_ARG(N >= 1 && N <= (1 << 20), "N must be in [1, 2^20]");
  FDE_ARG(leaf >= 1, "leaf must be >= 1");
  FDE_ARG(levels != nullptr, "levels is NULL");
  fde::Tree t;
  t.build(N, leaf);
  *levels = t.L;
  FDE_ARG(h_lo != nullptr && h_hi != nullptr, "NULL node arrays");
  FDE_ARG(cap >= (int)t.lo.size(), "capacity too small (2^(levels+1) - 1 nodes)");
  for (size_t i = 0; i < t.lo.size(); ++i) {
    h_lo[i] = t.lo[i];
    h_hi[i] = t.hi[i];
  }
  return FDE_OK;
}

extern "C" const char* fde_strerror(fde_status s) {
  switch (s) {
    case FDE_OK: return "ok";
    case FDE_ERR_ARG: return "invalid argument";
    case FDE_ERR_NOMEM: return "out of device memory";
    case FDE_ERR_NOCONV: return "iteration cap reached without convergence";
    case FDE_ERR_NUMERIC: return "non-finite or singular data";
    case FDE_ERR_CUDA: return "CUDA error";
  }
  return "unknown status";
}

extern "C" const char* fde_last_error(void) { return g_err; }
