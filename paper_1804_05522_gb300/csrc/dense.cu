// Batched dense kernels: SIMT GEMM with per-batch descriptors, batched
// Gauss–Jordan inversion, conversions.
#include <cstdint>

#include "dense.cuh"

namespace fde {

// ---------------------------------------------------------------- GEMM
// 64x64 output tile per CTA, 256 threads, 4x4 outputs per thread, BK = 16.
// Thread (tx, ty) owns rows tx + 16 i and columns ty + 16 j of the tile so
// that stores of a fixed (i, j) are contiguous in column-major C.
template <typename T, bool TA, bool TB>
__global__ void __launch_bounds__(256) gemm_batched_kernel(const GemmDesc<T>* __restrict__ descs, T alpha,
                                                          T beta) {
  const GemmDesc<T> d = descs[blockIdx.z];
  const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
  if (m0 >= d.m || n0 >= d.n) return;
  __shared__ T As[16][64 + 1];
  __shared__ T Bs[16][64 + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  for (int k0 = 0; k0 < d.k; k0 += 16) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = threadIdx.x + 256 * r;
      int mm, kk;
      if (!TA) {
        mm = e & 63;
        kk = e >> 6;
      } else {
        kk = e & 15;
        mm = e >> 4;
      }
      const int gm = m0 + mm, gk = k0 + kk;
      T v = T(0);
      if (gm < d.m && gk < d.k) {
        if (TA) {
          v = d.A[gk + (size_t)gm * d.lda];
        } else {
          const long long col = d.kblk ? (long long)(gk / d.kblk) * d.kstr + (long long)(gk % d.kblk) * d.lda
                                       : (long long)gk * d.lda;
          v = d.A[gm + col];
        }
      }
      As[kk][mm] = v;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = threadIdx.x + 256 * r;
      int kk, nn;
      if (!TB) {
        kk = e & 15;
        nn = e >> 4;
      } else {
        nn = e & 63;
        kk = e >> 6;
      }
      const int gn = n0 + nn, gk = k0 + kk;
      T v = T(0);
      if (gn < d.n && gk < d.k) {
        if (TB) {
          const long long col = d.kblk ? (long long)(gk / d.kblk) * d.kstr + (long long)(gk % d.kblk) * d.ldb
                                       : (long long)gk * d.ldb;
          v = d.B[gn + col];
        } else {
          v = d.B[gk + (size_t)gn * d.ldb];
        }
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
  // beta C: every load before the first store (a store in between would order
  // the next load behind it, as the compiler cannot rule out aliasing)
  T cv[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gm = m0 + tx + 16 * i, gn = n0 + ty + 16 * j;
      cv[i][j] = (beta != T(0) && gm < d.m && gn < d.n) ? d.C[gm + (size_t)gn * d.ldc] : T(0);
    }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int gn = n0 + ty + 16 * j;
    if (gn >= d.n) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gm = m0 + tx + 16 * i;
      if (gm >= d.m) continue;
      d.C[gm + (size_t)gn * d.ldc] = alpha * acc[i][j] + beta * cv[i][j];
    }
  }
}

template <typename T>
fde_status gemm_batch_upload(DevPool& pool, const std::vector<GemmDesc<T>>& h, bool ta, bool tb, T alpha,
                             T beta, GemmBatch<T>* out, cudaStream_t st) {
  GemmBatch<T> b;
  b.ta = ta;
  b.tb = tb;
  b.alpha = alpha;
  b.beta = beta;
  b.batch = (int)h.size();
  auto vec_ok = [](const T* p, int ld, int kblk, long long kstr) {
    return ((uintptr_t)p % 16) == 0 && ld % 4 == 0 && (kblk == 0 || kstr % 4 == 0);
  };
  b.vec_a = b.vec_b = b.batch > 0;
  std::vector<GemmDesc<T>> hd(h);
  for (auto& d : hd) {
    if (d.kblk > 0) {
      // division by the invariant kblk as a multiply-shift (Granlund and
      // Montgomery, "Division by invariant integers using multiplication", 1994):
      // l = ceil(log2 kblk), m = ceil(2^(32+l) / kblk) is exact for numerators < 2^32
      int l = 0;
      while ((1ll << l) < d.kblk) ++l;
      const unsigned long long two = 1ull << (32 + l);
      d.kmagic = (two + (unsigned long long)d.kblk - 1ull) / (unsigned long long)d.kblk;
      d.kshift = 32 + l;
      for (int k = 0; k < d.k + 64; ++k)
        if ((int)(((unsigned long long)k * d.kmagic) >> d.kshift) != k / d.kblk) {
          set_error("gemm_batch_upload: multiply-shift division by %d failed at %d", d.kblk, k);
          return FDE_ERR_ARG;
        }
    }
  }
  for (const auto& d : hd) {
    b.vec_a = b.vec_a && vec_ok(d.A, d.lda, ta ? 0 : d.kblk, d.kstr);
    b.vec_b = b.vec_b && vec_ok(d.B, d.ldb, tb ? d.kblk : 0, d.kstr);
    b.max_m = d.m > b.max_m ? d.m : b.max_m;
    b.max_ldc = d.ldc > b.max_ldc ? d.ldc : b.max_ldc;
    b.max_n = d.n > b.max_n ? d.n : b.max_n;
    b.max_k = d.k > b.max_k ? d.k : b.max_k;
    b.flops += 2.0 * d.m * d.n * d.k;
  }
  if (b.batch > 0) {
    FDE_TRY(pool.alloc(&b.d_desc, h.size()));
    FDE_CUDA(cudaMemcpyAsync(b.d_desc, hd.data(), hd.size() * sizeof(GemmDesc<T>), cudaMemcpyHostToDevice, st));
    // descriptors live in pageable host memory owned by the caller's vector:
    // make sure the copy has consumed them before returning.
    FDE_CUDA(cudaStreamSynchronize(st));
  }
  *out = b;
  return FDE_OK;
}

template <typename T>
fde_status gemm_batch_run(const GemmBatch<T>& b, cudaStream_t st) {
  if (b.batch == 0 || b.max_m == 0 || b.max_n == 0) return FDE_OK;
  if constexpr (sizeof(T) == 4) {
    bool used = false;
    FDE_TRY(tc_gemm_run(reinterpret_cast<const GemmBatch<float>&>(b), st, &used));
    if (used) return FDE_OK;
  }
  for (int z0 = 0; z0 < b.batch; z0 += 65535) {
    int nz = b.batch - z0 < 65535 ? b.batch - z0 : 65535;
    dim3 grid(ceil_div(b.max_m, 64), ceil_div(b.max_n, 64), nz);
    const GemmDesc<T>* d = b.d_desc + z0;
    ProfScope ps(sizeof(T) == 4 ? "gemm32" : "gemm64", st, z0 == 0 ? b.flops : 0.0, 1);
    if (!b.ta && !b.tb)
      gemm_batched_kernel<T, false, false><<<grid, 256, 0, st>>>(d, b.alpha, b.beta);
    else if (b.ta && !b.tb)
      gemm_batched_kernel<T, true, false><<<grid, 256, 0, st>>>(d, b.alpha, b.beta);
    else if (!b.ta && b.tb)
      gemm_batched_kernel<T, false, true><<<grid, 256, 0, st>>>(d, b.alpha, b.beta);
    else
      gemm_batched_kernel<T, true, true><<<grid, 256, 0, st>>>(d, b.alpha, b.beta);
    FDE_LAUNCH("gemm_batched_kernel");
  }
  return FDE_OK;
}

// ------------------------------------------------------------- inversion
// One CTA per matrix.  W = [A | I] (n x 2n, column-major, ld = n) in global
// scratch; Gauss–Jordan with partial pivoting; A <- right half.
template <typename T>
__global__ void __launch_bounds__(256) gj_inverse_kernel(T* A, int ld, size_t stride, const int* __restrict__ dn,
                                                        int nmax, T* work, int* flag) {
  const int b = blockIdx.x;
  const int n = dn[b];
  T* a = A + (size_t)b * stride;
  T* w = work + (size_t)b * nmax * 2 * nmax;
  __shared__ T colk[256];
  __shared__ T rowk[512];
  __shared__ T redv[256];
  __shared__ int redi[256];
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  for (int e = threadIdx.x; e < n * 2 * n; e += blockDim.x) {
    int i = e % n, j = e / n;
    w[i + (size_t)j * n] = (j < n) ? a[i + (size_t)j * ld] : (i == j - n ? T(1) : T(0));
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    // pivot search on column k, rows k..n-1 (lowest index on ties)
    T best = T(-1);
    int bi = k;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
      T v = fabs(w[i + (size_t)k * n]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
    redv[threadIdx.x] = best;
    redi[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        T v2 = redv[threadIdx.x + s];
        int i2 = redi[threadIdx.x + s];
        if (v2 > redv[threadIdx.x] || (v2 == redv[threadIdx.x] && i2 < redi[threadIdx.x])) {
          redv[threadIdx.x] = v2;
          redi[threadIdx.x] = i2;
        }
      }
      __syncthreads();
    }
    const int piv = redi[0];
    if (!(redv[0] > T(0))) {
      if (threadIdx.x == 0) s_bad = 1;
      __syncthreads();
      break;
    }
    // swap rows k and piv
    if (piv != k)
      for (int j = threadIdx.x; j < 2 * n; j += blockDim.x) {
        T t = w[k + (size_t)j * n];
        w[k + (size_t)j * n] = w[piv + (size_t)j * n];
        w[piv + (size_t)j * n] = t;
      }
    __syncthreads();
    const T p = w[k + (size_t)k * n];
    for (int j = threadIdx.x; j < 2 * n; j += blockDim.x) rowk[j] = w[k + (size_t)j * n] / p;
    for (int i = threadIdx.x; i < n; i += blockDim.x) colk[i] = w[i + (size_t)k * n];
    __syncthreads();
    for (int e = threadIdx.x; e < n * 2 * n; e += blockDim.x) {
      int i = e % n, j = e / n;
      if (i == k)
        w[i + (size_t)j * n] = rowk[j];
      else
        w[i + (size_t)j * n] -= colk[i] * rowk[j];
    }
    __syncthreads();
  }
  if (s_bad) {
    if (threadIdx.x == 0) atomicExch(flag, 1);
    return;
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e % n, j = e / n;
    a[i + (size_t)j * ld] = w[i + (size_t)(j + n) * n];
  }
}

template <typename T>
fde_status batched_inverse(T* A, int ld, size_t stride, const int* d_n, int batch, int nmax, T* work,
                           int* d_flag, cudaStream_t st) {
  if (batch == 0) return FDE_OK;
  if (nmax > 256) {
    set_error("batched_inverse: size %d > 256", nmax);
    return FDE_ERR_ARG;
  }
  gj_inverse_kernel<T><<<batch, 256, 0, st>>>(A, ld, stride, d_n, nmax, work, d_flag);
  FDE_LAUNCH("gj_inverse_kernel");
  return FDE_OK;
}

// ------------------------------------------------------------ conversion
template <typename Tin, typename Tout>
__global__ void convert_kernel(const Tin* __restrict__ x, Tout* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (Tout)x[i];
}

template <typename Tin, typename Tout>
fde_status convert(const Tin* x, Tout* y, size_t n, cudaStream_t st) {
  if (n == 0) return FDE_OK;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  convert_kernel<Tin, Tout><<<blocks, 256, 0, st>>>(x, y, n);
  FDE_LAUNCH("convert_kernel");
  return FDE_OK;
}

template <typename Tin, typename Tout>
__global__ void copy2d_kernel(const Tin* __restrict__ X, int ldx, Tout* __restrict__ Y, int ldy, int m, int n) {
  size_t total = (size_t)m * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(e % m), j = (int)(e / m);
    Y[i + (size_t)j * ldy] = (Tout)X[i + (size_t)j * ldx];
  }
}

template <typename Tin, typename Tout>
fde_status copy2d(const Tin* X, int ldx, Tout* Y, int ldy, int m, int n, cudaStream_t st) {
  if (m == 0 || n == 0) return FDE_OK;
  size_t total = (size_t)m * n;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  copy2d_kernel<Tin, Tout><<<blocks, 256, 0, st>>>(X, ldx, Y, ldy, m, n);
  FDE_LAUNCH("copy2d_kernel");
  return FDE_OK;
}

#define INST(T)                                                                                            \
  template fde_status gemm_batch_upload<T>(DevPool&, const std::vector<GemmDesc<T>>&, bool, bool, T, T,     \
                                           GemmBatch<T>*, cudaStream_t);                                   \
  template fde_status gemm_batch_run<T>(const GemmBatch<T>&, cudaStream_t);                                \
  template fde_status batched_inverse<T>(T*, int, size_t, const int*, int, int, T*, int*, cudaStream_t);
INST(double)
INST(float)
#undef INST
template fde_status convert<double, float>(const double*, float*, size_t, cudaStream_t);
template fde_status convert<float, double>(const float*, double*, size_t, cudaStream_t);
template fde_status copy2d<double, float>(const double*, int, float*, int, int, int, cudaStream_t);
template fde_status copy2d<float, double>(const float*, int, double*, int, int, int, cudaStream_t);
template fde_status copy2d<double, double>(const double*, int, double*, int, int, int, cudaStream_t);
template fde_status copy2d<float, float>(const float*, int, float*, int, int, int, cudaStream_t);

}  // namespace fde
