// Batched dense kernels: SIMT GEMM with per-batch descriptors, batched
// Gauss–Jordan inversion, conversions.
#include <atomic>
#include <cstdint>
#include <cstdlib>

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

// FDE_SKINNY=0 turns the skinny kernel below off (comparisons);
// set_skinny_force (fde_gemm_f32's explicit modes) overrides both ways.
static std::atomic<int> g_skinny_force{-1};
void set_skinny_force(int v) { g_skinny_force.store(v); }
static bool skinny_mode() {
  const int f = g_skinny_force.load();
  if (f >= 0) return f != 0;
  static const bool on = []() {
    const char* e = getenv("FDE_SKINNY");
    return !(e && e[0] == '0');
  }();
  return on;
}

// ------------------------------------------------------------ skinny GEMM
// FP32 products with one dimension of at most 64 (the fADI right-hand-side
// factors and the root-level rational application, n = 16..34; the
// rank-sized products Vᵀ X, m <= 64).  Written on a "long x skinny" view:
//   C'(l, c) = alpha sum_k A'(l, k) B'(k, c) + beta C'(l, c),  l < L, c < S <= SC,
// with A'(l, k) = A[l * al + k * ak], B'(k, c) = B[k * bk + c * bc],
// C'(l, c) = C[l * cl + c * cc]: for n <= 64 the problem itself (L = m), for
// m <= 64 its transpose (L = n, A' = op(B)ᵀ, B' = op(A)ᵀ, C' = Cᵀ).
// Tile 128 (l) x SC (c), k in steps of 16 prefetched in registers; 128
// threads, thread (tl, tc) owns rows 8 tl..8 tl + 7 and columns
// tc (SC/8)..: exact FP32 products (no tensor-core rounding), every column
// of the skinny dimension used (SC is the next multiple of 16).
constexpr int kSkL = 128, kSkK = 16, kSkThreads = 128;

template <int SC, bool A_LCONT, bool B_KCONT>
__global__ void __launch_bounds__(kSkThreads, SC <= 32 ? 4 : 2) gemm_skinny_kernel(const GemmDesc<float>* __restrict__ descs,
                                                                  bool transposed, bool ta, bool tb, float alpha,
                                                                  float beta) {
  constexpr int RC = SC / 8;
  constexpr int LDA_S = kSkL + 4, LDB_S = SC + 4;  // padded shared rows (16-byte aligned)
  __shared__ __align__(16) float As[kSkK][LDA_S];
  __shared__ __align__(16) float Bs[kSkK][LDB_S];
  const GemmDesc<float> d = descs[blockIdx.y];
  // strides of the long x skinny view
  long long al, ak, bk, bc, cl, cc;
  int L, S;
  if (!transposed) {
    L = d.m; S = d.n;
    al = ta ? d.lda : 1; ak = ta ? 1 : d.lda;
    bk = tb ? d.ldb : 1; bc = tb ? 1 : d.ldb;
    cl = 1; cc = d.ldc;
  } else {
    L = d.n; S = d.m;
    al = tb ? 1 : d.ldb; ak = tb ? d.ldb : 1;
    bk = ta ? 1 : d.lda; bc = ta ? d.lda : 1;
    cl = d.ldc; cc = 1;
  }
  const int K = d.k;
  const int l0 = blockIdx.x * kSkL;
  if (l0 >= L) return;
  const int t = threadIdx.x, tl = t & 15, tc = t >> 4;
  // register prefetch of one k-tile: 16 A' values, SC / 8 B' values per thread.
  // Element q of this thread: A_LCONT: (l, k) = (t, q); else (t / 16 + 8 q, t % 16),
  // i.e. a base address plus q steps of a fixed stride.
  const int la = A_LCONT ? t : (t >> 4), ka = A_LCONT ? 0 : (t & 15);
  const int dla = A_LCONT ? 0 : 8, dka = A_LCONT ? 1 : 0;
  const long long astep = A_LCONT ? ak : 8 * al;
  // A' and B' come from op(B) and op(A) in the transposed view
  const float* Ap = transposed ? d.B : d.A;
  const float* Bp = transposed ? d.A : d.B;
  const float* abase = Ap + (long long)(l0 + la) * al + (long long)ka * ak;
  float ra[16], rb[RC];
  auto load = [&](int k0) {
    const float* ap = abase + (long long)k0 * ak;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int gl = l0 + la + dla * q, gk = k0 + ka + dka * q;
      ra[q] = (gl < L && gk < K) ? ap[q * astep] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < RC; ++q) {
      const int e = t + kSkThreads * q;  // e < 16 * SC
      const int c = B_KCONT ? (e >> 4) : (e % SC), kk = B_KCONT ? (e & 15) : (e / SC);
      const int gk = k0 + kk;
      rb[q] = (c < S && gk < K) ? Bp[(long long)gk * bk + (long long)c * bc] : 0.f;
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int q = 0; q < 16; ++q) As[ka + dka * q][la + dla * q] = ra[q];
#pragma unroll
    for (int q = 0; q < RC; ++q) {
      const int e = t + kSkThreads * q;
      const int c = B_KCONT ? (e >> 4) : (e % SC), kk = B_KCONT ? (e & 15) : (e / SC);
      Bs[kk][c] = rb[q];
    }
  };
  float acc[8][RC];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < RC; ++j) acc[i][j] = 0.f;
  load(0);
  for (int k0 = 0; k0 < K; k0 += kSkK) {
    __syncthreads();  // the previous tile's readers are done
    stash();
    __syncthreads();
    if (k0 + kSkK < K) load(k0 + kSkK);  // in flight during the products below
#pragma unroll
    for (int kk = 0; kk < kSkK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][8 * tl]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][8 * tl + 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float b[RC];
#pragma unroll
      for (int j = 0; j < RC; ++j) b[j] = Bs[kk][tc * RC + j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < RC; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
  }
  // per row: the RC loads of beta C' before its stores
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gl = l0 + 8 * tl + i;
    if (gl >= L) break;
    float cv[RC];
#pragma unroll
    for (int j = 0; j < RC; ++j) {
      const int c = tc * RC + j;
      cv[j] = (beta != 0.f && c < S) ? d.C[(long long)gl * cl + (long long)c * cc] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < RC; ++j) {
      const int c = tc * RC + j;
      if (c < S) d.C[(long long)gl * cl + (long long)c * cc] = alpha * acc[i][j] + beta * cv[j];
    }
  }
}

// Pipelined variant for the common layout: A m-contiguous (ta = 0), B
// k-contiguous (tb = 0), both 16-byte aligned with leading dimensions that
// are multiples of 4 (the root-level rational application streams its
// stacked operator, ~1 GB, from HBM).  NST k-tiles of A' (16 x 128) and B'
// (stored column-major, SC x 16) in flight through cp.async, zero-filled at
// the ragged edges; the arithmetic is the kernel above's.
constexpr int kSkStages = 4;

__device__ __forceinline__ void sk_cp16(uint32_t dst, const float* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void sk_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void sk_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int SC>
constexpr int sk_stage_floats() {
  return kSkK * (kSkL + 4) + SC * (kSkK + 4);
}

template <int SC>
__global__ void __launch_bounds__(kSkThreads, 3) gemm_skinny_pipe_kernel(const GemmDesc<float>* __restrict__ descs,
                                                                          float alpha, float beta) {
  constexpr int RC = SC / 8, LDA_S = kSkL + 4, LDB_S = kSkK + 4, STAGE = sk_stage_floats<SC>();
  extern __shared__ __align__(16) float skm[];
  const GemmDesc<float> d = descs[blockIdx.y];
  const int L = d.m, S = d.n, K = d.k;
  const int l0 = blockIdx.x * kSkL;
  if (l0 >= L) return;
  const int t = threadIdx.x, tl = t & 15, tc = t >> 4;
  const int nkt = (K + kSkK - 1) / kSkK;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(skm);
  auto issue = [&](int kt) {
    if (kt < nkt) {
      const int k0 = kt * kSkK;
      const uint32_t st = sbase + (uint32_t)((kt % kSkStages) * STAGE) * 4u;
      // A': 16 k rows of 128 l, 16-byte chunks of 4 l
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = t + kSkThreads * q, kk = c >> 5, l4 = (c & 31) * 4;
        const int gl = l0 + l4, gk = k0 + kk;
        int nv = L - gl;
        nv = gk < K ? (nv < 0 ? 0 : nv > 4 ? 4 : nv) : 0;
        const float* src = nv > 0 ? d.A + (long long)gl + (long long)gk * d.lda : d.A;
        sk_cp16(st + (uint32_t)(kk * LDA_S + l4) * 4u, src, 4 * nv);
      }
      // B': SC columns of 16 k, chunks of 4 k
      for (int c = t; c < SC * 4; c += kSkThreads) {
        const int col = c >> 2, k4 = (c & 3) * 4, gk = k0 + k4;
        int nv = K - gk;
        nv = col < S ? (nv < 0 ? 0 : nv > 4 ? 4 : nv) : 0;
        const float* src = nv > 0 ? d.B + (long long)gk + (long long)col * d.ldb : d.B;
        sk_cp16(st + (uint32_t)(kSkK * LDA_S + col * LDB_S + k4) * 4u, src, 4 * nv);
      }
    }
    sk_commit();
  };
  float acc[8][RC];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < RC; ++j) acc[i][j] = 0.f;
#pragma unroll
  for (int s0 = 0; s0 < kSkStages - 1; ++s0) issue(s0);
  for (int kt = 0; kt < nkt; ++kt) {
    sk_wait<kSkStages - 2>();  // this thread's copies of k-tile kt have landed
    __syncthreads();           // everyone's have; the stage of k-tile kt - 1 is free
    issue(kt + kSkStages - 1);
    const float* As = skm + (kt % kSkStages) * STAGE;
    const float* Bs = As + kSkK * LDA_S;
#pragma unroll
    for (int kk = 0; kk < kSkK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(As + kk * LDA_S + 8 * tl);
      const float4 a1 = *reinterpret_cast<const float4*>(As + kk * LDA_S + 8 * tl + 4);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float bv[RC];
#pragma unroll
      for (int j = 0; j < RC; ++j) bv[j] = Bs[(tc * RC + j) * LDB_S + kk];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < RC; ++j) acc[i][j] = fmaf(a[i], bv[j], acc[i][j]);
    }
  }
  sk_wait<0>();
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gl = l0 + 8 * tl + i;
    if (gl >= L) break;
    float cv[RC];
#pragma unroll
    for (int j = 0; j < RC; ++j) {
      const int c = tc * RC + j;
      cv[j] = (beta != 0.f && c < S) ? d.C[(long long)gl + (long long)c * d.ldc] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < RC; ++j) {
      const int c = tc * RC + j;
      if (c < S) d.C[(long long)gl + (long long)c * d.ldc] = alpha * acc[i][j] + beta * cv[j];
    }
  }
}

template <int SC>
static fde_status launch_skinny_pipe(const GemmBatch<float>& b, cudaStream_t st) {
  const size_t smem = (size_t)kSkStages * sk_stage_floats<SC>() * sizeof(float);
  static const cudaError_t attr =
      cudaFuncSetAttribute(gemm_skinny_pipe_kernel<SC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  FDE_CUDA(attr);
  for (int z0 = 0; z0 < b.batch; z0 += 65535) {
    const int nz = b.batch - z0 < 65535 ? b.batch - z0 : 65535;
    const dim3 grid(ceil_div(b.max_m, kSkL), nz);
    gemm_skinny_pipe_kernel<SC><<<grid, kSkThreads, smem, st>>>(b.d_desc + z0, b.alpha, b.beta);
  }
  return FDE_OK;
}

template <int SC>
static void launch_skinny(const GemmBatch<float>& b, bool transposed, bool a_lcont, bool b_kcont, int L,
                          cudaStream_t st) {
  for (int z0 = 0; z0 < b.batch; z0 += 65535) {
    const int nz = b.batch - z0 < 65535 ? b.batch - z0 : 65535;
    const dim3 grid(ceil_div(L, kSkL), nz);
    const GemmDesc<float>* d = b.d_desc + z0;
    if (a_lcont && b_kcont)
      gemm_skinny_kernel<SC, true, true><<<grid, kSkThreads, 0, st>>>(d, transposed, b.ta, b.tb, b.alpha, b.beta);
    else if (a_lcont)
      gemm_skinny_kernel<SC, true, false><<<grid, kSkThreads, 0, st>>>(d, transposed, b.ta, b.tb, b.alpha, b.beta);
    else if (b_kcont)
      gemm_skinny_kernel<SC, false, true><<<grid, kSkThreads, 0, st>>>(d, transposed, b.ta, b.tb, b.alpha, b.beta);
    else
      gemm_skinny_kernel<SC, false, false><<<grid, kSkThreads, 0, st>>>(d, transposed, b.ta, b.tb, b.alpha, b.beta);
  }
}

// Runs an FP32 batch on a skinny kernel if one dimension is small enough:
// n <= 40 with m >= 128, or m <= 64 with n >= 128 (no two-level k panels).
// With A m-contiguous and B k-contiguous, aligned, the pipelined kernel takes
// any n <= 40; otherwise the register-prefetch kernel takes n <= limit_n (32 in
// the library's own dispatch: the n = 34 root-level rational application
// streams a 1 GB operand from HBM, which one-tile register prefetch does not
// hide, 16 against 28 TFLOP/s on the tensor cores).
static fde_status skinny_gemm_run(const GemmBatch<float>& b, int limit_n, cudaStream_t st, bool* used) {
  *used = false;
  if (b.any_kblk) return FDE_OK;
  bool transposed;
  int S, L;
  if (b.max_n <= 40 && b.max_m >= kSkL) {
    transposed = false;
    S = b.max_n;
    L = b.max_m;
  } else if (b.max_m <= 64 && b.max_n >= kSkL) {
    transposed = true;
    S = b.max_m;
    L = b.max_n;
  } else {
    return FDE_OK;
  }
  // which index of A' and B' is contiguous (see the kernel's view)
  const bool a_lcont = transposed ? b.tb : !b.ta;
  const bool b_kcont = transposed ? b.ta : !b.tb;
  ProfScope ps("gemm32", st, b.flops, 1);
  if (!transposed && !b.ta && !b.tb && b.vec_a && b.vec_b && S <= 40) {
    if (S <= 16)
      FDE_TRY(launch_skinny_pipe<16>(b, st));
    else if (S <= 32)
      FDE_TRY(launch_skinny_pipe<32>(b, st));
    else
      FDE_TRY(launch_skinny_pipe<40>(b, st));
    FDE_LAUNCH("gemm_skinny_pipe_kernel");
    *used = true;
    return FDE_OK;
  }
  if (S > limit_n && !transposed) return FDE_OK;  // (the pipelined kernel only, above)
  if (S <= 16)
    launch_skinny<16>(b, transposed, a_lcont, b_kcont, L, st);
  else if (S <= 32)
    launch_skinny<32>(b, transposed, a_lcont, b_kcont, L, st);
  else if (S <= 48)
    launch_skinny<48>(b, transposed, a_lcont, b_kcont, L, st);
  else
    launch_skinny<64>(b, transposed, a_lcont, b_kcont, L, st);
  FDE_LAUNCH("gemm_skinny_kernel");
  *used = true;
  return FDE_OK;
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
    b.any_kblk = b.any_kblk || d.kblk > 0;
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
    // batches with packed operands go to the tensor cores when they are eligible
    if (skinny_mode() && !b.pk_a && !b.pk_b) {
      const int limit_n = g_skinny_force.load() == 1 ? 40 : 32;
      FDE_TRY(skinny_gemm_run(reinterpret_cast<const GemmBatch<float>&>(b), limit_n, st, &used));
      if (used) return FDE_OK;
    }
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
