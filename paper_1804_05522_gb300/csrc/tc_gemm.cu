// Batched FP32 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
//   C = alpha op(A) op(B) + beta C      (column-major, per-batch descriptors)
//
// Tile 128 x 128 x 32.  Operand tiles are staged in shared memory in the
// canonical K-major layout with 128-byte swizzle (8-row x 128-byte atoms,
// 1024 bytes apart), double buffered; one elected thread issues
// tcgen05.mma.kind::tf32 (M=128, N=128, K=8 per instruction) accumulating in
// tensor memory; completion of each stage is signalled by tcgen05.commit on an
// mbarrier.  The epilogue reads the accumulator with tcgen05.ld (one warp per
// 32-lane quarter) and writes C with coalesced stores.
// Precision: mode 1 = TF32 inputs (inputs rounded to TF32), mode 3 = 3xTF32
// split (a = a_hi + a_lo, products hi*hi + hi*lo + lo*hi) which keeps FP32-level
// accuracy.  Accumulation is FP32.
#include <stdint.h>

#include "dense.cuh"

namespace fde {

namespace tc {

// Raised by a kernel whose bounded mbarrier wait ran out (read by the host).
__device__ int g_wait_timeout;

constexpr int BM = 128, BN = 128, BK = 32;
constexpr int TILE_BYTES = BM * BK * 4;  // 16 KB (A or B tile, TF32)
constexpr uint32_t kSpinLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ uint32_t mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok;
}
// bounded wait: returns false (and raises the timeout flag) if the phase never completes
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < kSpinLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(&g_wait_timeout, 1);
  return false;
}
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 32 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,"
      "%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1u << 46;             // version
  d |= (uint64_t)2u << 61;             // SWIZZLE_128B
  return d;
}
// Instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = 128.
__host__ __device__ constexpr uint32_t idesc_tf32() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// round to TF32 (nearest, ties away) and the remainder
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of element (row r, k c) inside a 128 x 32 K-major SW128 tile.
__device__ __forceinline__ uint32_t sw_off(int r, int c) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((c >> 2) ^ (r & 7)) & 7) << 4) + ((c & 3) << 2));
}

// Load a 128 (rows) x 32 (k) tile of op(X) into hi (and lo) tiles.
// kcontig: element (row, k) sits at X[k_off(k) + row*ld] (k contiguous);
// else at X[row + k_off(k)] with k_off(k) = column address of k (two-level).
template <bool KCONTIG>
__device__ __forceinline__ void load_tile(const float* __restrict__ X, int ld, int kblk, long long kstr, int row0,
                                          int nrows, int k0, int K, uint8_t* hi, uint8_t* lo, bool split) {
  const int tid = threadIdx.x;  // 128 threads: one row each
  const int r = tid;
  const int grow = row0 + r;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + 4 * j + q;
      float x = 0.f;
      if (grow < nrows && k < K) {
        if (KCONTIG) {
          x = X[(size_t)k + (size_t)grow * ld];
        } else {
          const long long col = kblk ? (long long)(k / kblk) * kstr + (long long)(k % kblk) * ld : (long long)k * ld;
          x = X[(long long)grow + col];
        }
      }
      v[q] = x;
    }
    float4 h, l;
    h.x = to_tf32(v[0]);
    h.y = to_tf32(v[1]);
    h.z = to_tf32(v[2]);
    h.w = to_tf32(v[3]);
    const uint32_t off = sw_off(r, 4 * j);
    *reinterpret_cast<float4*>(hi + off) = h;
    if (split) {
      l.x = to_tf32(v[0] - h.x);
      l.y = to_tf32(v[1] - h.y);
      l.z = to_tf32(v[2] - h.z);
      l.w = to_tf32(v[3] - h.w);
      *reinterpret_cast<float4*>(lo + off) = l;
    }
  }
}

// 128 threads per CTA; grid (ceil(m/128), ceil(n/128), batch).
template <bool TA, bool TB>
__global__ void __launch_bounds__(128) tc_gemm_kernel(const GemmDesc<float>* __restrict__ descs, float alpha, float beta,
                                                      int split) {
  const GemmDesc<float> d = descs[blockIdx.z];
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if (m0 >= d.m || n0 >= d.n) return;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t base_u32 = smem_u32(smem_raw);
  const uint32_t pad = ((base_u32 + 1023u) & ~1023u) - base_u32;
  uint8_t* sm = smem_raw + pad;  // 1024-byte aligned
  const int ntile = split ? 4 : 2;  // A_hi, B_hi (, A_lo, B_lo) per stage
  uint8_t* stage[2] = {sm, sm + ntile * TILE_BYTES};
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bars[0]), 1);
    mbar_init(smem_u32(&bars[1]), 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(&tmem_base), BN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const int nk = (d.k + BK - 1) / BK;
  bool ok = true;
  for (int kt = 0; kt < nk; ++kt) {
    const int b = kt & 1;
    if (kt >= 2) ok = ok && mbar_wait(smem_u32(&bars[b]), (uint32_t)(((kt - 2) >> 1) & 1));
    uint8_t* st = stage[b];
    const int k0 = kt * BK;
    // A: rows = m (op(A) is m x k); B: rows = n (op(B)ᵀ is n x k)
    load_tile<TA>(d.A, d.lda, TA ? 0 : d.kblk, d.kstr, m0, d.m, k0, d.k, st, st + 2 * TILE_BYTES, split);
    load_tile<!TB>(d.B, d.ldb, TB ? d.kblk : 0, d.kstr, n0, d.n, k0, d.k, st + TILE_BYTES, st + 3 * TILE_BYTES, split);
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t a_hi = smem_u32(st), b_hi = smem_u32(st + TILE_BYTES);
      const uint32_t a_lo = smem_u32(st + 2 * TILE_BYTES), b_lo = smem_u32(st + 3 * TILE_BYTES);
#pragma unroll
      for (int kk = 0; kk < BK / 8; ++kk) {
        const uint32_t off = kk * 32;  // 8 TF32 = 32 bytes along k inside the swizzle atom
        const uint32_t acc0 = (kt > 0 || kk > 0) ? 1u : 0u;
        mma_tf32(tmem, sw128_desc(a_hi + off), sw128_desc(b_hi + off), idesc_tf32(), acc0);
        if (split) {
          mma_tf32(tmem, sw128_desc(a_hi + off), sw128_desc(b_lo + off), idesc_tf32(), 1u);
          mma_tf32(tmem, sw128_desc(a_lo + off), sw128_desc(b_hi + off), idesc_tf32(), 1u);
        }
      }
      mma_commit(smem_u32(&bars[b]));
    }
  }
  // wait for the last stage (its commit covers all earlier MMAs)
  if (nk > 0) ok = ok && mbar_wait(smem_u32(&bars[(nk - 1) & 1]), (uint32_t)(((nk - 1) >> 1) & 1));
  tc_fence_after();
  const bool all_ok = __syncthreads_and(ok ? 1 : 0) != 0;
  if (all_ok && nk > 0) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t tw = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      float v[32];
      tmem_ld32(tw + c0, v);
      if (row < d.m) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = n0 + c0 + j;
          if (col < d.n) {
            float* c = d.C + row + (size_t)col * d.ldc;
            *c = (beta == 0.f) ? alpha * v[j] : alpha * v[j] + beta * (*c);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, BN);
}

}  // namespace tc

static int g_tc_mode = -1;  // -1: not read yet; 0 off; 1 tf32; 3 3xtf32

int tc_mode() {
  if (g_tc_mode < 0) {
    const char* e = getenv("FDE_TC");
    g_tc_mode = e ? atoi(e) : 3;
    if (g_tc_mode != 0 && g_tc_mode != 1 && g_tc_mode != 3) g_tc_mode = 3;
  }
  return g_tc_mode;
}
void set_tc_mode(int m) { g_tc_mode = m; }

fde_status tc_error_flag(int* out) {
  *out = 0;
  FDE_CUDA(cudaMemcpyFromSymbol(out, tc::g_wait_timeout, sizeof(int)));
  return FDE_OK;
}

// Kernel attributes are set once, before any stream capture.
fde_status tc_prepare() {
  static bool done = false;
  if (done) return FDE_OK;
  const int smax = 1024 + 8 * tc::TILE_BYTES;
  FDE_CUDA(cudaFuncSetAttribute(tc::tc_gemm_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
  FDE_CUDA(cudaFuncSetAttribute(tc::tc_gemm_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
  FDE_CUDA(cudaFuncSetAttribute(tc::tc_gemm_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
  FDE_CUDA(cudaFuncSetAttribute(tc::tc_gemm_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
  done = true;
  return FDE_OK;
}

// Runs the batch on the tensor cores; returns FDE_OK without launching if the
// batch is better left to the SIMT kernel (*used = false).
fde_status tc_gemm_run(const GemmBatch<float>& b, cudaStream_t st, bool* used) {
  *used = false;
  const int mode = tc_mode();
  if (mode == 0 || b.max_m < 64 || b.max_n < 32 || b.max_k < 32) return FDE_OK;
  FDE_TRY(tc_prepare());
  const int split = (mode == 3) ? 1 : 0;
  const size_t smem = 1024 + 2 * (size_t)(split ? 4 : 2) * tc::TILE_BYTES;
  const int which = (b.ta ? 2 : 0) + (b.tb ? 1 : 0);
  auto kern = (which == 0) ? tc::tc_gemm_kernel<false, false>
              : (which == 1) ? tc::tc_gemm_kernel<false, true>
              : (which == 2) ? tc::tc_gemm_kernel<true, false>
                             : tc::tc_gemm_kernel<true, true>;
  for (int z0 = 0; z0 < b.batch; z0 += 65535) {
    const int nz = b.batch - z0 < 65535 ? b.batch - z0 : 65535;
    dim3 grid(ceil_div(b.max_m, tc::BM), ceil_div(b.max_n, tc::BN), nz);
    ProfScope ps("gemm32tc", st, z0 == 0 ? b.flops : 0.0, 1);
    kern<<<grid, 128, smem, st>>>(b.d_desc + z0, b.alpha, b.beta, split);
    FDE_LAUNCH("tc_gemm_kernel");
  }
  *used = true;
  return FDE_OK;
}

}  // namespace fde
