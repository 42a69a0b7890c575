// Batched FP32 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
//   C = alpha op(A) op(B) + beta C      (column-major, per-batch descriptors)
//
// Tile 128 x BN x 32 (BN = 32, 64 or 128), persistent CTAs (one per SM).  Operand tiles are staged in shared
// memory in the canonical K-major layout with 128-byte swizzle (8-row x
// 128-byte atoms, 1024 bytes apart) in a ring of slots filled by eight loader
// warps; one elected thread issues tcgen05.mma.kind::tf32 (M = 128, N = BN,
// K = 8 per instruction) accumulating in tensor memory, and tcgen05.commit on
// per-slot mbarriers hands each slot back to the loaders.  The epilogue reads
// the accumulator with tcgen05.ld and writes C with coalesced stores.
// Precision: mode 1 = TF32 inputs (inputs rounded to TF32), mode 3 = 3xTF32
// split (a = a_hi + a_lo, products hi*hi + hi*lo + lo*hi) which keeps FP32-level
// accuracy.  Per batch, the operands may instead be BF16 (kind::f16, K = 16
// per instruction): rounded to BF16 (one product), or split into BF16 hi and
// lo (three products, about 16 significant bits).  A BF16 tile uses the same
// slot geometry as a TF32 one: each 128-byte row holds the tile's 32 k as 16
// pairs in its first 64 logical bytes.  Accumulation is FP32.
#include <stdint.h>

#include <cuda_bf16.h>

#include <atomic>
#include <mutex>

#include "dense.cuh"

namespace fde {

namespace tc {

// Counts the bounded mbarrier waits that ran out (read by the host; it only
// grows, so a caller compares it with the value it saw before its launches).
__device__ unsigned int g_wait_timeout;
// Iteration limit of the pipeline's bounded waits (host-settable so that tests
// can make them run out; kSpinLimit by default).
constexpr uint32_t kSpinLimit = 1u << 26;
__device__ uint32_t g_spin_limit = kSpinLimit;

constexpr int BM = 128, BK = 32;

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
  atomicAdd(&g_wait_timeout, 1u);
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
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// Two FP32 values as a BF16 pair (round to nearest even), e0 in the low half,
// and the pair of their exact FP32 remainders rounded to BF16 in *lo.
__device__ __forceinline__ uint32_t bf16_pair(float e0, float e1, uint32_t* lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(e0, e1);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(e0 - hf.x, e1 - hf.y);
  *lo = *reinterpret_cast<const uint32_t*>(&l);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
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
// The same with 64-byte swizzle: K-major, 64-byte rows, 8-row groups 512 bytes
// apart (dense BF16 tiles: 32 k per row).
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512u >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1u << 46;             // version
  d |= (uint64_t)4u << 61;             // SWIZZLE_64B
  return d;
}
// Byte offset of 4-byte unit u (0..15) of row r in a K-major SW64 tile (rows in
// 8-row groups of 512 bytes, 16-byte chunks XOR-swizzled by (r / 2) mod 4).
__host__ __device__ __forceinline__ uint32_t sw64_off(int r, int u) {
  return (uint32_t)((r >> 3) * 512 + (r & 7) * 64 + ((((u >> 2) ^ (r >> 1)) & 3) << 4) + ((u & 3) << 2));
}
// round to TF32 (nearest, ties away)
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of element (row r, k c) inside a K-major SW128 tile (rows in
// 8-row groups of 1024 bytes, 32 FP32 k per 128-byte row, 16-byte chunks
// XOR-swizzled by the row within the group).
__device__ __forceinline__ uint32_t sw_off(int r, int c) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((c >> 2) ^ (r & 7)) & 7) << 4) + ((c & 3) << 2));
}
// Byte offset of 16-byte chunk c (rows 4c..4c+3) of k row kl in a raw
// row-contiguous stage of R rows: R / 4 chunks per k row, the chunk column
// XOR-ed with kl / 4 (mod 8) so that 8 different k quads of one chunk column
// fall in 8 different bank groups (R / 4 is a multiple of 8).
template <int R>
__device__ __forceinline__ uint32_t mn_raw_off(int kl, int c) {
  return (uint32_t)((kl * (R / 4) + (c ^ ((kl >> 2) & 7))) << 4);
}


constexpr int kLoaders = 256;              // 8 warps: global -> shared, then the epilogue
constexpr int kMaxSlots = 8;               // MMA slots (TF32 hi / lo tiles)

__device__ __forceinline__ void cp_async4(uint32_t dst, const float* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Adds tx bytes that the current phase of an mbarrier must also see land.
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bulk asynchronous copy global -> shared of `bytes` (multiple of 16, both
// addresses 16-byte aligned) whose completion counts as tx bytes on `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const float* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}

// Asynchronous copy of an R x 32 tile of op(X) (element (row, k): X[k + row*ld]
// when KCONTIG, else X[row + col(k)], col(k) = k*ld or the two-level panel
// address) into a raw stage at dst; out-of-range elements are zero-filled.
// Every loader thread copies exactly the 16-byte chunks that it converts
// afterwards (tile_convert / tile_convert_mn), so it only waits for its own
// copies and never for the other loaders.
//  - row-contiguous X: the raw stage holds per k a row of R values in 16-byte
//    chunks, chunk c of k row kl at column c ^ (kl / 4 mod 8) (mn_raw_off);
//    thread block b = (kg = b mod 8, mg = b / 8) owns rows 4mg..4mg+3 x k
//    4kg..4kg+3, four 16-byte copies (64 contiguous bytes per 4 lanes).
//  - k-contiguous X: the raw stage already has the swizzled K-major layout of
//    the MMA operand; chunk ch = (row ch / 8, k quad ch % 8), 8 lanes copy one
//    row's 128 bytes.
template <int R, bool KCONTIG>
__device__ __forceinline__ void tile_copy(uint32_t dst, const float* __restrict__ X, int ld, int kblk, long long kstr,
                                          unsigned long long kmagic, int kshift, int row0, int nrows, int k0, int K,
                                          bool vec) {
  if (!KCONTIG) {
    constexpr int NB = (R / 4) * 8;  // 4 x 4 blocks of the tile
#pragma unroll
    for (int i = 0; i < (NB + kLoaders - 1) / kLoaders; ++i) {
      const int b = threadIdx.x + kLoaders * i;
      if (b >= NB) break;
      const int kg = b & 7, mg = b >> 3;
      const int grow = row0 + 4 * mg;
      int nrow = nrows - grow;
      nrow = nrow < 0 ? 0 : nrow > 4 ? 4 : nrow;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const int kl = 4 * kg + kk, kabs = k0 + kl;
        const uint32_t o = dst + mn_raw_off<R>(kl, mg);
        const int nvalid = kabs < K ? nrow : 0;
        long long col = 0;
        if (nvalid > 0) {
          if (kblk) {
            const int q = (int)(((unsigned long long)kabs * kmagic) >> kshift);
            col = (long long)q * kstr + (long long)(kabs - q * kblk) * ld;
          } else {
            col = (long long)kabs * ld;
          }
        }
        const float* p = X + col + grow;
        if (vec) {
          cp_async16_zfill(o, nvalid > 0 ? p : X, 4 * nvalid);
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c) cp_async4(o + 4 * c, c < nvalid ? p + c : X, c < nvalid);
        }
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < R / 32; ++i) {
      const int ch = threadIdx.x + kLoaders * i, r = ch >> 3, kq = ch & 7;
      const int grow = row0 + r, kk = k0 + 4 * kq;
      const float* p = X + (size_t)grow * ld + kk;
      const uint32_t o = dst + sw_off(r, 4 * kq);
      if (vec && grow < nrows && kk + 3 < K) {
        cp_async16(o, p);
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const bool ok = grow < nrows && kk + c < K;
          cp_async4(o + 4 * c, ok ? p + c : X, ok);
        }
      }
    }
  }
}

// Raw FP32 tile -> TF32 hi (and the remainder lo in split mode),
// same swizzled offsets; thread t converts 16-byte chunks t, t + 256, ...
// (the chunks tile_copy<R, true> gave it)
// BF16 operands (bf): the four k of the chunk become two pairs (8 bytes) at
// pair positions 2 kq, 2 kq + 1 of the row, i.e. logical bytes 8 kq .. 8 kq + 7.
template <int R>
__device__ __forceinline__ void tile_convert(const uint8_t* raw, uint8_t* hi, uint8_t* lo, bool split, bool bf) {
#pragma unroll
  for (int i = 0; i < R / 32; ++i) {
    const int ch = threadIdx.x + kLoaders * i, r = ch >> 3, kq = ch & 7;
    const uint32_t off = sw_off(r, 4 * kq);
    const float4 v = *reinterpret_cast<const float4*>(raw + off);
    if (bf) {
      const uint32_t o2 = sw_off(r, 2 * kq);
      uint2 hv, lv;
      hv.x = bf16_pair(v.x, v.y, &lv.x);
      hv.y = bf16_pair(v.z, v.w, &lv.y);
      *reinterpret_cast<uint2*>(hi + o2) = hv;
      if (split) *reinterpret_cast<uint2*>(lo + o2) = lv;
      continue;
    }
    float4 h;
    h.x = to_tf32(v.x);
    h.y = to_tf32(v.y);
    h.z = to_tf32(v.z);
    h.w = to_tf32(v.w);
    *reinterpret_cast<float4*>(hi + off) = h;
    if (split) {
      // the remainder is exact in FP32; the MMA reads its top 19 bits
      // (truncation to TF32), which leaves an error below 2^-21 |v|
      float4 l;
      l.x = v.x - h.x;
      l.y = v.y - h.y;
      l.z = v.z - h.z;
      l.w = v.w - h.w;
      *reinterpret_cast<float4*>(lo + off) = l;
    }
  }
}

// Row-contiguous raw stage (mn_raw_off) -> swizzled K-major TF32 hi (and lo).
// Thread block (kg = b mod 8, mg = b / 8): rows 4mg..4mg+3 x k 4kg..4kg+3,
// read as four 16-byte row segments and transposed in registers.  The 8
// lanes of a quarter warp share mg and take kg = 0..7: their reads hit
// chunk columns mg ^ kg and their stores the swizzled chunks kg ^ (row mod 8),
// 8 distinct bank groups either way, in a fixed order.
template <int R>
__device__ __forceinline__ void tile_convert_mn(const uint8_t* raw, uint8_t* hi, uint8_t* lo, bool split, bool bf) {
  constexpr int NB = (R / 4) * 8;
#pragma unroll
  for (int i = 0; i < (NB + kLoaders - 1) / kLoaders; ++i) {
    const int b = threadIdx.x + kLoaders * i;
    if (b >= NB) break;
    const int kg = b & 7, mg = b >> 3;
    float4 q[4];  // q[kk] = rows 4mg..4mg+3 at k = 4kg + kk
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) q[kk] = *reinterpret_cast<const float4*>(raw + mn_raw_off<R>(4 * kg + kk, mg));
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const uint32_t off = sw_off(4 * mg + rr, 4 * kg);
      float4 x, h;
      x.x = rr == 0 ? q[0].x : rr == 1 ? q[0].y : rr == 2 ? q[0].z : q[0].w;
      x.y = rr == 0 ? q[1].x : rr == 1 ? q[1].y : rr == 2 ? q[1].z : q[1].w;
      x.z = rr == 0 ? q[2].x : rr == 1 ? q[2].y : rr == 2 ? q[2].z : q[2].w;
      x.w = rr == 0 ? q[3].x : rr == 1 ? q[3].y : rr == 2 ? q[3].z : q[3].w;
      if (bf) {
        const uint32_t o2 = sw_off(4 * mg + rr, 2 * kg);
        uint2 hv, lv;
        hv.x = bf16_pair(x.x, x.y, &lv.x);
        hv.y = bf16_pair(x.z, x.w, &lv.y);
        *reinterpret_cast<uint2*>(hi + o2) = hv;
        if (split) *reinterpret_cast<uint2*>(lo + o2) = lv;
        continue;
      }
      h.x = to_tf32(x.x);
      h.y = to_tf32(x.y);
      h.z = to_tf32(x.z);
      h.w = to_tf32(x.w);
      *reinterpret_cast<float4*>(hi + off) = h;
      if (split) {
        float4 l;  // exact remainder, truncated to TF32 by the MMA (see tile_convert)
        l.x = x.x - h.x;
        l.y = x.y - h.y;
        l.z = x.z - h.z;
        l.w = x.w - h.w;
        *reinterpret_cast<float4*>(lo + off) = l;
      }
    }
  }
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = BN.
template <int BN>
__host__ __device__ constexpr uint32_t idesc_tf32_n() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// Instruction descriptor for kind::f16: D = F32, A = B = BF16, both K-major,
// M = 128, N = BN.
template <int BN>
__host__ __device__ constexpr uint32_t idesc_bf16_n() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int BN>
__host__ __device__ constexpr int raw_bytes() {
  return (BM + BN) * BK * 4;
}

// 32 consecutive accumulator columns of this thread's lane, without waiting
// (tcgen05.wait::ld before the registers are used)
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,"
      "%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// bounded wait that gives up at once when another role has already failed
__device__ __forceinline__ bool mbar_wait_f(uint32_t bar, uint32_t parity, volatile int* fail) {
  const uint32_t limit = g_spin_limit;
  for (uint32_t it = 0; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && *fail) return false;
  }
  atomicAdd(&g_wait_timeout, 1u);
  *fail = 1;
  return false;
}

// A position in the stream of k-tiles of one CTA: tile t (flattened index),
// k-tile kt of its nk, the tile's problem d and origin (m0, n0).
struct KStream {
  int t, kt, nk, m0, n0;
  GemmDesc<float> d;
};
// Moves s to the first tile at or after s.t (stepping by gridDim.x) that has
// work (inside its problem, k > 0), at k-tile 0; false at the end.
template <int BN>
__device__ __forceinline__ bool next_tile(KStream& s, const GemmDesc<float>* __restrict__ descs, int tiles, int mt,
                                          int nt) {
  for (; s.t < tiles; s.t += gridDim.x) {
    const int z = s.t / (mt * nt), rem = s.t - z * (mt * nt), ni = rem / mt, mi = rem - ni * mt;
    s.d = descs[z];
    s.m0 = mi * BM;
    s.n0 = ni * BN;
    if (s.m0 >= s.d.m || s.n0 >= s.d.n || s.d.k <= 0) continue;
    s.nk = (s.d.k + BK - 1) / BK;
    s.kt = 0;
    return true;
  }
  return false;
}

// The same walk for the conversion side, which needs only the tile and its
// k-tile count (m, n, k of the problem are read, not the whole descriptor).
struct KPos {
  int t, kt, nk;
};
template <int BN>
__device__ __forceinline__ bool next_pos(KPos& s, const GemmDesc<float>* __restrict__ descs, int tiles, int mt,
                                         int nt) {
  for (; s.t < tiles; s.t += gridDim.x) {
    const int z = s.t / (mt * nt), rem = s.t - z * (mt * nt), ni = rem / mt, mi = rem - ni * mt;
    const int m = descs[z].m, n = descs[z].n, k = descs[z].k;
    if (mi * BM >= m || ni * BN >= n || k <= 0) continue;
    s.nk = (k + BK - 1) / BK;
    s.kt = 0;
    return true;
  }
  return false;
}

constexpr int kEpiWarps = 4;                                   // one per TMEM lane quarter
constexpr int kPThreads = kLoaders + 32 * kEpiWarps + 32;      // loaders, epilogue, MMA
constexpr int kEpiWarp0 = kLoaders / 32;                       // warps 8..11
constexpr int kMmaWarp = kEpiWarp0 + kEpiWarps;                // warp 12

// Persistent warp-specialised batched GEMM: one CTA per SM walks the tiles
// t = blockIdx.x, blockIdx.x + gridDim.x, ... of the flattened
// (batch, n tile, m tile) space (m fastest, so neighbouring CTAs share B).
//  - Warps 0-7 (loaders) copy the op(A) (128 x 32) and op(B) (BN x 32) tiles
//    with cp.async into a ring of RAW raw FP32 stages, RAW k-tiles ahead of
//    the k-tile g they convert (g counts k-tiles over all tiles of the CTA);
//    each thread waits for its own copies of g, rounds them to TF32 (hi, and
//    lo = remainder in split mode) into MMA slot g % mslots once the slot's
//    `empty` barrier says its MMAs are done, and arrives on its `full` barrier.
//  - Warp 12 waits on `full`, issues the tcgen05 MMAs of the slot (one
//    elected thread) into accumulator buffer b = (tile count) & 1 in TMEM and
//    commits them to `empty`; after the last k-tile it commits to tfull[b].
//  - Warps 8-11 (epilogue) wait on tfull[b], read buffer b (warp = lane
//    quarter), release it on tempty[b] and write C; meanwhile the MMAs of the
//    next tile fill the other buffer.
// Every mbarrier wait is bounded; after a failure the roles skip their work
// but keep the loop structure (no barrier is left waiting) and count the
// expiry in g_wait_timeout.  Before the TMEM is freed the issuing thread
// commits once more to a drain barrier and waits for it (bounded by the fixed
// kSpinLimit), so that no MMA it launched is still writing the accumulators.
// Registers: the 13 warps sit 4/3/3/3 on the four SM sub-partitions, whose
// register files hold 16K each, so a thread gets at most 128.
template <int BN, int RAW, bool TA, bool TB>
__global__ void __launch_bounds__(kPThreads, 1)
    tc_gemm_kernel(const GemmDesc<float>* __restrict__ descs, int batch, int mt, int nt, float alpha, float beta,
                   int split, int mslots, int vec_a, int vec_b, int pk_a, int pk_b, int bf) {
  constexpr int A_BYTES = BM * BK * 4, B_BYTES = BN * BK * 4;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t base_u32 = smem_u32(smem_raw);
  const uint32_t pad = ((base_u32 + 1023u) & ~1023u) - base_u32;
  uint8_t* sm = smem_raw + pad;  // 1024-byte aligned
  // MMA slot: A_hi | A_lo | B_hi | B_lo (lo only in split mode), so that a
  // packed operand's hi and lo tiles arrive in one bulk copy; raw stages after the slots
  const int slot_bytes = (A_BYTES + B_BYTES) * (split ? 2 : 1);
  const int a_lo_off = A_BYTES, b_hi_off = split ? 2 * A_BYTES : A_BYTES, b_lo_off = b_hi_off + B_BYTES;
  // packed BF16 operands arrive dense (64-byte rows, SW64; hi then lo), half
  // the bytes of a TF32 or converted BF16 tile
  const bool dense_a = bf && pk_a, dense_b = bf && pk_b;
  const uint32_t a_copy = (uint32_t)(dense_a ? BM * 64 : A_BYTES) * (split ? 2u : 1u);
  const uint32_t b_copy = (uint32_t)(dense_b ? BN * 64 : B_BYTES) * (split ? 2u : 1u);
  uint8_t* raw = sm + (size_t)mslots * slot_bytes;
  __shared__ __align__(8) uint64_t full_bar[kMaxSlots], empty_bar[kMaxSlots], tfull[2], tempty[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  volatile int* fail = &s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < mslots; ++s) {
      mbar_init(smem_u32(&full_bar[s]), kLoaders / 32);  // one arrival per loader warp
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&tfull[b]), 1);
      mbar_init(smem_u32(&tempty[b]), kEpiWarps);
    }
    mbar_init(smem_u32(&drain), 1);
    s_fail = 0;
    fence_barrier_init();
  }
  // per buffer: columns [0, BN) hi*hi; in split mode [BN, 2BN) the hi*lo +
  // lo*hi corrections (summed into the hi*hi accumulator they would lose
  // their low bits to its alignment)
  const uint32_t tcols = split ? 2 * BN : BN;
  if (warp == kMmaWarp) {
    tmem_alloc(smem_u32(&tmem_base), 2 * tcols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const int tiles = batch * mt * nt;

  if (warp < kLoaders / 32) {
    // ---------------- loaders
    // The k-tiles of all tiles of this CTA form one stream; the copies run
    // RAW positions ahead of the conversion, across tile boundaries, so a
    // tile with few k-tiles does not pay the memory latency in a prologue.
    // Position p uses raw stage p % RAW and MMA slot p % mslots.
    KStream is;  // the next position to copy
    KPos cv;     // the position being converted
    cv.t = is.t = blockIdx.x;
    bool is_ok = next_tile<BN>(is, descs, tiles, mt, nt);
    bool cv_ok = next_pos<BN>(cv, descs, tiles, mt, nt);
    int p_issue = 0;
    auto issue = [&]() {
      // copies of position p_issue (an empty group past the end of the stream)
      if (is_ok) {
        const uint32_t dst = smem_u32(raw + (size_t)(p_issue % RAW) * raw_bytes<BN>());
        const GemmDesc<float>& d = is.d;
        const int a_kblk = TA ? 0 : d.kblk, b_kblk = TB ? d.kblk : 0;
        if (!pk_a)
          tile_copy<BM, TA>(dst, d.A, d.lda, a_kblk, d.kstr, d.kmagic, d.kshift, is.m0, d.m, is.kt * BK, d.k,
                            vec_a != 0);
        if (!pk_b)
          tile_copy<BN, !TB>(dst + A_BYTES, d.B, d.ldb, b_kblk, d.kstr, d.kmagic, d.kshift, is.n0, d.n, is.kt * BK,
                             d.k, vec_b != 0);
        if (++is.kt == is.nk) {
          is.t += gridDim.x;
          is_ok = next_tile<BN>(is, descs, tiles, mt, nt);
        }
      }
      cp_async_commit();
      ++p_issue;
    };
#pragma unroll 1
    for (int i = 0; i < RAW; ++i) issue();
    bool ok = true;
    // last position whose packed tiles were copied into each slot (thread 0)
    int last_bulk[kMaxSlots];
#pragma unroll
    for (int s2 = 0; s2 < kMaxSlots; ++s2) last_bulk[s2] = -1;
    for (int gg = 0; cv_ok; ++gg) {
      cp_async_wait<RAW - 1>();  // this thread's copies of position gg have landed
      const int ms = gg % mslots;
      if (gg >= mslots) {
        // one lane per warp polls the slot's `empty` barrier
        int got = 1;
        if (lane == 0 && ok) got = mbar_wait_f(smem_u32(&empty_bar[ms]), (uint32_t)((gg / mslots - 1) & 1), fail);
        ok = ok && __shfl_sync(0xffffffffu, got, 0) != 0;
      }
      uint8_t* slot = sm + (size_t)ms * slot_bytes;
      if (threadIdx.x == 0 && ok && (pk_a || pk_b)) {
        // packed operands: the slot is free, copy their hi | lo tiles into it;
        // the `full` barrier also waits for these bytes (this warp has not
        // arrived on it yet)
        const int z = cv.t / (mt * nt), rem = cv.t - z * (mt * nt), ni = rem / mt, mi = rem - ni * mt;
        const uint32_t fb = smem_u32(&full_bar[ms]);
        mbar_expect_tx(fb, (pk_a ? a_copy : 0u) + (pk_b ? b_copy : 0u));
        if (pk_a)
          bulk_g2s(smem_u32(slot), descs[z].Apk + ((size_t)mi * cv.nk + cv.kt) * (2 * BM * BK), a_copy, fb);
        if (pk_b)
          bulk_g2s(smem_u32(slot + b_hi_off), descs[z].Bpk + ((size_t)ni * cv.nk + cv.kt) * (2 * BN * BK), b_copy,
                   fb);
        last_bulk[ms] = gg;
      }
      if (ok) {
        const uint8_t* rs = raw + (size_t)(gg % RAW) * raw_bytes<BN>();
        if (!pk_a) {
          if (TA)
            tile_convert<BM>(rs, slot, slot + a_lo_off, split != 0, bf != 0);
          else
            tile_convert_mn<BM>(rs, slot, slot + a_lo_off, split != 0, bf != 0);
        }
        if (!pk_b) {
          if (!TB)
            tile_convert<BN>(rs + A_BYTES, slot + b_hi_off, slot + b_lo_off, split != 0, bf != 0);
          else
            tile_convert_mn<BN>(rs + A_BYTES, slot + b_hi_off, slot + b_lo_off, split != 0, bf != 0);
        }
        fence_proxy_async();  // this thread's tiles -> visible to the tensor core
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&full_bar[ms]));
      // this thread's chunks of raw stage gg % RAW are free again: refill
      issue();
      if (++cv.kt == cv.nk) {
        cv.t += gridDim.x;
        cv_ok = next_pos<BN>(cv, descs, tiles, mt, nt);
      }
    }
    cp_async_wait<0>();
    if (threadIdx.x == 0 && (pk_a || pk_b)) {
      // no bulk copy may still be writing this CTA's shared memory when it
      // exits (after a failed wait the MMA warp may not have consumed them)
      for (int s2 = 0; s2 < mslots; ++s2)
        if (last_bulk[s2] >= 0) mbar_wait(smem_u32(&full_bar[s2]), (uint32_t)((last_bulk[s2] / mslots) & 1));
    }
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int g = 0, lt = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int z = t / (mt * nt), rem = t - z * (mt * nt), ni = rem / mt, mi = rem - ni * mt;
        const GemmDesc<float> d = descs[z];
        if (mi * BM >= d.m || ni * BN >= d.n) continue;
        const int nk = (d.k + BK - 1) / BK;
        const int b = lt & 1, u = lt >> 1;
        const uint32_t acc = tmem + (uint32_t)b * tcols;
        // the epilogue has drained this buffer (its previous use)
        if (ok && u > 0) ok = mbar_wait_f(smem_u32(&tempty[b]), (uint32_t)((u - 1) & 1), fail);
        tc_fence_after();
        for (int kt = 0; kt < nk; ++kt) {
          const int gg = g + kt, s = gg % mslots;
          if (ok) ok = mbar_wait_f(smem_u32(&full_bar[s]), (uint32_t)((gg / mslots) & 1), fail);
          if (!ok) break;
          tc_fence_after();
          uint8_t* slot = sm + (size_t)s * slot_bytes;
          const uint32_t a_hi = smem_u32(slot), b_hi = smem_u32(slot + b_hi_off);
          const uint32_t a_lo = smem_u32(slot + a_lo_off);
          if (bf) {
            // BF16: K = 16 per instruction, 32 bytes along the row; the tile's
            // 32 k are the row's first 64 logical bytes (converted tiles,
            // SW128) or the whole 64-byte row (packed tiles, SW64)
            const uint32_t a_lo_b = dense_a ? a_hi + BM * 64 : a_lo;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint32_t off = kk * 32;
              const uint32_t acc0 = (kt > 0 || kk > 0) ? 1u : 0u;
              const uint64_t dah = dense_a ? sw64_desc(a_hi + off) : sw128_desc(a_hi + off);
              const uint64_t dbh = dense_b ? sw64_desc(b_hi + off) : sw128_desc(b_hi + off);
              if (split) {
                const uint64_t dal = dense_a ? sw64_desc(a_lo_b + off) : sw128_desc(a_lo_b + off);
                mma_bf16(acc, dah, dbh, idesc_bf16_n<2 * BN>(), acc0);
                mma_bf16(acc + BN, dal, dbh, idesc_bf16_n<BN>(), 1u);
              } else {
                mma_bf16(acc, dah, dbh, idesc_bf16_n<BN>(), acc0);
              }
            }
            mma_commit(smem_u32(&empty_bar[s]));
            continue;
          }
#pragma unroll
          for (int kk = 0; kk < BK / 8; ++kk) {
            const uint32_t off = kk * 32;  // 8 TF32 = 32 bytes along k inside the swizzle atom
            const uint32_t acc0 = (kt > 0 || kk > 0) ? 1u : 0u;
            if (split) {
              // B_lo follows B_hi in the slot with the same 8-row swizzle
              // atoms, so [B_hi; B_lo] is one K-major operand of 2 BN rows:
              // one N = 2 BN MMA gives A_hi B_hi in columns [0, BN) and the
              // A_hi B_lo correction in [BN, 2 BN), where A_lo B_hi adds (two
              // instructions per k-step instead of three; an MMA issues in
              // about the same time for N = 64 .. 256)
              mma_tf32(acc, sw128_desc(a_hi + off), sw128_desc(b_hi + off), idesc_tf32_n<2 * BN>(), acc0);
              mma_tf32(acc + BN, sw128_desc(a_lo + off), sw128_desc(b_hi + off), idesc_tf32_n<BN>(), 1u);
            } else {
              mma_tf32(acc, sw128_desc(a_hi + off), sw128_desc(b_hi + off), idesc_tf32_n<BN>(), acc0);
            }
          }
          mma_commit(smem_u32(&empty_bar[s]));
        }
        // completes once every MMA issued so far has finished
        mma_commit(smem_u32(&tfull[b]));
        g += nk;
        ++lt;
      }
      // drain: after a failed wait the epilogue may not have waited for the
      // last tfull, so wait here until every MMA of this thread is done
      mma_commit(smem_u32(&drain));
      mbar_wait(smem_u32(&drain), 0u);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue (warp = TMEM lane quarter)
    const int quarter = warp - kEpiWarp0;  // == warp % 4
    int lt = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
      const int z = t / (mt * nt), rem = t - z * (mt * nt), ni = rem / mt, mi = rem - ni * mt;
      const GemmDesc<float> d = descs[z];
      const int m0 = mi * BM, n0 = ni * BN;
      if (m0 >= d.m || n0 >= d.n) continue;
      const int nk = (d.k + BK - 1) / BK;
      const int b = lt & 1, u = lt >> 1;
      int got = 1;
      if (lane == 0 && ok) got = mbar_wait_f(smem_u32(&tfull[b]), (uint32_t)(u & 1), fail);
      ok = ok && __shfl_sync(0xffffffffu, got, 0) != 0;
      tc_fence_after();
      const int row = m0 + quarter * 32 + lane;
      const uint32_t tw = tmem + (uint32_t)b * tcols + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        if (ok && nk > 0) {
          uint32_t r0[32], r1[32];
          tmem_ld32_nowait(tw + c0, r0);
          if (split) tmem_ld32_nowait(tw + BN + c0, r1);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r0[j]) + (split ? __uint_as_float(r1[j]) : 0.f);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = 0.f;
        }
        // beta C: all 32 loads are issued before any store of this chunk (a
        // store between them would order each load behind it, since the
        // compiler cannot rule out that the columns alias)
        float cv[32];
        const bool rowok = ok && row < d.m;
        // column j of the chunk at cbase[j * ldc]: one 64-bit base, 32-bit offsets
        float* cbase = d.C + (rowok ? row + (size_t)(n0 + c0) * d.ldc : 0);
        const int ncol = d.n - (n0 + c0);
#pragma unroll
        for (int j = 0; j < 32; ++j) cv[j] = (beta != 0.f && rowok && j < ncol) ? cbase[j * d.ldc] : 0.f;
        if (c0 + 32 >= BN) {
          // the last TMEM read of this buffer: hand it back to the MMA warp
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&tempty[b]));
        }
        if (rowok) {
          // the stores recompute their addresses from an opaque copy of the
          // base instead of keeping the 32 load addresses live
          float* sbase;
          asm("mov.b64 %0, %1;" : "=l"(sbase) : "l"(cbase));
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < ncol) sbase[j * d.ldc] = alpha * v[j] + beta * cv[j];
        }
      }
      ++lt;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    __syncwarp();
    tmem_dealloc(tmem, 2 * tcols);
  }
}

template <int BN>
constexpr size_t slot_bytes(int split) {
  return (size_t)(BM * BK * 4 + BN * BK * 4) * (split ? 2 : 1);
}
// dynamic bytes after the 1 KB alignment pad; 1 KB more stays free for the
// kernel's static shared memory (227 KB per block in all)
constexpr size_t kSmemBudget = 227 * 1024 - 2048;

// Raw stages per tile width: the rest of the budget after two MMA slots of the
// 3xTF32 split (BN = 128: 3 x 32 KB + 2 x 64 KB; 64: 5 x 24 + 2 x 48; 32:
// 7 x 20 + 2 x 40), so narrow tiles, whose long k loops stream their operand
// from memory, keep more copies in flight.
template <int BN>
constexpr int raw_stages() {
  return BN >= 128 ? 3 : BN >= 64 ? 5 : 7;
}
template <int BN>
int mslots_for(int split) {
  int s = (int)((kSmemBudget - (size_t)raw_stages<BN>() * raw_bytes<BN>()) / slot_bytes<BN>(split));
  return s > kMaxSlots ? kMaxSlots : s;
}

}  // namespace tc

static std::atomic<int> g_tc_mode{-1};  // -1: not read yet; 0 off; 1 tf32; 3 3xtf32

int tc_mode() {
  int m = g_tc_mode.load();
  if (m < 0) {
    const char* e = getenv("FDE_TC");
    m = e ? atoi(e) : 3;
    if (m != 0 && m != 1 && m != 3) m = 3;
    g_tc_mode.store(m);
  }
  return m;
}
void set_tc_mode(int m) { g_tc_mode.store(m); }

fde_status tc_error_flag(int* out) {
  *out = 0;
  unsigned int n = 0;
  FDE_CUDA(cudaMemcpyFromSymbol(&n, tc::g_wait_timeout, sizeof(n)));
  *out = (int)n;
  return FDE_OK;
}

// Device address of the expired-wait counter (current device), for callers
// that read it asynchronously on their stream.
fde_status tc_timeout_counter(unsigned int** ptr) {
  FDE_CUDA(cudaGetSymbolAddress((void**)ptr, tc::g_wait_timeout));
  return FDE_OK;
}

fde_status tc_set_wait_limit(unsigned int iters) {
  const uint32_t v = iters ? iters : tc::kSpinLimit;
  FDE_CUDA(cudaMemcpyToSymbol(tc::g_spin_limit, &v, sizeof(v)));
  return FDE_OK;
}

template <int BN, bool TA, bool TB>
static fde_status set_attr() {
  FDE_CUDA(cudaFuncSetAttribute(tc::tc_gemm_kernel<BN, tc::raw_stages<BN>(), TA, TB>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(1024 + tc::kSmemBudget)));
  return FDE_OK;
}

static fde_status tc_prepare_once();

// Kernel attributes are set once (thread-safe), before any stream capture.
fde_status tc_prepare() {
  static std::once_flag once;
  static fde_status status = FDE_OK;
  std::call_once(once, []() { status = tc_prepare_once(); });
  return status;
}

static fde_status tc_prepare_once() {
  FDE_TRY((set_attr<32, false, false>()));
  FDE_TRY((set_attr<32, false, true>()));
  FDE_TRY((set_attr<32, true, false>()));
  FDE_TRY((set_attr<32, true, true>()));
  FDE_TRY((set_attr<64, false, false>()));
  FDE_TRY((set_attr<64, false, true>()));
  FDE_TRY((set_attr<64, true, false>()));
  FDE_TRY((set_attr<64, true, true>()));
  FDE_TRY((set_attr<128, false, false>()));
  FDE_TRY((set_attr<128, false, true>()));
  FDE_TRY((set_attr<128, true, false>()));
  FDE_TRY((set_attr<128, true, true>()));
  return FDE_OK;
}

template <int BN>
static fde_status launch_bn(const GemmBatch<float>& b, int split, int bf, cudaStream_t st) {
  constexpr int RAW = tc::raw_stages<BN>();
  // both operands packed: no raw stages are used, so the whole budget goes to
  // MMA slots (a deeper ring of bulk copies in flight)
  const bool no_raw = b.pk_a && b.pk_b;
  int mslots = tc::mslots_for<BN>(split);
  if (no_raw) {
    const int s2 = (int)(tc::kSmemBudget / tc::slot_bytes<BN>(split));
    mslots = s2 > tc::kMaxSlots ? tc::kMaxSlots : s2;
  }
  const size_t smem = 1024 + (size_t)mslots * tc::slot_bytes<BN>(split) +
                      (no_raw ? (size_t)0 : (size_t)RAW * tc::raw_bytes<BN>());
  const int which = (b.ta ? 2 : 0) + (b.tb ? 1 : 0);
  auto kern = (which == 0) ? tc::tc_gemm_kernel<BN, RAW, false, false>
              : (which == 1) ? tc::tc_gemm_kernel<BN, RAW, false, true>
              : (which == 2) ? tc::tc_gemm_kernel<BN, RAW, true, false>
                             : tc::tc_gemm_kernel<BN, RAW, true, true>;
  const int mt = ceil_div(b.max_m, tc::BM), nt = ceil_div(b.max_n, BN);
  const long long tiles = (long long)b.batch * mt * nt;
  if (tiles > 0x7fffffffLL) {
    set_error("tensor-core GEMM: %lld tiles", tiles);
    return FDE_ERR_ARG;
  }
  int dev = 0, sms = 0;
  FDE_CUDA(cudaGetDevice(&dev));
  FDE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = (int)(tiles < sms ? tiles : sms);
  ProfScope ps("gemm32tc", st, b.flops, 1);
  kern<<<grid, tc::kPThreads, smem, st>>>(b.d_desc, b.batch, mt, nt, b.alpha, b.beta, split, mslots,
                                          b.vec_a ? 1 : 0, b.vec_b ? 1 : 0, b.pk_a ? 1 : 0, b.pk_b ? 1 : 0, bf);
  FDE_LAUNCH("tc_gemm_kernel");
  return FDE_OK;
}

static fde_status repack_run(const GemmBatch<float>& b, int bn, cudaStream_t st);

// Runs the batch on the tensor cores; returns FDE_OK without launching if the
// batch is better left to the SIMT kernel (*used = false).
fde_status tc_gemm_run(const GemmBatch<float>& b, cudaStream_t st, bool* used) {
  *used = false;
  const int mode = tc_mode();
  // (the epilogue addresses the 32 columns of a chunk with 32-bit offsets j * ldc)
  if (mode == 0 || b.max_m < 64 || b.max_n < 16 || b.max_k < 32 || b.max_ldc > (1 << 26)) return FDE_OK;
  FDE_TRY(tc_prepare());
  const int bf = b.kind == kTcDefault ? 0 : 1;
  const int split = b.kind == kTcBF16x3 ? 1 : b.kind == kTcBF16 ? 0 : (mode == 3) ? 1 : 0;
  const int bn = tc_bn_for(b.max_n);
  if (b.pk_b && b.pk_bn != bn) {
    set_error("tensor-core GEMM: B packed for BN = %d, launch needs %d", b.pk_bn, bn);
    return FDE_ERR_ARG;
  }
  if (b.rp_a_n || b.rp_b_n) FDE_TRY(repack_run(b, bn, st));
  if (bn == 32)
    FDE_TRY(launch_bn<32>(b, split, bf, st));
  else if (bn == 64)
    FDE_TRY(launch_bn<64>(b, split, bf, st));
  else
    FDE_TRY(launch_bn<128>(b, split, bf, st));
  *used = true;
  return FDE_OK;
}

int tc_bn_for(int max_n) { return max_n <= 32 ? 32 : max_n <= 64 ? 64 : 128; }

namespace {
// One packed tile per block: (problem z, row tile r, k tile t) -> dst, hi then lo.
struct PackJob {
  int z, r, t;
  float* dst;
};
// Tile rows R x 32 k of op(X), X = A (IS_B false) or B, read with the same
// addressing as the GEMM (transposes, two-level k), rounded to TF32 hi and
// the exact remainder lo, written at the swizzled K-major offsets of the
// shared-memory tile; zeros outside the problem.
template <bool IS_B>
__global__ void __launch_bounds__(256) pack_tiles_kernel(const GemmDesc<float>* __restrict__ descs,
                                                         const PackJob* __restrict__ jobs, int R, int trans, int bf) {
  // the tile (R <= 128 rows x 32 k) is read into shared memory with coalesced
  // loads (consecutive threads along the operand's contiguous dimension), then
  // written as the MMA's shared-memory image one 16-byte chunk per thread,
  // the 8 (4 for BF16) chunks of a row by consecutive threads
  __shared__ float t[128][tc::BK + 1];
  const PackJob jb = jobs[blockIdx.x];
  const GemmDesc<float> d = descs[jb.z];
  const float* X = IS_B ? d.B : d.A;
  const int ld = IS_B ? d.ldb : d.lda, nrows = IS_B ? d.n : d.m;
  // k-contiguous when op(A) = Aᵀ (A: trans) or op(B) = B (B: !trans)
  const bool kcontig = IS_B ? !trans : trans;
  const bool two_level = d.kblk > 0 && !kcontig;
  const int row0 = jb.r * R, k0 = jb.t * tc::BK;
  for (int e = threadIdx.x; e < R * tc::BK; e += blockDim.x) {
    int r, c;
    if (kcontig) {
      r = e / tc::BK;
      c = e % tc::BK;
    } else {
      r = e % R;
      c = e / R;
    }
    const int row = row0 + r, k = k0 + c;
    float v = 0.f;
    if (row < nrows && k < d.k) {
      if (kcontig) {
        v = X[(size_t)row * ld + k];
      } else {
        long long col = (long long)k * ld;
        if (two_level) {
          const int q = k / d.kblk;
          col = (long long)q * d.kstr + (long long)(k - q * d.kblk) * ld;
        }
        v = X[col + row];
      }
    }
    t[r][c] = v;
  }
  __syncthreads();
  uint8_t* hi = reinterpret_cast<uint8_t*>(jb.dst);
  if (bf) {
    // BF16: dense 64-byte rows in the SW64 layout (pair p of row r: k = 2p,
    // 2p + 1), the hi tile (R x 64 bytes) then the lo tile; chunk q of a row
    // holds pairs 4q .. 4q + 3
    uint8_t* lo = hi + (size_t)R * 64;
    for (int e = threadIdx.x; e < R * 4; e += blockDim.x) {
      const int r = e >> 2, q = e & 3;
      uint4 hv, lv;
      hv.x = tc::bf16_pair(t[r][8 * q + 0], t[r][8 * q + 1], &lv.x);
      hv.y = tc::bf16_pair(t[r][8 * q + 2], t[r][8 * q + 3], &lv.y);
      hv.z = tc::bf16_pair(t[r][8 * q + 4], t[r][8 * q + 5], &lv.z);
      hv.w = tc::bf16_pair(t[r][8 * q + 6], t[r][8 * q + 7], &lv.w);
      const uint32_t off = tc::sw64_off(r, 4 * q);
      *reinterpret_cast<uint4*>(hi + off) = hv;
      *reinterpret_cast<uint4*>(lo + off) = lv;
    }
    return;
  }
  uint8_t* lo = hi + (size_t)R * tc::BK * 4;
  for (int e = threadIdx.x; e < R * 8; e += blockDim.x) {
    const int r = e >> 3, q = e & 7;
    float4 h, l;
    h.x = tc::to_tf32(t[r][4 * q + 0]);
    h.y = tc::to_tf32(t[r][4 * q + 1]);
    h.z = tc::to_tf32(t[r][4 * q + 2]);
    h.w = tc::to_tf32(t[r][4 * q + 3]);
    l.x = t[r][4 * q + 0] - h.x;
    l.y = t[r][4 * q + 1] - h.y;
    l.z = t[r][4 * q + 2] - h.z;
    l.w = t[r][4 * q + 3] - h.w;
    const uint32_t off = tc::sw_off(r, 4 * q);
    *reinterpret_cast<float4*>(hi + off) = h;
    *reinterpret_cast<float4*>(lo + off) = l;
  }
}
}  // namespace

// Refreshes the packed tiles of the batch's repacked operands from their
// current values.
static fde_status repack_run(const GemmBatch<float>& b, int bn, cudaStream_t st) {
  const int bf = b.kind == kTcDefault ? 0 : 1;
  const double bytes = 12.0 * 32.0 * ((double)b.rp_a_n * 128 + (double)b.rp_b_n * bn);  // read 4, write 8 per element
  ProfScope ps("pack", st, bytes, 0);
  if (b.rp_a_n) {
    pack_tiles_kernel<false><<<(unsigned)b.rp_a_n, 256, 0, st>>>(b.d_desc, (const PackJob*)b.rp_a_jobs, 128,
                                                                  b.ta ? 1 : 0, bf);
    FDE_LAUNCH("pack_tiles_kernel");
  }
  if (b.rp_b_n) {
    pack_tiles_kernel<true><<<(unsigned)b.rp_b_n, 256, 0, st>>>(b.d_desc, (const PackJob*)b.rp_b_jobs, bn,
                                                                 b.tb ? 1 : 0, bf);
    FDE_LAUNCH("pack_tiles_kernel");
  }
  return FDE_OK;
}

fde_status gemm_batch_pack(DevPool& pool, GemmBatch<float>* b, bool pack_a, bool pack_b, size_t* budget,
                           cudaStream_t st, bool repack_a, bool repack_b) {
  const int mode = tc_mode();
  if (b->batch == 0 || mode == 0 || (!pack_a && !pack_b)) return FDE_OK;
  if (b->max_m < 64 || b->max_n < 16 || b->max_k < 32 || b->max_ldc > (1 << 26)) return FDE_OK;
  std::vector<GemmDesc<float>> h(b->batch);
  FDE_CUDA(cudaMemcpy(h.data(), b->d_desc, h.size() * sizeof(GemmDesc<float>), cudaMemcpyDeviceToHost));
  const int bn = tc_bn_for(b->max_n);
  // tile counts and bytes
  size_t na = 0, nb = 0;
  for (const auto& d : h) {
    const size_t nk = (size_t)ceil_div(d.k, tc::BK);
    if (pack_a) na += (size_t)ceil_div(d.m, 128) * nk;
    if (pack_b) nb += (size_t)ceil_div(d.n, bn) * nk;
  }
  const size_t bytes = (na * 2 * 128 * tc::BK + nb * 2 * (size_t)bn * tc::BK) * sizeof(float);
  if (bytes > *budget) return FDE_OK;
  *budget -= bytes;
  float *pa = nullptr, *pb = nullptr;
  if (na) FDE_TRY(pool.alloc(&pa, na * 2 * 128 * tc::BK));
  if (nb) FDE_TRY(pool.alloc(&pb, nb * 2 * (size_t)bn * tc::BK));
  std::vector<PackJob> ja, jbv;
  size_t oa = 0, ob = 0;
  for (int z = 0; z < b->batch; ++z) {
    GemmDesc<float>& d = h[z];
    const int nk = ceil_div(d.k, tc::BK);
    if (pack_a) {
      d.Apk = pa + oa;
      for (int r = 0; r < ceil_div(d.m, 128); ++r)
        for (int t = 0; t < nk; ++t) {
          ja.push_back({z, r, t, pa + oa});
          oa += 2 * 128 * tc::BK;
        }
    }
    if (pack_b) {
      d.Bpk = pb + ob;
      for (int r = 0; r < ceil_div(d.n, bn); ++r)
        for (int t = 0; t < nk; ++t) {
          jbv.push_back({z, r, t, pb + ob});
          ob += 2 * (size_t)bn * tc::BK;
        }
    }
  }
  DevPool scratch;
  if (!ja.empty()) {
    PackJob* dj;
    FDE_TRY((repack_a ? pool : scratch).alloc(&dj, ja.size()));
    if (repack_a) {
      b->rp_a_jobs = dj;
      b->rp_a_n = (int)ja.size();
    }
    FDE_CUDA(cudaMemcpyAsync(dj, ja.data(), ja.size() * sizeof(PackJob), cudaMemcpyHostToDevice, st));
    pack_tiles_kernel<false><<<(unsigned)ja.size(), 256, 0, st>>>(b->d_desc, dj, 128, b->ta ? 1 : 0,
                                                                 b->kind == kTcDefault ? 0 : 1);
    FDE_LAUNCH("pack_tiles_kernel");
  }
  if (!jbv.empty()) {
    PackJob* dj;
    FDE_TRY((repack_b ? pool : scratch).alloc(&dj, jbv.size()));
    if (repack_b) {
      b->rp_b_jobs = dj;
      b->rp_b_n = (int)jbv.size();
    }
    FDE_CUDA(cudaMemcpyAsync(dj, jbv.data(), jbv.size() * sizeof(PackJob), cudaMemcpyHostToDevice, st));
    pack_tiles_kernel<true><<<(unsigned)jbv.size(), 256, 0, st>>>(b->d_desc, dj, bn, b->tb ? 1 : 0,
                                                                 b->kind == kTcDefault ? 0 : 1);
    FDE_LAUNCH("pack_tiles_kernel");
  }
  FDE_CUDA(cudaStreamSynchronize(st));
  FDE_CUDA(cudaMemcpy(b->d_desc, h.data(), h.size() * sizeof(GemmDesc<float>), cudaMemcpyHostToDevice));
  b->pk_a = b->pk_a || pack_a;
  b->pk_b = b->pk_b || pack_b;
  if (pack_b) b->pk_bn = bn;
  return FDE_OK;
}

}  // namespace fde

extern "C" fde_status fde_gemm_f32(int ta, int tb, int m, int n, int k, float alpha, const float* A, int lda,
                                   long long strideA, const float* B, int ldb, long long strideB, float beta,
                                   float* C, int ldc, long long strideC, int batch, int kblk, long long kstr,
                                   int mode, void* stream) {
  using namespace fde;
  FDE_ARG(m >= 0 && n >= 0 && k >= 0 && batch >= 0, "negative size");
  FDE_ARG(A != nullptr && B != nullptr && C != nullptr, "NULL matrix");
  FDE_ARG(mode == -1 || mode == 0 || mode == 1 || mode == 3 || mode == 4 || (mode >= 5 && mode <= 11),
          "mode must be -1, 0, 1, 3, 4 or 5 .. 11");
  FDE_ARG(kblk >= 0 && (kblk == 0 || kstr >= 0), "bad kblk / kstr");
  FDE_ARG(ldc >= (m > 1 ? m : 1), "ldc < m");
  FDE_ARG(lda >= 1 && ldb >= 1, "bad lda / ldb");
  if (batch == 0 || m == 0 || n == 0) return FDE_OK;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<GemmDesc<float>> h;
  for (int i = 0; i < batch; ++i) {
    GemmDesc<float> d{A + (size_t)i * strideA, B + (size_t)i * strideB, C + (size_t)i * strideC, m, n, k, lda, ldb,
                      ldc};
    d.kblk = kblk;
    d.kstr = kstr;
    h.push_back(d);
  }
  DevPool scratch;
  GemmBatch<float> gb;
  FDE_TRY(gemm_batch_upload(scratch, h, ta != 0, tb != 0, alpha, beta, &gb, st));
  int before = 0;
  FDE_CUDA(cudaStreamSynchronize(st));
  FDE_TRY(tc_error_flag(&before));
  const int saved = tc_mode();
  if (mode >= 0) {
    set_tc_mode(mode >= 4 ? 3 : mode);
    set_skinny_force(mode == 4 ? 1 : 0);
  }
  if (mode >= 8) gb.kind = (mode == 8 || mode == 11) ? kTcBF16 : kTcBF16x3;
  if ((mode >= 5 && mode <= 7) || mode >= 10) {
    size_t budget = (size_t)1 << 40;
    const bool pa = mode >= 10 || mode != 6, pb = mode >= 10 || mode != 5;
    const fde_status ps = gemm_batch_pack(scratch, &gb, pa, pb, &budget, st);
    if (ps != FDE_OK) {
      set_tc_mode(saved);
      set_skinny_force(-1);
      return ps;
    }
  }
  const fde_status s = gemm_batch_run(gb, st);
  set_tc_mode(saved);
  set_skinny_force(-1);
  FDE_TRY(s);
  FDE_CUDA(cudaStreamSynchronize(st));
  int flag = 0;
  FDE_TRY(tc_error_flag(&flag));
  if (flag != before) {
    set_error("tensor-core GEMM: a bounded wait expired");
    return FDE_ERR_CUDA;
  }
  return FDE_OK;
}

extern "C" fde_status fde_set_wait_limit(unsigned int iters) {
  using namespace fde;
  FDE_TRY(tc_set_wait_limit(iters));
  return FDE_OK;
}
