// Shared host/device helpers for the fde_hodlr library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string>
#include <vector>

#include "../../include/fde_hodlr.h"

namespace fde {

// ------------------------------------------------------------ error plumbing
void set_error(const char* fmt, ...);
fde_status cuda_status(cudaError_t e, const char* what, const char* file, int line);

#define FDE_CUDA(call)                                                          \
  do {                                                                          \
    cudaError_t e__ = (call);                                                   \
    if (e__ != cudaSuccess) return ::fde::cuda_status(e__, #call, __FILE__, __LINE__); \
  } while (0)

void count_launch();
void count_launches(size_t n);
void count_suspend(bool on);  // nested: stop / resume counting on this thread
bool prof_enabled();
// Host-side failure injection (fde_fail_alloc_after): true when this device
// allocation is the one that must fail.
bool alloc_fail_now();

// Brackets a kernel launch with CUDA events when profiling is on.
// work: algorithmic FLOPs (kind 1) or bytes (kind 0) of the bracketed launches.
struct ProfScope {
  const char* fam;
  cudaStream_t st;
  cudaEvent_t a;
  double work;
  int kind;
  ProfScope(const char* family, cudaStream_t st, double work = 0.0, int kind = 1);
  ~ProfScope();
};

// Checks the launch just issued and counts it.
#define FDE_LAUNCH(what)                                                        \
  do {                                                                          \
    ::fde::count_launch();                                                      \
    cudaError_t e__ = cudaGetLastError();                                       \
    if (e__ != cudaSuccess) return ::fde::cuda_status(e__, what, __FILE__, __LINE__); \
  } while (0)

#define FDE_TRY(expr)                                                           \
  do {                                                                          \
    fde_status s__ = (expr);                                                    \
    if (s__ != FDE_OK) return s__;                                              \
  } while (0)

#define FDE_ARG(cond, msg)                                                      \
  do {                                                                          \
    if (!(cond)) {                                                              \
      ::fde::set_error("argument error: %s", msg);                              \
      return FDE_ERR_ARG;                                                       \
    }                                                                           \
  } while (0)

// ---------------------------------------------------------- device memory
// A handle-owned list of cudaMalloc'd buffers; freed together.
struct DevPool {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  template <typename T>
  fde_status alloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    if (alloc_fail_now()) {
      set_error("device allocation of %zu bytes refused (injected failure)", n * sizeof(T));
      return FDE_ERR_NOMEM;
    }
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, n * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
      return FDE_ERR_NOMEM;
    }
    ptrs.push_back(q);
    bytes += n * sizeof(T);
    *p = static_cast<T*>(q);
    return FDE_OK;
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
    bytes = 0;
  }
  ~DevPool() { release(); }
};

inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

// --------------------------------------------------------- device helpers
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (any blockDim multiple of 32, <= 1024); result to all threads.
template <typename T>
__device__ T block_sum(T v, T* sh /* >= 32 */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T r = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
  if (wid == 0) r = warp_sum(r);
  if (threadIdx.x == 0) sh[0] = r;
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

// Tree layout of a HODLR partition (§3.4.1, Eq. (HODLRpart)): node id
// 2^l - 1 + p for node p of level l; children of node p are 2p, 2p+1.
struct Tree {
  int N = 0, leaf = 0, L = 0;          // L = number of splits (levels 0..L)
  std::vector<int> lo, hi;             // per node id
  int nodes_at(int l) const { return 1 << l; }
  int id(int l, int p) const { return (1 << l) - 1 + p; }
  int nleaves() const { return 1 << L; }
  int maxleaf = 0;                     // largest leaf size
  void build(int N_, int leaf_) {
    N = N_;
    leaf = leaf_;
    L = 0;
    while ((N + (1 << L) - 1) / (1 << L) > leaf) ++L;  // ceil(N/2^L) <= leaf
    int total = (1 << (L + 1)) - 1;
    lo.assign(total, 0);
    hi.assign(total, 0);
    lo[0] = 0;
    hi[0] = N;
    for (int l = 0; l < L; ++l)
      for (int p = 0; p < (1 << l); ++p) {
        int i = id(l, p), a = lo[i], b = hi[i], m = a + (b - a) / 2;
        lo[id(l + 1, 2 * p)] = a;
        hi[id(l + 1, 2 * p)] = m;
        lo[id(l + 1, 2 * p + 1)] = m;
        hi[id(l + 1, 2 * p + 1)] = b;
      }
    maxleaf = 0;
    for (int p = 0; p < nleaves(); ++p) {
      int i = id(L, p);
      if (hi[i] - lo[i] > maxleaf) maxleaf = hi[i] - lo[i];
    }
  }
};

double now_seconds();

}  // namespace fde
