// hodlr_matvec_noalloc: y = A x for a built HODLR operator with no device
// allocation on the call path.
//
// hodlr_matvec allocates its per-level coupling products z = Vᵀx and GEMM
// descriptor arrays on every call and synchronises the stream to release
// them.  This variant computes the same product with three small kernels and
// keeps the coupling products in one file-scope device array, so a call only
// launches kernels on the caller's stream and returns.
//
// Scratch: g_mv_scratch holds kMvScratchDoubles doubles (4 MiB).  A call needs
// max over levels l of 2^l * 2 * K_l * nrhs doubles (K_l the padded level rank
// from hodlr_get_info); larger requests are rejected with FDE_ERR_ARG before
// anything is launched.  Every scratch element a kernel reads was written
// earlier in the same call, so nothing has to start at zero.
//
// All calls on a device share the one array: two calls in flight at the same
// time on that device (different streams, or different host threads) race
// on it.  Issue them on one stream, or otherwise order them.
#include <mutex>

#include "hodlr_internal.cuh"

namespace {

constexpr size_t kMvScratchDoubles = size_t(1) << 19;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_mv_scratch[kMvScratchDoubles];

std::mutex g_mv_mu;
double* g_mv_ptr[kMaxDevices] = {};

// Device address of g_mv_scratch on the current device, looked up once per
// device.
fde_status scratch_ptr(double** out) {
  int dev = 0;
  FDE_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    fde::set_error("hodlr_matvec_noalloc: device ordinal %d beyond the %d supported", dev, kMaxDevices);
    return FDE_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_mv_mu);
  if (!g_mv_ptr[dev]) {
    void* p = nullptr;
    FDE_CUDA(cudaGetSymbolAddress(&p, g_mv_scratch));
    g_mv_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_mv_ptr[dev];
  return FDE_OK;
}

// Range [lo, hi) of node p at level l of the bisection tree over [0, N):
// each split puts floor((hi - lo) / 2) rows in the left child.
__device__ __forceinline__ void node_range(int N, int l, int p, int& lo, int& hi) {
  lo = 0;
  hi = N;
  for (int b = l - 1; b >= 0; --b) {
    const int m = lo + (hi - lo) / 2;
    if ((p >> b) & 1) lo = m;
    else hi = m;
  }
}

// Leaves: y[lo:hi, c] = D_q x[lo:hi, c].  Block per (leaf q, column c).
__global__ void mv_leaf_kernel(const double* __restrict__ D, int lmax, int N, int L, const double* __restrict__ x,
                               double* __restrict__ y, int ld) {
  extern __shared__ double xs[];
  const int q = blockIdx.x, c = blockIdx.y;
  int lo, hi;
  node_range(N, L, q, lo, hi);
  const int n = hi - lo;
  const double* xc = x + (size_t)c * ld + lo;
  for (int j = threadIdx.x; j < n; j += blockDim.x) xs[j] = xc[j];
  __syncthreads();
  const double* Dq = D + (size_t)q * lmax * lmax;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s = fma(Dq[i + (size_t)j * lmax], xs[j], s);
    y[(size_t)c * ld + lo + i] = s;
  }
}

// Level l, z = Vᵀ x per node half.  blockIdx.x = 2q + h: h = 0 takes rows
// [mid, hi) (the product feeds rows [lo, mid) through A12), h = 1 takes rows
// [lo, mid) (feeds rows [mid, hi) through A21).  blockIdx.y = k, blockIdx.z = c.
// z layout: z[((c * 2^(l+1)) + b) * K + k].
__global__ void mv_vtx_kernel(const double* __restrict__ V, int K, int N, int l, const double* __restrict__ x,
                              int ld, double* __restrict__ z) {
  __shared__ double red[32];
  const int b = blockIdx.x, q = b >> 1, h = b & 1, k = blockIdx.y, c = blockIdx.z;
  int lo, hi;
  node_range(N, l, q, lo, hi);
  const int mid = lo + (hi - lo) / 2;
  const int r0 = h == 0 ? mid : lo, r1 = h == 0 ? hi : mid;
  const double* vk = V + (size_t)k * N;
  const double* xc = x + (size_t)c * ld;
  double s = 0.0;
  for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) s = fma(vk[r], xc[r], s);
  s = fde::block_sum(s, red);
  if (threadIdx.x == 0) z[((size_t)c * (2u << l) + b) * K + k] = s;
}

// Level l, y += U z: thread per (row, column).
__global__ void mv_uz_kernel(const double* __restrict__ U, int K, int N, int l, const double* __restrict__ z,
                             double* __restrict__ y, int ld) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y;
  if (r >= N) return;
  int lo = 0, hi = N, q = 0;
  for (int s = 0; s < l; ++s) {
    const int m = lo + (hi - lo) / 2;
    if (r >= m) {
      lo = m;
      q = 2 * q + 1;
    } else {
      hi = m;
      q = 2 * q;
    }
  }
  const int mid = lo + (hi - lo) / 2;
  const int b = 2 * q + (r >= mid ? 1 : 0);
  const double* zb = z + ((size_t)c * (2u << l) + b) * K;
  double s = 0.0;
  for (int k = 0; k < K; ++k) s = fma(U[r + (size_t)k * N], zb[k], s);
  y[(size_t)c * ld + r] += s;
}

}  // namespace

extern "C" fde_status hodlr_matvec_noalloc(hodlr_t h, const double* d_x, double* d_y, int nrhs, int ldx,
                                           void* stream) {
  FDE_ARG(h != nullptr, "handle is NULL");
  FDE_ARG(d_x != nullptr && d_y != nullptr && d_x != d_y, "bad vectors");
  FDE_ARG(nrhs >= 1 && nrhs <= 65535 && ldx >= h->tree.N, "bad nrhs / ldx");
  const fde::Tree& tr = h->tree;
  const int N = tr.N, L = tr.L;
  size_t need = 0;
  for (int l = 0; l < L; ++l) {
    const size_t n = ((size_t)2 << l) * (size_t)h->K[l] * (size_t)nrhs;
    if (n > need) need = n;
  }
  if (need > kMvScratchDoubles) {
    fde::set_error("argument error: hodlr_matvec_noalloc needs %zu scratch doubles, its static scratch holds %zu "
                   "(reduce nrhs)", need, kMvScratchDoubles);
    return FDE_ERR_ARG;
  }
  double* z = nullptr;
  FDE_TRY(scratch_ptr(&z));
  cudaStream_t st = (cudaStream_t)stream;
  const int threads_leaf = tr.maxleaf >= 256 ? 256 : ((tr.maxleaf + 31) / 32) * 32;
  mv_leaf_kernel<<<dim3(tr.nleaves(), nrhs), threads_leaf, (size_t)tr.maxleaf * sizeof(double), st>>>(
      h->D, h->lmax, N, L, d_x, d_y, ldx);
  FDE_LAUNCH("mv_leaf_kernel");
  for (int l = 0; l < L; ++l) {
    const int K = h->K[l];
    if (K == 0) continue;
    mv_vtx_kernel<<<dim3(2u << l, K, nrhs), 128, 0, st>>>(h->V[l], K, N, l, d_x, ldx, z);
    FDE_LAUNCH("mv_vtx_kernel");
    mv_uz_kernel<<<dim3((N + 255) / 256, nrhs), 256, 0, st>>>(h->U[l], K, N, l, z, d_y, ldx);
    FDE_LAUNCH("mv_uz_kernel");
  }
  return FDE_OK;
}
