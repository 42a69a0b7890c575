// Implicit-Euler time loop (1D: Eq. (system_FD); 2D: Eq. (sylv-timestepping)).
#include <math.h>

#include <algorithm>
#include <vector>

#include "hodlr_internal.cuh"

struct sylv_s;
namespace fde {
fde_status sylv_step_internal(sylv_s* s, const double* C, double* X, cudaStream_t st, double* relres, int* sweeps);
}
using namespace fde;

namespace {

constexpr int kMaxSrc = 8;
struct SrcW {
  double w[kMaxSrc];
};

// C = U + dt Σ_l w_l FL[:,l] FR[:,l]ᵀ   (source at the new time level)
__global__ void rhs2d_kernel(const double* __restrict__ U, const double* __restrict__ FL,
                             const double* __restrict__ FR, int N, int r, SrcW w, double dt, double* __restrict__ C) {
  const size_t total = (size_t)N * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % N), j = (int)(e / N);
    double f = 0.0;
    for (int l = 0; l < r; ++l) f += w.w[l] * FL[i + (size_t)l * N] * FR[j + (size_t)l * N];
    C[e] = U[e] + dt * f;
  }
}
// b = u + dt Σ_l w_l FL[:,l]
__global__ void rhs1d_kernel(const double* __restrict__ u, const double* __restrict__ FL, int N, int r, SrcW w,
                             double dt, double* __restrict__ b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double f = 0.0;
    for (int l = 0; l < r; ++l) f += w.w[l] * FL[i + (size_t)l * N];
    b[i] = u[i] + dt * f;
  }
}
// r = b - y ; acc += |r|^2
__global__ void sub_kernel(const double* __restrict__ b, const double* __restrict__ y, double* __restrict__ r, int N) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) r[i] = b[i] - y[i];
}
// x += d ; acc[0] += |d|^2, acc[1] += |x|^2
__global__ void add_norms_kernel(double* __restrict__ x, const double* __restrict__ d, int N, double* acc) {
  __shared__ double sh[32];
  double sd = 0.0, sx = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double v = x[i] + d[i];
    x[i] = v;
    sd += d[i] * d[i];
    sx += v * v;
  }
  sd = block_sum(sd, sh);
  sx = block_sum(sx, sh);
  if (threadIdx.x == 0) {
    acc[0] = sd;
    acc[1] = sx;
  }
}

SrcW weights(const fde_run_params* p, double t) {
  SrcW w{};
  for (int l = 0; l < p->rank; ++l) w.w[l] = p->h_amp[l] + p->h_sin_amp[l] * sin(p->h_omega[l] * t);
  return w;
}

struct Guard {
  hodlr_t ax = nullptr, ay = nullptr;
  sylv_t s = nullptr;
  ~Guard() {
    sylv_free(s);
    hodlr_free(ax);
    hodlr_free(ay);
  }
};

}  // namespace

extern "C" fde_status fde_run(const fde_run_params* p, const double* d_U0, double* d_Uout, void* stream,
                              fde_run_stats* stats) {
  FDE_ARG(p != nullptr, "params is NULL");
  FDE_ARG(d_U0 != nullptr && d_Uout != nullptr, "NULL state buffer");
  FDE_ARG(p->dim == 1 || p->dim == 2, "dim must be 1 or 2");
  FDE_ARG(p->steps >= 1, "steps must be >= 1");
  FDE_ARG(p->rank >= 0 && p->rank <= kMaxSrc, "source rank must be in [0, 8]");
  FDE_ARG(p->rank == 0 || (p->h_src_left && p->h_amp && p->h_sin_amp && p->h_omega), "NULL source arrays");
  FDE_ARG(p->dim == 1 || p->rank == 0 || p->h_src_right, "NULL right source factor");
  FDE_ARG(p->prec == FDE_FP64 || p->prec == FDE_FP32_REFINE, "unknown precision");
  if (p->dim == 2) FDE_ARG(p->op_x.N == p->op_y.N && p->op_x.leaf == p->op_y.leaf, "op_x / op_y differ in N or leaf");
  cudaStream_t st = (cudaStream_t)stream;
  const int N = p->op_x.N;
  const double dt = p->op_x.dt;
  Guard g;
  DevPool pool;
  const double t0 = now_seconds();
  FDE_TRY(hodlr_build(&p->op_x, stream, &g.ax));
  double *FL = nullptr, *FR = nullptr;
  const int r = p->rank;
  if (r > 0) {
    FDE_TRY(pool.alloc(&FL, (size_t)N * r));
    FDE_CUDA(cudaMemcpy(FL, p->h_src_left, (size_t)N * r * sizeof(double), cudaMemcpyHostToDevice));
    if (p->dim == 2) {
      FDE_TRY(pool.alloc(&FR, (size_t)N * r));
      FDE_CUDA(cudaMemcpy(FR, p->h_src_right, (size_t)N * r * sizeof(double), cudaMemcpyHostToDevice));
    }
  }
  fde_run_stats s{};
  if (p->dim == 1) {
    FDE_TRY(hodlr_factor(g.ax, stream));
    double *u, *b, *y, *rr, *acc;
    FDE_TRY(pool.alloc(&u, N));
    FDE_TRY(pool.alloc(&b, N));
    FDE_TRY(pool.alloc(&y, N));
    FDE_TRY(pool.alloc(&rr, N));
    FDE_TRY(pool.alloc(&acc, 2));
    FDE_CUDA(cudaMemcpyAsync(u, d_U0, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    FDE_CUDA(cudaStreamSynchronize(st));
    const double t1 = now_seconds();
    s.setup_s = t1 - t0;
    const int nb = std::min(1024, ceil_div(N, 256));
    for (int m = 1; m <= p->steps; ++m) {
      rhs1d_kernel<<<nb, 256, 0, st>>>(u, FL, N, r, weights(p, m * dt), dt, b);
      FDE_LAUNCH("rhs1d_kernel");
      // refinement: x = u (warm start); r = b - A x; δ = Â^{-1} r; x += δ
      int sw = 0;
      double rel = 0.0;
      for (sw = 1; sw <= 10; ++sw) {
        FDE_TRY(fd_apply_dense(g.ax, u, y, 0, st));
        sub_kernel<<<nb, 256, 0, st>>>(b, y, rr, N);
        FDE_LAUNCH("sub_kernel");
        FDE_TRY(hodlr_solve(g.ax, rr, rr, 1, N, stream));
        add_norms_kernel<<<1, 1024, 0, st>>>(u, rr, N, acc);
        FDE_LAUNCH("add_norms_kernel");
        double a[2];
        FDE_CUDA(cudaMemcpyAsync(a, acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        FDE_CUDA(cudaStreamSynchronize(st));
        if (!std::isfinite(a[0])) {
          set_error("fde_run: non-finite iterate");
          return FDE_ERR_NUMERIC;
        }
        rel = (a[1] > 0.0) ? sqrt(a[0] / a[1]) : sqrt(a[0]);
        if (rel <= 1e-13) break;
      }
      if (sw > 10) {
        set_error("fde_run: 1D refinement did not converge (last update %.3e)", rel);
        return FDE_ERR_NOCONV;
      }
      s.sweeps_total += sw;
      s.sweeps_max = std::max(s.sweeps_max, sw);
    }
    FDE_CUDA(cudaMemcpyAsync(d_Uout, u, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    FDE_CUDA(cudaStreamSynchronize(st));
    s.solve_s = now_seconds() - t1;
  } else {
    FDE_TRY(hodlr_build(&p->op_y, stream, &g.ay));
    FDE_TRY(sylv_create(g.ax, g.ay, p->prec, stream, &g.s));
    const size_t NN = (size_t)N * N;
    double *U, *C;
    FDE_TRY(pool.alloc(&U, NN));
    FDE_TRY(pool.alloc(&C, NN));
    FDE_CUDA(cudaMemcpyAsync(U, d_U0, NN * sizeof(double), cudaMemcpyDeviceToDevice, st));
    FDE_CUDA(cudaStreamSynchronize(st));
    const double t1 = now_seconds();
    s.setup_s = t1 - t0;
    const int nb = (int)std::min<size_t>((NN + 255) / 256, 152 * 32);
    for (int m = 0; m < p->steps; ++m) {
      rhs2d_kernel<<<nb, 256, 0, st>>>(U, FL, FR, N, r, weights(p, (m + 1) * dt), dt, C);
      FDE_LAUNCH("rhs2d_kernel");
      double rel = 0.0;
      int sw = 0;
      FDE_TRY(sylv_step_internal(g.s, C, U, st, &rel, &sw));
      s.sweeps_total += sw;
      s.sweeps_max = std::max(s.sweeps_max, sw);
      s.relres_max = std::max(s.relres_max, rel);
    }
    FDE_CUDA(cudaMemcpyAsync(d_Uout, U, NN * sizeof(double), cudaMemcpyDeviceToDevice, st));
    FDE_CUDA(cudaStreamSynchronize(st));
    s.solve_s = now_seconds() - t1;
    hodlr_info_t iy;
    hodlr_get_info(g.ay, &iy);
    s.kmax_y = iy.kmax;
  }
  hodlr_info_t ix;
  hodlr_get_info(g.ax, &ix);
  s.kmax_x = ix.kmax;
  s.steps_per_s = p->steps / std::max(s.solve_s, 1e-12);
  if (stats) *stats = s;
  return FDE_OK;
}
