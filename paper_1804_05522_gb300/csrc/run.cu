// Implicit-Euler time loop (1D: Eq. (system_FD); 2D: Eq. (sylv-timestepping)).
#include <math.h>

#include <algorithm>
#include <vector>

#include "hodlr_internal.cuh"

struct sylv_s;
namespace fde {
bool sylv_graph_steps(sylv_s* s);
fde_status sylv_step_graph(sylv_s* s, const double* C, double* X, cudaStream_t st, const double* C_prev);
fde_status sylv_graph_collect(sylv_s* s, cudaStream_t st, int* steps, int* sweeps_total, int* sweeps_max,
                              double* relres_max);
fde_status sylv_step_internal(sylv_s* s, const double* C, double* X, cudaStream_t st, double* relres, int* sweeps,
                              const double* C_prev);
}
using namespace fde;

namespace {

constexpr int kMaxSrc = 8;
struct SrcW {
  double w[kMaxSrc];
};

// C = U + dt F   (a dense source at the new time level)
__global__ void rhs_dense_kernel(const double* __restrict__ U, const double* __restrict__ F, int N, int ldf,
                                 double dt, double* __restrict__ C) {
  const size_t total = (size_t)N * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % N), j = (int)(e / N);
    C[e] = U[e] + dt * F[i + (size_t)j * ldf];
  }
}

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
__global__ void sub_kernel(const double* __restrict__ b, const double* __restrict__ y, double* __restrict__ r, int N) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) r[i] = b[i] - y[i];
}
// x += d ; acc[0] = |d|^2, acc[1] = |x|^2
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

// Max-abs and sum of squares of x[0, n), deterministic: each block writes
// (max |x|, Σ x²) of its grid-stride share to part[2 b], part[2 b + 1];
// norms_final_kernel (one block) combines them in block order.
constexpr int kNormBlocks = 1024;
__global__ void norms_part_kernel(const double* __restrict__ x, size_t n, double* __restrict__ part) {
  __shared__ double sh[32];
  double m = 0.0, q = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    m = fmax(m, fabs(v));
    q += v * v;
  }
  q = block_sum(q, sh);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double shm[32];
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, shm[w]);
    part[2 * blockIdx.x] = mm;
    part[2 * blockIdx.x + 1] = q;
  }
}
__global__ void norms_final_kernel(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double sh[32];
  double m = 0.0, q = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    m = fmax(m, part[2 * b]);
    q += part[2 * b + 1];
  }
  q = block_sum(q, sh);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double shm[32];
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, shm[w]);
    out[0] = mm;
    out[1] = q;
  }
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

struct fde_runner_s {
  fde_run_params p{};
  std::vector<double> amp, samp, om;
  hodlr_t ax = nullptr, ay = nullptr;
  sylv_t s = nullptr;
  DevPool pool;
  double *U = nullptr, *C = nullptr, *FL = nullptr, *FR = nullptr;
  double* C2 = nullptr;          // previous step's right-hand side (2D)
  double* F = nullptr;           // caller-supplied dense source (fde_runner_step_source)
  bool have_prev = false;        // C2 / the solver's residual belong to the current U
  double *y = nullptr, *rr = nullptr, *acc = nullptr;
  double* Rres = nullptr;        // exact residual of the last step (fde_runner_residual)
  double* npart = nullptr;       // per-block partial norms, and the two final values
  bool c_valid = false;          // C holds the right-hand side of the current state's step
  int N = 0, step = 0;
  fde_run_stats stats{};
  // pipelined host I/O (fde_runner_step_source_async / fde_runner_state_async):
  // copy streams for uploads (cs) and read-backs (cs_out), so that an upload
  // never queues behind a read-back that waits for a step; two device source
  // buffers and a snapshot of the state
  cudaStream_t cs = nullptr, cs_out = nullptr;
  double* Fb[2] = {nullptr, nullptr};
  double* Usnap = nullptr;
  int fk = 0;
  cudaEvent_t ev_fready[2] = {nullptr, nullptr}, ev_fused[2] = {nullptr, nullptr};
  cudaEvent_t ev_snap = nullptr, ev_d2h = nullptr;
  bool pending = false;          // launched whole-step graphs not collected yet
  ~fde_runner_s() {
    if (cs) cudaStreamSynchronize(cs);
    for (int k = 0; k < 2; ++k) {
      if (ev_fready[k]) cudaEventDestroy(ev_fready[k]);
      if (ev_fused[k]) cudaEventDestroy(ev_fused[k]);
    }
    if (ev_snap) cudaEventDestroy(ev_snap);
    if (ev_d2h) cudaEventDestroy(ev_d2h);
    if (cs_out) {
      cudaStreamSynchronize(cs_out);
      cudaStreamDestroy(cs_out);
    }
    if (cs) cudaStreamDestroy(cs);
    sylv_free(s);
    hodlr_free(ax);
    hodlr_free(ay);
  }
  SrcW weights(double t) const {
    SrcW w{};
    for (int l = 0; l < p.rank; ++l) w.w[l] = amp[l] + samp[l] * sin(om[l] * t);
    return w;
  }
};

static fde_status check_run(const fde_run_params* p) {
  FDE_ARG(p != nullptr, "params is NULL");
  FDE_ARG(p->dim == 1 || p->dim == 2, "dim must be 1 or 2");
  FDE_ARG(p->steps >= 0, "steps must be >= 0");
  FDE_ARG(p->rank >= 0 && p->rank <= kMaxSrc, "source rank must be in [0, 8]");
  FDE_ARG(p->rank == 0 || (p->h_src_left && p->h_amp && p->h_sin_amp && p->h_omega), "NULL source arrays");
  FDE_ARG(p->dim == 1 || p->rank == 0 || p->h_src_right, "NULL right source factor");
  FDE_ARG(p->prec == FDE_FP64 || p->prec == FDE_FP32_REFINE || (p->prec == FDE_BF16_REFINE && p->dim == 2),
          "unknown precision (FDE_BF16_REFINE: 2D only)");
  if (p->dim == 2) FDE_ARG(p->op_x.N == p->op_y.N && p->op_x.leaf == p->op_y.leaf, "op_x / op_y differ in N or leaf");
  // the implicit-Euler step: I + ... in 1D (Eq. (system_FD)), 1/2 I + ... per side in 2D (Eq. (sylv-timestepping))
  if (p->dim == 1) FDE_ARG(p->op_x.shift == 1.0, "1D: op_x.shift must be 1");
  if (p->dim == 2) FDE_ARG(p->op_x.shift == 0.5 && p->op_y.shift == 0.5, "2D: op_x.shift and op_y.shift must be 1/2");
  return FDE_OK;
}

static fde_status copy_state(double* dst, const double* src, size_t n, cudaStream_t st) {
  const bool dd = is_device_ptr(dst), sd = is_device_ptr(src);
  const cudaMemcpyKind k = sd ? (dd ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost)
                              : (dd ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost);
  FDE_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), k, st));
  if (!dd || !sd) FDE_CUDA(cudaStreamSynchronize(st));
  return FDE_OK;
}

static fde_status runner_create(const fde_run_params* p, const double* U0, cudaStream_t st, fde_runner_s* R) {
  R->p = *p;
  const int N = p->op_x.N, r = p->rank;
  R->N = N;
  R->amp.assign(p->h_amp, p->h_amp + r);
  R->samp.assign(p->h_sin_amp, p->h_sin_amp + r);
  R->om.assign(p->h_omega, p->h_omega + r);
  R->p.h_amp = R->p.h_sin_amp = R->p.h_omega = nullptr;
  R->p.h_src_left = R->p.h_src_right = nullptr;
  const double t0 = now_seconds();
  FDE_TRY(hodlr_build(&p->op_x, st, &R->ax));
  DevPool& pool = R->pool;
  if (r > 0) {
    FDE_TRY(pool.alloc(&R->FL, (size_t)N * r));
    FDE_CUDA(cudaMemcpy(R->FL, p->h_src_left, (size_t)N * r * sizeof(double), cudaMemcpyHostToDevice));
    if (p->dim == 2) {
      FDE_TRY(pool.alloc(&R->FR, (size_t)N * r));
      FDE_CUDA(cudaMemcpy(R->FR, p->h_src_right, (size_t)N * r * sizeof(double), cudaMemcpyHostToDevice));
    }
  }
  const size_t n = (p->dim == 1) ? (size_t)N : (size_t)N * N;
  FDE_TRY(pool.alloc(&R->U, n));
  FDE_TRY(pool.alloc(&R->C, n));
  if (p->dim == 1) {
    FDE_TRY(hodlr_factor(R->ax, st));
    FDE_TRY(pool.alloc(&R->y, N));
    FDE_TRY(pool.alloc(&R->rr, N));
    FDE_TRY(pool.alloc(&R->acc, 2));
  } else {
    FDE_TRY(hodlr_build(&p->op_y, st, &R->ay));
    FDE_TRY(sylv_create(R->ax, R->ay, p->prec, st, &R->s));
    FDE_TRY(pool.alloc(&R->C2, n));
  }
  FDE_TRY(copy_state(R->U, U0, n, st));
  FDE_CUDA(cudaStreamSynchronize(st));
  R->stats.setup_s = now_seconds() - t0;
  hodlr_info_t ix;
  hodlr_get_info(R->ax, &ix);
  R->stats.kmax_x = ix.kmax;
  if (R->ay) {
    hodlr_get_info(R->ay, &ix);
    R->stats.kmax_y = ix.kmax;
  }
  return FDE_OK;
}

// Statistics and errors of the whole-step graphs launched since the last
// collection (one host synchronisation).
static fde_status collect_graph_steps(fde_runner_s* R, cudaStream_t st) {
  int steps = 0, total = 0, mx = 0;
  double rel = 0.0;
  const fde_status s = sylv_graph_collect(R->s, st, &steps, &total, &mx, &rel);
  if (s != FDE_OK) {
    R->have_prev = false;
    R->c_valid = false;
    return s;
  }
  R->stats.sweeps_total += total;
  R->stats.sweeps_max = std::max(R->stats.sweeps_max, mx);
  R->stats.relres_max = std::max(R->stats.relres_max, rel);
  return FDE_OK;
}

// Steps launched by fde_runner_step_source_async and not collected yet.
static fde_status flush_async(fde_runner_s* r, cudaStream_t st) {
  if (!r->pending) return FDE_OK;
  r->pending = false;
  return collect_graph_steps(r, st);
}

static fde_status runner_advance(fde_runner_s* R, int nsteps, cudaStream_t st) {
  const int N = R->N, r = R->p.rank;
  const double dt = R->p.op_x.dt;
  const double t1 = now_seconds();
  if (R->p.dim == 1) {
    const int nb = std::min(1024, ceil_div(N, 256));
    for (int i = 0; i < nsteps; ++i) {
      const int m = R->step + 1;
      rhs1d_kernel<<<nb, 256, 0, st>>>(R->U, R->FL, N, r, R->weights(m * dt), dt, R->C);
      FDE_LAUNCH("rhs1d_kernel");
      // refinement: x = u (warm start); r = b - A x; δ = Â^{-1} r; x += δ
      // Stop when the error left is estimated below 1e-13 (the update itself,
      // or rho |δ| / (1 - rho) with the observed contraction rho < 1/2), or
      // when the updates stop shrinking at <= 1e-11: the FP64 rounding floor of
      // the residual for an ill-conditioned operator has been reached.
      int sw = 0;
      double rel = 0.0, prev = -1.0;
      bool done = false;
      for (sw = 1; sw <= 10; ++sw) {
        FDE_TRY(fd_apply_dense(R->ax, R->U, R->y, 0, st));
        sub_kernel<<<nb, 256, 0, st>>>(R->C, R->y, R->rr, N);
        FDE_LAUNCH("sub_kernel");
        FDE_TRY(hodlr_solve(R->ax, R->rr, R->rr, 1, N, st));
        add_norms_kernel<<<1, 1024, 0, st>>>(R->U, R->rr, N, R->acc);
        FDE_LAUNCH("add_norms_kernel");
        double a[2];
        FDE_CUDA(cudaMemcpyAsync(a, R->acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        FDE_CUDA(cudaStreamSynchronize(st));
        if (!std::isfinite(a[0])) {
          set_error("fde_run: non-finite iterate");
          return FDE_ERR_NUMERIC;
        }
        rel = (a[1] > 0.0) ? sqrt(a[0] / a[1]) : sqrt(a[0]);
        if (rel <= 1e-13) done = true;
        if (!done && prev > 0.0) {
          const double rho = rel / prev;
          if (rho < 0.5 && rel * rho / (1.0 - rho) <= 1e-13) done = true;
          if (rho >= 0.5 && rel <= 1e-11) done = true;
        }
        prev = rel;
        if (done) break;
      }
      if (!done) {
        set_error("fde_run: 1D refinement did not converge (last update %.3e)", rel);
        return FDE_ERR_NOCONV;
      }
      R->stats.sweeps_total += sw;
      R->stats.sweeps_max = std::max(R->stats.sweeps_max, sw);
      R->step = m;
      R->c_valid = true;
    }
  } else {
    const size_t NN = (size_t)N * N;
    const int nb = (int)std::min<size_t>((NN + 255) / 256, 152 * 32);
    const bool graph = sylv_graph_steps(R->s);
    for (int i = 0; i < nsteps; ++i) {
      const int m = R->step;
      std::swap(R->C, R->C2);  // C2 <- previous right-hand side
      rhs2d_kernel<<<nb, 256, 0, st>>>(R->U, R->FL, R->FR, N, r, R->weights((m + 1) * dt), dt, R->C);
      FDE_LAUNCH("rhs2d_kernel");
      if (graph) {
        // the whole step is one graph launch; its results are collected below
        fde_status s = sylv_step_graph(R->s, R->C, R->U, st, R->have_prev ? R->C2 : nullptr);
        R->have_prev = (s == FDE_OK);
        R->c_valid = (s == FDE_OK);
        FDE_TRY(s);
        R->step = m + 1;
        continue;
      }
      double rel = 0.0;
      int sw = 0;
      fde_status s = sylv_step_internal(R->s, R->C, R->U, st, &rel, &sw, R->have_prev ? R->C2 : nullptr);
      R->have_prev = (s == FDE_OK);
      R->c_valid = (s == FDE_OK);
      FDE_TRY(s);
      R->stats.sweeps_total += sw;
      R->stats.sweeps_max = std::max(R->stats.sweeps_max, sw);
      R->stats.relres_max = std::max(R->stats.relres_max, rel);
      R->step = m + 1;
    }
    if (graph) FDE_TRY(collect_graph_steps(R, st));
  }
  FDE_CUDA(cudaStreamSynchronize(st));
  R->stats.solve_s += now_seconds() - t1;
  return FDE_OK;
}

extern "C" fde_status fde_runner_create(const fde_run_params* p, const double* U0, void* stream, fde_runner_t* out) {
  FDE_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  FDE_TRY(check_run(p));
  FDE_ARG(U0 != nullptr, "U0 is NULL");
  fde_runner_s* R = new fde_runner_s();
  fde_status s = runner_create(p, U0, (cudaStream_t)stream, R);
  if (s != FDE_OK) {
    delete R;
    return s;
  }
  *out = R;
  return FDE_OK;
}

extern "C" fde_status fde_runner_advance(fde_runner_t r, int nsteps, void* stream) {
  FDE_ARG(r != nullptr, "runner is NULL");
  FDE_ARG(nsteps >= 0, "nsteps must be >= 0");
  FDE_TRY(flush_async(r, (cudaStream_t)stream));
  return runner_advance(r, nsteps, (cudaStream_t)stream);
}

extern "C" fde_status fde_runner_step_source(fde_runner_t r, const double* F, int ldf, void* stream) {
  FDE_ARG(r != nullptr && F != nullptr, "NULL argument");
  FDE_ARG(r->p.dim == 2, "fde_runner_step_source is for 2D runners");
  const int N = r->N;
  FDE_ARG(ldf >= N, "ldf < N");
  FDE_TRY(flush_async(r, (cudaStream_t)stream));
  cudaStream_t st = (cudaStream_t)stream;
  const double t1 = now_seconds();
  const double dt = r->p.op_x.dt;
  const double* Fd = F;
  if (!is_device_ptr(F)) {
    if (!r->F) FDE_TRY(r->pool.alloc(&r->F, (size_t)N * N));
    FDE_CUDA(cudaMemcpy2DAsync(r->F, (size_t)N * sizeof(double), F, (size_t)ldf * sizeof(double),
                               (size_t)N * sizeof(double), N, cudaMemcpyHostToDevice, st));
    Fd = r->F;
    ldf = N;
  }
  const size_t NN = (size_t)N * N;
  const int nb = (int)std::min<size_t>((NN + 255) / 256, 152 * 32);
  std::swap(r->C, r->C2);  // C2 <- previous right-hand side
  rhs_dense_kernel<<<nb, 256, 0, st>>>(r->U, Fd, N, ldf, dt, r->C);
  FDE_LAUNCH("rhs_dense_kernel");
  if (sylv_graph_steps(r->s)) {
    // one graph launch; collected (one synchronisation) before returning
    fde_status s = sylv_step_graph(r->s, r->C, r->U, st, r->have_prev ? r->C2 : nullptr);
    r->have_prev = (s == FDE_OK);
    r->c_valid = (s == FDE_OK);
    FDE_TRY(s);
    FDE_TRY(collect_graph_steps(r, st));
    r->step += 1;
    r->stats.solve_s += now_seconds() - t1;
    return FDE_OK;
  }
  double rel = 0.0;
  int sw = 0;
  fde_status s = sylv_step_internal(r->s, r->C, r->U, st, &rel, &sw, r->have_prev ? r->C2 : nullptr);
  r->have_prev = (s == FDE_OK);
  r->c_valid = (s == FDE_OK);
  FDE_TRY(s);
  r->stats.sweeps_total += sw;
  r->stats.sweeps_max = std::max(r->stats.sweeps_max, sw);
  r->stats.relres_max = std::max(r->stats.relres_max, rel);
  r->step += 1;
  r->stats.solve_s += now_seconds() - t1;
  return FDE_OK;
}

// ------------------------------------------------ pipelined host I/O
static fde_status io_prepare(fde_runner_s* r, cudaStream_t st) {
  if (r->cs) return FDE_OK;
  const size_t NN = (size_t)r->N * r->N;
  FDE_TRY(r->pool.alloc(&r->Fb[0], NN));
  FDE_TRY(r->pool.alloc(&r->Fb[1], NN));
  FDE_TRY(r->pool.alloc(&r->Usnap, NN));
  FDE_CUDA(cudaStreamCreateWithFlags(&r->cs, cudaStreamNonBlocking));
  FDE_CUDA(cudaStreamCreateWithFlags(&r->cs_out, cudaStreamNonBlocking));
  for (int k = 0; k < 2; ++k) {
    FDE_CUDA(cudaEventCreateWithFlags(&r->ev_fready[k], cudaEventDisableTiming));
    FDE_CUDA(cudaEventCreateWithFlags(&r->ev_fused[k], cudaEventDisableTiming));
    FDE_CUDA(cudaEventRecord(r->ev_fused[k], st));
  }
  FDE_CUDA(cudaEventCreateWithFlags(&r->ev_snap, cudaEventDisableTiming));
  FDE_CUDA(cudaEventCreateWithFlags(&r->ev_d2h, cudaEventDisableTiming));
  FDE_CUDA(cudaEventRecord(r->ev_d2h, st));
  return FDE_OK;
}

extern "C" fde_status fde_runner_step_source_async(fde_runner_t r, const double* F, int ldf, void* stream) {
  FDE_ARG(r != nullptr && F != nullptr, "NULL argument");
  FDE_ARG(r->p.dim == 2, "fde_runner_step_source_async is for 2D runners");
  const int N = r->N;
  FDE_ARG(ldf >= N, "ldf < N");
  cudaStream_t st = (cudaStream_t)stream;
  if (!sylv_graph_steps(r->s)) return fde_runner_step_source(r, F, ldf, stream);
  FDE_TRY(io_prepare(r, st));
  const double t1 = now_seconds();
  const double* Fd = F;
  int k = -1;
  if (!is_device_ptr(F)) {
    // the copy of this step's source runs on the copy stream, into the
    // buffer the step before last used, while earlier steps compute
    k = r->fk;
    r->fk ^= 1;
    FDE_CUDA(cudaStreamWaitEvent(r->cs, r->ev_fused[k], 0));
    FDE_CUDA(cudaMemcpy2DAsync(r->Fb[k], (size_t)N * sizeof(double), F, (size_t)ldf * sizeof(double),
                               (size_t)N * sizeof(double), N, cudaMemcpyHostToDevice, r->cs));
    FDE_CUDA(cudaEventRecord(r->ev_fready[k], r->cs));
    FDE_CUDA(cudaStreamWaitEvent(st, r->ev_fready[k], 0));
    Fd = r->Fb[k];
    ldf = N;
  }
  const size_t NN = (size_t)N * N;
  const int nb = (int)std::min<size_t>((NN + 255) / 256, 152 * 32);
  std::swap(r->C, r->C2);
  rhs_dense_kernel<<<nb, 256, 0, st>>>(r->U, Fd, N, ldf, r->p.op_x.dt, r->C);
  FDE_LAUNCH("rhs_dense_kernel");
  if (k >= 0) FDE_CUDA(cudaEventRecord(r->ev_fused[k], st));
  fde_status s = sylv_step_graph(r->s, r->C, r->U, st, r->have_prev ? r->C2 : nullptr);
  r->have_prev = (s == FDE_OK);
  r->c_valid = (s == FDE_OK);
  FDE_TRY(s);
  r->pending = true;
  r->step += 1;
  r->stats.solve_s += now_seconds() - t1;
  return FDE_OK;
}

extern "C" fde_status fde_runner_state_async(fde_runner_t r, double* U_out, void* stream) {
  FDE_ARG(r != nullptr && U_out != nullptr, "NULL argument");
  const size_t n = (r->p.dim == 1) ? (size_t)r->N : (size_t)r->N * r->N;
  cudaStream_t st = (cudaStream_t)stream;
  if (r->p.dim == 1 || is_device_ptr(U_out)) {
    FDE_CUDA(cudaMemcpyAsync(U_out, r->U, n * sizeof(double), is_device_ptr(U_out) ? cudaMemcpyDeviceToDevice
                                                                                    : cudaMemcpyDeviceToHost, st));
    return FDE_OK;
  }
  FDE_TRY(io_prepare(r, st));
  // snapshot on the compute stream (once the previous read-back has left the
  // snapshot buffer), read back on the copy stream while the next steps run
  FDE_CUDA(cudaStreamWaitEvent(st, r->ev_d2h, 0));
  FDE_CUDA(cudaMemcpyAsync(r->Usnap, r->U, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  FDE_CUDA(cudaEventRecord(r->ev_snap, st));
  FDE_CUDA(cudaStreamWaitEvent(r->cs_out, r->ev_snap, 0));
  FDE_CUDA(cudaMemcpyAsync(U_out, r->Usnap, n * sizeof(double), cudaMemcpyDeviceToHost, r->cs_out));
  FDE_CUDA(cudaEventRecord(r->ev_d2h, r->cs_out));
  return FDE_OK;
}

extern "C" fde_status fde_runner_sync(fde_runner_t r, void* stream) {
  FDE_ARG(r != nullptr, "runner is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (r->cs) FDE_CUDA(cudaStreamSynchronize(r->cs));
  if (r->cs_out) FDE_CUDA(cudaStreamSynchronize(r->cs_out));
  FDE_CUDA(cudaStreamSynchronize(st));
  if (r->pending) {
    r->pending = false;
    FDE_TRY(collect_graph_steps(r, st));
  }
  return FDE_OK;
}

extern "C" fde_status fde_runner_load(fde_runner_t r, const double* U, int step_index, void* stream) {
  FDE_ARG(r != nullptr && U != nullptr, "NULL argument");
  FDE_ARG(step_index >= 0, "step_index must be >= 0");
  FDE_TRY(flush_async(r, (cudaStream_t)stream));
  const size_t n = (r->p.dim == 1) ? (size_t)r->N : (size_t)r->N * r->N;
  FDE_TRY(copy_state(r->U, U, n, (cudaStream_t)stream));
  r->step = step_index;
  r->have_prev = false;
  r->c_valid = false;
  return FDE_OK;
}

// Rebuilds the runner's operators for the diagonals D_±^{(m+1)} of the next
// step (Eq. (system_FD) with time-dependent coefficients): HODLR build and
// factorisation in 1D; both HODLR operators and the Sylvester solver in 2D.
// The stored residual history belongs to the old operator, so the next step
// starts from U^{(m)} with an exact residual.
static fde_status runner_set_coeffs(fde_runner_s* R, const double* dpx, const double* dmx, const double* dpy,
                                    const double* dmy, cudaStream_t st) {
  const double t0 = now_seconds();
  fde_op_params ox = R->p.op_x;
  ox.d_plus = dpx;
  ox.d_minus = dmx;
  hodlr_t ax = nullptr, ay = nullptr;
  sylv_t sv = nullptr;
  fde_status s = hodlr_build(&ox, st, &ax);
  if (s == FDE_OK && R->p.dim == 1) s = hodlr_factor(ax, st);
  if (s == FDE_OK && R->p.dim == 2) {
    fde_op_params oy = R->p.op_y;
    oy.d_plus = dpy;
    oy.d_minus = dmy;
    s = hodlr_build(&oy, st, &ay);
    if (s == FDE_OK) s = sylv_create(ax, ay, R->p.prec, st, &sv);
  }
  if (s != FDE_OK) {
    sylv_free(sv);
    hodlr_free(ay);
    hodlr_free(ax);
    return s;
  }
  sylv_free(R->s);
  hodlr_free(R->ay);
  hodlr_free(R->ax);
  R->ax = ax;
  R->ay = ay;
  R->s = sv;
  R->have_prev = false;
  R->c_valid = false;
  hodlr_info_t ix;
  hodlr_get_info(R->ax, &ix);
  R->stats.kmax_x = std::max(R->stats.kmax_x, ix.kmax);
  if (R->ay) {
    hodlr_get_info(R->ay, &ix);
    R->stats.kmax_y = std::max(R->stats.kmax_y, ix.kmax);
  }
  R->stats.solve_s += now_seconds() - t0;
  return FDE_OK;
}

extern "C" fde_status fde_runner_set_coefficients(fde_runner_t r, const double* d_plus_x, const double* d_minus_x,
                                                  const double* d_plus_y, const double* d_minus_y, void* stream) {
  FDE_ARG(r != nullptr && d_plus_x != nullptr && d_minus_x != nullptr, "NULL argument");
  FDE_ARG(r->p.dim == 1 || (d_plus_y != nullptr && d_minus_y != nullptr), "2D needs the y coefficients");
  FDE_TRY(flush_async(r, (cudaStream_t)stream));
  return runner_set_coeffs(r, d_plus_x, d_minus_x, d_plus_y, d_minus_y, (cudaStream_t)stream);
}

extern "C" fde_status fde_runner_flop_model(fde_runner_t r, double* method_flops, double* impl_flops) {
  FDE_ARG(r != nullptr && r->p.dim == 2, "needs a 2D runner");
  return sylv_flop_model(r->s, method_flops, impl_flops);
}

extern "C" fde_status fde_runner_residual(fde_runner_t r, double* relres, double* maxabs, double* fro,
                                          void* stream) {
  FDE_ARG(r != nullptr && relres != nullptr && maxabs != nullptr, "NULL argument");
  FDE_TRY(flush_async(r, (cudaStream_t)stream));
  FDE_ARG(r->c_valid, "no step since fde_runner_create / fde_runner_load");
  cudaStream_t st = (cudaStream_t)stream;
  const int N = r->N;
  const size_t n = (r->p.dim == 1) ? (size_t)N : (size_t)N * N;
  if (!r->npart) FDE_TRY(r->pool.alloc(&r->npart, 2 * (size_t)kNormBlocks + 4));
  const double* Rv;
  if (r->p.dim == 1) {
    // r = b - A u with the exact (dense-structured) operator
    const int nb = std::min(1024, ceil_div(N, 256));
    FDE_TRY(fd_apply_dense(r->ax, r->U, r->y, 0, st));
    sub_kernel<<<nb, 256, 0, st>>>(r->C, r->y, r->rr, N);
    FDE_LAUNCH("sub_kernel");
    Rv = r->rr;
  } else {
    if (!r->Rres) FDE_TRY(r->pool.alloc(&r->Rres, n));
    FDE_TRY(sylv_residual(r->s, r->C, r->U, r->Rres, N, stream));
    Rv = r->Rres;
  }
  const int nb = (int)std::min<size_t>((n + 255) / 256, kNormBlocks);
  double* fin = r->npart + 2 * kNormBlocks;
  norms_part_kernel<<<nb, 256, 0, st>>>(Rv, n, r->npart);
  FDE_LAUNCH("norms_part_kernel");
  norms_final_kernel<<<1, 1024, 0, st>>>(r->npart, nb, fin);
  FDE_LAUNCH("norms_final_kernel");
  norms_part_kernel<<<nb, 256, 0, st>>>(r->C, n, r->npart);
  FDE_LAUNCH("norms_part_kernel");
  norms_final_kernel<<<1, 1024, 0, st>>>(r->npart, nb, fin + 2);
  FDE_LAUNCH("norms_final_kernel");
  double h[4];
  FDE_CUDA(cudaMemcpyAsync(h, fin, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  FDE_CUDA(cudaStreamSynchronize(st));
  *maxabs = h[0];
  *relres = h[3] > 0.0 ? sqrt(h[1] / h[3]) : sqrt(h[1]);
  if (fro) *fro = sqrt(h[1]);
  return FDE_OK;
}

extern "C" fde_status fde_runner_state(fde_runner_t r, double* U_out, void* stream) {
  FDE_ARG(r != nullptr && U_out != nullptr, "NULL argument");
  FDE_TRY(flush_async(r, (cudaStream_t)stream));
  const size_t n = (r->p.dim == 1) ? (size_t)r->N : (size_t)r->N * r->N;
  return copy_state(U_out, r->U, n, (cudaStream_t)stream);
}

extern "C" fde_status fde_runner_stats(fde_runner_t r, fde_run_stats* stats) {
  FDE_ARG(r != nullptr && stats != nullptr, "NULL argument");
  *stats = r->stats;
  const int done = r->stats.sweeps_total > 0 ? r->step : 0;
  stats->steps_per_s = (r->stats.solve_s > 0.0) ? done / r->stats.solve_s : 0.0;
  return FDE_OK;
}

extern "C" void fde_runner_free(fde_runner_t r) { delete r; }

extern "C" fde_status fde_run(const fde_run_params* p, const double* d_U0, double* d_Uout, void* stream,
                              fde_run_stats* stats) {
  FDE_TRY(check_run(p));
  FDE_ARG(d_U0 != nullptr && d_Uout != nullptr, "NULL state buffer");
  FDE_ARG(p->steps >= 1, "steps must be >= 1");
  fde_runner_t r = nullptr;
  FDE_TRY(fde_runner_create(p, d_U0, stream, &r));
  fde_status s = fde_runner_advance(r, p->steps, stream);
  if (s == FDE_OK) s = fde_runner_state(r, d_Uout, stream);
  if (s == FDE_OK && stats) {
    fde_runner_stats(r, stats);
    stats->steps_per_s = p->steps / std::max(stats->solve_s, 1e-12);
  }
  fde_runner_free(r);
  return s;
}
