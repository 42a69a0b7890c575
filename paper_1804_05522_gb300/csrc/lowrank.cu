// The 2D time loop with the solution kept in factored form (§4.1, §4.2):
//   U^{(m)} = W Zᵀ,  C = U^{(m)} + Δt F^{(m+1)} = L Rᵀ,
// L Rᵀ recompressed by QR + SVD, the low-rank Sylvester equation
//   A_x X + X A_yᵀ = L Rᵀ                     (Eq. (sylv-timestepping))
// solved in factored form by factored ADI on the whole operators, with
// shifted HODLR factorisations of A_x and A_y (§3.5) and Zolotarev shifts for
// their spectral intervals (§3.3), the accumulated factors recompressed after
// every two shifts, and U^{(m+1)} the solution recompressed to its ε-rank.
// Everything in FP64, with fixed shapes (rank capacity kRcap, zero columns
// beyond the current rank) so that one step's launches after the right-hand
// side are captured once as a CUDA graph.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "hodlr_internal.cuh"

namespace fde {
namespace {

constexpr int kRcap = 32;     // rank capacity of every factor (3 kRcap <= kRecompMax)
constexpr int kMaxSrcLR = 8;  // source terms

struct SrcWL {
  double w[kMaxSrcLR];
};

// L = [W | Δt F_L diag(w)],  R = [Z | F_R]   (N x (kRcap + r) each, ld N)
__global__ void lr_rhs_kernel(const double* __restrict__ W, const double* __restrict__ Z,
                              const double* __restrict__ FL, const double* __restrict__ FR, int N, int r, SrcWL w,
                              double dt, double* __restrict__ L, double* __restrict__ R) {
  const size_t total = (size_t)N * (kRcap + r);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % N), c = (int)(e / N);
    if (c < kRcap) {
      L[e] = W[i + (size_t)c * N];
      R[e] = Z[i + (size_t)c * N];
    } else {
      const int l = c - kRcap;
      L[e] = dt * w.w[l] * FL[i + (size_t)l * N];
      R[e] = FR[i + (size_t)l * N];
    }
  }
}

// One fADI step's factor updates: Z <- c Z ; G <- G - Z ; H <- H - c W; the
// step's factors go to column block `slot` of Lc, Rc (N x 3 kRcap), and with
// copy_x the accumulated solution factors XL, XR to block 0.
__global__ void lr_fadi_kernel(double* __restrict__ Zb, double* __restrict__ G, double* __restrict__ H,
                               const double* __restrict__ Wb, const double* __restrict__ XL,
                               const double* __restrict__ XR, double* __restrict__ Lc, double* __restrict__ Rc,
                               size_t n, double c, int slot, int copy_x) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double z = c * Zb[e], wv = Wb[e];
    G[e] -= z;
    H[e] -= c * wv;
    Lc[(size_t)slot * n + e] = z;
    Rc[(size_t)slot * n + e] = wv;
    if (copy_x) {
      Lc[e] = XL[e];
      Rc[e] = XR[e];
    }
  }
}

__global__ void lr_zero_kernel(double* __restrict__ a, double* __restrict__ b, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    a[e] = 0.0;
    b[e] = 0.0;
  }
}

int grid_n(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 152 * 16); }

}  // namespace
}  // namespace fde

using namespace fde;

struct fde_lowrank_s {
  fde_run_params p{};
  std::vector<double> amp, samp, om;
  hodlr_t ax = nullptr, ay = nullptr;
  DevPool pool;
  int N = 0, r_src = 0, step = 0, J = 0;
  double eps = 0.0;
  std::vector<double> a, b;               // shifts: (A_y + a_j I), (A_x + b_j I)
  std::vector<Fact<double>> fx, fy;       // shifted factorisations
  std::vector<Plan<double>> px, py;       // Zb = (A_x + b_j)^{-1} G, Wb = (A_y + a_j)^{-1} H
  double *W = nullptr, *Z = nullptr;      // state factors, N x kRcap
  double *FL = nullptr, *FR = nullptr;    // source factors, N x r
  double *L = nullptr, *R = nullptr;      // right-hand side factors, N x (kRcap + r) (destroyed by the QR)
  double *G = nullptr, *H = nullptr;      // fADI right-hand side factors, N x kRcap
  double *Zb = nullptr, *Wb = nullptr;    // one fADI step's solves
  double *XL = nullptr, *XR = nullptr;    // accumulated solution factors
  double *Lc = nullptr, *Rc = nullptr;    // [XL | Zb_j | Zb_j+1], [XR | Wb_j | Wb_j+1], N x 3 kRcap
  RecompJob* jobs = nullptr;              // 0: right-hand side, 1: accumulation, 2: final
  int* ranks = nullptr;                   // kept ranks of the three jobs, then their uncapped maxima
  RecompWork wk{};                        // workspace of the recompressions
  TsqrPlan* tp[3] = {nullptr, nullptr, nullptr};  // their TSQR plans
  cudaStream_t gs = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t graph_kernels = 0;
  int rank = 0;
  ~fde_lowrank_s() {
    for (auto* t : tp) tsqr_plan_free(t);
    if (exec) cudaGraphExecDestroy(exec);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (gs) cudaStreamDestroy(gs);
    hodlr_free(ax);
    hodlr_free(ay);
  }
  SrcWL weights(double t) const {
    SrcWL w{};
    for (int l = 0; l < r_src; ++l) w.w[l] = amp[l] + samp[l] * sin(om[l] * t);
    return w;
  }
};

namespace {

// The step after the right-hand side factors: recompression of L Rᵀ, the fADI
// sweep with a recompression after every two shifts, the final truncation.
fde_status lr_step_body(fde_lowrank_s* S, cudaStream_t st) {
  const int N = S->N;
  const size_t nf = (size_t)N * kRcap;
  // truncation: eps relative to ||C||_2 and to ||X||_2 (as the paper's single
  // tolerance); the accumulation keeps 100 x more than the final truncation
  const double rel_rhs = S->eps, rel_acc = 0.01 * S->eps, rel_fin = S->eps;
  FDE_TRY(tsqr_run(S->tp[0], 0.0, rel_rhs, st));
  lr_zero_kernel<<<grid_n(nf), 256, 0, st>>>(S->XL, S->XR, nf);
  FDE_LAUNCH("lr_zero_kernel");
  // two fADI steps per recompression of [XL | Z_j | Z_j+1] [XR | W_j | W_j+1]ᵀ
  for (int j = 0; j < S->J; j += 2) {
    for (int k = 0; k < 2; ++k) {
      if (j + k < S->J) {
        FDE_TRY(plan_run(S->px[j + k], st));
        FDE_TRY(plan_run(S->py[j + k], st));
        lr_fadi_kernel<<<grid_n(nf), 256, 0, st>>>(S->Zb, S->G, S->H, S->Wb, S->XL, S->XR, S->Lc, S->Rc, nf,
                                                   S->a[j + k] + S->b[j + k], 1 + k, k == 0);
        FDE_LAUNCH("lr_fadi_kernel");
      } else {
        lr_zero_kernel<<<grid_n(nf), 256, 0, st>>>(S->Lc + 2 * nf, S->Rc + 2 * nf, nf);
        FDE_LAUNCH("lr_zero_kernel");
      }
    }
    FDE_TRY(tsqr_run(S->tp[1], 0.0, rel_acc, st));
  }
  FDE_TRY(tsqr_run(S->tp[2], 0.0, rel_fin, st));
  return FDE_OK;
}

fde_status lr_capture(fde_lowrank_s* S) {
  FDE_CUDA(cudaStreamCreateWithFlags(&S->gs, cudaStreamNonBlocking));
  FDE_CUDA(cudaEventCreateWithFlags(&S->ev_in, cudaEventDisableTiming));
  FDE_CUDA(cudaEventCreateWithFlags(&S->ev_out, cudaEventDisableTiming));
  cudaGraph_t g = nullptr;
  FDE_CUDA(cudaStreamBeginCapture(S->gs, cudaStreamCaptureModeThreadLocal));
  count_suspend(true);
  fde_status s = lr_step_body(S, S->gs);
  const cudaError_t e = cudaStreamEndCapture(S->gs, &g);
  count_suspend(false);
  if (s != FDE_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (s != FDE_OK) return s;
    FDE_CUDA(e);
  }
  size_t n = 0;
  FDE_CUDA(cudaGraphGetNodes(g, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  if (n) FDE_CUDA(cudaGraphGetNodes(g, nodes.data(), &n));
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    FDE_CUDA(cudaGraphNodeGetType(nd, &t));
    if (t == cudaGraphNodeTypeKernel) ++S->graph_kernels;
  }
  const cudaError_t ei = cudaGraphInstantiate(&S->exec, g, 0);
  cudaGraphDestroy(g);
  FDE_CUDA(ei);
  return FDE_OK;
}

fde_status lr_create(const fde_run_params* p, const double* hW0, const double* hZ0, int r0, double eps,
                     cudaStream_t st, fde_lowrank_s* S) {
  S->p = *p;
  const int N = p->op_x.N, r = p->rank;
  S->N = N;
  S->r_src = r;
  S->eps = eps;
  S->amp.assign(p->h_amp, p->h_amp + r);
  S->samp.assign(p->h_sin_amp, p->h_sin_amp + r);
  S->om.assign(p->h_omega, p->h_omega + r);
  // spectral intervals of the whole operators and the Zolotarev shifts
  double a_, b_, c_, d_;
  FDE_TRY(fde_block_interval(&p->op_x, 0, N, &a_, &b_));
  FDE_TRY(fde_block_interval(&p->op_y, 0, N, &c_, &d_));
  std::vector<double> al(64), be(64);
  double ratio = 0.0;
  int J = 0;
  // the fADI error stays well below the truncation (its rounding floor is
  // about 1e-11 relative for these operators)
  FDE_TRY(fde_fadi_shifts(a_, b_, c_, d_, std::max(1e-2 * eps, 1e-12), 64, &J, al.data(), be.data(), &ratio));
  S->J = J;
  S->a.assign(al.begin(), al.begin() + J);
  S->b.resize(J);
  for (int j = 0; j < J; ++j) S->b[j] = -be[j];
  FDE_TRY(hodlr_build(&p->op_x, st, &S->ax));
  FDE_TRY(hodlr_build(&p->op_y, st, &S->ay));
  DevPool& pool = S->pool;
  const size_t nf = (size_t)N * kRcap;
  FDE_TRY(pool.alloc(&S->W, nf));
  FDE_TRY(pool.alloc(&S->Z, nf));
  FDE_TRY(pool.alloc(&S->FL, (size_t)N * std::max(r, 1)));
  FDE_TRY(pool.alloc(&S->FR, (size_t)N * std::max(r, 1)));
  FDE_TRY(pool.alloc(&S->L, (size_t)N * (kRcap + r)));
  FDE_TRY(pool.alloc(&S->R, (size_t)N * (kRcap + r)));
  FDE_TRY(pool.alloc(&S->G, nf));
  FDE_TRY(pool.alloc(&S->H, nf));
  FDE_TRY(pool.alloc(&S->Zb, nf));
  FDE_TRY(pool.alloc(&S->Wb, nf));
  FDE_TRY(pool.alloc(&S->XL, nf));
  FDE_TRY(pool.alloc(&S->XR, nf));
  FDE_TRY(pool.alloc(&S->Lc, 3 * nf));
  FDE_TRY(pool.alloc(&S->Rc, 3 * nf));
  {
    const int rw = 3 * kRcap;
    FDE_TRY(pool.alloc(&S->wk.tau, 2 * (size_t)rw));
    FDE_TRY(pool.alloc(&S->wk.R, 2 * (size_t)rw * rw));
    FDE_TRY(pool.alloc(&S->wk.C, 2 * (size_t)rw * kRcap));
    FDE_TRY(pool.alloc(&S->wk.rank, 1));
  }
  FDE_TRY(pool.alloc(&S->ranks, 6));
  FDE_CUDA(cudaMemsetAsync(S->ranks, 0, 6 * sizeof(int), st));
  if (r > 0) {
    FDE_CUDA(cudaMemcpy(S->FL, p->h_src_left, (size_t)N * r * sizeof(double), cudaMemcpyHostToDevice));
    FDE_CUDA(cudaMemcpy(S->FR, p->h_src_right, (size_t)N * r * sizeof(double), cudaMemcpyHostToDevice));
  }
  FDE_CUDA(cudaMemsetAsync(S->W, 0, nf * sizeof(double), st));
  FDE_CUDA(cudaMemsetAsync(S->Z, 0, nf * sizeof(double), st));
  FDE_CUDA(cudaMemcpyAsync(S->W, hW0, (size_t)N * r0 * sizeof(double), cudaMemcpyHostToDevice, st));
  FDE_CUDA(cudaMemcpyAsync(S->Z, hZ0, (size_t)N * r0 * sizeof(double), cudaMemcpyHostToDevice, st));
  S->rank = r0;
  // recompression jobs: 0: L Rᵀ -> G Hᵀ; 1: [XL | Zb] [XR | Wb]ᵀ -> XL XRᵀ; 2: XL XRᵀ -> W Zᵀ
  std::vector<RecompJob> jb(3);
  jb[0] = {S->L, S->R, S->G, S->H, N, N, N, S->ranks + 0, S->ranks + 3};
  jb[1] = {S->Lc, S->Rc, S->XL, S->XR, N, N, N, S->ranks + 1, S->ranks + 4};
  jb[2] = {S->XL, S->XR, S->W, S->Z, N, N, N, S->ranks + 2, S->ranks + 5};
  FDE_TRY(pool.alloc(&S->jobs, 3));
  FDE_CUDA(cudaMemcpy(S->jobs, jb.data(), 3 * sizeof(RecompJob), cudaMemcpyHostToDevice));
  FDE_TRY(recompress_prepare(3 * kRcap));
  FDE_TRY(tsqr_prepare(3 * kRcap));
  const int rj[3] = {kRcap + r, 3 * kRcap, kRcap};
  for (int k = 0; k < 3; ++k) FDE_TRY(tsqr_plan_create(jb[k], S->jobs + k, rj[k], kRcap, S->wk, pool, &S->tp[k]));
  // shifted factorisations and their solve plans (kRcap columns)
  S->fx.resize(J);
  S->fy.resize(J);
  S->px.resize(J);
  S->py.resize(J);
  double *zx, *wx, *zy, *wy;
  FDE_TRY(pool.alloc(&zx, solve_scratch_elems(S->ax, kRcap, 0)));
  FDE_TRY(pool.alloc(&wx, solve_scratch_elems(S->ax, kRcap, 0)));
  FDE_TRY(pool.alloc(&zy, solve_scratch_elems(S->ay, kRcap, 0)));
  FDE_TRY(pool.alloc(&wy, solve_scratch_elems(S->ay, kRcap, 0)));
  for (int j = 0; j < J; ++j) {
    FDE_TRY(hodlr_factorize(S->ax, S->b[j], 0, &S->fx[j], st, &pool));
    FDE_TRY(hodlr_factorize(S->ay, S->a[j], 0, &S->fy[j], st, &pool));
    FDE_TRY(build_solve_plan<double>(S->ax, S->fx[j], S->ax->V, S->G, N, S->Zb, N, kRcap, 0, nullptr, zx, wx, pool,
                                     &S->px[j], st));
    FDE_TRY(build_solve_plan<double>(S->ay, S->fy[j], S->ay->V, S->H, N, S->Wb, N, kRcap, 0, nullptr, zy, wy, pool,
                                     &S->py[j], st));
  }
  FDE_CUDA(cudaStreamSynchronize(st));
  return lr_capture(S);
}

}  // namespace

extern "C" fde_status fde_lowrank_create(const fde_run_params* p, const double* h_W0, const double* h_Z0, int r0,
                                         double eps, void* stream, fde_lowrank_t* out) {
  FDE_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  FDE_ARG(p != nullptr && p->dim == 2, "a 2D time loop is required");
  FDE_ARG(p->op_x.N == p->op_y.N && p->op_x.leaf == p->op_y.leaf, "op_x / op_y differ in N or leaf");
  FDE_ARG(p->op_x.shift == 0.5 && p->op_y.shift == 0.5, "op_x.shift and op_y.shift must be 1/2");
  FDE_ARG(p->op_x.N > p->op_x.leaf && p->op_x.N >= 3 * kRcap, "N must exceed the leaf size and 96");
  FDE_ARG(p->rank >= 0 && p->rank <= kMaxSrcLR, "source rank must be in [0, 8]");
  FDE_ARG(p->rank == 0 || (p->h_src_left && p->h_src_right && p->h_amp && p->h_sin_amp && p->h_omega),
          "NULL source arrays");
  FDE_ARG(h_W0 != nullptr && h_Z0 != nullptr && r0 >= 1 && r0 <= kRcap, "initial factors: 1 <= r0 <= 32");
  FDE_ARG(eps > 0.0 && eps < 1.0, "eps must be in (0, 1)");
  fde_lowrank_s* S = new fde_lowrank_s();
  fde_status s = lr_create(p, h_W0, h_Z0, r0, eps, (cudaStream_t)stream, S);
  if (s != FDE_OK) {
    delete S;
    return s;
  }
  *out = S;
  return FDE_OK;
}

extern "C" fde_status fde_lowrank_advance(fde_lowrank_t S, int nsteps, void* stream) {
  FDE_ARG(S != nullptr, "handle is NULL");
  FDE_ARG(nsteps >= 0, "nsteps must be >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  const int N = S->N;
  const double dt = S->p.op_x.dt;
  for (int i = 0; i < nsteps; ++i) {
    const size_t total = (size_t)N * (kRcap + S->r_src);
    lr_rhs_kernel<<<grid_n(total), 256, 0, st>>>(S->W, S->Z, S->FL, S->FR, N, S->r_src,
                                                 S->weights((S->step + 1) * dt), dt, S->L, S->R);
    FDE_LAUNCH("lr_rhs_kernel");
    FDE_CUDA(cudaEventRecord(S->ev_in, st));
    FDE_CUDA(cudaStreamWaitEvent(S->gs, S->ev_in, 0));
    FDE_CUDA(cudaGraphLaunch(S->exec, S->gs));
    FDE_CUDA(cudaEventRecord(S->ev_out, S->gs));
    FDE_CUDA(cudaStreamWaitEvent(st, S->ev_out, 0));
    count_launches(S->graph_kernels);
    S->step += 1;
  }
  // ranks: kept (0..2) and uncapped maxima (3..5); a truncation that had to
  // drop singular values above its tolerance makes the result meaningless
  int rk[6];
  FDE_CUDA(cudaMemcpyAsync(rk, S->ranks, sizeof(rk), cudaMemcpyDeviceToHost, st));
  FDE_CUDA(cudaStreamSynchronize(st));
  S->rank = rk[2];
  if (rk[3] > kRcap || rk[4] > kRcap || rk[5] > kRcap) {
    set_error("fde_lowrank_advance: rank %d above the capacity %d", std::max(rk[3], std::max(rk[4], rk[5])), kRcap);
    return FDE_ERR_NOCONV;
  }
  return FDE_OK;
}

extern "C" fde_status fde_lowrank_factors(fde_lowrank_t S, double* W, double* Z, int cap, int* rank, void* stream) {
  FDE_ARG(S != nullptr && W != nullptr && Z != nullptr && rank != nullptr, "NULL argument");
  FDE_ARG(cap >= 1, "cap must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  FDE_CUDA(cudaStreamSynchronize(st));
  *rank = S->rank;
  const int nc = std::min(cap, kRcap);
  FDE_CUDA(cudaMemcpyAsync(W, S->W, (size_t)S->N * nc * sizeof(double), cudaMemcpyDefault, st));
  FDE_CUDA(cudaMemcpyAsync(Z, S->Z, (size_t)S->N * nc * sizeof(double), cudaMemcpyDefault, st));
  FDE_CUDA(cudaStreamSynchronize(st));
  return FDE_OK;
}

extern "C" fde_status fde_lowrank_info(fde_lowrank_t S, int* shifts, int* rank_max) {
  FDE_ARG(S != nullptr, "handle is NULL");
  if (shifts) *shifts = S->J;
  if (rank_max) {
    int rk[6];
    FDE_CUDA(cudaMemcpy(rk, S->ranks, sizeof(rk), cudaMemcpyDeviceToHost));
    *rank_max = std::max(rk[3], std::max(rk[4], rk[5]));
  }
  return FDE_OK;
}

extern "C" void fde_lowrank_free(fde_lowrank_t S) { delete S; }
