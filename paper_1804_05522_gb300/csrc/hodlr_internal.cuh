// Internal representation of a HODLR operator and of its factorisation.
#pragma once
#include "common.cuh"
#include "dense.cuh"

namespace fde {

// Factorisation of A + sigma I restricted to the subtrees rooted at level
// lmin (levels lmin..L):  A_l = A_{l+1} (I + A_{l+1}^{-1} O_l), O_l the
// level-l off-diagonal part, so that
//   (A + sigma I)^{-1} = Π_{l=lmin}^{L-1} (I + Ut_l V_lᵀ)^{-1} · blkdiag(D_p + sigma I)^{-1}
// with Ut_l = A_{l+1}^{-1} U_l and, per node, the capacitance matrix
//   K = [[I, V12ᵀ Ut2], [V21ᵀ Ut1, I]]  (Sherman–Morrison–Woodbury).
// Leaf blocks and capacitance matrices are kept as explicit inverses so that
// every solve is a sequence of batched GEMMs.
template <typename T>
struct Fact {
  double sigma = 0.0;
  int lmin = 0;
  T* Dinv = nullptr;               // nleaves x (lmax x lmax), ld lmax
  std::vector<T*> Ut;              // per level l >= lmin: N x K_l, ld N
  std::vector<T*> Kinv;            // per level l >= lmin: 2^l x (2K_l)^2, ld 2K_l
};

// One step of a precomputed solve: a batched GEMM or a strided copy.
template <typename T>
struct PlanOp {
  int kind = 0;                    // 0 = gemm, 1 = copy
  GemmBatch<T> g;
  const T* src = nullptr;
  T* dst = nullptr;
  int ld_src = 0, ld_dst = 0, m = 0, n = 0;
};
template <typename T>
struct Plan {
  std::vector<PlanOp<T>> ops;
};
// Host-side form of a plan step (descriptors not yet uploaded), so that
// independent plans can be merged into shared launches.
template <typename T>
struct HostOp {
  int kind = 0;  // 0 = gemm, 1 = copy
  std::vector<GemmDesc<T>> d;
  bool ta = false, tb = false;
  T alpha = T(1), beta = T(0);
  const T* src = nullptr;
  T* dst = nullptr;
  int ld_src = 0, ld_dst = 0, m = 0, n = 0;
};
template <typename T>
fde_status plan_run(const Plan<T>& p, cudaStream_t st);

}  // namespace fde

struct hodlr_s {
  fde_op_params p{};
  double c = 0, norm2 = 0, aca_tol = 0, blk_tol = 0;
  int kaca = 0, aca_conv = 0, rcap = 0, lmax = 0;
  fde::Tree tree;
  fde::DevPool pool;
  double* g = nullptr;             // g_0..g_{N+1}
  double* dp = nullptr;            // d_+ (N)
  double* dm = nullptr;            // d_- (N)
  double* U0 = nullptr;            // ACA factors of T21: N2 x kaca, N1 x kaca
  double* V0 = nullptr;
  std::vector<int> aca_rows, aca_cols;
  std::vector<int> K;              // per level l < L: padded rank
  std::vector<double*> U, V;       // per level: N x rcap (ld N), first K[l] columns used
  std::vector<int> rank12, rank21; // per internal node id
  double* D = nullptr;             // leaves: nleaves x lmax x lmax (ld lmax), FP64
  int* d_leaf_n = nullptr;         // leaf sizes (device)
  std::vector<int> leaf_n, leaf_lo;
  // FP32 copies for the mixed-precision solver (created on demand)
  std::vector<float*> U32, V32;
  float* D32 = nullptr;
  fde::Fact<double>* f0 = nullptr; // sigma = 0, lmin = 0 (hodlr_factor)
  fde::Plan<double>* solve_plan = nullptr;
  double* solve_tmp = nullptr;
  int solve_plan_ncols = 0;
  const double* solve_plan_x = nullptr;
  int solve_plan_ld = 0;
  ~hodlr_s();
};

namespace fde {

// Factorise A + sigma I for levels lmin..L into F (FP64).  Memory comes from
// `pool` (the handle's own pool when NULL).
fde_status hodlr_factorize(hodlr_s* h, double sigma, int lmin, Fact<double>* F, cudaStream_t st,
                           DevPool* pool = nullptr);
// Demote an FP64 factorisation to FP32 (allocates in pool).
fde_status fact_demote(hodlr_s* h, const Fact<double>& F, Fact<float>* G, DevPool& pool, cudaStream_t st);
// y = A x (trans 0) or Aᵀ x (trans 1) for the exact operator, FP64, O(N²).
fde_status fd_apply_dense(hodlr_s* h, const double* x, double* y, int trans, cudaStream_t st);
// FP32 copies of the level factors and leaves.
fde_status hodlr_make_fp32(hodlr_s* h, cudaStream_t st);

// Plan for Y = (A_node + sigma I)^{-1} X for all nodes of level lvl0 at once
// (X, Y: N x ncols, leading dimensions ldx, ldy).  If Y == X the solve runs
// in tmp (N x ncols, ld N) and is copied back.  z/w scratch is sized by
// solve_scratch_elems().  Level factors V: per-level pointers of type T.
template <typename T>
fde_status build_solve_plan(const hodlr_s* h, const Fact<T>& F, const std::vector<T*>& V, const T* X, int ldx,
                            T* Y, int ldy, int ncols, int lvl0, T* tmp, T* zbuf, T* wbuf, DevPool& pool,
                            Plan<T>* out, cudaStream_t st);
template <typename T>
fde_status build_solve_spec(const hodlr_s* h, const Fact<T>& F, const std::vector<T*>& V, const T* X, int ldx, T* Y,
                            int ldy, int ncols, int lvl0, T* tmp, T* zbuf, T* wbuf, std::vector<HostOp<T>>* ops);
// Upload a list of specs; specs with the same step count are merged step by
// step into single launches (their steps must agree in kind/transposes/scalars).
template <typename T>
fde_status upload_specs(const std::vector<std::vector<HostOp<T>>>& specs, DevPool& pool, Plan<T>* out,
                        cudaStream_t st);
size_t solve_scratch_elems(const hodlr_s* h, int ncols, int lvl0);

// QR + SVD recompression U Vᵀ -> U' V'ᵀ (§4.1), one CTA per job: Uin (m x r)
// and Vin (n x r) are overwritten by their Householder QR; Uout, Vout get
// rcap columns, zero beyond the kept rank, which counts the singular values
// above max(abstol, reltol σ_max) (capped at rcap).  *rank_out = kept rank;
// rank_full (may be NULL) receives the uncapped count by atomic maximum.
struct RecompJob {
  double* Uin;
  double* Vin;
  double* Uout;
  double* Vout;
  int m, n, ld;  // rows of U, rows of V, leading dimension of all four
  int* rank_out;
  int* rank_full = nullptr;
};
constexpr int kRecompMax = 96;  // largest r (shared memory 3 r² + 3 r doubles)
// Workspace of recompress_split for njobs jobs of rank r, capacity rcap:
// tau 2 njobs r, R 2 njobs r², C 2 njobs r rcap doubles, rank njobs ints.
struct RecompWork {
  double* tau;
  double* R;
  double* C;
  int* rank;
};
// recompress_jobs in three launches (QR of each factor in its own CTA, the
// small core, the products with the Householder factors in their own CTAs).
fde_status recompress_split(const RecompJob* d_jobs, int njobs, int r, int rcap, double abstol, double reltol,
                            const RecompWork& wk, cudaStream_t st);
// The core of recompress_split alone: R_U, R_V (r x r each, ld r) in wk.R,
// the kept factors to wk.C, the rank to wk.rank[0] and the job's rank fields.
fde_status recompress_core(const RecompJob* d_job, int r, int rcap, double abstol, double reltol,
                           const RecompWork& wk, cudaStream_t st);
// The same recompression for one job with m = n >= 128 rows, the QR spread over
// many CTAs (tsqr.cu).  A plan fixes the job's buffers and shapes (device
// workspace from `pool`); tsqr_run launches it (no allocation, capturable).
struct TsqrPlan;
fde_status tsqr_prepare(int rmax);  // once, before any capture
fde_status tsqr_plan_create(const RecompJob& job, const RecompJob* d_job, int r, int rcap, const RecompWork& wk,
                            DevPool& pool, TsqrPlan** out);
fde_status tsqr_run(const TsqrPlan* plan, double abstol, double reltol, cudaStream_t st);
void tsqr_plan_free(TsqrPlan* plan);
fde_status recompress_prepare(int rmax);  // once, before launches (and before any capture)
fde_status recompress_jobs(const RecompJob* d_jobs, int njobs, int r, int rcap, double abstol, double reltol,
                           cudaStream_t st);

}  // namespace fde
