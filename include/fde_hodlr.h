/*
 * fde_hodlr.h -- C ABI of the GB300 (sm_103a) HODLR solvers for the shifted
 * Grünwald–Letnikov discretisation of space-fractional diffusion
 * (Massei, Mazza, Robol, "Fast solvers for two-dimensional fractional
 * diffusion equations using rank structured matrices", arXiv:1804.05522).
 *
 * What is computed
 *   1D (§2.2.1, Eq. (system_FD)): one implicit-Euler step is the dense system
 *        A u = b,   A = s I + (Δt/h^α) (D_+ T_α + D_- T_αᵀ),   s = 1,
 *   with T_α = -[g_{i-j+1}] the lower Hessenberg Toeplitz matrix of
 *   Eq. (toeplitz_FD) and g_k the Grünwald–Letnikov weights (Eq. (Grun)).
 *   2D (§4.2, Eq. (sylv-timestepping)): one step is the Sylvester equation
 *        A_x X + X A_yᵀ = C,   A_{x,y} as above with s = 1/2,
 *   C = U^{(m)} + Δt F^{(m+1)}.
 *
 * How (all on one GPU, no CPU fallback)
 *   hodlr_build  : g_k on the device; the top-level subdiagonal Toeplitz block
 *                  compressed once by ACA and restricted to every level
 *                  (§3.4.2), D_± scaling applied to the factors, per-block
 *                  QR+SVD recompression at ε||A||_2 (§3.4.1).
 *   hodlr_factor : HODLR factorisation (§3.5) in telescoping form: explicit
 *                  leaf inverses and one small capacitance inverse per
 *                  internal node, so that solves are batched GEMMs,
 *                  O(k N log N) per right-hand side.
 *   sylv_step    : divide and conquer over the HODLR tree (Conclusions,
 *                  D&C for HODLR right-hand sides) with leaf Bartels–Stewart
 *                  and low-rank corrections solved by factored ADI, wrapped in
 *                  FP64 iterative refinement against the exact structured
 *                  residual.
 *
 * Conventions (every entry point)
 *   - Matrices are column-major; X[i + j*ld] = u(x_i, y_j).
 *   - Pointers named d_* are DEVICE pointers, h_* HOST pointers; where either
 *     is accepted it says so.  Caller buffers are borrowed and must stay valid
 *     until the work on `stream` that uses them has completed.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *   - Handles own all of their device memory and free it in *_free.
 *   - No call aborts, traps or spins without bound.  Argument errors are
 *     detected on the host before any launch and return FDE_ERR_ARG; a failed
 *     allocation returns FDE_ERR_NOMEM; an iteration that hits its cap returns
 *     FDE_ERR_NOCONV; NaN/Inf in inputs or residuals returns FDE_ERR_NUMERIC;
 *     any other CUDA error returns FDE_ERR_CUDA (fde_last_error() has text).
 *   - Calls on one handle must not overlap (one stream per handle).
 */
#ifndef FDE_HODLR_H
#define FDE_HODLR_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FDE_OK = 0,
  FDE_ERR_ARG = 1,
  FDE_ERR_NOMEM = 2,
  FDE_ERR_NOCONV = 3,
  FDE_ERR_NUMERIC = 4,
  FDE_ERR_CUDA = 5
} fde_status;

/* Precision of the inner HODLR/D&C solver.  Refinement residuals and the
 * solution iterate are always FP64. */
typedef enum {
  FDE_FP64 = 0,         /* all inner kernels in FP64                    */
  FDE_FP32_REFINE = 1,  /* inner kernels in FP32, FP64 refinement        */
  FDE_BF16_REFINE = 2   /* 2D only: as FDE_FP32_REFINE, but the low-rank */
                        /* products of the divide-and-conquer levels     */
                        /* (fADI applications and updates, §3.3-§3.4)    */
                        /* take BF16 operands on the tensor cores (FP32  */
                        /* accumulation), split into BF16 hi + lo (three */
                        /* products); environment FDE_BF16_SPLIT=0 rounds */
                        /* them to BF16 instead (one product, more       */
                        /* refinement sweeps); leaf solves stay FP32;    */
                        /* FP64 refinement to the same tolerance         */
} fde_prec;

/* One 1D operator  A = shift*I + (dt/h^alpha) (D_+ T_alpha + D_- T_alphaᵀ)
 * (§2.2.1, Eq. (system_FD)).  d_plus / d_minus are the diagonals of D_±
 * sampled by the caller (host or device pointers, length N, finite, >= 0).
 * Requirements: N >= 2, 1 < alpha <= 2, h > 0, dt > 0, shift > 0,
 * 8 <= leaf <= 256, 0 < tol < 1 (truncation tolerance ε, relative to
 * ||A||_2, §3.4.1). */
typedef struct {
  int N;
  double alpha;
  double h;
  double dt;
  double shift;
  const double* d_plus;
  const double* d_minus;
  int leaf;
  double tol;
} fde_op_params;

typedef struct hodlr_s* hodlr_t;
typedef struct sylv_s* sylv_t;

/* Summary of a built HODLR operator (read back for checks and reports). */
typedef struct {
  int N, leaf, levels, nleaves;
  int kmax;              /* largest off-diagonal rank after recompression */
  int aca_rank;          /* rank of the ACA of the top-level Toeplitz block */
  int aca_converged;     /* 1 if ACA met its tolerance                     */
  double norm2;          /* power-iteration estimate of ||A||_2            */
  double c;              /* dt / h^alpha                                   */
  double aca_tol;        /* absolute ACA tolerance used                    */
} hodlr_info_t;

/* Build the HODLR representation of the operator.  Owns its memory.
 * Errors: FDE_ERR_ARG (bad parameters, NULL out), FDE_ERR_NOMEM,
 * FDE_ERR_NUMERIC (non-finite d_±), FDE_ERR_NOCONV (ACA hit its rank cap). */
fde_status hodlr_build(const fde_op_params* p, void* stream, hodlr_t* out);

/* Factorise A (§3.5), level by level from the leaves up: A_l = A_{l+1} +
 * [U12 V21ᵀ; U21 V12ᵀ] (the level-l couplings) is inverted by the
 * Sherman–Morrison–Woodbury identity, which needs A_{l+1}^{-1} U (computed
 * with the levels below) and the inverse of a 2k x 2k capacitance matrix per
 * node; leaves are inverted explicitly.  All inverses by Gauss–Jordan with
 * partial pivoting.  Idempotent. */
fde_status hodlr_factor(hodlr_t h, void* stream);

/* x = A^{-1} b for nrhs right-hand sides (device pointers, leading dim ldb >= N;
 * b and x may alias).  Requires hodlr_factor.  FP64. */
fde_status hodlr_solve(hodlr_t h, const double* d_b, double* d_x, int nrhs, int ldb, void* stream);

/* y = A x (HODLR matvec, FP64, device pointers), for checks. */
fde_status hodlr_matvec(hodlr_t h, const double* d_x, double* d_y, int nrhs, int ldx, void* stream);

/* y = A x like hodlr_matvec, without allocating device memory.  The paper has
 * no counterpart: this entry point is for callers that must not allocate on
 * the call path (a loop with a fixed memory budget, or a process whose device
 * memory another allocator already owns), since hodlr_matvec allocates its
 * coupling products and descriptor arrays per call and synchronises `stream`
 * to free them.  This call only enqueues kernels on `stream` and returns.
 *
 * x, y: device pointers, column-major N x nrhs, leading dimension ldx >= N,
 * x != y; the caller owns both.  Scratch is one static device array of
 * 2^19 doubles (4 MiB) per device; a call needs max_l 2^(l+1) K_l nrhs doubles
 * (K_l the padded level rank, hodlr_get_info) and larger requests return
 * FDE_ERR_ARG before anything is launched.  Nothing has to be zeroed first.
 * The first call on a device looks up the array's address; make that first
 * call before any stream capture.  Calls that overlap in time on one device
 * (two streams, two host threads) race on the shared scratch: order them. */
fde_status hodlr_matvec_noalloc(hodlr_t h, const double* d_x, double* d_y, int nrhs, int ldx, void* stream);

fde_status hodlr_get_info(hodlr_t h, hodlr_info_t* info);

/* Writes the dense N x N matrix represented by the HODLR (column-major,
 * device pointer, ld >= N).  For checks at small N. */
fde_status hodlr_to_dense(hodlr_t h, double* d_A, int ld, void* stream);

/* Copies the GL weights g_0..g_{N+1} (host pointer, N+2 doubles). */
fde_status hodlr_get_weights(hodlr_t h, double* h_g);

/* Copies the ACA pivot sequence (host pointers, capacity cap each) and its
 * length.  rows index the block rows N1..N-1 from 0, cols the columns 0..N1-1. */
fde_status hodlr_get_aca_pivots(hodlr_t h, int* h_rows, int* h_cols, int cap, int* h_k);

/* Copies the tree layout: node ranges [lo, hi) in level order, 2^(L+1)-1
 * entries each (host pointers). */
fde_status hodlr_get_tree(hodlr_t h, int* h_lo, int* h_hi, int cap);

void hodlr_free(hodlr_t h);

/* The tree hodlr_build uses for N and leaf, on the host (no device work, no
 * GPU needed): a node [lo, hi) splits into [lo, lo + (hi-lo)/2) and
 * [lo + (hi-lo)/2, hi) (Eq. (HODLRpart)); every node of a level splits while
 * ceil(N / 2^l) > leaf, so all leaves sit on level *levels and have size
 * <= leaf.  Nodes are written in level order (id 2^l - 1 + p) into h_lo /
 * h_hi (host, capacity cap >= 2^(*levels + 1) - 1).  *levels is set before
 * the capacity check, so a call with cap = 0 returns FDE_ERR_ARG and the
 * depth.  Errors: FDE_ERR_ARG for N outside [1, 2^20], leaf < 1, NULL
 * pointers or a small capacity. */
fde_status fde_tree_layout(int N, int leaf, int* h_lo, int* h_hi, int cap, int* levels);

/* ------------------------------------------------------------------ 2D -- */
/* Prepare the Sylvester solver for A_x X + X A_yᵀ = C (Eq. (sylv-timestepping)).
 * Ax and Ay must have the same N and leaf, N > leaf, and be built with shift
 * 1/2 (FDE_ERR_ARG otherwise).  Computes the real Schur forms of every leaf
 * block, the fADI shifts per level and the shifted factorisations.  The
 * handle keeps references to Ax, Ay: free it before them. */
fde_status sylv_create(hodlr_t Ax, hodlr_t Ay, int prec, void* stream, sylv_t* out);

/* Refinement controls (defaults set by sylv_create). */
typedef struct {
  int max_sweeps;        /* cap on refinement sweeps (FDE_ERR_NOCONV beyond) */
  double tol_update;     /* stop when the error left after the last update,
                            estimated as ||δX_k||_F or, once the sweeps
                            contract (rho = ||δX_k|| / ||δX_{k-1}|| < 1/2),
                            as rho ||δX_k||_F / (1 - rho), is
                            <= tol_update ||X||_F                          */
  double tol_relres;     /* or when ||R||_F <= tol_relres ||C||_F            */
  int fixed_sweeps;      /* > 0: run exactly this many sweeps, no host sync   */
} sylv_refine_t;
fde_status sylv_get_refine(sylv_t s, sylv_refine_t* r);
fde_status sylv_set_refine(sylv_t s, const sylv_refine_t* r);

/* Solve A_x X + X A_yᵀ = C.  d_C, d_X: device FP64, column-major N x N,
 * leading dimension ld >= N.  On entry X holds the initial guess (e.g. the
 * previous time step; zeros are fine); on exit the refined solution.
 * relres_out (host, may be NULL) receives ||C - A_x X - X A_yᵀ||_F / ||C||_F
 * computed in FP64 from the structured operators; sweeps_out (host, may be
 * NULL) the number of refinement sweeps.  Errors: FDE_ERR_NUMERIC (non-finite
 * C, iterate or residual), FDE_ERR_NOCONV (max_sweeps reached), FDE_ERR_CUDA
 * (also when a bounded wait of the tensor-core GEMM expired during the step;
 * with fixed_sweeps > 0 this is only checked when relres_out is requested). */
fde_status sylv_step(sylv_t s, const double* d_C, double* d_X, int ld, void* stream,
                     double* relres_out, int* sweeps_out);

/* One application of the inner (unrefined) D&C solver: X = S(C).  For checks. */
fde_status sylv_inner_solve(sylv_t s, const double* d_C, double* d_X, int ld, void* stream);

/* R = C - A_x X - X A_yᵀ in FP64 (structured, FFT based).  For checks. */
fde_status sylv_residual(sylv_t s, const double* d_C, const double* d_X, double* d_R, int ld, void* stream);

/* Work model of one inner solve (one refinement sweep), host only, no device
 * work.  *method_flops: the tensor-core-eligible flops the method itself needs
 * (§3.4 divide and conquer with §3.3 fADI by shifted HODLR solves): the leaf
 * Bartels–Stewart transforms 4 n_i n_j (n_i + n_j) per leaf pair; per level and
 * node pair the X0-dependent right-hand-side factors, J shifted HODLR solves of
 * the 2K-column factors (2 n s + 4 K s log2(s/n) per column) and the rank
 * 2J(K_x + K_y) update, with the counted leaf sizes, level ranks K and shift
 * counts J.  *impl_flops: Σ 2 m n k of the batched GEMMs the implementation
 * launches per inner solve.  Errors: FDE_ERR_ARG (NULL argument). */
fde_status sylv_flop_model(sylv_t s, double* method_flops, double* impl_flops);

void sylv_free(sylv_t s);

/* ------------------------------------------- fADI shifts (host only) -- */
/* The two host steps by which sylv_create chooses the factored-ADI shifts
 * (§3.3) of every D&C level; neither launches device work nor needs a GPU.
 *
 * fde_block_interval: an interval [lam_lo, lam_hi] holding the real parts of
 * all eigenvalues of the diagonal block A[lo:hi, lo:hi] (0 <= lo < hi <= N) of
 * the operator of Eq. (system_FD) described by p (p->d_plus / d_minus must be
 * HOST pointers here; leaf and tol are not used).  A is an M-matrix (positive
 * diagonal, non-positive off-diagonal entries, diagonally dominant; §2.2.1),
 * so by Gershgorin lam_lo = the smallest row sum of the block and
 * lam_hi = max_i (2 a_ii - row sum_i).  sylv_create takes, per level, the
 * union of these intervals over the level's nodes, for A_x ([a, b]) and A_y
 * ([c, d]).
 *
 * fde_fadi_shifts: for A X + X Bᵀ = G Hᵀ with spec(A) in [a, b] and spec(B)
 * in [c, d] (0 < a < b, 0 < c < d), the Zolotarev problem for E = [a, b] and
 * F = [-d, -c] mapped by a Möbius transform to [k, 1] ∪ [-1, -k], whose optimal
 * zeros are Jacobi dn values.  J is the smallest count <= jmax (1..64) whose
 * ratio max_E |r| / min_F |r|, r(z) = Π_j (z - alpha_j) / (z - beta_j), on 400
 * log-spaced points per interval, is <= target (0 < target < 1); J = jmax if
 * none is.  h_alpha / h_beta (host, length >= jmax) receive the J zeros
 * (in E) and poles (in F); *ratio the ratio for J.  sylv_create uses
 * jmax = 64 and target 1e-13 (FP64 inner solver) or 1e-5 (FP32).
 *
 * Errors: FDE_ERR_ARG for NULL pointers, device pointers for d_plus /
 * d_minus, or arguments outside the ranges above. */
fde_status fde_block_interval(const fde_op_params* p, int lo, int hi, double* lam_lo, double* lam_hi);
fde_status fde_fadi_shifts(double a, double b, double c, double d, double target, int jmax, int* J,
                           double* h_alpha, double* h_beta, double* ratio);

/* ------------------------------------------------------------ time loop -- */
/* Source f(x[,y],t) = Σ_l w_l(t) F_L[:,l] (⊗ F_R[:,l]),
 * w_l(t) = amp_l + sin_amp_l * sin(omega_l * t), sampled at the new time level
 * t_{m+1} = (m+1) dt (implicit Euler). */
typedef struct {
  int dim;                       /* 1 or 2                                       */
  fde_op_params op_x;            /* shift must be 1 (1D) or 1/2 (2D), else ARG   */
  fde_op_params op_y;            /* 2D only                                      */
  int steps;                     /* number of implicit-Euler steps M             */
  int rank;                      /* number of source terms r (0 allowed)         */
  const double* h_src_left;      /* host, N x r column-major                     */
  const double* h_src_right;     /* host, N x r column-major (2D only)           */
  const double* h_amp;           /* host, r                                      */
  const double* h_sin_amp;       /* host, r                                      */
  const double* h_omega;         /* host, r                                      */
  int prec;                      /* fde_prec                                     */
  int use_graph;                 /* reserved, ignored: with the FP32 inner       */
                                 /* solver every 2D step runs as one CUDA graph  */
                                 /* launch (refinement decisions on the device), */
                                 /* otherwise the inner solve is one graph per   */
                                 /* sweep; FDE_STEP_GRAPH=0 selects the latter   */
} fde_run_params;

typedef struct {
  double setup_s;                /* build + factor + Schur + shift factors       */
  double solve_s;                /* time-stepping loop                           */
  double steps_per_s;
  int sweeps_total;              /* refinement sweeps over all steps             */
  int sweeps_max;
  double relres_max;             /* worst final FP64 relative residual           */
  int kmax_x, kmax_y;
} fde_run_stats;

/* Run M implicit-Euler steps from U0 (device, N (1D) or N x N (2D),
 * column-major, ld = N) into U_out (device, same shape; may alias U0).
 * 2D with the FP32 inner solver: each step is one CUDA graph launch whose
 * refinement loop (stopping tests, choice of residual form) is decided on
 * the device, and the host synchronises once per call (fde_runner_advance:
 * once per call as well); an error of any step (FDE_ERR_NUMERIC,
 * FDE_ERR_NOCONV, an expired tensor-core wait as FDE_ERR_CUDA) is returned
 * by the call that launched it, and the state is then undefined until
 * fde_runner_load. */
fde_status fde_run(const fde_run_params* p, const double* d_U0, double* d_U_out, void* stream,
                   fde_run_stats* stats);

/* Stateful form of fde_run for callers that advance the state themselves.
 * fde_runner_create does the whole setup (build, factorisations, Schur forms,
 * shift factorisations) from U0 (host or device, same shape as in fde_run).
 * fde_runner_advance runs nsteps implicit-Euler steps on `stream`.
 * fde_runner_load / fde_runner_state copy the state in / out (host or device
 * pointers; ld = N); load also sets the time level to step_index.
 * Stats accumulate over all advances. */
typedef struct fde_runner_s* fde_runner_t;
fde_status fde_runner_create(const fde_run_params* p, const double* U0, void* stream, fde_runner_t* out);
fde_status fde_runner_advance(fde_runner_t r, int nsteps, void* stream);
fde_status fde_runner_load(fde_runner_t r, const double* U, int step_index, void* stream);
/* One 2D step with a caller-supplied source at the new time level instead of
 * the low-rank one of the parameters: C = U^{(m)} + dt F (Eq.
 * (sylv-timestepping) with a general F^{(m+1)}).  F: N x N column-major,
 * leading dimension ldf >= N, host (copied on `stream`) or device pointer.
 * Keeps the time-loop state (residual reuse, predictor) like
 * fde_runner_advance; fde_runner_load resets it. */
fde_status fde_runner_step_source(fde_runner_t r, const double* F, int ldf, void* stream);
fde_status fde_runner_state(fde_runner_t r, double* U_out, void* stream);
/* Pipelined host I/O for serving loops that feed a source field and read the
 * state back every step.  fde_runner_step_source_async is
 * fde_runner_step_source without host synchronisation: with a host F the
 * copy runs on the runner's own upload stream into one of two device buffers
 * while the previous steps compute (F must be page-locked for the copy to be
 * asynchronous, and must stay unchanged until fde_runner_sync).
 * fde_runner_state_async enqueues a device snapshot of the state on `stream`
 * and its copy into U_out (host, page-locked; a device pointer is copied on
 * `stream`) on the runner's read-back stream, overlapping the next steps; U_out is valid
 * after fde_runner_sync.  fde_runner_sync waits for all three streams and returns
 * the first error of the steps launched since the last synchronisation (the
 * state is then undefined until fde_runner_load); the synchronous calls on
 * the runner do the same first.  Without whole-step graphs (FP64 inner
 * solver, FDE_STEP_GRAPH=0) the step call is the synchronous one. */
fde_status fde_runner_step_source_async(fde_runner_t r, const double* F, int ldf, void* stream);
fde_status fde_runner_state_async(fde_runner_t r, double* U_out, void* stream);
fde_status fde_runner_sync(fde_runner_t r, void* stream);
/* Time-dependent coefficients (Eq. (system_FD) with D_±^{(m)}): the diagonals
 * of D_± for the NEXT step, sampled by the caller at its new time level
 * t_{m+1} (host or device pointers, length N, finite, >= 0; d_plus_y /
 * d_minus_y for 2D, ignored in 1D).  The runner rebuilds its operators (HODLR
 * build and factorisation in 1D; both HODLR operators and the Sylvester solver
 * in 2D) and starts the next step from U^{(m)} with an exact residual, since
 * its residual history belongs to the old operator.  The coefficients stay
 * in force until the next call.  The rebuild's time counts in the runner's
 * solve time.  On an error the old operators are kept. */
fde_status fde_runner_set_coefficients(fde_runner_t r, const double* d_plus_x, const double* d_minus_x,
                                       const double* d_plus_y, const double* d_minus_y, void* stream);
/* Exact FP64 residual of the runner's current state against the right-hand
 * side of the step that produced it (Eq. (system_FD) in 1D: b - A u; Eq.
 * (sylv-timestepping) in 2D: C - A_x U - U A_yᵀ, Toeplitz products by FFT),
 * whatever residual form the refinement used inside the step.  *relres
 * (host) = ||R||_F / ||C||_F, *maxabs (host) = max |R_ij|, *fro (host, may be
 * NULL) = ||R||_F; deterministic.  For the exact solution U* of that step's
 * equation: with the smallest row sums m_x, m_y of A_x, A_y (both
 * M-matrices, §2.2.1; fde_block_interval over [0, N) gives them as lam_lo),
 * max|U - U*| <= maxabs / (m_x + m_y); with λ_min((A + Aᵀ)/2) >= θ_x, θ_y,
 * ||U - U*||_F <= fro / (θ_x + θ_y).  Synchronises `stream`.  FDE_ERR_ARG if
 * no step was taken since fde_runner_create / fde_runner_load. */
fde_status fde_runner_residual(fde_runner_t r, double* relres, double* maxabs, double* fro, void* stream);
/* sylv_flop_model of a 2D runner's Sylvester solver (per refinement sweep).
 * FDE_ERR_ARG for a 1D runner or a NULL argument. */
fde_status fde_runner_flop_model(fde_runner_t r, double* method_flops, double* impl_flops);
fde_status fde_runner_stats(fde_runner_t r, fde_run_stats* stats);
void fde_runner_free(fde_runner_t r);

/* -------------------------------------------------- factored 2D loop -- */
/* The paper's own 2D time loop with the solution kept in factored form
 * (§4.1, §4.2): U^{(m)} = W Zᵀ, the right-hand side C = U^{(m)} + Δt F^{(m+1)}
 * = L Rᵀ recompressed by QR + SVD (singular values <= eps ||C||_2 dropped),
 * the low-rank Sylvester equation A_x X + X A_yᵀ = L Rᵀ
 * (Eq. (sylv-timestepping)) solved in factored form by factored ADI on the
 * whole operators (shifted HODLR factorisations, Zolotarev shifts for their
 * spectral intervals, §3.3; the accumulated factors recompressed after every
 * two shifts), and U^{(m+1)} = X truncated to its eps-rank.  FP64.  The source
 * is the low-rank one of p (dim 2; p->op_x / op_y d_plus / d_minus HOST
 * pointers; N >= 96); h_W0, h_Z0 (host, N x r0 column-major, 1 <= r0 <= 32)
 * give U^{(0)} = W0 Z0ᵀ.  Every factor has a capacity of 32 columns: a step
 * whose solution needs more returns FDE_ERR_NOCONV from fde_lowrank_advance.
 * fde_lowrank_factors copies W and Z (N x min(cap, 32) each, host or device,
 * zero beyond *rank) and the current rank.  fde_lowrank_info: number of fADI
 * shifts and the largest rank seen.  One CUDA graph launch per step after the
 * right-hand side; fde_lowrank_advance synchronises once per call. */
typedef struct fde_lowrank_s* fde_lowrank_t;
fde_status fde_lowrank_create(const fde_run_params* p, const double* h_W0, const double* h_Z0, int r0, double eps,
                              void* stream, fde_lowrank_t* out);
fde_status fde_lowrank_advance(fde_lowrank_t r, int nsteps, void* stream);
fde_status fde_lowrank_factors(fde_lowrank_t r, double* W, double* Z, int cap, int* rank, void* stream);
fde_status fde_lowrank_info(fde_lowrank_t r, int* shifts, int* rank_max);
void fde_lowrank_free(fde_lowrank_t r);

/* ------------------------------------------------------------- batches -- */
/* Many independent instances (1D and 2D, uneven N, α, coefficients), e.g. a
 * batch of problems served together.  fde_batch_create builds one time-loop
 * runner per instance (params[i], initial state d_U0[i]: device pointers,
 * copied); with opts->autotune the HODLR leaf size of each (dim, N, prec)
 * bucket is chosen by timing trial steps of its first instance over
 * {32, 64, 128, 256} (1D) or {64, 128, 256} (2D) and cached for the process
 * (params' leaf is used otherwise).  fde_batch_advance advances every instance
 * nsteps with opts->threads host worker threads, each on its own CUDA stream,
 * and returns when all are done (errors name the instance).  Instances are
 * indexed in the order given. */
typedef struct fde_batch_s* fde_batch_t;
typedef struct {
  int threads;   /* concurrent host workers / CUDA streams, 1..64   */
  int autotune;  /* 1: pick the leaf size per bucket by trial steps */
} fde_batch_opts;
fde_status fde_batch_create(const fde_run_params* params, const double* const* d_U0, int count,
                            const fde_batch_opts* opts, void* stream, fde_batch_t* out);
fde_status fde_batch_advance(fde_batch_t b, int nsteps);
fde_status fde_batch_state(fde_batch_t b, int i, double* U_out, void* stream);
fde_status fde_batch_info(fde_batch_t b, int i, int* leaf, fde_run_stats* stats);
fde_status fde_batch_timing(fde_batch_t b, double* setup_s, double* tune_s, double* solve_s,
                            long long* instance_steps);
void fde_batch_free(fde_batch_t b);

/* Batched FP32 GEMM of the FP32 inner solver (the dense products of the
 * Sylvester divide-and-conquer, §3.3-§3.4), exposed for checks:
 *   C_i = alpha op(A_i) op(B_i) + beta C_i,  i < batch,
 * column-major device matrices, X_i = X + i * strideX.  op(A) is m x k,
 * op(B) k x n.  kblk > 0 selects two-level addressing along k for a
 * non-transposed A and a transposed B: column k sits at
 * (k / kblk) * kstr + (k % kblk) * ld.  mode: 0 SIMT FP32 FMA, 1 tcgen05 TF32,
 * 3 tcgen05 3xTF32 (hi/lo split, FP32-level accuracy), 4 the skinny SIMT FP32
 * kernel (one dimension <= 64: n <= 40 with m >= 128, or m <= 64 with
 * n >= 128, no two-level k; other shapes as mode 3), -1 the library's own
 * dispatch (the skinny kernel for n <= 32 or m <= 64, then the tensor
 * cores), 5 / 6 / 7 3xTF32 with A / B / both operands packed first (pre-split
 * into TF32 hi and lo tiles in the kernel's shared-memory layout and loaded by
 * bulk asynchronous copies, as the solver does for its constant operands);
 * 8 BF16 operands (tcgen05 kind::f16, FP32 accumulation), 9 BF16 hi/lo split
 * (three products, about 16 significant bits), 10 / 11 modes 9 / 8 with both
 * operands packed first; batches too small
 * for the tensor cores (m < 64, n < 16 or k < 32) take a SIMT kernel.
 * Allocates the descriptor array and synchronises `stream`.  FDE_ERR_CUDA if
 * a tensor-core wait expired.  Not thread-safe: while it runs, a mode other
 * than -1 overrides the library's process-wide kernel choice, which calls on
 * other threads (fde_batch_advance workers) would also see. */
fde_status fde_gemm_f32(int ta, int tb, int m, int n, int k, float alpha, const float* A, int lda,
                        long long strideA, const float* B, int ldb, long long strideB, float beta, float* C,
                        int ldc, long long strideC, int batch, int kblk, long long kstr, int mode, void* stream);

/* Instrumentation.  fde_launch_count: kernels launched by this library in
 * this process so far.  fde_prof_enable(1) makes the library bracket the
 * launches of its main kernel families with CUDA events on their stream;
 * fde_prof_query returns the summed device time (ms) and launch count of a
 * family ("gemm32", "gemm32tc", "gemm64", "trsyl32", "trsyl64", "fft_apply",
 * "fft_df", "fft_f32", "schur", "recompress", "fadi_axpy", "transpose",
 * "refine", "pack"; an unknown name reads as no launches), synchronising the events
 * it reads;
 * fde_prof_reset clears the records. */
unsigned long long fde_launch_count(void);
void fde_prof_enable(int on);
/* work (may be NULL): algorithmic work of the recorded launches, FLOPs when
 * *work_kind == 1 (FP32 for *32 families, FP64 otherwise), DRAM bytes when
 * *work_kind == 0 (work_kind may be NULL). */
fde_status fde_prof_query(const char* family, double* ms, long long* launches, double* work, int* work_kind);
void fde_prof_reset(void);

/* Host-side failure injection, for tests of the error paths; neither call
 * makes a device fault.  The paper has no counterpart.
 *
 * fde_fail_alloc_after(n): after n more device allocations by this library
 * (n >= 0; 0 = the next one), one allocation fails as if cudaMalloc had run
 * out of memory, and the call that made it returns FDE_ERR_NOMEM; the hook
 * then disarms itself.  n < 0 disarms it.  Process-wide.
 *
 * fde_set_wait_limit(iters): iteration limit of the tensor-core GEMM's
 * bounded mbarrier waits on the current device (0 restores the default,
 * 2^26).  A limit far below what a wait needs makes the waits run out: the
 * kernel then skips its remaining work, waits for its tensor-core operations
 * to finish, frees its tensor memory and counts the expiry in a device
 * counter; sylv_step (at its next host synchronisation) and fde_gemm_f32
 * return FDE_ERR_CUDA.  Results of the affected calls are meaningless. */
void fde_fail_alloc_after(long long n);
fde_status fde_set_wait_limit(unsigned int iters);

const char* fde_strerror(fde_status s);
/* Text of the last error on the calling thread (never NULL). */
const char* fde_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FDE_HODLR_H */
