"""Plain FP64 CPU oracle for the shifted Grünwald–Letnikov fractional-diffusion
solvers of Massei, Mazza, Robol, "Fast solvers for two-dimensional fractional
diffusion equations using rank structured matrices" (arXiv:1804.05522).

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA path and never calls it.

Every function is slow on purpose: it writes the definition out (dense
matrices, dense LU, real-Schur Bartels–Stewart, Kronecker brute force), using
numpy / scipy LAPACK routines only as single library steps.

Parity status per function (what pins it, see tests/test_oracle_pins.py):
  gl_weights                 pinned: closed Γ form, g_1=-α, ordering, partial
                             sums, α∈{1,2} exact cases
  gl_toeplitz / fd_operator  pinned: α=2 Laplacian, SDD, M-matrix signs,
                             manufactured-solution first-order convergence
  hodlr_tree                 pinned: brute-force enumeration of the split rule
  norm2_power                pinned: vs dense SVD
  aca_partial_pivot          pinned: exact recovery of exactly-low-rank inputs
  truncate_lowrank           pinned: prescribed singular values
  hodlr_reference            pinned: per-block SVD error bound, rank bounds
  eps_rank                   pinned: prescribed singular values
  beckermann_bound and the   pinned: the Lemma's own hypothesis (Hilbert
  qsrank bounds                matrix, PSD Hankel) from both sides; SVD
                               ranks of T and A below the bounds; both
                               qsrank bounds hand-evaluated at fixed
                               (N, ε, norms)
  solve_dense / fde1d_run    pinned: residual / library cross-check,
                             manufactured-solution first-order convergence
  sylvester_bartels_stewart  pinned: Kronecker brute force, α=2 DST closed form
  SchurSylvester             pinned: Kronecker brute force, reused Schur forms
  quasi_triangular_sylvester pinned: Kronecker brute force on Schur forms with
                               2 x 2 blocks, every cut (base 1 .. 8)
  fde2d_rhs / fde2d_run      pinned: Kronecker steps, manufactured 2D solution
                             (first order), exactness for a solution linear
                             in t (source at the new time level)
  apply_fd_operator_fft      pinned: dense product
  min_row_sum /              pinned: dense row sums; ||K^{-1}||_∞ of the
  sylvester_error_bound        dense Kronecker matrix; the bound holds and is
                               attained for a constant error
  sym_part_exceeds /         pinned: eigenvalues of the symmetric part on
  sylvester_error_bound_fro    both sides of θ; ||K^{-1}||_2 of the dense
                               Kronecker matrix; the bound holds for random
                               errors
  sylvester_residual         pinned: X = 0, Kronecker solution, Kronecker
                             product of a perturbation
  lowrank_from_dense         pinned: prescribed singular values
  fde2d_rhs_factors          pinned: the dense right-hand side
  fde2d_lowrank_run          pinned: reduces to fde2d_run below rounding;
                             error and rank follow eps
  fde1d_run_tv / fde2d_run_tv pinned: reduce to the constant runs;
                             exactness for a solution linear in t with the
                             operator at the new level; manufactured
                             solution with time-dependent coefficients
  fe_weights / fe_stiffness  pinned: α=2 FE Laplacian, 50-digit evaluation,
                             quadrature of Eq. (fe-int), structure and
                             definiteness, manufactured-solution convergence
  fe_mass                    pinned: quadrature
  fe2d_operator              pinned: Kronecker brute force of
                             Eq. (sylv-timestepping-fe)
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
from scipy.linalg import lapack


# ---------------------------------------------------------------------------
# §2.1, Eq. (Grun) and §3.4.2: Grünwald–Letnikov weights
# ---------------------------------------------------------------------------
def gl_weights(alpha: float, K: int) -> np.ndarray:
    """g_0..g_K of g_k = (-1)^k binom(α, k), Eq. (Grun), §2.1.

    Evaluated by the recurrence of §3.4.2 written as g_k = g_{k-1} (1 - (α+1)/k):
    one correctly rounded division, subtraction and multiplication per step,
    in that order (Python floats are IEEE doubles and are never contracted).
    """
    g = np.empty(K + 1, dtype=np.float64)
    g[0] = 1.0
    a1 = alpha + 1.0
    prev = 1.0
    for k in range(1, K + 1):
        q = a1 / float(k)
        f = 1.0 - q
        prev = prev * f
        g[k] = prev
    return g


def gl_toeplitz(alpha: float, N: int) -> np.ndarray:
    """T_{α,N} = -[g_{i-j+1}]  (lower Hessenberg Toeplitz, Eq. (toeplitz_FD), §2.2.1)."""
    g = gl_weights(alpha, N)
    T = np.zeros((N, N))
    for i in range(N):
        for j in range(0, min(N, i + 2)):
            T[i, j] = -g[i - j + 1]
    return T


def fd_scale(op) -> float:
    """c = Δt / Δx^α, the factor in front of D_+T + D_-Tᵀ in Eq. (system_FD)."""
    return op.dt * op.h ** (-op.alpha)


def fd_operator(op) -> np.ndarray:
    """Dense A = s I + (Δt/Δx^α)(D_+ T + D_- Tᵀ), Eq. (system_FD) §2.2.1.

    s = 1 gives the 1D implicit-Euler matrix; s = 1/2 gives each factor of the
    2D Kronecker form of §4.2 (I⊗(½I - ΔtM) + (½I - ΔtM)⊗I).
    """
    T = gl_toeplitz(op.alpha, op.N)
    c = fd_scale(op)
    return op.shift * np.eye(op.N) + c * (op.d_plus[:, None] * T + op.d_minus[:, None] * T.T)


# ---------------------------------------------------------------------------
# §3.4.1, Eq. (HODLRpart): HODLR partition
# ---------------------------------------------------------------------------
def hodlr_tree(N: int, leaf: int):
    """Node ranges [lo, hi) per level; a node of size n splits into ⌊n/2⌋, ⌈n/2⌉
    (Eq. (HODLRpart)).  Reading of 'until we reach a minimal dimension': every
    node of a level splits while the largest node of that level exceeds `leaf`,
    so all leaves sit on one level and have size <= leaf.
    """
    levels = [[(0, N)]]
    while max(hi - lo for lo, hi in levels[-1]) > leaf:
        nxt = []
        for lo, hi in levels[-1]:
            mid = lo + (hi - lo) // 2
            nxt.append((lo, mid))
            nxt.append((mid, hi))
        levels.append(nxt)
    return levels


# ---------------------------------------------------------------------------
# §3.4.1: truncation relative to ||A||_2
# ---------------------------------------------------------------------------
def norm2_power(A: np.ndarray, iters: int = 30) -> float:
    """Estimate of ||A||_2 by `iters` power steps on AᵀA from the normalised
    all-ones vector (the paper does not say how ||A||_2 is obtained)."""
    n = A.shape[1]
    v = np.full(n, 1.0 / math.sqrt(n))
    s = 0.0
    for _ in range(iters):
        w = A.T @ (A @ v)
        s = float(np.linalg.norm(w))
        if s == 0.0:
            return 0.0
        v = w / s
    return math.sqrt(s)


def eps_rank(Y: np.ndarray, abstol: float) -> int:
    """Number of singular values above `abstol` (ε-rank with ε||X|| = abstol, §3)."""
    if Y.size == 0:
        return 0
    s = np.linalg.svd(Y, compute_uv=False)
    return int(np.sum(s > abstol))


def truncate_lowrank(U: np.ndarray, V: np.ndarray, abstol: float):
    """Recompression of U Vᵀ: reduced QR of both factors, SVD of the small core,
    drop singular values <= abstol (§4.1, the QR+SVD recompression cited there).
    Returns (U', V') with U' = Q_U W Σ, V' = Q_V Z."""
    if U.shape[1] == 0:
        return U.copy(), V.copy()
    Qu, Ru = np.linalg.qr(U)
    Qv, Rv = np.linalg.qr(V)
    W, s, Zt = np.linalg.svd(Ru @ Rv.T)
    r = int(np.sum(s > abstol))
    return (Qu @ W[:, :r]) * s[:r], Qv @ Zt[:r].T


# ---------------------------------------------------------------------------
# Adaptive cross approximation (replaces the two-sided Lanczos of §3.4.2)
# ---------------------------------------------------------------------------
def aca_partial_pivot(row_fn, col_fn, m: int, n: int, abstol: float, maxrank: int):
    """Textbook ACA with partial pivoting on an m x n matrix given by its rows
    and columns.

    Operation order (fixed so that another FP64 implementation can reproduce the
    pivots exactly):
      * residual row:    r = a(i*,:) ; for l < k: r = r - u_l[i*] * v_l   (mul, then sub)
      * column pivot:    j* = first argmax over unused columns of |r_j|
      * v_k = r / r[j*]
      * residual column: c = a(:,j*) ; for l < k: c = c - u_l * v_l[j*]
      * u_k = c
      * stop after term k when (Σ u_k²)(Σ v_k²) <= abstol², both sums taken
        sequentially from index 0 (products rounded before the add)
      * next row pivot:  first argmax over unused rows of |u_k|
    A residual row that is exactly zero marks the row used and moves to the
    lowest-index unused row.  Returns (U (m x k), V (n x k), rows, cols, converged).
    """
    U, V, rows, cols = [], [], [], []
    used_r = np.zeros(m, dtype=bool)
    used_c = np.zeros(n, dtype=bool)
    i_star = 0
    tol2 = abstol * abstol
    converged = False
    while len(U) < maxrank:
        r = np.array(row_fn(i_star), dtype=np.float64)
        for l in range(len(U)):
            r = r - U[l][i_star] * V[l]
        used_r[i_star] = True
        absr = np.where(used_c, -1.0, np.abs(r))
        j_star = int(np.argmax(absr))
        if absr[j_star] <= 0.0:
            free = np.flatnonzero(~used_r)
            if free.size == 0:
                converged = True
                break
            i_star = int(free[0])
            continue
        v = r / r[j_star]
        c = np.array(col_fn(j_star), dtype=np.float64)
        for l in range(len(U)):
            c = c - U[l] * V[l][j_star]
        u = c
        used_c[j_star] = True
        U.append(u)
        V.append(v)
        rows.append(i_star)
        cols.append(j_star)
        su = np.cumsum(u * u)[-1]
        sv = np.cumsum(v * v)[-1]
        if su * sv <= tol2:
            converged = True
            break
        absu = np.where(used_r, -1.0, np.abs(u))
        i_next = int(np.argmax(absu))
        if absu[i_next] < 0.0:
            converged = True
            break
        i_star = i_next
    k = len(U)
    Um = np.stack(U, 1) if k else np.zeros((m, 0))
    Vm = np.stack(V, 1) if k else np.zeros((n, 0))
    return Um, Vm, rows, cols, converged


def toeplitz_lower_block_entries(g: np.ndarray, N: int):
    """Row / column accessors of the top-level subdiagonal block T21 of
    T_{α,N}: rows N1..N-1, columns 0..N1-1, entries -g_{N1+i-j+1}
    (§3.4.2: T21 contains every lower off-diagonal block by restriction;
    entries as in the proof of Lemma lem:fd-qsrank)."""
    N1 = N // 2
    N2 = N - N1

    def row(i):
        return -g[N1 + i - np.arange(N1) + 1]

    def col(j):
        return -g[N1 + np.arange(N2) - j + 1]

    return N1, N2, row, col


def hodlr_reference(A: np.ndarray, leaf: int, eps: float, normA: float | None = None):
    """Definition of the HODLR approximation of §3.4.1: each off-diagonal block
    of Eq. (HODLRpart), at every level, truncated at ε||A||_2 by its SVD.
    Returns (tree, {(lo,hi): (rank12, rank21)}, abstol)."""
    N = A.shape[0]
    tree = hodlr_tree(N, leaf)
    nrm = norm2_power(A) if normA is None else normA
    abstol = eps * nrm
    ranks = {}
    for lvl in tree[:-1]:
        for lo, hi in lvl:
            mid = lo + (hi - lo) // 2
            ranks[(lo, hi)] = (eps_rank(A[lo:mid, mid:hi], abstol), eps_rank(A[mid:hi, lo:mid], abstol))
    return tree, ranks, abstol


# ---------------------------------------------------------------------------
# Lemma beckermann, Lemma lem:fd-qsrank, Corollary cor:fd-qsrank (§3.2)
# ---------------------------------------------------------------------------
def beckermann_bound(N: int, eps: float) -> int:
    """𝔅(N, ε) = 2 + 2⌈(2/π²) log(4N/π) log(16/ε)⌉ (Lemma beckermann)."""
    return 2 + 2 * math.ceil((2.0 / math.pi ** 2) * math.log(4.0 * N / math.pi) * math.log(16.0 / eps))


def qsrank_bound_T(N: int, eps: float) -> int:
    """qsrank_ε(T_{α,N}) <= 𝔅(N, ε/2) (Lemma lem:fd-qsrank)."""
    return beckermann_bound(N, eps / 2.0)


def qsrank_bound_M(N: int, eps: float, normM: float, normT: float, maxD: float) -> int:
    """qsrank_ε(M) <= 1 + 𝔅(N, ε̂/2), ε̂ = ||M|| ε / (||T|| max||D±||) (Corollary cor:fd-qsrank)."""
    eps_hat = normM * eps / (normT * maxD)
    return 1 + beckermann_bound(N, eps_hat / 2.0)


# ---------------------------------------------------------------------------
# §3.5: 1D time stepping — dense LU oracle
# ---------------------------------------------------------------------------
def solve_dense(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """x = A^{-1} b by dense LU with partial pivoting (LAPACK getrf/getrs)."""
    lu, piv = sla.lu_factor(A)
    return sla.lu_solve((lu, piv), B)


def fde1d_run(w, steps: int | None = None):
    """Implicit Euler, Eq. (system_FD): A u^{(m)} = u^{(m-1)} + Δt f^{(m)}, m = 1..M,
    f sampled at the new time level t_m = m Δt.  Returns u^{(M)}."""
    op = w.ops[0]
    A = fd_operator(op)
    lu, piv = sla.lu_factor(A)
    u = w.u0.copy()
    M = w.steps if steps is None else steps
    for m in range(1, M + 1):
        b = u + w.dt * w.source(m * w.dt)
        u = sla.lu_solve((lu, piv), b)
    return u


# ---------------------------------------------------------------------------
# §4.2, Eq. (sylv-timestepping): 2D step as a Sylvester equation
# ---------------------------------------------------------------------------
def sylvester_bartels_stewart(A: np.ndarray, B: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Solve A X + X Bᵀ = C by Bartels–Stewart: real Schur forms A = Q S Qᵀ,
    B = Z R Zᵀ (LAPACK gees), quasi-triangular S Y + Y Rᵀ = Qᵀ C Z (LAPACK trsyl),
    X = Q Y Zᵀ."""
    S, Q = sla.schur(A, output="real")
    R, Z = sla.schur(B, output="real")
    Ct = Q.T @ C @ Z
    Y, scale, info = lapack.dtrsyl(S, R, Ct, trana="N", tranb="T", isgn=1)
    if info < 0:
        raise RuntimeError(f"dtrsyl info={info}")
    return Q @ (Y / scale) @ Z.T


def quasi_triangular_sylvester(S: np.ndarray, R: np.ndarray, F: np.ndarray, base: int = 128) -> np.ndarray:
    """S Y + Y Rᵀ = F for upper quasi-triangular S (m x m) and R (n x n), the
    middle stage of Bartels–Stewart, in the recursive block form of the same
    back substitution (Jonsson & Kågström, ACM TOMS 28, 2002): the larger side
    is cut in two where no 2 x 2 diagonal block is split,
      S = [S11 S12; 0 S22]:  S22 Y2 + Y2 Rᵀ = F2,  then  S11 Y1 + Y1 Rᵀ = F1 - S12 Y2;
      R = [R11 R12; 0 R22]:  S Y2 + Y2 R22ᵀ = F2,  then  S Y1 + Y1 R11ᵀ = F1 - Y2 R12ᵀ
    (Y = [Y1; Y2] resp. [Y1, Y2]); problems of at most `base` rows and
    columns go to LAPACK trsyl.  Same result as trsyl on the whole problem up
    to rounding order, with the couplings as matrix products (base >= 2, so
    that every cut leaves two non-empty parts)."""
    if base < 2:
        raise ValueError("base must be at least 2")
    m, n = F.shape
    if m == 0 or n == 0:
        return np.zeros_like(F)
    if m <= base and n <= base:
        Y, scale, info = lapack.dtrsyl(S, R, F, trana="N", tranb="T", isgn=1)
        if info < 0 or scale != 1.0:
            raise RuntimeError(f"dtrsyl info={info} scale={scale}")
        return Y

    def cut(T, k):
        h = k // 2
        if h > 0 and T[h, h - 1] != 0.0:  # inside a 2 x 2 block
            h += 1
        return h

    if m >= n:
        h = cut(S, m)
        Y2 = quasi_triangular_sylvester(S[h:, h:], R, F[h:], base)
        Y1 = quasi_triangular_sylvester(S[:h, :h], R, F[:h] - S[:h, h:] @ Y2, base)
        return np.vstack([Y1, Y2])
    h = cut(R, n)
    Y2 = quasi_triangular_sylvester(S, R[h:, h:], F[:, h:], base)
    Y1 = quasi_triangular_sylvester(S, R[:h, :h], F[:, :h] - Y2 @ R[:h, h:].T, base)
    return np.hstack([Y1, Y2])


class SchurSylvester:
    """Bartels–Stewart with the two real Schur forms computed once (the
    coefficients of Eq. (sylv-timestepping) do not depend on time).  With
    `base`, the quasi-triangular stage runs in the recursive block form
    (quasi_triangular_sylvester); without, as one LAPACK trsyl call."""

    def __init__(self, A: np.ndarray, B: np.ndarray, base: int | None = None):
        self.S, self.Q = sla.schur(A, output="real")
        self.R, self.Z = sla.schur(B, output="real")
        self.base = base

    def solve(self, C: np.ndarray) -> np.ndarray:
        Ct = self.Q.T @ C @ self.Z
        if self.base is not None:
            return self.Q @ quasi_triangular_sylvester(self.S, self.R, Ct, self.base) @ self.Z.T
        Y, scale, info = lapack.dtrsyl(self.S, self.R, Ct, trana="N", tranb="T", isgn=1)
        if info < 0:
            raise RuntimeError(f"dtrsyl info={info}")
        return self.Q @ (Y / scale) @ self.Z.T


def sylvester_kron(A: np.ndarray, B: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Kronecker brute force: (I ⊗ A + B ⊗ I) vec X = vec C with column-major
    vec (vec(A X Bᵀ) = (B ⊗ A) vec X, §4.2)."""
    n, m = C.shape
    K = np.kron(np.eye(m), A) + np.kron(B, np.eye(n))
    x = np.linalg.solve(K, C.reshape(-1, order="F"))
    return x.reshape((n, m), order="F")


def fde2d_rhs(w, U: np.ndarray, m: int) -> np.ndarray:
    """C = U^{(m)} + Δt F^{(m+1)} (Eq. (sylv-timestepping) with the Δt of the
    implicit Euler step written out; F sampled at t_{m+1} = (m+1) Δt)."""
    return U + w.dt * w.source((m + 1) * w.dt)


def fde2d_run(w, steps: int | None = None, return_all: bool = False, base: int | None = None):
    """M implicit-Euler steps of the 2D problem, each one Sylvester equation
    A_x U^{(m+1)} + U^{(m+1)} A_yᵀ = U^{(m)} + Δt F^{(m+1)} (Eq. (sylv-timestepping)).
    base: see SchurSylvester (large N: LAPACK trsyl on the whole problem is
    memory-bound and takes tens of minutes per step at N = 4096)."""
    Ax = fd_operator(w.ops[0])
    Ay = fd_operator(w.ops[1])
    solver = SchurSylvester(Ax, Ay, base)
    U = w.u0.copy()
    M = w.steps if steps is None else steps
    hist = []
    for m in range(M):
        U = solver.solve(fde2d_rhs(w, U, m))
        if return_all:
            hist.append(U.copy())
    return (U, hist) if return_all else U


# ---------------------------------------------------------------------------
# §4.1-§4.2: the 2D time loop with the solution kept in factored form
# ---------------------------------------------------------------------------
def lowrank_from_dense(X: np.ndarray, eps: float):
    """X ≈ W Zᵀ from the SVD of X, singular values <= eps·σ_1 dropped (the
    ε-rank of §3 with ε relative to ||X||_2).  W carries the singular values."""
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    if s.size == 0 or s[0] == 0.0:
        return np.zeros((X.shape[0], 0)), np.zeros((X.shape[1], 0))
    r = int(np.sum(s > eps * s[0]))
    return U[:, :r] * s[:r], Vt[:r].T


def fde2d_rhs_factors(w, W: np.ndarray, Z: np.ndarray, m: int):
    """Outer factors (L, R) of C = U^{(m)} + Δt F^{(m+1)} = L Rᵀ, with
    U^{(m)} = W Zᵀ and F^{(m+1)} = F_L diag(w(t_{m+1})) F_Rᵀ (§4.1: both terms
    are low rank, so their sum is, before recompression)."""
    wt = w.source_weights((m + 1) * w.dt)
    return np.hstack([W, w.dt * w.src_left * wt]), np.hstack([Z, w.src_right])


def fde2d_lowrank_run(w, eps: float, steps: int | None = None):
    """The 2D scheme with U^{(m)} in factored form (§4.1, §4.2), step by step:
      1. factors of C = U^{(m)} + Δt F^{(m+1)} (fde2d_rhs_factors);
      2. recompression of the sum: reduced QR of both factors, SVD of the small
         core, singular values <= eps·||C||_2 dropped (truncate_lowrank);
      3. the Sylvester equation A_x X + X A_yᵀ = L Rᵀ (Eq. (sylv-timestepping)),
         solved here exactly by Bartels–Stewart in place of a low-rank solver
         that reaches the solution within its tolerance (§4.3);
      4. U^{(m+1)} = X truncated to its ε-rank (lowrank_from_dense).
    eps is relative to the 2-norm at both truncations (the paper states one
    tolerance for the solver and none for the recompressions).  Returns the
    factors (W, Z) of U^{(M)}."""
    solver = SchurSylvester(fd_operator(w.ops[0]), fd_operator(w.ops[1]))
    W, Z = lowrank_from_dense(w.u0, eps)
    M = w.steps if steps is None else steps
    for m in range(M):
        L, R = fde2d_rhs_factors(w, W, Z, m)
        _, Ru = np.linalg.qr(L)
        _, Rv = np.linalg.qr(R)
        normC = float(np.linalg.svd(Ru @ Rv.T, compute_uv=False)[0])
        L, R = truncate_lowrank(L, R, eps * normC)
        X = solver.solve(L @ R.T)
        W, Z = lowrank_from_dense(X, eps)
    return W, Z


# ---------------------------------------------------------------------------
# Eq. (system_FD) with time-dependent coefficients D_±^{(m)}
# ---------------------------------------------------------------------------
def _with_coeffs(op, dp: np.ndarray, dm: np.ndarray):
    return type(op)(op.N, op.alpha, op.h, op.dt, op.shift, dp, dm, op.leaf, op.tol)


def fde1d_run_tv(w, coeff, steps: int | None = None):
    """Implicit Euler with D_±^{(m)} sampled at the new time level t_m = m Δt
    (Eq. (system_FD)): every step forms A^{(m)} and solves
    A^{(m)} u^{(m)} = u^{(m-1)} + Δt f^{(m)} by dense LU.  coeff(t) -> (d_+, d_-)."""
    op = w.ops[0]
    u = w.u0.copy()
    M = w.steps if steps is None else steps
    for m in range(1, M + 1):
        t = m * w.dt
        dp, dm = coeff(t)
        u = solve_dense(fd_operator(_with_coeffs(op, dp, dm)), u + w.dt * w.source(t))
    return u


def fde2d_run_tv(w, coeff_x, coeff_y, steps: int | None = None):
    """The 2D step of Eq. (sylv-timestepping) with each side's coefficients at
    the new time level t_{m+1}: A_x^{(m+1)} U + U A_y^{(m+1)ᵀ} = U^{(m)} + Δt F^{(m+1)},
    a new pair of Schur forms per step (Bartels–Stewart)."""
    U = w.u0.copy()
    M = w.steps if steps is None else steps
    for m in range(M):
        t = (m + 1) * w.dt
        Ax = fd_operator(_with_coeffs(w.ops[0], *coeff_x(t)))
        Ay = fd_operator(_with_coeffs(w.ops[1], *coeff_y(t)))
        U = sylvester_bartels_stewart(Ax, Ay, fde2d_rhs(w, U, m))
    return U


# ---------------------------------------------------------------------------
# §2.2.2 and Eq. (fe-int): finite elements with hat functions on a uniform grid
# ---------------------------------------------------------------------------
def fe_weights(alpha: float, K: int) -> np.ndarray:
    """w_{-1}, w_0, ..., w_K (index k + 1) with (M_+)_{ij} = h^{1-α}/Γ(4-α) w_{i-j}
    for the left Riemann–Liouville stiffness of Eq. (fe-int) on hat functions
    φ_j (height 1, nodes x_j = j h).

    Derivation from Eq. (fe-int): g_j = I^{2-α} φ_j (the RL integral of the hat)
    is (1/h)/Γ(4-α) times the second difference of (x - x_{j-1} - m h)_+^{3-α}
    over m = 0, 1, 2; integrating φ_i g_j'' by parts twice turns φ_i'' into
    (δ_{x_{i-1}} - 2 δ_{x_i} + δ_{x_{i+1}})/h.  So w_k is the fourth central
    difference of t_+^γ, γ = 3 - α:
        w_k = Σ_{m=-2..2} (1, -4, 6, -4, 1)_m (k + m)_+^γ,
    zero for k <= -2.  Far from the diagonal the five terms cancel to
    O(k^{γ-4}) (the instability of the explicit symbol that the paper's
    footnote in its finite-element experiment points out), so for k >= 3
    the difference is evaluated as its expansion in powers of 1/k, which
    converges for k > 2:
        w_k = Σ_{n = 4, 6, ...} binom(γ, n) (2^{n+1} - 8) k^{γ-n}
    (odd moments of the symmetric stencil vanish; Σ_m c_m m^n = 2^{n+1} - 8
    for even n >= 2, which is 0 for n = 2), summed until the terms are below
    rounding."""
    g = 3.0 - alpha
    w = np.zeros(K + 2)
    stencil = (1.0, -4.0, 6.0, -4.0, 1.0)
    for idx in range(K + 2):
        k = idx - 1
        if k < 3:
            w[idx] = sum(c * (k + m) ** g for m, c in zip(range(-2, 3), stencil) if k + m > 0)
        else:
            s, n, binom = 0.0, 0, 1.0
            # binom(γ, n) by the recurrence binom(γ, n) = binom(γ, n-1) (γ - n + 1) / n
            while True:
                n += 1
                binom *= (g - n + 1) / n
                if n >= 4 and n % 2 == 0:
                    term = binom * (2.0 ** (n + 1) - 8.0) * k ** (g - n)
                    s += term
                    if abs(term) <= 1e-18 * abs(s):
                        break
            w[idx] = s
    return w


def fe_mass(N: int, h: float) -> np.ndarray:
    """M_{ij} = <φ_i, φ_j> for hat functions: h (1/6, 2/3, 1/6) tridiagonal."""
    return h * (np.diag(np.full(N, 2.0 / 3.0)) + np.diag(np.full(N - 1, 1.0 / 6.0), 1)
                + np.diag(np.full(N - 1, 1.0 / 6.0), -1))


def fe_stiffness(alpha: float, N: int, h: float) -> np.ndarray:
    """K = M_+ + M_-, the stiffness of ∂^α_+ + ∂^α_- with constant unit
    coefficients (§2.2.2); M_- = M_+ᵀ on a uniform grid (reflection x -> -x)."""
    w = fe_weights(alpha, N)
    Mp = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            if i - j >= -1:
                Mp[i, j] = w[i - j + 1]
    Mp *= h ** (1.0 - alpha) / math.gamma(4.0 - alpha)
    return Mp + Mp.T


def fe2d_operator(alpha: float, N: int, h: float, dt: float) -> np.ndarray:
    """One side of Eq. (sylv-timestepping-fe) brought to the form of
    Eq. (sylv-timestepping) by M^{-1} (the paper's first approach):
    M^{-1}(1/2 M - Δt K)."""
    M = fe_mass(N, h)
    return np.linalg.solve(M, 0.5 * M - dt * fe_stiffness(alpha, N, h))


# ---------------------------------------------------------------------------
# Structured operator application for residual certificates at large N
# ---------------------------------------------------------------------------
def _fftconv(a: np.ndarray, b: np.ndarray, axis: int) -> np.ndarray:
    """Linear convolution along `axis` by zero-padded FFT (numpy library FFT)."""
    n = a.shape[0] + b.shape[axis] - 1
    P = 1 << (n - 1).bit_length()
    fa = np.fft.rfft(a, P)
    fb = np.fft.rfft(b, P, axis=axis)
    shape = [1] * b.ndim
    shape[axis] = fa.shape[0]
    return np.fft.irfft(fb * fa.reshape(shape), P, axis=axis)


def apply_fd_operator_fft(op, X: np.ndarray, axis: int = 0) -> np.ndarray:
    """A applied along `axis` of X (A X for axis 0, X Aᵀ for axis 1) with
    A = s I + c (D_+ T + D_- Tᵀ), Eq. (system_FD).  (T x)_i = -Σ_m g_m x_{i+1-m}
    and (Tᵀ x)_i = -Σ_m g_m x_{i-1+m}, both as FFT convolutions."""
    N = op.N
    g = gl_weights(op.alpha, N + 1)
    c = fd_scale(op)
    Xa = np.moveaxis(X, axis, 0)
    conv = _fftconv(g, Xa, 0)
    Tx = -conv[1:N + 1]
    convr = _fftconv(g, Xa[::-1], 0)
    Ttx = -convr[N - np.arange(N)]
    dp = op.d_plus.reshape((-1,) + (1,) * (Xa.ndim - 1))
    dm = op.d_minus.reshape((-1,) + (1,) * (Xa.ndim - 1))
    Y = op.shift * Xa + c * (dp * Tx + dm * Ttx)
    return np.moveaxis(Y, 0, axis)


def sylvester_residual(opx, opy, X: np.ndarray, C: np.ndarray) -> float:
    """||C - A_x X - X A_yᵀ||_F / ||C||_F with both products taken structurally."""
    R = C - apply_fd_operator_fft(opx, X, 0) - apply_fd_operator_fft(opy, X, 1)
    return float(np.linalg.norm(R) / np.linalg.norm(C))


def min_row_sum(op) -> float:
    """Smallest row sum of A = s I + c (D_+ T + D_- Tᵀ) (Eq. (system_FD)), from
    A applied to the all-ones vector (structured product)."""
    return float(np.min(apply_fd_operator_fft(op, np.ones((op.N, 1)), 0)))


def sylvester_error_bound(opx, opy, r_maxabs: float) -> float:
    """Bound on max|X - X*| for A_x X + X A_yᵀ = C from the largest residual
    entry r_maxabs = max|C - A_x X - X A_yᵀ|.

    A_x and A_y are M-matrices with positive row sums (§2.2.1: non-positive
    off-diagonal entries, strict diagonal dominance), so the Kronecker matrix
    K = I ⊗ A_x + A_y ⊗ I of §4.2 is one too, with row sums
    rowsum_x(i) + rowsum_y(j) >= μ := min rowsum_x + min rowsum_y.  Then
    K^{-1} >= 0 and K^{-1} 1 <= 1/μ, so ||K^{-1}||_∞ <= 1/μ and
    max|X - X*| = ||K^{-1} vec R||_∞ <= r_maxabs / μ.  Over an implicit-Euler
    loop whose right-hand sides are formed from the loop's own states, the
    errors of the steps add: e_m = K^{-1}(e_{m-1} - r_m), and μ >= s_x + s_y = 1."""
    return r_maxabs / (min_row_sum(opx) + min_row_sum(opy))


def sym_part_exceeds(op, theta: float) -> bool:
    """True when the symmetric part (A + Aᵀ)/2 of A (Eq. (system_FD)) minus
    θ I is positive definite, i.e. λ_min((A + Aᵀ)/2) > θ: Cholesky
    factorisation (LAPACK potrf) of the dense matrix succeeds."""
    A = fd_operator(op)
    S = 0.5 * (A + A.T) - theta * np.eye(op.N)
    try:
        sla.cholesky(S, lower=True, check_finite=False)
    except np.linalg.LinAlgError:
        return False
    return True


def sylvester_error_bound_fro(r_fro: float, theta_x: float, theta_y: float) -> float:
    """Bound on ||X - X*||_F for A_x X + X A_yᵀ = C from ||R||_F, when
    λ_min((A_x + A_xᵀ)/2) >= θ_x and λ_min((A_y + A_yᵀ)/2) >= θ_y: the
    symmetric part of K = I ⊗ A_x + A_y ⊗ I (§4.2) is then >= (θ_x + θ_y) I,
    so ||K v|| ||v|| >= vᵀ K v >= (θ_x + θ_y) ||v||² and
    ||X - X*||_F = ||K^{-1} vec R|| <= ||R||_F / (θ_x + θ_y).  Over an
    implicit-Euler loop (e_m = K^{-1}(e_{m-1} - r_m)) with θ_x + θ_y >= 1
    the bounds of the steps add."""
    return r_fro / (theta_x + theta_y)
