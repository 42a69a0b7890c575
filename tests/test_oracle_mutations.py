"""The oracle's pins catch plausible mistakes: each case plants one mistake in
the oracle (on the CPU, for the duration of the test only) and checks that a
pin of tests/test_oracle_pins.py then fails."""
import copy
import math

import numpy as np
import pytest

from oracle import fde_oracle as O
import tests.test_oracle_pins as P

_orig = {name: getattr(O, name) for name in dir(O) if callable(getattr(O, name))}


def _gl_shifted_order(alpha, K):
    return _orig["gl_weights"](alpha - 0.01, K)


def _toeplitz_transposed(alpha, N):
    return _orig["gl_toeplitz"](alpha, N).T


def _operator_without_minus(op):
    o2 = copy.copy(op)
    o2.d_minus = 0.0 * op.d_minus
    return _orig["fd_operator"](o2)


def _scale_wrong_power(op):
    return _orig["fd_scale"](op) * op.h


def _bs_untransposed(A, B, C):
    return _orig["sylvester_bartels_stewart"](A, B.T, C)


def _rhs_old_level(w, U, m):
    return U + w.dt * w.source(m * w.dt)


def _fft_wrong_shift(op, X, axis=0):
    o2 = copy.copy(op)
    o2.shift = 2.0 * op.shift
    return _orig["apply_fd_operator_fft"](o2, X, axis)


def _aca_signed_pivot(row_fn, col_fn, m, n, abstol, maxrank):
    """ACA whose column pivot is the largest residual entry, not the largest
    magnitude (a dropped |.|), otherwise the oracle's sequence."""
    U, V, rows, cols = [], [], [], []
    used_r = np.zeros(m, dtype=bool)
    used_c = np.zeros(n, dtype=bool)
    i_star = 0
    while len(U) < maxrank:
        r = np.array(row_fn(i_star), dtype=float)
        for l in range(len(U)):
            r = r - U[l][i_star] * V[l]
        used_r[i_star] = True
        cand = np.where(used_c, -np.inf, r)
        j_star = int(np.argmax(cand))
        if r[j_star] == 0.0:
            free = np.flatnonzero(~used_r)
            if free.size == 0:
                break
            i_star = int(free[0])
            continue
        v = r / r[j_star]
        c = np.array(col_fn(j_star), dtype=float)
        for l in range(len(U)):
            c = c - U[l] * V[l][j_star]
        used_c[j_star] = True
        U.append(c)
        V.append(v)
        rows.append(i_star)
        cols.append(j_star)
        if np.sum(c * c) * np.sum(v * v) <= abstol * abstol:
            break
        absu = np.where(used_r, -1.0, np.abs(c))
        if absu.max() < 0.0:
            break
        i_star = int(np.argmax(absu))
    k = len(U)
    return (np.stack(U, 1) if k else np.zeros((m, 0)), np.stack(V, 1) if k else np.zeros((n, 0)), rows, cols, True)


def _truncate_scaled(U, V, abstol):
    a, b = _orig["truncate_lowrank"](U, V, abstol)
    return a, 1.0001 * b


def _beckermann_pi(N, eps):
    return 2 + 2 * math.ceil((2.0 / math.pi) * math.log(4.0 * N / math.pi) * math.log(16.0 / eps))



def _qsrank_T_full_eps(N, eps):
    return _orig["beckermann_bound"](N, eps)


def _qsrank_M_one_plus(N, eps, normM, normT, maxD):
    return _orig["qsrank_bound_M"](N, eps, normM, normT, maxD) - 2


def _qsrank_M_inverted(N, eps, normM, normT, maxD):
    return _orig["qsrank_bound_M"](N, eps, normT * maxD, normM, 1.0)


def _min_row_sum_max(op):
    return float(np.max(_orig["apply_fd_operator_fft"](op, np.ones((op.N, 1)), 0)))


def _sym_part_always(op, theta):
    return True

def _norm_squared(A, iters=30):
    return _orig["norm2_power"](A, iters) ** 2


def _tree_ceil_first(N, leaf):
    levels = [[(0, N)]]
    while max(hi - lo for lo, hi in levels[-1]) > leaf:
        nxt = []
        for lo, hi in levels[-1]:
            mid = lo + (hi - lo + 1) // 2
            nxt += [(lo, mid), (mid, hi)]
        levels.append(nxt)
    return levels


def _fe_gamma(alpha, N, h):
    return _orig["fe_stiffness"](alpha, N, h) * math.gamma(4 - alpha) / math.gamma(3 - alpha)


def _fe_lumped(N, h):
    return h * np.eye(N)


def _tv_old_level(w, cx, cy, steps=None):
    U = w.u0.copy()
    M = w.steps if steps is None else steps
    for m in range(M):
        t = m * w.dt
        Ax = O.fd_operator(O._with_coeffs(w.ops[0], *cx(t)))
        Ay = O.fd_operator(O._with_coeffs(w.ops[1], *cy(t)))
        U = O.sylvester_bartels_stewart(Ax, Ay, O.fde2d_rhs(w, U, m))
    return U


def _lowrank_unscaled(X, eps):
    W, Z = _orig["lowrank_from_dense"](X, eps)
    n = np.linalg.norm(W, axis=0)
    return W / np.where(n > 0, n, 1.0), Z


def _residual_untransposed(opx, opy, X, C):
    R = C - O.apply_fd_operator_fft(opx, X, 0) - X @ O.fd_operator(opy)
    return float(np.linalg.norm(R) / np.linalg.norm(C))


def _fde1d_old_level(w, steps=None):
    op = w.ops[0]
    A = O.fd_operator(op)
    u = w.u0.copy()
    M = w.steps if steps is None else steps
    for m in range(1, M + 1):
        u = O.solve_dense(A, u + w.dt * w.source((m - 1) * w.dt))
    return u


def _kron_swapped(A, B, C):
    n, m = C.shape
    K = np.kron(A, np.eye(m)) + np.kron(np.eye(n), B)
    return np.linalg.solve(K, C.reshape(-1, order="F")).reshape((n, m), order="F")


def _hodlr_reference_abs(A, leaf, eps, normA=None):
    return _orig["hodlr_reference"](A, leaf, eps, normA=1.0)


def _rhs_factors_old_level(w, W, Z, m):
    return _orig["fde2d_rhs_factors"](w, W, Z, m - 1)


def _fe2d_without_mass(alpha, N, h, dt):
    M = O.fe_mass(N, h)
    return 0.5 * np.eye(N) - dt * O.fe_stiffness(alpha, N, h)


def _fe_weights_series_sign(alpha, K):
    w = _orig["fe_weights"](alpha, K).copy()
    w[4:] = -w[4:]  # k >= 3: the series part
    return w


def _block_entries_shifted(g, N):
    N1, N2, row, col = _orig["toeplitz_lower_block_entries"](g, N)
    return N1, N2, (lambda i: -g[N1 + i - np.arange(N1)]), (lambda j: -g[N1 + np.arange(N2) - j])


def _schur_untransposed_init(self, A, B):
    _orig["SchurSylvester"].__init__(self, A, B.T)


def _eps_rank_scaled(Y, abstol):
    return _orig["eps_rank"](Y, 10.0 * abstol)


class _SchurUntransposed:
    def __init__(self, A, B):
        self.inner = _orig["SchurSylvester"](A, B.T)

    def solve(self, C):
        return self.inner.solve(C)


def _lowrank_run_absolute(w, eps, steps=None):
    return _orig["fde2d_lowrank_run"](w, eps * 1e-3, steps)


def _tv1d_old_level(w, coeff, steps=None):
    op = w.ops[0]
    u = w.u0.copy()
    M = w.steps if steps is None else steps
    for m in range(1, M + 1):
        dp, dm = coeff((m - 1) * w.dt)
        u = O.solve_dense(O.fd_operator(O._with_coeffs(op, dp, dm)), u + w.dt * w.source(m * w.dt))
    return u


def _solve_transposed(A, B):
    return _orig["solve_dense"](A.T, B)


def _qts_coupling_sign(S, R, F, base=128):
    """The recursive quasi-triangular stage with the S coupling added instead
    of subtracted, otherwise the oracle's recursion."""
    m, n = F.shape
    if m <= base and n <= base:
        return _orig["quasi_triangular_sylvester"](S, R, F, base)
    if m >= n:
        h = m // 2 + (1 if S[m // 2, m // 2 - 1] != 0.0 else 0)
        Y2 = _qts_coupling_sign(S[h:, h:], R, F[h:], base)
        Y1 = _qts_coupling_sign(S[:h, :h], R, F[:h] + S[:h, h:] @ Y2, base)
        return np.vstack([Y1, Y2])
    h = n // 2 + (1 if R[n // 2, n // 2 - 1] != 0.0 else 0)
    Y2 = _qts_coupling_sign(S, R[h:, h:], F[:, h:], base)
    Y1 = _qts_coupling_sign(S, R[:h, :h], F[:, :h] - Y2 @ R[:h, h:].T, base)
    return np.hstack([Y1, Y2])


def _qts_wrong_r_block(S, R, F, base=128):
    """The recursive quasi-triangular stage with the R coupling taken from the
    lower-left block of R (zero for a quasi-triangular R, so the coupling is
    dropped) instead of R12 transposed."""
    m, n = F.shape
    if m <= base and n <= base:
        return _orig["quasi_triangular_sylvester"](S, R, F, base)
    if m >= n:
        h = m // 2 + (1 if S[m // 2, m // 2 - 1] != 0.0 else 0)
        Y2 = _qts_wrong_r_block(S[h:, h:], R, F[h:], base)
        Y1 = _qts_wrong_r_block(S[:h, :h], R, F[:h] - S[:h, h:] @ Y2, base)
        return np.vstack([Y1, Y2])
    h = n // 2 + (1 if R[n // 2, n // 2 - 1] != 0.0 else 0)
    Y2 = _qts_wrong_r_block(S, R[h:, h:], F[:, h:], base)
    Y1 = _qts_wrong_r_block(S, R[:h, :h], F[:, :h] - Y2 @ R[h:, :h], base)
    return np.hstack([Y1, Y2])


def _qts_splits_2x2(S, R, F, base=128):
    """The recursive quasi-triangular stage cutting at k // 2 even inside a
    2 x 2 diagonal block (the subdiagonal entry is then lost from both halves)."""
    m, n = F.shape
    if m <= base and n <= base:
        return _orig["quasi_triangular_sylvester"](S, R, F, base)
    if m >= n:
        h = m // 2
        Y2 = _qts_splits_2x2(S[h:, h:], R, F[h:], base)
        Y1 = _qts_splits_2x2(S[:h, :h], R, F[:h] - S[:h, h:] @ Y2, base)
        return np.vstack([Y1, Y2])
    h = n // 2
    Y2 = _qts_splits_2x2(S, R[h:, h:], F[:, h:], base)
    Y1 = _qts_splits_2x2(S, R[:h, :h], F[:, :h] - Y2 @ R[:h, h:].T, base)
    return np.hstack([Y1, Y2])


MUTATIONS = [
    ("gl_weights", _gl_shifted_order, lambda: P.test_gl_first_weights_exact(1.5)),
    ("gl_toeplitz", _toeplitz_transposed, lambda: P.test_toeplitz_structure(1.3)),
    ("fd_operator", _operator_without_minus, lambda: P.test_fd_operator_sdd_and_signs(1.0)),
    ("fd_scale", _scale_wrong_power, P.test_manufactured_solution_first_order),
    ("sylvester_bartels_stewart", _bs_untransposed, P.test_bartels_stewart_vs_kronecker_random),
    ("fde2d_rhs", _rhs_old_level, P.test_fde2d_time_exact_linear_in_time),
    ("apply_fd_operator_fft", _fft_wrong_shift, P.test_fft_operator_matches_dense),
    ("aca_partial_pivot", _aca_signed_pivot, P.test_aca_hand_worked),
    ("truncate_lowrank", _truncate_scaled, P.test_truncate_lowrank_prescribed_spectrum),
    ("beckermann_bound", _beckermann_pi, lambda: P.test_beckermann_bound_on_psd_hankel(256)),
    ("norm2_power", _norm_squared, P.test_norm2_power),
    ("sym_part_exceeds", _sym_part_always, P.test_sym_part_and_frobenius_error_bound),
    ("min_row_sum", _min_row_sum_max, P.test_mmatrix_error_bound),
    ("qsrank_bound_T", _qsrank_T_full_eps, P.test_qsrank_bounds_hand_evaluated),
    ("qsrank_bound_M", _qsrank_M_one_plus, P.test_qsrank_bounds_hand_evaluated),
    ("qsrank_bound_M", _qsrank_M_inverted, P.test_qsrank_bounds_hand_evaluated),
    ("hodlr_tree", _tree_ceil_first, lambda: P.test_hodlr_tree(1000, 64)),
    ("fe_stiffness", _fe_gamma, P.test_fe_stiffness_by_quadrature),
    ("fe_mass", _fe_lumped, P.test_fe_stiffness_by_quadrature),
    ("fde2d_run_tv", _tv_old_level, P.test_time_dependent_coefficients_at_new_level),
    ("lowrank_from_dense", _lowrank_unscaled, P.test_lowrank_from_dense_prescribed_spectrum),
    ("sylvester_residual", _residual_untransposed, P.test_sylvester_residual_definition),
    ("fde1d_run", _fde1d_old_level, P.test_fde1d_time_exact_linear_in_time),
    ("sylvester_kron", _kron_swapped, P.test_bartels_stewart_vs_kronecker_random),
    ("hodlr_reference", _hodlr_reference_abs, P.test_hodlr_reference_known_ranks),
    ("fde2d_rhs_factors", _rhs_factors_old_level, P.test_rhs_factors_match_dense_rhs),
    ("fe2d_operator", _fe2d_without_mass, P.test_fe2d_operator_generalized_sylvester),
    ("fe_weights", _fe_weights_series_sign, lambda: P.test_fe_weights_against_high_precision(1.5)),
    ("toeplitz_lower_block_entries", _block_entries_shifted, lambda: P.test_aca_toeplitz_block(1.5, 512)),
    ("eps_rank", _eps_rank_scaled, P.test_eps_rank_prescribed_spectrum),
    ("SchurSylvester", _SchurUntransposed, P.test_schur_sylvester_reuse_vs_kronecker),
    ("fde2d_lowrank_run", _lowrank_run_absolute, P.test_lowrank_run_error_follows_eps),
    ("fde1d_run_tv", _tv1d_old_level, P.test_time_dependent_1d_coefficients_at_new_level),
    ("solve_dense", _solve_transposed, P.test_solve_dense_residual),
    ("quasi_triangular_sylvester", _qts_coupling_sign, P.test_quasi_triangular_sylvester_recursive_vs_kronecker),
    ("quasi_triangular_sylvester", _qts_wrong_r_block, P.test_quasi_triangular_sylvester_recursive_vs_kronecker),
    ("quasi_triangular_sylvester", _qts_splits_2x2, P.test_quasi_triangular_sylvester_recursive_vs_kronecker),
]


@pytest.mark.parametrize("name,mutant,pin", MUTATIONS, ids=[f"{m[0]}-{m[1].__name__}" for m in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, name, mutant, pin):
    monkeypatch.setattr(O, name, mutant)
    with pytest.raises(AssertionError):
        pin()
