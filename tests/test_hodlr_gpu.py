"""GPU parity of the HODLR construction, factorisation and solve against the
CPU oracle (through the C ABI)."""
import numpy as np
import pytest

from oracle import fde_oracle as O
from paper_1804_05522_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    """Column-major device copy of a host matrix as a flat tensor."""
    return torch.from_numpy(np.asarray(a, dtype=np.float64).ravel(order="F").copy()).to("cuda")


def _host(t, m, n):
    return t.cpu().numpy().reshape((m, n), order="F")


def _build(lib, op):
    p = lib.op_params(op)
    h = lib.hodlr_build(p)
    return h


CASES = [
    dict(N=1024, alpha=1.5, leaf=64, tol=1e-10, shift=1.0),   # 1D workload shape
    dict(N=1000, alpha=1.3, leaf=64, tol=1e-10, shift=0.5),   # uneven splits
    dict(N=129, alpha=1.7, leaf=64, tol=1e-8, shift=1.0),     # ragged leaves 32/33
    dict(N=300, alpha=1.8, leaf=32, tol=1e-12, shift=0.5),
    dict(N=64, alpha=1.2, leaf=64, tol=1e-10, shift=1.0),     # single leaf, no levels
]


def _op(case, dt=1.0 / 32):
    w = I.fd1d(N=case["N"], alpha=case["alpha"], steps=int(round(1 / dt)), leaf=case["leaf"], tol=case["tol"])
    op = w.ops[0]
    op.shift = case["shift"]
    return op


@pytest.mark.parametrize("case", CASES)
def test_weights_tree_norm(lib, case):
    op = _op(case)
    h = _build(lib, op)
    try:
        g = lib.hodlr_get_weights(h, op.N)
        # bit-exact: same recurrence, same operation order
        np.testing.assert_array_equal(g, O.gl_weights(op.alpha, op.N + 1))
        info = lib.hodlr_get_info(h)
        tree = O.hodlr_tree(op.N, op.leaf)
        assert info.levels == len(tree) - 1
        lo, hi = lib.hodlr_get_tree(h, info.levels)
        flat = [n for lvl in tree for n in lvl]
        np.testing.assert_array_equal(lo, [a for a, b in flat])
        np.testing.assert_array_equal(hi, [b for a, b in flat])
        A = O.fd_operator(op)
        assert abs(info.norm2 - O.norm2_power(A)) <= 1e-12 * info.norm2
    finally:
        lib.hodlr_free(h)


@pytest.mark.parametrize("case", CASES[:4])
def test_aca_pivots_bitexact(lib, case):
    op = _op(case)
    h = _build(lib, op)
    try:
        info = lib.hodlr_get_info(h)
        rows, cols = lib.hodlr_get_aca_pivots(h)
        g = O.gl_weights(op.alpha, op.N + 1)
        N1, N2, row, col = O.toeplitz_lower_block_entries(g, op.N)
        U, V, orows, ocols, conv = O.aca_partial_pivot(row, col, N2, N1, info.aca_tol, min(N1, N2, 90))
        assert info.aca_rank == len(orows)
        np.testing.assert_array_equal(rows, orows)
        np.testing.assert_array_equal(cols, ocols)
        assert bool(info.aca_converged) == bool(conv)
    finally:
        lib.hodlr_free(h)


@pytest.mark.parametrize("case", CASES)
def test_hodlr_blocks_within_tolerance(lib, case):
    op = _op(case)
    h = _build(lib, op)
    try:
        info = lib.hodlr_get_info(h)
        N = op.N
        Ad = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        lib.hodlr_to_dense(h, Ad.data_ptr(), N)
        torch.cuda.synchronize()
        Ah = Ad.cpu().numpy().T  # column-major -> numpy (row index first)
        A = O.fd_operator(op)
        tree = O.hodlr_tree(N, op.leaf)
        abstol = op.tol * info.norm2
        for lvl in tree[:-1]:
            for lo, hi in lvl:
                mid = lo + (hi - lo) // 2
                for (r0, r1, c0, c1) in ((lo, mid, mid, hi), (mid, hi, lo, mid)):
                    err = np.linalg.norm(A[r0:r1, c0:c1] - Ah[r0:r1, c0:c1], 2)
                    assert err <= 1.01 * abstol, (lo, hi, err, abstol)
        for lo, hi in tree[-1]:
            np.testing.assert_allclose(Ah[lo:hi, lo:hi], A[lo:hi, lo:hi], rtol=1e-14, atol=1e-14 * info.norm2)
        # ranks respect the rank bound of Corollary cor:fd-qsrank
        if info.levels > 0:
            T = O.gl_toeplitz(op.alpha, N)
            bound = O.qsrank_bound_M(N, op.tol, np.linalg.norm(A, 2), np.linalg.norm(T, 2),
                                     max(op.d_plus.max(), op.d_minus.max()))
            assert info.kmax <= bound
    finally:
        lib.hodlr_free(h)


@pytest.mark.parametrize("case", CASES)
def test_hodlr_solve_and_matvec(lib, case):
    op = _op(case)
    h = _build(lib, op)
    try:
        lib.hodlr_factor(h)
        N = op.N
        info = lib.hodlr_get_info(h)
        A = O.fd_operator(op)
        B = I.random_matrix(N, 3, seed=N)
        Bd = _dev(B)
        Xd = torch.zeros_like(Bd)
        lib.hodlr_solve(h, Bd.data_ptr(), Xd.data_ptr(), 3, N)
        Yd = torch.zeros_like(Bd)
        lib.hodlr_matvec(h, Bd.data_ptr(), Yd.data_ptr(), 3, N)
        torch.cuda.synchronize()
        X = _host(Xd, N, 3)
        Y = _host(Yd, N, 3)
        # matvec: HODLR error is at most ε||A|| per block, summed over the levels
        eps = op.tol
        L = info.levels
        assert np.linalg.norm(Y - A @ B) <= (2 * L + 1) * eps * info.norm2 * np.linalg.norm(B) + 1e-13 * np.linalg.norm(A @ B)
        # solve: backward error of the HODLR solve against the exact operator
        R = A @ X - B
        assert np.linalg.norm(R) <= (2 * L + 2) * eps * info.norm2 * np.linalg.norm(X) + 1e-12 * np.linalg.norm(B)
        Xo = O.solve_dense(A, B)
        kappa = np.linalg.cond(A)
        assert np.linalg.norm(X - Xo) <= 10 * kappa * (2 * L + 2) * eps * np.linalg.norm(Xo) + 1e-12 * np.linalg.norm(Xo)
    finally:
        lib.hodlr_free(h)


@pytest.mark.parametrize("case", [CASES[1], CASES[2]])
def test_hodlr_solve_padded_leading_dimension(lib, case):
    """hodlr_solve with ldb > N, out of place and in place: the N rows match
    the dense solve within the HODLR backward-error bound, and the padding
    rows of the output are left as they were."""
    op = _op(case)
    h = _build(lib, op)
    try:
        lib.hodlr_factor(h)
        N, ld, nrhs = op.N, op.N + 9, 2
        info = lib.hodlr_get_info(h)
        A = O.fd_operator(op)
        B = I.random_matrix(N, nrhs, seed=N + 1)
        Bpad = np.full((ld, nrhs), 5.0)
        Bpad[:N] = B
        Xpad = np.full((ld, nrhs), -2.0)
        Bd, Xd = _dev(Bpad), _dev(Xpad)
        lib.hodlr_solve(h, Bd.data_ptr(), Xd.data_ptr(), nrhs, ld)  # out of place
        lib.hodlr_solve(h, Bd.data_ptr(), Bd.data_ptr(), nrhs, ld)  # in place
        torch.cuda.synchronize()
        bound = (2 * info.levels + 2) * op.tol * info.norm2
        for out, pad in ((_host(Xd, ld, nrhs), -2.0), (_host(Bd, ld, nrhs), 5.0)):
            X = out[:N]
            assert np.linalg.norm(A @ X - B) <= bound * np.linalg.norm(X) + 1e-12 * np.linalg.norm(B)
            assert np.all(out[N:] == pad)
    finally:
        lib.hodlr_free(h)


def test_alpha2_degenerate_case(lib):
    """α = 2, the upper end of the allowed orders: T is the second-difference
    matrix, the top-level block has a single nonzero, so ACA takes one term and
    then skips zero residual rows (the oracle's pivots, bit for bit), every
    off-diagonal block has rank exactly 1, and the solve matches the dense one."""
    w = I.fd1d(N=300, alpha=2.0, steps=32, leaf=32, tol=1e-10)
    op = w.ops[0]
    h = _build(lib, op)
    try:
        info = lib.hodlr_get_info(h)
        rows, cols = lib.hodlr_get_aca_pivots(h)
        g = O.gl_weights(op.alpha, op.N + 1)
        N1, N2, row, col = O.toeplitz_lower_block_entries(g, op.N)
        U, V, orows, ocols, conv = O.aca_partial_pivot(row, col, N2, N1, info.aca_tol, min(N1, N2, 90))
        assert info.aca_rank == len(orows) == 1 and bool(info.aca_converged) and conv
        np.testing.assert_array_equal(rows, orows)
        np.testing.assert_array_equal(cols, ocols)
        assert info.kmax == 1
        lib.hodlr_factor(h)
        N = op.N
        A = O.fd_operator(op)
        B = I.random_matrix(N, 2, seed=77)
        Bd = _dev(B)
        Xd = torch.zeros_like(Bd)
        lib.hodlr_solve(h, Bd.data_ptr(), Xd.data_ptr(), 2, N)
        torch.cuda.synchronize()
        X = _host(Xd, N, 2)
        Xo = O.solve_dense(A, B)
        assert np.linalg.norm(X - Xo) <= 1e-10 * np.linalg.norm(Xo)
    finally:
        lib.hodlr_free(h)
