"""Error paths of the C ABI on the GPU, every failure injected on the host
(non-finite inputs, iteration caps, a refused allocation, a wait limit far
below what the tensor-core pipeline needs): each call returns its status and
the library stays usable afterwards.  No test faults, traps or hangs the GPU:
an expired wait ends the kernel through its own bounded-wait exit."""
import numpy as np
import pytest

from oracle import fde_oracle as O
from paper_1804_05522_gb300 import binding as B
from paper_1804_05522_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float64).ravel(order="F").copy()).to("cuda")


def _status(fn, *args):
    try:
        fn(*args)
    except B.FdeError as e:
        return e.status
    return B.FDE_OK


def _pair(lib, w, prec):
    ax = lib.hodlr_build(lib.op_params(w.ops[0]))
    ay = lib.hodlr_build(lib.op_params(w.ops[1]))
    return ax, ay, lib.sylv_create(ax, ay, prec)


def _free(lib, ax, ay, s):
    lib.sylv_free(s)
    lib.hodlr_free(ax)
    lib.hodlr_free(ay)


@pytest.mark.parametrize("where", ["d_plus", "d_minus"])
def test_nonfinite_coefficient_is_numeric(lib, where):
    op = I.fd1d(N=256, leaf=32).ops[0]
    dp, dm = op.d_plus.copy(), op.d_minus.copy()
    (dp if where == "d_plus" else dm)[17] = np.nan
    op.d_plus, op.d_minus = dp, dm
    s, h = lib.hodlr_build_status(lib.op_params(op))
    assert s == B.FDE_ERR_NUMERIC and not h, lib.last_error()


def test_nonfinite_rhs_is_numeric(lib):
    w = I.fd2d(N=128, alpha=(1.3, 1.7), steps=50, leaf=32)
    ax, ay, s = _pair(lib, w, B.FDE_FP32_REFINE)
    try:
        C = O.fde2d_rhs(w, w.u0, 0)
        C[5, 9] = np.inf
        Cd = _dev(C)
        Xd = torch.zeros_like(Cd)
        assert _status(lib.sylv_step, s, Cd.data_ptr(), Xd.data_ptr(), 128) == B.FDE_ERR_NUMERIC
        # the handle still solves a finite right-hand side
        Cd = _dev(O.fde2d_rhs(w, w.u0, 0))
        relres, _ = lib.sylv_step(s, Cd.data_ptr(), Xd.data_ptr(), 128)
        assert relres < 1e-10
    finally:
        _free(lib, ax, ay, s)


def test_sweep_cap_is_noconv(lib):
    """One refinement sweep of the FP32 inner solver cannot reach the FP64
    stopping test from a zero initial guess."""
    w = I.fd2d(N=256, alpha=(1.3, 1.7), steps=50, leaf=64)
    ax, ay, s = _pair(lib, w, B.FDE_FP32_REFINE)
    try:
        r = lib.sylv_get_refine(s)
        r.max_sweeps = 1
        lib.sylv_set_refine(s, r)
        Cd = _dev(O.fde2d_rhs(w, w.u0, 0))
        Xd = torch.zeros_like(Cd)
        assert _status(lib.sylv_step, s, Cd.data_ptr(), Xd.data_ptr(), 256) == B.FDE_ERR_NOCONV
        r.max_sweeps = 12
        lib.sylv_set_refine(s, r)
        Xd.zero_()
        relres, sweeps = lib.sylv_step(s, Cd.data_ptr(), Xd.data_ptr(), 256)
        assert relres < 1e-10 and sweeps > 1
    finally:
        _free(lib, ax, ay, s)


def test_aca_rank_cap_is_noconv(lib):
    """A truncation tolerance far below rounding: the ACA of the top-level
    Toeplitz block can never meet it and stops at its rank cap."""
    op = I.fd1d(N=1024, leaf=64).ops[0]
    op.tol = 1e-300
    s, h = lib.hodlr_build_status(lib.op_params(op))
    assert s == B.FDE_ERR_NOCONV and not h, lib.last_error()


@pytest.mark.parametrize("after", [0, 3, 40])
def test_injected_allocation_failure(lib, after):
    """A refused device allocation anywhere in the setup of a 2D solver comes
    back as FDE_ERR_NOMEM and leaks nothing that later calls trip over."""
    w = I.fd2d(N=128, alpha=(1.3, 1.7), steps=50, leaf=32)
    lib.fail_alloc_after(after)
    try:
        st = B.FDE_OK
        try:
            ax, ay, s = _pair(lib, w, B.FDE_FP32_REFINE)
            _free(lib, ax, ay, s)
        except B.FdeError as e:
            st = e.status
    finally:
        lib.fail_alloc_after(-1)
    assert st == B.FDE_ERR_NOMEM
    ax, ay, s = _pair(lib, w, B.FDE_FP32_REFINE)
    _free(lib, ax, ay, s)


def test_expired_gemm_wait_is_reported(lib):
    """The tensor-core GEMM's mbarrier waits are bounded.  With the limit set
    to a few iterations they run out: the kernel exits through its failure
    path (drains its MMAs, frees its tensor memory), and sylv_step returns
    FDE_ERR_CUDA instead of a converged-looking result.  With the default
    limit restored the same handle solves correctly."""
    N = 256
    w = I.fd2d(N=N, alpha=(1.3, 1.7), steps=50, leaf=64)
    ax, ay, s = _pair(lib, w, B.FDE_FP32_REFINE)
    try:
        C = O.fde2d_rhs(w, w.u0, 0)
        Cd = _dev(C)
        Xd = torch.zeros_like(Cd)
        lib.set_wait_limit(2)
        try:
            st = _status(lib.sylv_step, s, Cd.data_ptr(), Xd.data_ptr(), N)
            torch.cuda.synchronize()
        finally:
            lib.set_wait_limit(0)
        assert st == B.FDE_ERR_CUDA, st
        assert "expired" in lib.last_error()
        Xd.zero_()
        relres, _ = lib.sylv_step(s, Cd.data_ptr(), Xd.data_ptr(), N)
        X = Xd.cpu().numpy().reshape((N, N), order="F")
        Xo = O.sylvester_bartels_stewart(O.fd_operator(w.ops[0]), O.fd_operator(w.ops[1]), C)
        assert np.linalg.norm(X - Xo) <= 1e-10 * np.linalg.norm(Xo) and relres < 1e-10
    finally:
        _free(lib, ax, ay, s)


def test_whole_step_graph_errors(lib):
    """Errors inside a whole-step graph (the device controller records them,
    the host reads them once the launched steps are collected): a non-finite
    source field gives FDE_ERR_NUMERIC, an expired tensor-core wait
    FDE_ERR_CUDA; afterwards the runner, reloaded, steps correctly."""
    N = 256
    w = I.fd2d(N=N, alpha=(1.3, 1.7), steps=50, leaf=64)
    U0 = _dev(w.u0)
    r = lib.runner_create(lib.run_params(w, prec=B.FDE_FP32_REFINE), U0.data_ptr())
    try:
        lib.runner_advance(r, 2)
        F = np.zeros((N, N))
        F[3, 4] = np.nan
        assert _status(lib.runner_step_source, r, F.ctypes.data, N) == B.FDE_ERR_NUMERIC
        lib.runner_load(r, U0.data_ptr(), 0)
        lib.set_wait_limit(2)
        try:
            st = _status(lib.runner_advance, r, 2)
        finally:
            lib.set_wait_limit(0)
        assert st == B.FDE_ERR_CUDA, st
        lib.runner_load(r, U0.data_ptr(), 0)
        lib.runner_advance(r, 3)
        X = torch.empty_like(U0)
        lib.runner_state(r, X.data_ptr())
        torch.cuda.synchronize()
        Xo = O.fde2d_run(w, steps=3)
        got = X.cpu().numpy().reshape((N, N), order="F")
        assert np.linalg.norm(got - Xo) <= 1e-8 * np.linalg.norm(Xo)
    finally:
        lib.runner_free(r)
