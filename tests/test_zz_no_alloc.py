"""hodlr_matvec_noalloc (static device scratch, no allocation on the call
path) against hodlr_matvec, through the C ABI.  Collected last on purpose: it
must pass both alone in a fresh process and after every other GPU test."""
import numpy as np
import pytest

from paper_1804_05522_gb300 import binding
from paper_1804_05522_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# Same arithmetic as hodlr_matvec up to summation order (FP64).
RTOL = 1e-13

CASES = [
    dict(N=1024, alpha=1.5, leaf=64, tol=1e-10, shift=1.0, nrhs=3, pad=0),
    dict(N=1000, alpha=1.3, leaf=64, tol=1e-10, shift=0.5, nrhs=2, pad=7),   # uneven splits, ld > N
    dict(N=129, alpha=1.7, leaf=64, tol=1e-8, shift=1.0, nrhs=1, pad=0),     # ragged leaves 32/33
    dict(N=64, alpha=1.2, leaf=64, tol=1e-10, shift=1.0, nrhs=4, pad=0),     # single leaf, no levels
    dict(N=4096, alpha=1.5, leaf=128, tol=1e-10, shift=0.5, nrhs=5, pad=0),  # 2D workload's 1D operator
]


def _op(case):
    w = I.fd1d(N=case["N"], alpha=case["alpha"], steps=32, leaf=case["leaf"], tol=case["tol"])
    op = w.ops[0]
    op.shift = case["shift"]
    return op


def _dev(a, ld):
    N, n = a.shape
    buf = np.zeros((ld, n))
    buf[:N] = a
    return torch.from_numpy(buf.ravel(order="F").copy()).to("cuda")


def _host(t, N, ld, n):
    return t.cpu().numpy().reshape((ld, n), order="F")[:N]


@pytest.mark.parametrize("case", CASES)
def test_noalloc_matches_matvec_twice(lib, case):
    op = _op(case)
    h = lib.hodlr_build(lib.op_params(op))
    try:
        N, n, ld = op.N, case["nrhs"], op.N + case["pad"]
        X1 = _dev(I.random_matrix(N, n, seed=N + 1), ld)
        X2 = _dev(I.random_matrix(N, n, seed=N + 2), ld)
        ref1, ref2, y1, y2 = (torch.zeros_like(X1) for _ in range(4))
        lib.hodlr_matvec(h, X1.data_ptr(), ref1.data_ptr(), n, ld)
        lib.hodlr_matvec(h, X2.data_ptr(), ref2.data_ptr(), n, ld)
        torch.cuda.synchronize()
        # two calls in a row on one stream, different inputs
        y1.fill_(np.nan)
        y2.fill_(np.nan)
        torch.cuda.synchronize()
        lib.hodlr_matvec_noalloc(h, X1.data_ptr(), y1.data_ptr(), n, ld)
        free0 = torch.cuda.mem_get_info()[0]
        lib.hodlr_matvec_noalloc(h, X2.data_ptr(), y2.data_ptr(), n, ld)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0
        for y, ref in ((y1, ref1), (y2, ref2)):
            Y, R = _host(y, N, ld, n), _host(ref, N, ld, n)
            assert np.all(np.isfinite(Y))
            assert np.linalg.norm(Y - R) <= RTOL * np.linalg.norm(R)
        # padding rows between N and ld are left untouched
        if ld > N:
            assert np.all(np.isnan(y1.cpu().numpy().reshape((ld, n), order="F")[N:]))
    finally:
        lib.hodlr_free(h)


def test_noalloc_rejects_oversized_request(lib):
    op = _op(CASES[0])
    h = lib.hodlr_build(lib.op_params(op))
    try:
        X = torch.zeros(op.N, dtype=torch.float64, device="cuda")
        Y = torch.zeros_like(X)
        # nrhs far beyond what 2^19 scratch doubles hold; rejected before any launch
        s = lib.dll.hodlr_matvec_noalloc(h, X.data_ptr(), Y.data_ptr(), 65535, op.N, 0)
        assert s == binding.FDE_ERR_ARG
        assert "static scratch" in lib.last_error()
    finally:
        lib.hodlr_free(h)
