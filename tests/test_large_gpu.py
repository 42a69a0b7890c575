"""N > 4096: the structured residual switches to block-Toeplitz FFTs (blocks of
4096 rows).  Checked against the oracle's FFT operator (itself pinned against
the dense operator) on ragged block counts; the refined steps that use it are
certified in tests/test_bench_parity_gpu.py."""
import numpy as np
import pytest

from oracle import fde_oracle as O
from paper_1804_05522_gb300 import binding as B
from paper_1804_05522_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float64).ravel(order="F").copy()).to("cuda")


def _host(t, m, n):
    return t.cpu().numpy().reshape((m, n), order="F")


class Pair:
    def __init__(self, lib, w, prec):
        self.lib = lib
        self.ax = lib.hodlr_build(lib.op_params(w.ops[0]))
        self.ay = lib.hodlr_build(lib.op_params(w.ops[1]))
        self.s = lib.sylv_create(self.ax, self.ay, prec)

    def close(self):
        self.lib.sylv_free(self.s)
        self.lib.hodlr_free(self.ax)
        self.lib.hodlr_free(self.ay)


@pytest.mark.parametrize("N", [4100, 8200])
def test_block_toeplitz_residual(lib, N):
    # 2 blocks (the second only 4 rows) and 3 blocks (ragged last block)
    w = I.fd2d(N=N, alpha=(1.2, 1.8), steps=20, leaf=128)
    P = Pair(lib, w, B.FDE_FP32_REFINE)
    try:
        X = I.random_matrix_fast(N, N, seed=21)
        C = I.random_matrix_fast(N, N, seed=22)
        Rd = torch.zeros(N * N, dtype=torch.float64, device="cuda")
        Cd, Xd = _dev(C), _dev(X)
        lib.sylv_residual(P.s, Cd.data_ptr(), Xd.data_ptr(), Rd.data_ptr(), N)
        torch.cuda.synchronize()
        AX = O.apply_fd_operator_fft(w.ops[0], X, 0)
        XA = O.apply_fd_operator_fft(w.ops[1], X, 1)
        Ro = C - AX - XA
        scale = np.linalg.norm(AX) + np.linalg.norm(XA)
        assert np.linalg.norm(_host(Rd, N, N) - Ro) <= 1e-13 * scale
    finally:
        P.close()
