"""Batches of independent instances (uneven N, alpha, coefficients; 1D and 2D)
advanced concurrently by host worker threads on separate streams, with the
leaf size autotuned per (dim, N) bucket: every instance against the oracle."""
import numpy as np
import pytest

from oracle import fde_oracle as O
from paper_1804_05522_gb300 import binding as B
from paper_1804_05522_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float64).ravel(order="F").copy()).to("cuda")


@pytest.mark.parametrize("autotune,threads", [(True, 3), (False, 1)])
def test_batch_matches_oracle(lib, autotune, threads):
    ws = I.batch(count=6, steps=20, sizes_log2=(6, 9), seed_index=1, leaf=32)
    steps = 4
    params = [lib.run_params(w, prec=B.FDE_FP32_REFINE if w.dim == 2 else B.FDE_FP64) for w in ws]
    U0 = [_dev(w.u0) for w in ws]
    b = lib.batch_create(params, [u.data_ptr() for u in U0], threads=threads, autotune=autotune)
    try:
        lib.batch_advance(b, steps)
        setup, tune, solve, inst = lib.batch_timing(b)
        assert inst == steps * len(ws) and solve > 0.0
        for i, w in enumerate(ws):
            n = w.N if w.dim == 1 else w.N * w.N
            out = torch.zeros(n, dtype=torch.float64, device="cuda")
            lib.batch_state(b, i, out.data_ptr())
            torch.cuda.synchronize()
            leaf, st = lib.batch_info(b, i)
            assert leaf in (8, 16, 32, 64, 128, 256)
            if w.dim == 1:
                ref = O.fde1d_run(w, steps=steps)
                err = np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(ref)
                assert err <= 1e-10, (i, w.N, err)
            else:
                ref = O.fde2d_run(w, steps=steps)
                got = out.cpu().numpy().reshape((w.N, w.N), order="F")
                err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
                assert err <= 1e-8, (i, w.N, err)
    finally:
        lib.batch_free(b)


def test_batch_bad_arguments(lib):
    w = I.fd1d(N=64)
    p = lib.run_params(w)
    U0 = _dev(w.u0)
    with pytest.raises(B.FdeError):
        lib.batch_create([p], [U0.data_ptr()], threads=0)
