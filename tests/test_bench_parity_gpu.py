"""The benchmarked configuration against the oracle, at the benchmark's size.

The 2D N = 4096 workload (α = 1.5, 1.5; Δt = 1/100; leaf 128) runs through the
time-loop runner with every default switch of the benchmark: FP32 inner solver
with blocked leaf Sylvester solves, the time-step predictor, exact residuals on
two consecutive steps of every 16 with double-float incremental residuals in
between, and FP32 last updates before them.  Its states are compared with

  - the oracle's own time loop (Bartels–Stewart per step, §4.2,
    Eq. (sylv-timestepping)): sampled entries, bilinear functionals and norms
    stored by tests/golden/make_fd2d_oracle.py at steps 2, 4, 8, 10, 16 (the
    last step of an incremental chain), 18 (a refresh step) and 20;
  - rigorous bounds on the error against the exact time loop, from the
    exact FP64 residuals of the steps: A_x and A_y are M-matrices (§2.2.1),
    so max|U - U*| <= max|R| / μ per step, μ the sum of their smallest row
    sums (oracle.sylvester_error_bound); and their symmetric parts exceed
    I/2, so ||U - U*||_F <= ||R||_F (oracle.sylvester_error_bound_fro).
    Both add over the loop.  The Frobenius bound must stay below the
    tolerance, and the oracle's values must lie inside both, widened by the
    oracle's own bounds of the same kind (stored with its values: with a
    condition near 1e4, its FP64 Bartels–Stewart is itself about 1e-11 off
    per step).

Above N = 4096 the same bound certifies the block-Toeplitz residual path."""
import os

import numpy as np
import pytest

from oracle import fde_oracle as O
from paper_1804_05522_gb300 import binding as B
from paper_1804_05522_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL = 1e-8  # relative error bound the refined FP32 path must meet at every checked step


def _golden(name):
    g = {}
    for line in open(os.path.join(GOLDEN, f"{name}_oracle.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        e = g.setdefault(int(f[1]), {"proj": {}, "ij": [], "val": []})
        if f[0] == "norm":
            e["fro"], e["maxabs"] = float(f[2]), float(f[3])
        elif f[0] == "bound":
            e["obound_max"], e["obound_fro"] = float(f[2]), float(f[3])
        elif f[0] == "proj":
            e["proj"][int(f[2])] = float(f[3])
        else:
            e["ij"].append((int(f[2]), int(f[3])))
            e["val"].append(float(f[4]))
    return g


def _mu(w):
    return O.min_row_sum(w.ops[0]) + O.min_row_sum(w.ops[1])


def _state(lib, r, N):
    X = torch.empty(N * N, dtype=torch.float64, device="cuda")
    lib.runner_state(r, X.data_ptr())
    torch.cuda.synchronize()
    return X.cpu().numpy().reshape((N, N), order="F")


def test_fd2d_n4096_default_run_vs_oracle(lib):
    name = "fd2d_n4096"
    w = I.WORKLOADS[name]()
    N = w.N
    gold = _golden(name)
    Uv, Vv = I.projection_vectors(N, 8, seed=0)
    mu = _mu(w)
    # λ_min of both symmetric parts above 1/2: the Frobenius bound applies
    # with θ_x + θ_y = 1 (oracle.sylvester_error_bound_fro)
    assert all(O.sym_part_exceeds(op, 0.5) for op in w.ops)
    U0 = torch.from_numpy(np.asarray(w.u0).ravel(order="F").copy()).to("cuda")
    r = lib.runner_create(lib.run_params(w, prec=B.FDE_FP32_REFINE), U0.data_ptr())
    try:
        bound = 0.0
        bound_fro = 0.0
        prev = w.u0.copy()
        for m in range(1, max(gold) + 1):
            lib.runner_advance(r, 1)
            rel, mx, fro = lib.runner_residual(r)
            bound += mx / mu
            bound_fro += O.sylvester_error_bound_fro(fro, 0.5, 0.5)
            if m in gold or m == 1:
                X = _state(lib, r, N)
            if m == 1:
                # the step's own Sylvester solve: error bound of this step
                assert mx / mu <= TOL * np.abs(X).max(), mx / mu
            if m == 1:
                # the device residual against the oracle's (CPU FFT operator)
                C = O.fde2d_rhs(w, prev, 0)
                Ro = C - O.apply_fd_operator_fft(w.ops[0], X, 0) - O.apply_fd_operator_fft(w.ops[1], X, 1)
                assert abs(mx - np.abs(Ro).max()) <= 1e-3 * np.abs(Ro).max() + 1e-11 * np.abs(C).max()
            if m not in gold:
                continue
            e = gold[m]
            ii = np.array([p[0] for p in e["ij"]])
            jj = np.array([p[1] for p in e["ij"]])
            err = X[ii, jj] - np.array(e["val"])
            rel_fro = np.sqrt(N * N * np.mean(err ** 2)) / e["fro"]
            assert rel_fro <= TOL, (m, rel_fro)
            assert np.abs(err).max() <= TOL * e["maxabs"], (m, np.abs(err).max())
            for k, v in e["proj"].items():
                assert abs(Uv[:, k] @ X @ Vv[:, k] - v) <= TOL * e["fro"], (m, k)
            assert abs(np.linalg.norm(X) - e["fro"]) <= TOL * e["fro"]
            # the accumulated residual bound is rigorous against the exact
            # loop, so the oracle's values must lie inside it (up to the
            # oracle's own rounding)
            assert np.abs(err).max() <= bound + e["obound_max"], (m, np.abs(err).max(), bound, e["obound_max"])
            # rigorous Frobenius bound against the exact loop, within the tolerance
            assert bound_fro <= TOL * e["fro"], (m, bound_fro / e["fro"])
            # the sampled entries estimate ||U - U_oracle||_F, so this one
            # allows for the sampling as well (a factor 2)
            assert rel_fro <= 2.0 * (bound_fro + e["obound_fro"]) / e["fro"], \
                (m, rel_fro, bound_fro / e["fro"], e["obound_fro"] / e["fro"])
    finally:
        lib.runner_free(r)


def test_fd2d_n16384_default_run_vs_oracle(lib):
    """The N = 16384 workload (α = 1.2, 1.8; leaf 256, block-Toeplitz FFT
    residual): its first two steps with every default switch against the
    oracle's Bartels–Stewart trajectory (tests/golden/fd2d_n16384_oracle.txt,
    46 minutes of oracle time).

    At this size ||A_y|| is near 1e7.  The FP64 Bartels–Stewart solution has a
    residual of a few 1e-7 ||C|| (backward stable: ~ε ||A|| ||X||), and even
    the evaluation of a residual in FP64 carries errors of order ε ||A||
    ||X||, so residual-based bounds certify about 1e-8 per step at best.  The
    refined GPU state's exact residual is at least ten times smaller than the
    oracle's; its summed Frobenius bound stays below 2e-8 per step; it agrees
    with the oracle's state within the tolerance plus the oracle's own bound;
    and their smooth components (bilinear functionals with the seeded unit
    vectors) agree to 1e-10."""
    name = "fd2d_n16384"
    w = I.WORKLOADS[name]()
    N = w.N
    gold = _golden(name)
    Uv, Vv = I.projection_vectors(N, 8, seed=0)
    assert all(O.sym_part_exceeds(op, 0.5) for op in w.ops)
    U0 = torch.from_numpy(np.asarray(w.u0).ravel(order="F").copy()).to("cuda")
    r = lib.runner_create(lib.run_params(w, prec=B.FDE_FP32_REFINE), U0.data_ptr())
    try:
        bound_fro, prev_obound = 0.0, 0.0
        for m in range(1, max(gold) + 1):
            lib.runner_advance(r, 1)
            rel, mx, fro = lib.runner_residual(r)
            bound_fro += O.sylvester_error_bound_fro(fro, 0.5, 0.5)
            if m not in gold:
                continue
            X = _state(lib, r, N)
            e = gold[m]
            # this step's residual against the oracle's (its bound's increment)
            assert fro <= 0.1 * (e["obound_fro"] - prev_obound), (m, fro, e["obound_fro"] - prev_obound)
            prev_obound = e["obound_fro"]
            assert bound_fro <= 2.0 * TOL * m * e["fro"], (m, bound_fro / e["fro"])
            ii = np.array([p[0] for p in e["ij"]])
            jj = np.array([p[1] for p in e["ij"]])
            err = X[ii, jj] - np.array(e["val"])
            rel_fro = np.sqrt(N * N * np.mean(err ** 2)) / e["fro"]
            assert rel_fro <= TOL + e["obound_fro"] / e["fro"], (m, rel_fro, e["obound_fro"] / e["fro"])
            assert abs(np.linalg.norm(X) - e["fro"]) <= TOL * e["fro"] + e["obound_fro"]
            for k, v in e["proj"].items():
                assert abs(Uv[:, k] @ X @ Vv[:, k] - v) <= 1e-10 * e["fro"], (m, k)
    finally:
        lib.runner_free(r)


def _certified_step(lib, N, steps, monkeypatch, resid=None):
    if resid:
        monkeypatch.setenv("FDE_RESID", resid)
    else:
        monkeypatch.delenv("FDE_RESID", raising=False)
    w = I.fd2d(N=N, alpha=(1.5, 1.5), steps=100, leaf=128)
    mu = _mu(w)
    U0 = torch.from_numpy(np.asarray(w.u0).ravel(order="F").copy()).to("cuda")
    r = lib.runner_create(lib.run_params(w, prec=B.FDE_FP32_REFINE), U0.data_ptr())
    try:
        bound = 0.0
        for m in range(1, steps + 1):
            if m == steps:
                prev = w.u0.copy() if m == 1 else _state(lib, r, N)
            lib.runner_advance(r, 1)
            rel, mx, fro = lib.runner_residual(r)
            bound += mx / mu
        X = _state(lib, r, N)
        # the last step's residual recomputed by the oracle on the CPU
        C = O.fde2d_rhs(w, prev, steps - 1)
        Ro = C - O.apply_fd_operator_fft(w.ops[0], X, 0) - O.apply_fd_operator_fft(w.ops[1], X, 1)
        assert abs(mx - np.abs(Ro).max()) <= 1e-3 * np.abs(Ro).max() + 1e-11 * np.abs(C).max()
        assert O.sylvester_error_bound(w.ops[0], w.ops[1], np.abs(Ro).max()) <= TOL * np.abs(X).max()
        return bound / np.abs(X).max(), X
    finally:
        lib.runner_free(r)


@pytest.mark.parametrize("resid", [None, "df", "fp64"])
def test_block_toeplitz_refined_step_certified(lib, monkeypatch, resid):
    """N = 6000 (2 blocks of the block-Toeplitz residual): one refined step
    from U^(0), certified by the oracle's residual and the M-matrix bound,
    with the default residual schedule, all double-float and all FP64."""
    b, _ = _certified_step(lib, 6000, 1, monkeypatch, resid)
    assert b <= TOL, b


def test_block_toeplitz_time_loop_certified(lib, monkeypatch):
    """N = 8200 (3 blocks, a ragged last one): 4 steps of the default time
    loop, the error against the exact loop bounded by the accumulated exact
    residuals."""
    b, _ = _certified_step(lib, 8200, 4, monkeypatch)
    assert b <= TOL, b
