"""Writes the stored expected values of an oracle 2D time loop:
tests/golden/<workload>_oracle.txt.

The oracle's own trajectory (oracle.fde2d_run: one Bartels–Stewart solve of
Eq. (sylv-timestepping), §4.2, per implicit-Euler step, its quasi-triangular
stage in the recursive block form with LAPACK trsyl on blocks of at most 256)
of a named workload is run from U^(0) for max(steps) steps.  For every requested step m the file
keeps, of U^(m):
  - the Frobenius and max-abs norms;
  - the bilinear functionals u_kᵀ U^(m) v_k for the seeded unit vectors of
    inputs.projection_vectors(N, 8, seed=0);
  - the entries at the seeded index pairs of inputs.sample_points(N, S, seed=0);
  - the oracle's own error bound against the exact loop: its FP64 residuals
    R_k = C_k - A_x U_k - U_k A_yᵀ (FFT operator, oracle.apply_fd_operator_fft)
    summed over steps k <= m as max|R_k| / μ (oracle.sylvester_error_bound)
    and ||R_k||_F / (θ_x + θ_y), θ = 1/2 (oracle.sylvester_error_bound_fro).
    At N = 4096 the Sylvester operator's condition (about 1e4) makes the
    oracle's own rounding about 1e-11 relative per step, which a comparison
    with another solver at that level has to allow for.
Only the oracle and the seeded input generators are called.

    python tests/golden/make_fd2d_oracle.py fd2d_n4096 4,8,10 2048
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import fde_oracle as O  # noqa: E402
from paper_1804_05522_gb300 import inputs as I  # noqa: E402

N_PROJ = 8


def main():
    name = sys.argv[1]
    steps = sorted(int(s) for s in sys.argv[2].split(","))
    nsamp = int(sys.argv[3]) if len(sys.argv) > 3 else 2048
    w = I.WORKLOADS[name]()
    N = w.N
    ii, jj = I.sample_points(N, nsamp, seed=0)
    Uv, Vv = I.projection_vectors(N, N_PROJ, seed=0)
    t0 = time.time()
    _, hist = O.fde2d_run(w, steps=steps[-1], return_all=True, base=256)
    wall = time.time() - t0
    # the oracle's own accumulated residual bounds
    bmax, bfro, prev = 0.0, 0.0, w.u0
    obound = {}
    for m in range(1, steps[-1] + 1):
        U = hist[m - 1]
        R = O.fde2d_rhs(w, prev, m - 1) - O.apply_fd_operator_fft(w.ops[0], U, 0) \
            - O.apply_fd_operator_fft(w.ops[1], U, 1)
        bmax += O.sylvester_error_bound(w.ops[0], w.ops[1], np.abs(R).max())
        bfro += O.sylvester_error_bound_fro(np.linalg.norm(R), 0.5, 0.5)
        obound[m] = (bmax, bfro)
        prev = U
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_oracle.txt")
    with open(out, "w") as f:
        f.write(f"# Oracle 2D time loop ({name}: N={N}, alpha=({w.ops[0].alpha},{w.ops[1].alpha}), "
                f"dt={w.dt!r}, from U^(0)), written by tests/golden/make_fd2d_oracle.py\n")
        f.write(f"# command: python tests/golden/make_fd2d_oracle.py {name} "
                f"{','.join(map(str, steps))} {nsamp}   ({wall:.0f} s of oracle time)\n")
        f.write("# rows: norm <step> <fro> <maxabs> | bound <step> <max-abs bound> <Frobenius bound> | "
                "proj <step> <k> <u_k^T U v_k> | entry <step> <i> <j> <U[i,j]>\n")
        for m in steps:
            U = hist[m - 1]
            f.write(f"norm {m} {np.linalg.norm(U):.17e} {np.max(np.abs(U)):.17e}\n")
            f.write(f"bound {m} {obound[m][0]:.6e} {obound[m][1]:.6e}\n")
            for k in range(N_PROJ):
                f.write(f"proj {m} {k} {Uv[:, k] @ U @ Vv[:, k]:.17e}\n")
            for i, j in zip(ii, jj):
                f.write(f"entry {m} {i} {j} {U[i, j]:.17e}\n")
    print(out, f"{wall:.0f} s")


if __name__ == "__main__":
    main()
