"""Writes the stored expected values of an oracle 2D time loop:
tests/golden/<workload>_oracle.txt.

The oracle's own trajectory (oracle.fde2d_run: one Bartels–Stewart solve of
Eq. (sylv-timestepping), §4.2, per implicit-Euler step) of a named workload is
run from U^(0) for max(steps) steps.  For every requested step m the file
keeps, of U^(m):
  - the Frobenius and max-abs norms;
  - the bilinear functionals u_kᵀ U^(m) v_k for the seeded unit vectors of
    inputs.projection_vectors(N, 8, seed=0);
  - the entries at the seeded index pairs of inputs.sample_points(N, S, seed=0).
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
    _, hist = O.fde2d_run(w, steps=steps[-1], return_all=True)
    wall = time.time() - t0
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_oracle.txt")
    with open(out, "w") as f:
        f.write(f"# Oracle 2D time loop ({name}: N={N}, alpha=({w.ops[0].alpha},{w.ops[1].alpha}), "
                f"dt={w.dt!r}, from U^(0)), written by tests/golden/make_fd2d_oracle.py\n")
        f.write(f"# command: python tests/golden/make_fd2d_oracle.py {name} "
                f"{','.join(map(str, steps))} {nsamp}   ({wall:.0f} s of oracle time)\n")
        f.write("# rows: norm <step> <fro> <maxabs> | proj <step> <k> <u_k^T U v_k> | "
                "entry <step> <i> <j> <U[i,j]>\n")
        for m in steps:
            U = hist[m - 1]
            f.write(f"norm {m} {np.linalg.norm(U):.17e} {np.max(np.abs(U)):.17e}\n")
            for k in range(N_PROJ):
                f.write(f"proj {m} {k} {Uv[:, k] @ U @ Vv[:, k]:.17e}\n")
            for i, j in zip(ii, jj):
                f.write(f"entry {m} {i} {j} {U[i, j]:.17e}\n")
    print(out, f"{wall:.0f} s")


if __name__ == "__main__":
    main()
