"""Writes tests/golden/sympart.txt: for named 2D workloads, whether the
symmetric part of each side's operator A = I/2 + c (D_+ T + D_- Tᵀ)
(Eq. (system_FD), §4.2) exceeds θ = 1/2, i.e. λ_min((A + Aᵀ)/2) > 1/2, by
the oracle's Cholesky test.  When both sides pass, ||X - X*||_F <= ||R||_F
for every Sylvester step of the workload (oracle.sylvester_error_bound_fro
with θ_x + θ_y = 1).  Only the oracle and the seeded input generators are
called.

    python tests/golden/make_sympart.py fd2d_n2048 fd2d_n4096 fd2d_n16384
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fde_oracle as O  # noqa: E402
from paper_1804_05522_gb300 import inputs as I  # noqa: E402

THETA = 0.5


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sympart.txt")
    rows = {}
    if os.path.exists(out):
        for line in open(out):
            if line.strip() and not line.startswith("#"):
                f = line.split()
                rows[(f[0], f[1])] = line.rstrip("\n")
    for name in sys.argv[1:]:
        w = I.WORKLOADS[name]()
        for side, op in zip("xy", w.ops):
            t0 = time.time()
            ok = O.sym_part_exceeds(op, THETA)
            rows[(name, side)] = f"{name} {side} {THETA} {int(ok)}   # {time.time() - t0:.0f} s"
            print(rows[(name, side)], flush=True)
    with open(out, "w") as f:
        f.write("# lambda_min((A + A^T)/2) > theta for each side of named 2D workloads (oracle Cholesky test),\n")
        f.write("# written by tests/golden/make_sympart.py\n")
        f.write("# columns: workload side theta holds\n")
        for k in sorted(rows):
            f.write(rows[k] + "\n")


if __name__ == "__main__":
    main()
