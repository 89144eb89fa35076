"""Writes tests/golden/oracle_iterations_n1023.txt: the oracle's own FGMRES
iteration counts on the 2D n=1023 benchmark problem (omega = 128 pi, layered
velocity, PML 20, b = 4, the first right-hand sides of the seeded 32-source
batch), restart 40, relative residual 1e-6.

Calls only the oracle (and the seeded input generator).  The CPU reference arm
of bench.py reads the counts, so that its extrapolated solve time uses the
oracle's iteration count and not the GPU path's.  Run from the repository root:

    python tests/golden/make_oracle_iterations.py [number of right-hand sides]
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import fgmres, operator, sweeping  # noqa: E402


def main(nr: int) -> None:
    P = W.problem_2d_n1023_layered(nrhs=nr)
    t0 = time.perf_counter()
    pc = sweeping.Preconditioner(2, P.n, P.omega, P.c, P.pml, P.b, P.C)
    A = operator.helmholtz_matrix(2, P.n, P.omega, P.c, P.pml, P.C)
    _, its, res = fgmres.solve(pc, A, P.f, tol=P.tol, restart=40)
    wall = time.perf_counter() - t0
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_iterations_n1023.txt")
    with open(out, "w") as fh:
        fh.write("# Oracle FGMRES(40) iteration counts, tolerance 1e-6, on the 2D n=1023 benchmark problem\n")
        fh.write("# (omega = 128 pi, 16 smoothed random layers, PML 20, b = 4, seed 1504), right-hand sides\n")
        fh.write("# 0 .. %d of the benchmark batch.  Written by tests/golden/make_oracle_iterations.py\n" % (nr - 1))
        fh.write("# (oracle only; %.0f s of CPU).  columns: rhs iterations final_relative_residual\n" % wall)
        for r in range(nr):
            fh.write(f"{r} {int(its[r])} {float(res[r]):.3e}\n")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 2)
