"""Write tests/golden/oracle_iters_c1.txt: the oracle's FGMRES(30) iteration
counts for the 2D workload T=20000, m=40, s=3 (periodic 100x100 split grid,
seed 0) at dt in {0.01, 0.1, 1}, rtol 1e-8, uncoupled shifted block ILU(0)
(Sec. 4.3.2) with FP64 factors.  Calls only the oracle.  The benchmark's CPU
baseline extrapolates its bounded oracle sample with these counts.

Run: python tests/golden/make_oracle_iters.py
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1701_07181_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_iters_c1.txt")


def main():
    P = inputs.config("c1", seed=0)
    ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M)
    lines = ["# oracle FGMRES(30) iterations, c1 workload (T=20000, m=40, s=3, seed 0),",
             "# rtol 1e-8, uncoupled shifted block ILU(0), FP64; written by make_oracle_iters.py",
             "# dt iters relres seconds"]
    for dt in (0.01, 0.1, 1.0):
        t = time.time()
        out = ref.solve(P.R, dt, rtol=1e-8, precond=oracle.PC_UNCOUPLED)
        lines.append("%g %d %.3e %.1f" % (dt, out["iters"], out["relres"], time.time() - t))
        print(lines[-1], flush=True)
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
