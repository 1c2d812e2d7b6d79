"""Write tests/golden/oracle_w_c1.txt: samples of the oracle's tightly
converged stage solution W of the 2D workload T=20000, m=40, s=3 (periodic
100x100 split grid, seed 0) at dt in {0.01, 0.1, 1}, for the benchmark's
report of each precision variant's error against the FP64 oracle.

For every dt the oracle (FP64, uncoupled shifted block ILU(0) of Sec. 4.3.2,
FGMRES(30) of Sec. 4, multi-core build: the same algorithm and operations
per row, threads over rows, stages and inner products) is run to a true
relative residual of 1e-12.  Stored: ||W||_2, max|W|, the length N, and
W at SAMPLES indices drawn without replacement by numpy's PCG64 with seed
2024 (the same indices for every dt), plus the index of max|W|.  Calls only
the oracle.

Run: python tests/golden/make_oracle_w_c1.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1701_07181_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_w_c1.txt")
SAMPLES = 1024
SEED = 2024


def sample_indices(N):
    return np.sort(np.random.default_rng(SEED).choice(N, SAMPLES, replace=False))


def main():
    P = inputs.config("c1", seed=0)
    ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, omp=True)
    N = P.s * P.T * P.m
    idx = sample_indices(N)
    lines = ["# oracle W samples, c1 workload (T=20000, m=40, s=3, seed 0), FP64, uncoupled shifted",
             "# block ILU(0), FGMRES(30) to true relres 1e-12; written by make_oracle_w_c1.py",
             "# header per dt: dt <dt> iters <k> relres <r> N <N> norm2 <||W||> amax <max|W|> argmax <i>",
             "# then one line per sample: <index> <W[index]> (%d samples, PCG64 seed %d)" % (SAMPLES, SEED)]
    for dt in (0.01, 0.1, 1.0):
        t = time.time()
        out = ref.solve(P.R, dt, rtol=1e-12, precond=oracle.PC_UNCOUPLED)
        W = out["x"]
        amax = int(np.argmax(np.abs(W)))
        lines.append("dt %g iters %d relres %.3e N %d norm2 %.17g amax %.17g argmax %d" %
                     (dt, out["iters"], out["relres"], N, np.linalg.norm(W), abs(W[amax]), amax))
        lines.extend("%d %.17g" % (q, W[q]) for q in idx)
        print(dt, out["iters"], out["relres"], "%.1f s" % (time.time() - t), flush=True)
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
