"""One factorisation + solve of a mid-size stage system, for profiler captures.

The benchmark workload (20000 triangles, m = 40, s = 3) holds about 5 GB on
the device and its level kernels run for milliseconds, which is too large for
multi-pass counter collection.  This driver runs the same kernels on a
smaller periodic split-quad mesh (default 60 x 60 quads = 7200 triangles,
m = 40, s = 3: inputs still larger than L2) with the benchmark's options
(FP32 factors, double-float Krylov vectors, two-colour ordering), so DRAM
counters per launch can be scaled to the full workload by the element count.

Usage: ``python profile_case.py [--nx 60 --ny 60 --m 40 --s 3 --solves 2 --matvec-variant V]``
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=60)
    ap.add_argument("--ny", type=int, default=60)
    ap.add_argument("--m", type=int, default=40)
    ap.add_argument("--s", type=int, default=3)
    ap.add_argument("--solves", type=int, default=2)
    ap.add_argument("--ordering", default="multicolor")
    ap.add_argument("--matvec-variant", type=int, default=-1,
                    help="pin the operator-product launch variant (-1: autotuned)")
    args = ap.parse_args(argv)
    import torch

    from paper_1701_07181_gb300 import inputs, irk
    P = inputs.make_problem(inputs.mesh_2d_periodic(args.nx, args.ny), args.m, args.s, 0.1, 6.0, seed=0)

    def dev(a):
        return torch.as_tensor(np.ascontiguousarray(a)).cuda()

    with irk.Solver(P.s, P.T, P.m, dev(P.row_ptr), dev(P.col_idx), dev(P.J), dev(P.M), factor_prec="fp32",
                    krylov="df64", timing=True, ordering=args.ordering,
                    kernel_options={"matvec_variant": args.matvec_variant}) as S:
        R = dev(P.R)
        for k in range(args.solves):
            W, it, rr, rc = S.solve(R, 0.1 * (k + 1))
            st = S.stats()
            print("T=%d m=%d s=%d dt=%.2f iters=%d relres=%.1e rc=%d factor_ms=%.3f matvec_variant=%d"
                  % (P.T, P.m, P.s, 0.1 * (k + 1), it, rr, rc, st["factor_ms"], st["matvec_variant"]))
            if rc not in (0, 1):
                raise SystemExit(1)


if __name__ == "__main__":
    main()
