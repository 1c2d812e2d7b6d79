"""Edge cases of the CUDA path against the FP64 oracle (through the C ABI).

* the largest block size the boundary accepts (m = 128 with binary32
  factors: the factorisation falls back from the staged and shared-memory
  fast kernels to the per-entry ones, the sweeps run two block rows per CTA;
  binary64 factors are refused above m = 120);
* a single element (T = 1: the block diagonal alone, no neighbours);
* elements without neighbours next to a two-colourable mesh: such a row sits
  in the first level of both sweeps, so the two-launch preconditioner must
  not be chosen; the level sweeps give the oracle's answer;
* five Radau IIA stages (order 9).
Bars as in test_gpu_parity: binary64 path W within 1e-10 of the oracle with
the same iteration count (+-1), mixed path within 1e-6 of a tight oracle
solve, both at rtol 1e-8.
"""
import numpy as np
import pytest

import oracle
from paper_1701_07181_gb300 import inputs
from _parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _irk():
    from paper_1701_07181_gb300 import irk
    return irk


def check(P, ordering="natural", sweep="auto", expect_two_colour=None, fp64_factors=True):
    irk = _irk()
    ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M)
    W_tight = ref.solve(P.R, P.dt, rtol=1e-12)["x"]
    if fp64_factors:
        out = ref.solve(P.R, P.dt, rtol=1e-8)
        with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, factor_prec="fp64", krylov="fp64") as S:
            W, it, rr, rc = S.solve(P.R, P.dt, rtol=1e-8)
        assert rc == 0 and rr <= 1e-8
        assert abs(it - out["iters"]) <= 1, (it, out["iters"])
        assert rel(W, out["x"]) <= (1e-10 if it == out["iters"] else 1e-6)
    with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, factor_prec="fp32", krylov="df64",
                    ordering=ordering, sweep=sweep) as S:
        W, it, rr, rc = S.solve(P.R, P.dt, rtol=1e-8)
        st = S.stats()
    assert rc == 0 and rr <= 1e-8
    assert rel(W, W_tight) <= 1e-6
    if expect_two_colour is not None:
        assert st["sweep_two_colour"] == expect_two_colour


def test_largest_block_size():
    """m = 128 with binary32 factors (binary64 Krylov and double-float
    Krylov); binary64 factors stop at m = 120, and set-up says so."""
    irk = _irk()
    P = inputs.make_problem(inputs.mesh_1d_chain(6), 128, 2, 0.1, 4.0, seed=3)
    check(P, fp64_factors=False)
    ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M)
    W_tight = ref.solve(P.R, P.dt, rtol=1e-12)["x"]
    with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, factor_prec="fp32", krylov="fp64") as S:
        W, it, rr, rc = S.solve(P.R, P.dt, rtol=1e-8)
    assert rc == 0 and rr <= 1e-8 and rel(W, W_tight) <= 1e-6
    with pytest.raises(irk.IrkError) as e:
        irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, factor_prec="fp64", krylov="fp64")
    assert e.value.code == -1


def test_single_element():
    P = inputs.make_problem([[]], 20, 3, 0.2, 4.0, seed=4)
    check(P)


def test_isolated_elements_keep_level_sweeps():
    base = inputs.mesh_2d_periodic(7, 5)
    T0 = len(base)
    nbrs = [list(x) for x in base] + [[] for _ in range(3)]  # three elements without neighbours
    P = inputs.make_problem(nbrs, 12, 3, 0.1, 4.0, seed=6)
    assert P.T == T0 + 3
    check(P, ordering="multicolor", sweep="levels", expect_two_colour=0)
    # the same mesh without them takes the two-launch form
    Q = inputs.make_problem(base, 12, 3, 0.1, 4.0, seed=6)
    check(Q, ordering="multicolor", sweep="levels", expect_two_colour=1)


def test_five_stages():
    P = inputs.make_problem(inputs.mesh_2d_periodic(7, 5), 12, 5, 0.1, 4.0, seed=7)
    check(P, ordering="multicolor")
