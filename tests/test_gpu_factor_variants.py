"""Inversion kernels of the factorisation's diagonal blocks.

The register-row Gauss-Jordan (block sizes 12, 20, 24, 40, 50) and the
shared-memory one (any size; IRK_GJ_ROWS=0 selects it) implement the same
partial pivoting (largest magnitude among the rows not yet used as pivots);
their preconditioner applications agree to rounding, and the binary64 one
matches the oracle's pivoted-LU preconditioner (same two-colour elimination
order) to 1e-11.  A singular
diagonal block is reported by both.
"""
import numpy as np
import pytest

import oracle
from paper_1701_07181_gb300 import inputs

from test_oracle_ordering import greedy_colouring_order

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _irk():
    from paper_1701_07181_gb300 import irk
    return irk


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("m", [12, 20, 24, 40, 50])
@pytest.mark.parametrize("fprec,bar", [("fp32", 1e-5), ("fp64", 1e-12)])
def test_register_rows_inverse_matches_shared_memory(monkeypatch, m, fprec, bar):
    irk = _irk()
    P = inputs.make_problem(inputs.mesh_2d_periodic(6, 5), m, 2, 0.3, 4.0, seed=m)
    V = np.random.default_rng(3).standard_normal(P.s * P.T * P.m)
    out = []
    for rows in ("1", "0"):
        monkeypatch.setenv("IRK_GJ_ROWS", rows)
        with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, factor_prec=fprec,
                        krylov="fp64" if fprec == "fp64" else "df64", ordering="multicolor") as S:
            S.factor(0.3)
            out.append(S.apply_precond(V))
    assert rel(out[0], out[1]) <= bar
    if fprec == "fp64":
        # the oracle's ILU(0) in the same (two-colour) elimination order
        perm, _ = greedy_colouring_order(P.row_ptr, P.col_idx)
        ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M).precond_apply_ordered(V, 0.3, perm=perm)
        assert rel(out[0], ref) <= 1e-11


@pytest.mark.parametrize("rows", ["1", "0"])
def test_singular_block_reported(monkeypatch, rows):
    irk = _irk()
    monkeypatch.setenv("IRK_GJ_ROWS", rows)
    P = inputs.make_problem(inputs.mesh_2d_periodic(4, 4), 12, 1, 0.3, 4.0, seed=1)
    M = P.M.copy()
    J = P.J.copy()
    # element 4 (first colour, so its block is inverted by the inversion
    # kernel of level 0): d M_4 - dt J_44 = 0 for s = 1 (d = 1/a_11 = 1,
    # shift 0) at dt = 0.5, exactly (powers of two)
    d4 = int(np.nonzero((np.repeat(np.arange(P.T), np.diff(P.row_ptr)) == 4) & (P.col_idx == 4))[0][0])
    J[d4] = M[4] / 0.5
    with irk.Solver(1, P.T, P.m, P.row_ptr, P.col_idx, J, M, factor_prec="fp32", krylov="df64",
                    ordering="multicolor") as S:
        with pytest.raises(irk.IrkError) as e:
            S.factor(0.5)
    assert e.value.code == -3
