"""Inversion kernels of the factorisation's diagonal blocks.

The register-row Gauss-Jordan (block sizes 12, 20, 24, 40, 50) and the
shared-memory one (any size; the kernel option factor_gj_rows = 0 selects it) implement the same
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
from _parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _irk():
    from paper_1701_07181_gb300 import irk
    return irk


@pytest.mark.parametrize("m", [12, 20, 24, 40, 50])
@pytest.mark.parametrize("fprec,bar", [("fp32", 1e-5), ("fp64", 1e-12)])
def test_register_rows_inverse_matches_shared_memory(m, fprec, bar):
    irk = _irk()
    P = inputs.make_problem(inputs.mesh_2d_periodic(6, 5), m, 2, 0.3, 4.0, seed=m)
    V = np.random.default_rng(3).standard_normal(P.s * P.T * P.m)
    out = []
    for rows in (1, 0):
        with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, factor_prec=fprec,
                        krylov="fp64" if fprec == "fp64" else "df64", ordering="multicolor",
                        kernel_options={"factor_gj_rows": rows}) as S:
            S.factor(0.3)
            out.append(S.apply_precond(V))
    assert rel(out[0], out[1]) <= bar
    if fprec == "fp64":
        # the oracle's ILU(0) in the same (two-colour) elimination order
        perm, _ = greedy_colouring_order(P.row_ptr, P.col_idx)
        ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M).precond_apply_ordered(V, 0.3, perm=perm)
        assert rel(out[0], ref) <= 1e-11


@pytest.mark.parametrize("rows", [1, 0])
def test_singular_block_reported(rows):
    irk = _irk()
    P = inputs.make_problem(inputs.mesh_2d_periodic(4, 4), 12, 1, 0.3, 4.0, seed=1)
    M = P.M.copy()
    J = P.J.copy()
    # element 4 (first colour, so its block is inverted by the inversion
    # kernel of level 0): d M_4 - dt J_44 = 0 for s = 1 (d = 1/a_11 = 1,
    # shift 0) at dt = 0.5, exactly (powers of two)
    d4 = int(np.nonzero((np.repeat(np.arange(P.T), np.diff(P.row_ptr)) == 4) & (P.col_idx == 4))[0][0])
    J[d4] = M[4] / 0.5
    with irk.Solver(1, P.T, P.m, P.row_ptr, P.col_idx, J, M, factor_prec="fp32", krylov="df64",
                    ordering="multicolor", kernel_options={"factor_gj_rows": rows}) as S:
        with pytest.raises(irk.IrkError) as e:
            S.factor(0.5)
    assert e.value.code == -3


def _mesh(kind):
    return {"2d": inputs.mesh_2d_periodic(7, 5), "3d": inputs.mesh_3d_periodic(3, 4, 3),
            "chain": inputs.mesh_1d_chain(37)}[kind]


@pytest.mark.parametrize("kind,s,m,order", [("2d", 3, 40, "multicolor"), ("2d", 2, 12, "natural"),
                                            ("3d", 2, 20, "multicolor"), ("3d", 3, 50, "multicolor"),
                                            ("chain", 1, 24, "natural"), ("2d", 2, 16, "multicolor")])
def test_fused_products_match_per_entry_kernel(kind, s, m, order):
    """Whole-row staged products (every update of a lower block lands on the
    row's diagonal block: no three elements pairwise adjacent in these
    meshes), in the compile-time block-size form (m = 12, 20, 24, 40, 50;
    m = 16 takes the generic form) and the generic form (factor_fused = 1),
    against the per-entry product kernel, every level through the separate
    inversion kernel: they differ only in the summation order of the Schur
    update, so their preconditioner applications agree to binary32 rounding;
    with double-float Krylov the fused factors also reach rtol 1e-8."""
    irk = _irk()
    P = inputs.make_problem(_mesh(kind), m, s, 0.3, 4.0, seed=5)
    V = np.random.default_rng(4).standard_normal(P.s * P.T * P.m)
    out, fused = [], []
    for mode in ("compiled", "generic", "off"):
        ko = {"factor_gj_split_min": 1, "factor_fused": {"compiled": 2, "generic": 1, "off": 0}[mode]}
        with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, precond="uncoupled", factor_prec="fp32",
                        krylov="df64", ordering=order, kernel_options=ko) as S:
            S.factor(0.3)
            out.append(S.apply_precond(V))
            fused.append(S.stats()["factor_fused_levels"])
            if mode != "off":
                W, it, rr, rc = S.solve(P.R, 0.3, rtol=1e-8)
                assert rc == 0 and rr <= 1e-8
                ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M)
                assert np.linalg.norm(P.R - ref.apply(W, 0.3)) / np.linalg.norm(P.R) <= 1e-8
    assert fused[0] >= 1 and fused[1] == fused[0] and fused[2] == 0
    assert rel(out[0], out[2]) <= 1e-5
    assert rel(out[1], out[2]) <= 1e-5


def test_coupled_preconditioner_keeps_per_entry_kernel():
    """With three stages the stage blocks of one element are pairwise coupled
    in the stage-coupled preconditioner, so a row's stage-0 and stage-1 lower
    entries are adjacent, updates reach off-diagonal blocks and the
    staged-row kernel must not be chosen."""
    irk = _irk()
    P = inputs.make_problem(_mesh("2d"), 12, 3, 0.3, 4.0, seed=5)
    with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, precond="coupled", factor_prec="fp32",
                    krylov="df64", ordering="multicolor", kernel_options={"factor_gj_split_min": 1}) as S:
        S.factor(0.3)
        assert S.stats()["factor_fused_levels"] == 0
        W, it, rr, rc = S.solve(P.R, 0.3, rtol=1e-8)
    assert rc == 0 and rr <= 1e-8

