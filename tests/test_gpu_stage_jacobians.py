"""One Jacobian per stage (Sec. 4.1: J_k evaluated at stage k's state;
irk_options.stage_jacobians = 1) against the oracle, whose operators take
the stages' Jacobians one after the other:

* operator product, both formulations, FP64 and double-float: <= 1e-13;
* FP64 preconditioner application of every kind the formulation allows:
  <= 1e-11 (the GPU's explicit D^{-1} vs the oracle's pivoted LU);
* solves at rtol 1e-8: binary64 iterations within one of the oracle's and
  W within 1e-10 of the oracle's W at the same rtol (same count); mixed
  precision W within 1e-6 of the oracle's tightly converged solution;
* the multi-request engine refuses the option.
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


def problem(s, m=12, seed=7, kind="2d"):
    nb = inputs.mesh_2d_periodic(7, 5) if kind == "2d" else inputs.mesh_3d_periodic(3, 3, 3)
    P = inputs.make_problem(nb, m, s, 0.2, 4.0, seed)
    rng = np.random.default_rng(seed + 100)
    # stage k's Jacobian: the shared one plus a stage-dependent perturbation
    Js = np.stack([P.J + 0.05 * (k + 1) * rng.standard_normal(P.J.shape) / np.sqrt(m) for k in range(s)])
    return P, Js


FORMS = {"transformed": oracle.FORM_TRANSFORMED, "untransformed": oracle.FORM_UNTRANSFORMED}


@pytest.mark.parametrize("krylov", ["fp64", "df64"])
@pytest.mark.parametrize("form", ["transformed", "untransformed"])
@pytest.mark.parametrize("s", [2, 3, 4])
def test_operator(krylov, form, s):
    irk = _irk()
    P, Js = problem(s)
    X = np.random.default_rng(1).standard_normal(s * P.T * P.m)
    ref = oracle.Problem(s, P.T, P.m, P.row_ptr, P.col_idx, Js, P.M).apply(X, 0.37, form=FORMS[form])
    with irk.Solver(s, P.T, P.m, P.row_ptr, P.col_idx, Js, P.M, precond="none", krylov=krylov, formulation=form,
                    stage_jacobians=True) as S:
        y = S.apply_operator(X, 0.37)
    assert rel(y, ref) <= 1e-13


@pytest.mark.parametrize("pc,form", [("uncoupled", "transformed"), ("coupled", "transformed"),
                                     ("coupled", "untransformed"), ("element", "transformed"),
                                     ("element", "untransformed")])
def test_fp64_preconditioner(pc, form):
    irk = _irk()
    P, Js = problem(3, m=8, kind="3d")
    opc = {"uncoupled": oracle.PC_UNCOUPLED, "coupled": oracle.PC_STAGE_MAJOR, "element": oracle.PC_ELEMENT_MAJOR}[pc]
    V = np.random.default_rng(2).standard_normal(3 * P.T * P.m)
    ref = oracle.Problem(3, P.T, P.m, P.row_ptr, P.col_idx, Js, P.M).precond_apply(V, 0.3, form=FORMS[form],
                                                                                     precond=opc)
    with irk.Solver(3, P.T, P.m, P.row_ptr, P.col_idx, Js, P.M, precond=pc, formulation=form, factor_prec="fp64",
                    krylov="fp64", stage_jacobians=True) as S:
        S.factor(0.3)
        z = S.apply_precond(V)
    assert rel(z, ref) <= 1e-11


@pytest.mark.parametrize("fprec,krylov,bar", [("fp64", "fp64", 1e-10), ("fp32", "df64", 1e-6)])
@pytest.mark.parametrize("form,pc", [("transformed", "uncoupled"), ("untransformed", "coupled")])
def test_solve(fprec, krylov, bar, form, pc):
    irk = _irk()
    P, Js = problem(3, m=12)
    ref = oracle.Problem(3, P.T, P.m, P.row_ptr, P.col_idx, Js, P.M)
    out = ref.solve(P.R, 0.2, rtol=1e-8, form=FORMS[form], precond=oracle.PC_UNCOUPLED if pc == "uncoupled"
                    else oracle.PC_STAGE_MAJOR)
    tight = ref.solve(P.R, 0.2, rtol=1e-13, form=FORMS[form], precond=oracle.PC_STAGE_MAJOR)["x"]
    with irk.Solver(3, P.T, P.m, P.row_ptr, P.col_idx, Js, P.M, precond=pc, formulation=form, factor_prec=fprec,
                    krylov=krylov, stage_jacobians=True) as S:
        W, it, rr, rc = S.solve(P.R, 0.2, rtol=1e-8)
    assert rc == 0 and rr <= 1e-8
    if fprec == "fp64":
        # same algorithm and arithmetic as the oracle at the same rtol
        assert abs(it - out["iters"]) <= 1
        if it == out["iters"]:
            assert rel(W, out["x"]) <= bar
    else:
        assert rel(W, tight) <= bar


def test_group_refuses_stage_jacobians():
    irk = _irk()
    import ctypes
    lib = irk.load()
    opt = irk.Options()
    lib.irk_default_options(ctypes.byref(opt))
    opt.factor_prec = 1
    opt.stage_jacobians = 1
    h = ctypes.c_void_p()
    rc = lib.irk_group_create(ctypes.byref(h), 3, None, 12, 100, 400, 4, ctypes.byref(opt))
    assert rc == -1  # IRK_ERR_INVALID
