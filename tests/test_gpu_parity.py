"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars (written in each test):
* operator product (Sec. 4.1, Table 2): ||y_gpu - y_ref|| / ||y_ref|| <= 1e-13,
  both for native FP64 and for double-float arithmetic;
* FP64 preconditioner (FP64 factors): <= 1e-11 relative (explicit D^{-1} on
  the GPU vs pivoted LU solves in the oracle: rounding only);
* FP32 / BF16 factors: the preconditioner is an approximation, pinned by the
  solve bar below;
* full solve at rtol 1e-8: FP64 path W within 1e-10 relative and iteration
  count within +-1 of the oracle; mixed paths W within 1e-6 relative.
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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def problem(kind, s, m=None, seed=11, dt=0.1, sigma=4.0):
    if kind == "2d":
        nb = inputs.mesh_2d_periodic(7, 5)  # 70 elements: several CTAs, ragged last group
    elif kind == "3d":
        nb = inputs.mesh_3d_periodic(3, 4, 3)
    elif kind == "chain":
        nb = inputs.mesh_1d_chain(37)  # boundary rows have one neighbour (ragged rows)
    elif kind == "c0":
        return inputs.config("c0", seed=seed)
    else:
        raise KeyError(kind)
    return inputs.make_problem(nb, m or 12, s, dt, sigma, seed)


def ref_of(P, J=None):
    return oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J if J is None else J, P.M)


def solver(P, host=False, **kw):
    irk = _irk()
    if host:
        return irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, **kw)
    return irk.Solver(P.s, P.T, P.m, dev(P.row_ptr), dev(P.col_idx), dev(P.J), dev(P.M), **kw)


@pytest.mark.parametrize("krylov", ["fp64", "df64", "fp64-dfop"])
@pytest.mark.parametrize("form", ["transformed", "untransformed"])
@pytest.mark.parametrize("kind,s,m", [("2d", 2, 12), ("3d", 3, 20), ("chain", 1, 7), ("chain", 5, 3),
                                      ("2d", 3, 40), ("c0", 2, 12), ("2d", 4, 1)])
def test_operator_matches_oracle(krylov, form, kind, s, m):
    P = problem(kind, s, m)
    ref = ref_of(P)
    X = np.random.default_rng(5).standard_normal(P.s * P.T * P.m)
    y_ref = ref.apply(X, 0.37, form=oracle.FORM_TRANSFORMED if form == "transformed" else 1)
    pc = "none"
    with solver(P, krylov=krylov, formulation=form, precond=pc) as S:
        y = S.apply_operator(dev(X), 0.37)
        torch.cuda.synchronize()
    assert rel(y, y_ref) <= 1e-13


def test_operator_host_memory_matches_device():
    P = problem("2d", 2)
    X = np.random.default_rng(1).standard_normal(P.s * P.T * P.m)
    with solver(P, host=True, krylov="df64") as S:
        y_host = S.apply_operator(X, 0.2)
    with solver(P, krylov="df64") as S:
        y_dev = S.apply_operator(dev(X), 0.2).cpu().numpy()
    np.testing.assert_array_equal(y_host, y_dev)


@pytest.mark.parametrize("pc,form", [("uncoupled", "transformed"), ("coupled", "transformed"),
                                     ("element", "transformed"), ("coupled", "untransformed"),
                                     ("element", "untransformed")])
@pytest.mark.parametrize("kind,s,m", [("2d", 2, 12), ("3d", 3, 8), ("chain", 3, 5)])
def test_fp64_preconditioner_matches_oracle(pc, form, kind, s, m):
    P = problem(kind, s, m)
    ref = ref_of(P)
    opc = {"uncoupled": oracle.PC_UNCOUPLED, "coupled": oracle.PC_STAGE_MAJOR,
           "element": oracle.PC_ELEMENT_MAJOR}[pc]
    f = 0 if form == "transformed" else 1
    V = np.random.default_rng(2).standard_normal(P.s * P.T * P.m)
    z_ref = ref.precond_apply(V, 0.3, form=f, precond=opc)
    with solver(P, precond=pc, formulation=form, factor_prec="fp64", krylov="fp64") as S:
        S.factor(0.3)
        z = S.apply_precond(dev(V))
        torch.cuda.synchronize()
    assert rel(z, z_ref) <= 1e-11


@pytest.mark.parametrize("fprec,bar", [("fp32", 1e-4), ("bf16", 5e-2)])
def test_low_precision_preconditioner_close_to_oracle(fprec, bar):
    P = problem("2d", 3, 12)
    ref = ref_of(P)
    V = np.random.default_rng(3).standard_normal(P.s * P.T * P.m)
    z_ref = ref.precond_apply(V, 0.3, precond=oracle.PC_UNCOUPLED)
    with solver(P, precond="uncoupled", factor_prec=fprec, krylov="df64") as S:
        S.factor(0.3)
        z = S.apply_precond(dev(V))
    assert rel(z, z_ref) <= bar


@pytest.mark.parametrize("pc,form", [("uncoupled", "transformed"), ("coupled", "transformed"),
                                     ("none", "transformed"), ("element", "untransformed")])
@pytest.mark.parametrize("kind,s,m", [("2d", 2, 12), ("3d", 3, 20), ("c0", 2, 12)])
def test_fp64_solve_matches_oracle(pc, form, kind, s, m):
    """P7: FP64 path, same iteration count +-1, W within 1e-10 of the oracle."""
    P = problem(kind, s, m)
    ref = ref_of(P)
    opc = {"uncoupled": oracle.PC_UNCOUPLED, "coupled": oracle.PC_STAGE_MAJOR, "none": oracle.PC_NONE,
           "element": oracle.PC_ELEMENT_MAJOR}[pc]
    f = 0 if form == "transformed" else 1
    out = ref.solve(P.R, P.dt, rtol=1e-8, form=f, precond=opc)
    with solver(P, precond=pc, formulation=form, factor_prec="fp64", krylov="fp64") as S:
        W, iters, relres, rc = S.solve(dev(P.R), P.dt, rtol=1e-8)
    assert rc == 0 and relres <= 1e-8
    assert abs(iters - out["iters"]) <= 1, (iters, out["iters"])
    # same Krylov path: rounding-level agreement; one iteration apart: both
    # iterates are within rtol of the solution
    assert rel(W, out["x"]) <= (1e-10 if iters == out["iters"] else 1e-6)


@pytest.mark.parametrize("fprec", ["fp32", "bf16", "fp64"])
@pytest.mark.parametrize("kind,s,m", [("2d", 3, 40), ("3d", 3, 20), ("c0", 2, 12), ("chain", 2, 9)])
def test_mixed_solve_within_1e6_of_oracle(fprec, kind, s, m):
    """Double-float Krylov + low-precision factors: W within 1e-6 relative of
    the FP64 oracle (solved tightly) at rtol 1e-8."""
    P = problem(kind, s, m)
    ref = ref_of(P)
    W_ref = ref.solve(P.R, P.dt, rtol=1e-12)["x"]
    with solver(P, precond="uncoupled", factor_prec=fprec, krylov="df64") as S:
        W, iters, relres, rc = S.solve(dev(P.R), P.dt, rtol=1e-8)
    assert rc == 0 and relres <= 1e-8
    assert rel(W, W_ref) <= 1e-6


@pytest.mark.parametrize("fprec", ["fp32", "bf16"])
@pytest.mark.parametrize("kind,s,m", [("2d", 3, 40), ("3d", 3, 20), ("c0", 2, 12)])
def test_split_precision_solve(fprec, kind, s, m):
    """Binary64 Krylov vectors, Gram-Schmidt and residual with the operator
    product alone in double-float (krylov="fp64-dfop"): W within 1e-6 of
    the FP64 oracle at rtol 1e-8, and the iteration count of the binary64
    path with the same factors within one."""
    P = problem(kind, s, m)
    ref = ref_of(P)
    W_ref = ref.solve(P.R, P.dt, rtol=1e-12)["x"]
    its = []
    for kry in ("fp64-dfop", "fp64"):
        with solver(P, precond="uncoupled", factor_prec=fprec, krylov=kry) as S:
            W, iters, relres, rc = S.solve(dev(P.R), P.dt, rtol=1e-8)
        assert rc == 0 and relres <= 1e-8
        assert rel(W, W_ref) <= 1e-6
        its.append(iters)
    assert abs(its[0] - its[1]) <= 1, its


@pytest.mark.parametrize("krylov", ["fp64", "df64", "fp64-dfop"])
@pytest.mark.parametrize("s,expect", [(1, 0.5), (2, 4.0 / 11.0), (3, 39.0 / 106.0)])
def test_scalar_problem_pade_on_gpu(krylov, s, expect):
    """u' = lambda u with dt*lambda = -1: u1 = u0 + dt w_s = R(-1) u0 (Sec. 4.1)."""
    T, m, dt, lam = 33, 2, 0.1, -10.0
    rp, ci = inputs.bsr_pattern([[] for _ in range(T)])
    J = np.stack([lam * np.eye(m)] * T)
    M = np.stack([np.eye(m)] * T)
    u0 = np.linspace(0.5, 2.0, T * m)
    R = np.concatenate([lam * u0] * s)
    irk = _irk()
    with irk.Solver(s, T, m, dev(rp), dev(ci), dev(J), dev(M), krylov=krylov) as S:
        W, iters, relres, rc = S.solve(dev(R), dt, rtol=1e-14)
    W = W.cpu().numpy()
    u1 = u0 + dt * W[(s - 1) * T * m:]
    tol = 1e-13 if krylov == "fp64" else 1e-12
    np.testing.assert_allclose(u1, expect * u0, rtol=tol, atol=0)


def test_transformed_equals_untransformed_on_gpu():
    """Sec. 4.1: W = (A (x) I) K from the two formulations on the GPU."""
    P = problem("2d", 3, 6)
    ref = ref_of(P)
    with solver(P, precond="coupled", krylov="fp64") as S:
        W, *_ = S.solve(dev(P.R), 0.5, rtol=1e-12)
    with solver(P, precond="element", formulation="untransformed", krylov="fp64") as S:
        K, *_ = S.solve(dev(P.R), 0.5, rtol=1e-12)
    K = K.cpu().numpy()
    AK = np.kron(ref.A, np.eye(P.n)) @ K
    assert rel(W, AK) <= 1e-10


def test_deterministic():
    P = problem("2d", 3, 12)
    with solver(P, precond="uncoupled", factor_prec="fp32", krylov="df64") as S:
        W1, *_ = S.solve(dev(P.R), 0.2)
        W2, *_ = S.solve(dev(P.R), 0.2)
    assert torch.equal(W1, W2)


def test_zero_rhs_and_not_converged():
    P = problem("2d", 2, 12)
    with solver(P, precond="uncoupled", krylov="df64", factor_prec="fp32", max_iter=2) as S:
        W, iters, relres, rc = S.solve(dev(np.zeros_like(P.R)), 0.1)
        assert rc == 0 and iters == 0 and not W.any()
        W, iters, relres, rc = S.solve(dev(P.R), 0.1, rtol=1e-14)
        assert rc == 1 and iters == 2 and relres > 1e-14


def test_singular_block_reported():
    P = problem("2d", 2, 4)
    irk = _irk()
    J = np.zeros_like(P.J)
    M = np.zeros_like(P.M)
    with solver(P, precond="uncoupled") as S:
        S.update_values(dev(J), dev(M))
        with pytest.raises(irk.IrkError) as e:
            S.factor(0.1)
        assert e.value.code == -3


def test_invalid_pattern_rejected():
    P = problem("2d", 2, 4)
    irk = _irk()
    ci = P.col_idx.copy()
    ci[0], ci[1] = ci[1], ci[0]  # unsorted row
    with pytest.raises(irk.IrkError) as e:
        irk.Solver(P.s, P.T, P.m, P.row_ptr, ci, P.J, P.M)
    assert e.value.code == -1


def test_precond_before_factor_is_state_error():
    P = problem("2d", 2, 4)
    irk = _irk()
    with solver(P, precond="uncoupled") as S:
        with pytest.raises(irk.IrkError) as e:
            S.apply_precond(dev(P.R))
        assert e.value.code == -7


@pytest.mark.parametrize("fprec,krylov", [("fp64", "fp64"), ("fp32", "df64")])
def test_large_blocks_3d_p3(fprec, krylov):
    """m = 100 (3D P3 x 5 variables): the factor and sweep kernels fall back to
    fewer buffers / warps per CTA to fit shared memory."""
    P = inputs.make_problem(inputs.mesh_3d_periodic(3), 100, 2, 0.1, 6.0, 17)
    ref = ref_of(P)
    W_ref = ref.solve(P.R, P.dt, rtol=1e-12)["x"]
    with solver(P, precond="uncoupled", factor_prec=fprec, krylov=krylov) as S:
        W, iters, relres, rc = S.solve(dev(P.R), P.dt, rtol=1e-8)
    assert rc == 0 and relres <= 1e-8
    assert rel(W, W_ref) <= 1e-6
