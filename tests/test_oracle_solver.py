"""Pins of the oracle's operators, block ILU(0) variants and FGMRES.

Pinned against: dense Kronecker assembly and a LAPACK solve (Sec. 4.1,
eq. big-irk / newton-system-2), the exact scalar IRK step R(z) u0 (Sec. 3,
Pade), the transformation W = (A (x) I) K (Sec. 4.1), exact LU on a block
tridiagonal chain (Sec. 4.2.1: ILU(0) drops nothing there), Alg. 2 and the
corrected Alg. 3 against the textbook ILU(0), and GMRES invariants.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import tableau
from paper_1701_07181_gb300 import inputs


def _problem(nbrs, m, s, dt=0.1, sigma=4.0, seed=3, per_stage_J=False):
    P = inputs.make_problem(nbrs, m, s, dt, sigma, seed)
    J = P.J
    if per_stage_J:
        rng = np.random.default_rng(seed + 100)
        J = np.stack([P.J + 0.05 * rng.standard_normal(P.J.shape) for _ in range(s)])
    return P, oracle.Problem(s, P.T, m, P.row_ptr, P.col_idx, J, P.M)


def _dense(P, pr):
    T, m, s = P.T, P.m, P.s
    n = T * m
    Md = np.zeros((n, n))
    for i in range(T):
        Md[i * m:(i + 1) * m, i * m:(i + 1) * m] = P.M[i]
    Js = []
    Jall = pr.J.reshape(-1, P.nnzb, m, m) if pr.jstride else pr.J.reshape(1, P.nnzb, m, m)
    for k in range(s):
        Jk = Jall[k if pr.jstride else 0]
        Jd = np.zeros((n, n))
        for i in range(T):
            for p in range(P.row_ptr[i], P.row_ptr[i + 1]):
                j = P.col_idx[p]
                Jd[i * m:(i + 1) * m, j * m:(j + 1) * m] = Jk[p]
        Js.append(Jd)
    return Md, Js


def _dense_transformed(P, pr, dt):
    Md, Js = _dense(P, pr)
    s, n = P.s, P.n
    B = np.kron(pr.Ainv, Md)
    for k in range(s):
        B[k * n:(k + 1) * n, k * n:(k + 1) * n] -= dt * Js[k]
    return B


def _dense_untransformed(P, pr, dt):
    Md, Js = _dense(P, pr)
    s, n = P.s, P.n
    B = np.kron(np.eye(s), Md)
    for k in range(s):
        for l in range(s):
            B[k * n:(k + 1) * n, l * n:(l + 1) * n] -= dt * pr.A[k, l] * Js[k]
    return B


MESHES = {
    "2d": lambda: inputs.mesh_2d_periodic(4, 3),
    "3d": lambda: inputs.mesh_3d_periodic(3),
    "chain": lambda: inputs.mesh_1d_chain(7),
}


@pytest.mark.parametrize("mesh", ["2d", "3d", "chain"])
@pytest.mark.parametrize("s", [1, 2, 3])
@pytest.mark.parametrize("per_stage", [False, True])
def test_operators_match_dense_kronecker(mesh, s, per_stage):
    P, pr = _problem(MESHES[mesh](), 3, s, per_stage_J=per_stage)
    x = np.random.default_rng(1).standard_normal(s * P.n)
    for form, dense in [(0, _dense_transformed), (1, _dense_untransformed)]:
        B = dense(P, pr, 0.37)
        y = pr.apply(x, 0.37, form=form)
        assert np.linalg.norm(y - B @ x) <= 1e-14 * np.linalg.norm(B @ x)


@pytest.mark.parametrize("pc", [oracle.PC_NONE, oracle.PC_UNCOUPLED, oracle.PC_STAGE_MAJOR,
                                oracle.PC_ELEMENT_MAJOR])
@pytest.mark.parametrize("s", [2, 3])
def test_gmres_matches_dense_solve(pc, s):
    """Sec. 4 / eq. big-irk: GMRES W vs pivoted dense solve of the full system."""
    P, pr = _problem(inputs.mesh_2d_periodic(4, 4), 6, s, dt=0.3)
    B = _dense_transformed(P, pr, 0.3)
    W = np.linalg.solve(B, P.R)
    out = pr.solve(P.R, 0.3, rtol=1e-12, precond=pc)
    assert out["rc"] == 0 and out["relres"] <= 1e-12
    kappa = np.linalg.cond(B)
    assert np.linalg.norm(out["x"] - W) <= 10 * 1e-12 * kappa * np.linalg.norm(W)


@pytest.mark.parametrize("pc", [oracle.PC_NONE, oracle.PC_STAGE_MAJOR, oracle.PC_ELEMENT_MAJOR])
def test_untransformed_gmres_matches_dense(pc):
    P, pr = _problem(inputs.mesh_3d_periodic(3), 4, 2, dt=0.2)
    B = _dense_untransformed(P, pr, 0.2)
    K = np.linalg.solve(B, P.R)
    out = pr.solve(P.R, 0.2, rtol=1e-12, form=oracle.FORM_UNTRANSFORMED, precond=pc)
    assert out["rc"] == 0
    assert np.linalg.norm(out["x"] - K) <= 1e-9 * np.linalg.norm(K)


@pytest.mark.parametrize("s", [2, 3, 4])
def test_transformed_equals_untransformed(s):
    """Sec. 4.1: W = (A (x) I_n) K, both systems solved tightly."""
    P, pr = _problem(inputs.mesh_2d_periodic(3, 3), 4, s, dt=0.5, per_stage_J=True)
    W = pr.solve(P.R, 0.5, rtol=1e-13, precond=oracle.PC_STAGE_MAJOR)["x"]
    K = pr.solve(P.R, 0.5, rtol=1e-13, form=1, precond=oracle.PC_ELEMENT_MAJOR)["x"]
    AK = (np.kron(pr.A, np.eye(P.n)) @ K)
    assert np.linalg.norm(W - AK) <= 1e-11 * np.linalg.norm(W)


@pytest.mark.parametrize("s,expect", [(1, 0.5), (2, 4.0 / 11.0), (3, 39.0 / 106.0)])
@pytest.mark.parametrize("pc", [oracle.PC_NONE, oracle.PC_UNCOUPLED, oracle.PC_STAGE_MAJOR])
def test_scalar_problem_gives_pade_value(s, expect, pc):
    """Whole pipeline on u' = lambda u (M = I, J = lambda I, no neighbours):
    the Newton system of eq. modified-IRK is B W = lambda u0 (1,..,1) and
    u1 = u0 + dt w_s = R(dt lambda) u0 (Sec. 4.1); at dt*lambda = -1 the
    (s-1, s) Pade value is 1/2, 4/11, 39/106."""
    T, m, dt, lam = 5, 2, 0.1, -10.0
    nbrs = [[] for _ in range(T)]
    rp, ci = inputs.bsr_pattern(nbrs)
    J = np.stack([lam * np.eye(m)] * T)
    M = np.stack([np.eye(m)] * T)
    pr = oracle.Problem(s, T, m, rp, ci, J, M)
    u0 = np.linspace(0.5, 2.0, T * m)
    R = np.concatenate([lam * u0] * s)
    W = pr.solve(R, dt, rtol=1e-14, precond=pc)["x"]
    u1 = u0 + dt * W[(s - 1) * T * m:]
    np.testing.assert_allclose(u1, expect * u0, rtol=1e-13, atol=0)


def _factor_product(rp, ci, F, b):
    """Dense L~ U~ from block factors (strict lower = L~, unit diagonal)."""
    nb = rp.size - 1
    L = np.eye(nb * b)
    U = np.zeros((nb * b, nb * b))
    for j in range(nb):
        for p in range(rp[j], rp[j + 1]):
            i = ci[p]
            blk = (slice(j * b, (j + 1) * b), slice(i * b, (i + 1) * b))
            if i < j:
                L[blk] = F[p]
            else:
                U[blk] = F[p]
    return L @ U


def _assembled_dense(rp, ci, V, b):
    nb = rp.size - 1
    D = np.zeros((nb * b, nb * b))
    for j in range(nb):
        for p in range(rp[j], rp[j + 1]):
            i = ci[p]
            D[j * b:(j + 1) * b, i * b:(i + 1) * b] = V[p]
    return D


@pytest.mark.parametrize("s", [1, 2, 3])
def test_ilu0_is_exact_lu_on_chain(s):
    """Sec. 4.2.1: on a non-periodic chain (block tridiagonal) ILU(0) drops
    nothing, so each shifted stage factor L~U~ equals d_k M - dt J."""
    P, pr = _problem(inputs.mesh_1d_chain(9), 5, s)
    alpha = tableau.shift_column_rule(pr.Ainv)
    for k in range(s):
        V = pr.assemble_shifted(k, pr.Ainv[k, k] + alpha[k], P.dt)
        F, _, _ = oracle.bilu0(P.row_ptr, P.col_idx, V)
        D = _assembled_dense(P.row_ptr, P.col_idx, V, P.m)
        LU = _factor_product(P.row_ptr, P.col_idx, F, P.m)
        assert np.abs(LU - D).max() <= 1e-13 * np.abs(D).max()


def test_single_stage_chain_converges_in_one_iteration():
    """s = 1 (Radau IIA s = 1 is backward Euler): the uncoupled preconditioner
    is the exact LU of the system on a chain, so GMRES takes one iteration."""
    P, pr = _problem(inputs.mesh_1d_chain(12), 6, 1)
    out = pr.solve(P.R, P.dt, rtol=1e-12, precond=oracle.PC_UNCOUPLED)
    assert out["iters"] == 1 and out["relres"] <= 1e-12


@pytest.mark.parametrize("s", [2, 3])
def test_element_major_ilu_on_chain_is_exact(s):
    """With (s*m)-blocks in element-major order the whole system is block
    tridiagonal on a chain, so its ILU(0) is exact: one GMRES iteration, for
    both formulations."""
    P, pr = _problem(inputs.mesh_1d_chain(10), 4, s)
    for form in (0, 1):
        out = pr.solve(P.R, P.dt, rtol=1e-12, form=form, precond=oracle.PC_ELEMENT_MAJOR)
        assert out["iters"] == 1, (form, out["iters"])


@pytest.mark.parametrize("mesh", ["2d", "3d"])
def test_alg2_equals_generic_ilu0(mesh):
    """Alg. 2 = textbook block ILU(0) (bitwise: same operations in the same
    order) on meshes where no two neighbours of an element are adjacent."""
    P, pr = _problem(MESHES[mesh](), 4, 2)
    V = pr.assemble_shifted(0, 5.0, P.dt)
    F1, d1, p1 = oracle.bilu0(P.row_ptr, P.col_idx, V)
    F2, d2, p2 = oracle.ilu_alg2(P.row_ptr, P.col_idx, V)
    np.testing.assert_array_equal(F1, F2)
    np.testing.assert_array_equal(d1, d2)
    np.testing.assert_array_equal(p1, p2)


def test_no_mutual_neighbours_on_generated_meshes():
    """The condition of Alg. 2 holds on the generated 2D and 3D meshes."""
    for nbrs in (inputs.mesh_2d_periodic(6, 5), inputs.mesh_3d_periodic(4)):
        sets = [set(x) for x in nbrs]
        for i, lst in enumerate(nbrs):
            for a in lst:
                for b in lst:
                    if a != b:
                        assert b not in sets[a]


@pytest.mark.parametrize("s", [2, 3, 4])
@pytest.mark.parametrize("mesh", ["2d", "3d"])
def test_alg3_corrected_equals_stage_major_ilu0(s, mesh):
    """Alg. 3 (corrected reading) = generic block ILU(0) of the stage-major
    assembled B of eq. big-irk, bitwise."""
    P, pr = _problem(MESHES[mesh](), 3, s)
    T, m = P.T, P.m
    rp2, ci2, V2 = pr.assemble_stage_major(P.dt)
    F, dlu, dpiv = oracle.bilu0(rp2, ci2, V2)
    # split storage for Alg. 3
    Bd = np.stack([pr.assemble_shifted(k, pr.Ainv[k, k], P.dt) for k in range(s)])
    Bo = np.zeros((s, s, T, m, m))
    for k in range(s):
        for l in range(s):
            if k != l:
                Bo[k, l] = pr.Ainv[k, l] * P.M
    Bd3, Bo3, dlu3, dpiv3 = oracle.ilu_alg3(s, P.row_ptr, P.col_idx, Bd, Bo)
    # compare block by block
    for k in range(s):
        for i in range(T):
            for p in range(rp2[k * T + i], rp2[k * T + i + 1]):
                col = ci2[p]
                l, j = divmod(int(col), T)
                if l == k:
                    q = P.row_ptr[i] + list(P.col_idx[P.row_ptr[i]:P.row_ptr[i + 1]]).index(j)
                    np.testing.assert_array_equal(F[p], Bd3[k, q])
                else:
                    np.testing.assert_array_equal(F[p], Bo3[k, l, i])
    np.testing.assert_array_equal(dlu, dlu3)
    np.testing.assert_array_equal(dpiv, dpiv3)


def test_gmres_invariants():
    """Residual estimate non-increasing within each cycle; at the end the true
    relative residual agrees with the final estimate; restarts happen."""
    P, pr = _problem(inputs.mesh_2d_periodic(5, 5), 6, 2, dt=0.5)
    restart = 8
    out = pr.solve(P.R, 0.5, rtol=1e-10, precond=oracle.PC_NONE, restart=restart, history=True)
    est = out["est"]
    assert out["cycles"] > 1 and out["relres"] <= 1e-10
    for c in range(out["cycles"]):
        seg = est[c * restart: (c + 1) * restart + 1]
        assert np.all(np.diff(seg) <= 1e-15 * seg[0]), c
    assert abs(out["relres"] - est[-1]) <= 1e-8 * max(est[-1], 1e-300) + 1e-14


def test_zero_rhs_and_initial_guess():
    P, pr = _problem(inputs.mesh_2d_periodic(3, 3), 3, 2)
    out = pr.solve(np.zeros_like(P.R), P.dt)
    assert out["iters"] == 0 and not out["x"].any()
    W = pr.solve(P.R, P.dt, rtol=1e-12)["x"]
    again = pr.solve(P.R, P.dt, rtol=1e-10, x0=W)
    assert again["iters"] == 0


def test_not_converged_is_reported():
    P, pr = _problem(inputs.mesh_2d_periodic(5, 5), 6, 3, dt=1.0)
    out = pr.solve(P.R, 1.0, rtol=1e-14, precond=oracle.PC_NONE, max_iter=3)
    assert out["rc"] == 1 and out["iters"] == 3 and out["relres"] > 1e-14


def test_preconditioner_quality_report(capsys):
    """Qualitative claims of Sec. 5.1.1 (reported, not asserted: they were made
    on flow problems, not on random blocks)."""
    P, pr = _problem(inputs.mesh_2d_periodic(8, 8), 12, 3, dt=0.5, sigma=4.0)
    res = {}
    for name, pc, shift in [("coupled", oracle.PC_STAGE_MAJOR, None),
                            ("uncoupled shifted", oracle.PC_UNCOUPLED, None),
                            ("uncoupled unshifted", oracle.PC_UNCOUPLED, np.zeros(3)),
                            ("none", oracle.PC_NONE, None)]:
        res[name] = pr.solve(P.R, 0.5, rtol=1e-8, precond=pc, shift=shift)["iters"]
    print("iterations:", res)
    assert all(v > 0 for v in res.values())
