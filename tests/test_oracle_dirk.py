"""Pins of the DIRK comparison schemes and of the oracle's Runge-Kutta steps
(Sec. 3, Table 1, App. A).

Independent checks: the order conditions of every rooted tree (elementary
weights), the stage order, the implicit-stage count and the leading error
coefficient printed in Table 1, L- and A-stability, the scalar test problem
(one step multiplies u0 by the stability function R(dt lambda)), brute-force
dense stage solves, and the observed convergence order against the matrix
exponential.
"""
import math
import os

import numpy as np
import pytest

from oracle import dirk, tableau
from paper_1701_07181_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SCHEMES = {"DIRK33": tableau.dirk33, "ESDIRK65": tableau.esdirk65}


def _rows():
    out = []
    for line in open(os.path.join(GOLDEN, "table1_dirk.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(line.split())
    return out


def rooted_trees(n):
    """All rooted trees with n vertices, each as a sorted tuple of subtrees."""
    if n == 1:
        return [()]
    out = set()

    def parts(total, max_first):
        # multisets of subtrees whose sizes sum to total (non-increasing sizes)
        if total == 0:
            yield ()
            return
        for size in range(min(total, max_first), 0, -1):
            for t in rooted_trees(size):
                for rest in parts(total - size, size):
                    if rest and len(rest[0]) == size and rest[0] > t:
                        continue
                    yield (t,) + rest

    for ch in parts(n - 1, n - 1):
        out.add(tuple(sorted(ch)))
    return sorted(out)


def order_of(t):
    return 1 + sum(order_of(u) for u in t)


def density(t):
    return order_of(t) * math.prod(density(u) for u in t)


def stage_weights(A, t):
    """Phi(t) per stage: product over the subtrees of A Phi(subtree)."""
    v = np.ones(A.shape[0])
    for u in t:
        v = v * (A @ stage_weights(A, u))
    return v


def test_tree_counts():
    # 1, 1, 2, 4, 9, 20 rooted trees of order 1..6 (OEIS A000081)
    assert [len(rooted_trees(n)) for n in range(1, 7)] == [1, 1, 2, 4, 9, 20]


def order_residuals(A, b, p):
    return [abs(b @ stage_weights(A, t) - 1.0 / density(t)) for n in range(1, p + 1) for t in rooted_trees(n)]


@pytest.mark.parametrize("row", _rows(), ids=lambda r: r[0])
def test_table1_dirk_rows(row):
    name, order, total, implicit, stage_order, coef = row
    order, total, implicit, stage_order = int(order), int(total), int(implicit), int(stage_order)
    A, b, c = SCHEMES[name]()
    assert A.shape == (total, total)
    assert np.all(np.triu(A, 1) == 0.0)
    assert int(np.count_nonzero(np.diag(A))) == implicit
    # order p: every tree of order <= p satisfied, some tree of order p + 1 not
    assert max(order_residuals(A, b, order)) < 1e-13
    assert max(abs(b @ stage_weights(A, t) - 1.0 / density(t)) for t in rooted_trees(order + 1)) > 1e-6
    # stage order q: sum_j a_ij c_j^(l-1) = c_i^l / l for l <= q, not for q + 1
    for l in range(1, stage_order + 1):
        np.testing.assert_allclose(A @ c ** (l - 1), c ** l / l, rtol=0, atol=1e-13)
    assert np.max(np.abs(A @ c ** stage_order - c ** (stage_order + 1) / (stage_order + 1))) > 1e-6
    # leading error coefficient of the stability function: e^z - R(z) = C z^(p+1) + ...
    C = 1.0 / math.factorial(order + 1) - b @ np.linalg.matrix_power(A, order) @ np.ones(total)
    assert float("%.2e" % abs(C)) == float(coef), (name, C)


@pytest.mark.parametrize("name", sorted(SCHEMES))
def test_l_and_a_stability(name):
    A, b, _ = SCHEMES[name]()
    for z in (-1e6, -1e8):
        assert abs(tableau.stability_function(A, b, z)) < 50.0 / abs(z)
    for y in np.linspace(-200, 200, 801):
        assert abs(tableau.stability_function(A, b, 1j * y)) <= 1.0 + 1e-12
    for x in (-0.1, -1.0, -10.0):
        for y in (0.0, 1.0, 30.0):
            assert abs(tableau.stability_function(A, b, x + 1j * y)) <= 1.0 + 1e-12


def test_dirk33_diagonal_is_the_l_stable_root():
    """Order 3 with three equal diagonal entries and b = last row admits three
    real diagonals, the roots of x^3 - 3x^2 + 3x/2 - 1/6; DIRK33's alpha is the
    middle one, the only one whose scheme is A-stable."""
    A, b, _ = tableau.dirk33()
    roots = np.sort(np.real(np.roots([1.0, -3.0, 1.5, -1.0 / 6.0])))
    assert abs(A[0, 0] - roots[1]) < 1e-15
    np.testing.assert_array_equal(b, A[-1])


def scalar_problem(lam):
    rp = np.array([0, 1], np.int32)
    ci = np.array([0], np.int32)
    return rp, ci, np.array([lam]), np.array([1.0])


@pytest.mark.parametrize("name", sorted(SCHEMES))
@pytest.mark.parametrize("z", [-0.3, -2.0, -40.0])
def test_scalar_step_is_stability_function(name, z):
    A, b, _ = SCHEMES[name]()
    rp, ci, J, M = scalar_problem(z / 0.5)
    out = dirk.dirk_step(1, 1, rp, ci, J, M, A, b, np.array([1.7]), 0.5, rtol=1e-14)
    R = tableau.stability_function(A, b, z).real
    assert abs(out["u1"][0] - 1.7 * R) < 1e-13 * max(1.0, abs(1.7 * R))


@pytest.mark.parametrize("s", [2, 3])
def test_scalar_irk_step_is_pade(s):
    A, b, _ = tableau.radau_iia(s)
    rp, ci, J, M = scalar_problem(-3.0)
    out = dirk.irk_step(1, 1, rp, ci, J, M, A, b, np.array([1.0]), 0.25, rtol=1e-14)
    assert abs(out["u1"][0] - tableau.stability_function(A, b, -0.75).real) < 1e-13


def dense(T, m, rp, ci, blocks):
    D = np.zeros((T * m, T * m))
    blocks = np.asarray(blocks).reshape(-1, m, m)
    for i in range(T):
        for p in range(rp[i], rp[i + 1]):
            D[i * m:(i + 1) * m, ci[p] * m:(ci[p] + 1) * m] = blocks[p]
    return D


@pytest.mark.parametrize("name", sorted(SCHEMES))
def test_dirk_step_matches_dense_stage_solves(name):
    """Chain mesh (block tridiagonal): ILU(0) of each stage matrix is its exact
    LU, so every implicit stage converges in one iteration; u1 equals the
    stage recurrence done with dense solves."""
    A, b, _ = SCHEMES[name]()
    P = inputs.make_problem(inputs.mesh_1d_chain(9), 4, 1, 0.2, 4.0, seed=3)
    u0 = np.random.default_rng(1).standard_normal(P.T * P.m)
    out = dirk.dirk_step(P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, A, b, u0, 0.2, rtol=1e-13)
    assert all(it <= 1 for it in out["iters"])
    Jd = dense(P.T, P.m, P.row_ptr, P.col_idx, P.J)
    Md = np.zeros_like(Jd)
    for i in range(P.T):
        Md[i * P.m:(i + 1) * P.m, i * P.m:(i + 1) * P.m] = P.M[i]
    K = []
    for k in range(len(b)):
        v = u0 + 0.2 * sum(A[k, j] * K[j] for j in range(k))
        K.append(np.linalg.solve(Md - 0.2 * A[k, k] * Jd, Jd @ v))
    u1 = u0 + 0.2 * sum(b[k] * K[k] for k in range(len(b)))
    assert np.linalg.norm(out["u1"] - u1) <= 1e-11 * np.linalg.norm(u1)


@pytest.mark.parametrize("name,p", [("DIRK33", 3), ("ESDIRK65", 5), ("RADAU35", 5)])
def test_convergence_order_against_exponential(name, p):
    """Global error after t = 1 against exp(t M^{-1} J) u0 on a small non-stiff
    system: halving dt divides it by about 2^p."""
    import scipy.linalg
    P = inputs.make_problem(inputs.mesh_1d_chain(4), 3, 1, 0.1, 0.5, seed=5)
    Jd = dense(P.T, P.m, P.row_ptr, P.col_idx, P.J)
    Md = np.zeros_like(Jd)
    for i in range(P.T):
        Md[i * P.m:(i + 1) * P.m, i * P.m:(i + 1) * P.m] = P.M[i]
    u0 = np.random.default_rng(2).standard_normal(P.T * P.m)
    exact = scipy.linalg.expm(np.linalg.solve(Md, Jd)) @ u0
    if name == "RADAU35":
        A, b, _ = tableau.radau_iia(3)
    else:
        A, b, _ = SCHEMES[name]()
    errs = []
    for nsteps in (4, 8):
        u = u0.copy()
        for _ in range(nsteps):
            if name == "RADAU35":
                u = dirk.irk_step(P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, A, b, u, 1.0 / nsteps, rtol=1e-14)["u1"]
            else:
                u = dirk.dirk_step(P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, A, b, u, 1.0 / nsteps, rtol=1e-14)["u1"]
        errs.append(np.linalg.norm(u - exact))
    rate = math.log2(errs[0] / errs[1])
    assert p - 0.6 < rate < p + 0.8, (name, errs, rate)


# ---------------------------------------------------------------------------
# step_outputs: K = (A^-1 (x) I) W and u1 = u0 + dt (b^T A^-1 (x) I) W (Sec. 4.1)

@pytest.mark.parametrize("s", [2, 3])
def test_step_outputs_radau_reduces_to_last_stage(s):
    """The paper's simplification for Radau IIA: b^T A^-1 = e_s, so
    u1 = u0 + dt w_s."""
    A, b, _ = tableau.radau_iia(s)
    rng = np.random.default_rng(s)
    W = rng.standard_normal((s, 50))
    u0 = rng.standard_normal(50)
    K, u1 = dirk.step_outputs(A, b, W, u0, 0.3)
    np.testing.assert_allclose(u1, u0 + 0.3 * W[-1], rtol=0, atol=1e-13)


def test_step_outputs_match_classical_rk_form():
    """With W = (A (x) I) K the transformed update equals the classical one,
    u1 = u0 + dt sum_i b_i k_i, and K maps back to W (any invertible A)."""
    rng = np.random.default_rng(11)
    s = 4
    A = rng.standard_normal((s, s)) + 3.0 * np.eye(s)
    b = rng.standard_normal(s)
    K0 = rng.standard_normal((s, 30))
    W = A @ K0
    u0 = rng.standard_normal(30)
    K, u1 = dirk.step_outputs(A, b, W, u0, 0.7)
    np.testing.assert_allclose(K, K0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(u1, u0 + 0.7 * (b @ K0), rtol=0, atol=1e-12)


@pytest.mark.parametrize("scheme", ["radau23", "radau35", "DIRK33", "ESDIRK65"])
def test_step_outputs_scalar_problem_is_stability_function(scheme):
    """u' = lam u: the stage solution of (A^-1 - dt lam I) W = lam u0 1 gives
    u1 = R(dt lam) u0 with the stability function R(z) = 1 + z b^T (I - zA)^-1 1;
    ESDIRK65's explicit first stage makes A singular, so its W comes from K."""
    A, b = {"radau23": tableau.radau23, "radau35": tableau.radau35,
            "DIRK33": tableau.dirk33, "ESDIRK65": tableau.esdirk65}[scheme]()[:2]
    A = np.asarray(A, dtype=np.float64)
    s = len(b)
    lam, dt, u0 = -2.5, 0.4, np.array([1.7])
    # stage derivatives k = lam (u0 + dt A k): (I - dt lam A) k = lam u0 1
    K = np.linalg.solve(np.eye(s) - dt * lam * A, lam * u0[0] * np.ones(s))
    W = (A @ K).reshape(s, 1)
    if abs(np.linalg.det(A)) > 1e-12:
        _, u1 = dirk.step_outputs(A, b, W, u0, dt)
    else:
        u1 = u0 + dt * (np.asarray(b) @ K)
    R = tableau.stability_function(A, b, dt * lam).real
    np.testing.assert_allclose(u1, R * u0, rtol=1e-13)
