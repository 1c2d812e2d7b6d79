"""DIRK steps through the C ABI (irk_dirk_*) against the oracle (Sec. 3).

* scalar test problem (T = m = 1, M = 1, J = lambda): u1 = R(dt lambda) u0
  with R the scheme's stability function, to 1e-12;
* 2D mesh, binary64 factors and Krylov: u1 within 1e-10 of the oracle's
  step, every stage's iteration count within 1;
* double-float Krylov with FP32 factors: u1 within 1e-6;
* block-tridiagonal chain: ILU(0) of each stage matrix is exact, so every
  implicit stage converges in one iteration and explicit stages report 0.
"""
import numpy as np
import pytest

from oracle import dirk as odirk
from oracle import tableau
from paper_1701_07181_gb300 import inputs
from _parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
SCHEMES = ["dirk33", "esdirk65"]


def _irk():
    from paper_1701_07181_gb300 import irk
    return irk


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("name", SCHEMES)
@pytest.mark.parametrize("krylov,fprec", [("fp64", "fp64"), ("df64", "fp32")])
def test_scalar_problem_gives_stability_function(name, krylov, fprec):
    irk = _irk()
    A, b, _ = getattr(tableau, name)()
    rp, ci = np.array([0, 1], np.int32), np.array([0], np.int32)
    for z in (-0.4, -3.0, -50.0):
        dt = 0.5
        with irk.Dirk(A, b, 1, 1, rp, ci, np.array([z / dt]), np.array([1.0]), krylov=krylov,
                      factor_prec=fprec) as D:
            u1, K, its, rr, rc = D.step(np.array([2.0]), dt, rtol=1e-13)
        R = tableau.stability_function(A, b, z).real
        assert rc == 0
        assert abs(u1[0] - 2.0 * R) <= 1e-12 * max(1.0, abs(2.0 * R)), (z, u1[0], 2 * R)


@pytest.mark.parametrize("name", SCHEMES)
def test_mesh_step_matches_oracle_fp64(name):
    irk = _irk()
    A, b, _ = getattr(tableau, name)()
    P = inputs.make_problem(inputs.mesh_2d_periodic(7, 5), 12, 1, 0.3, 4.0, seed=4)
    u0 = np.random.default_rng(9).standard_normal(P.T * P.m)
    ref = odirk.dirk_step(P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, A, b, u0, 0.3, rtol=1e-12)
    with irk.Dirk(A, b, P.T, P.m, dev(P.row_ptr), dev(P.col_idx), dev(P.J), dev(P.M), krylov="fp64",
                  factor_prec="fp64") as D:
        u1, K, its, rr, rc = D.step(dev(u0), 0.3, rtol=1e-12, want_K=True)
    u1 = u1.cpu().numpy()
    assert rc == 0 and rr <= 1e-12
    assert rel(u1, ref["u1"]) <= 1e-10
    np.testing.assert_allclose(K.cpu().numpy().reshape(len(b), -1), ref["K"], rtol=0,
                               atol=1e-10 * np.abs(ref["K"]).max())
    for a, r in zip(its, ref["iters"]):
        assert abs(a - r) <= 1, (its, ref["iters"])


@pytest.mark.parametrize("name", SCHEMES)
def test_mesh_step_mixed_precision(name):
    irk = _irk()
    A, b, _ = getattr(tableau, name)()
    P = inputs.make_problem(inputs.mesh_2d_periodic(9, 6), 24, 1, 0.1, 4.0, seed=6)
    u0 = np.random.default_rng(3).standard_normal(P.T * P.m)
    ref = odirk.dirk_step(P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, A, b, u0, 0.1, rtol=1e-12)
    with irk.Dirk(A, b, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, krylov="df64", factor_prec="fp32",
                  ordering="multicolor") as D:
        u1, _, its, rr, rc = D.step(u0, 0.1, rtol=1e-8)
    assert rc == 0 and rr <= 1e-8
    assert rel(u1, ref["u1"]) <= 1e-6


@pytest.mark.parametrize("name", SCHEMES)
def test_chain_one_iteration_per_implicit_stage(name):
    irk = _irk()
    A, b, _ = getattr(tableau, name)()
    P = inputs.make_problem(inputs.mesh_1d_chain(23), 5, 1, 0.2, 4.0, seed=8)
    u0 = np.random.default_rng(4).standard_normal(P.T * P.m)
    with irk.Dirk(A, b, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, krylov="fp64", factor_prec="fp64") as D:
        u1, _, its, rr, rc = D.step(u0, 0.2, rtol=1e-12)
    assert rc == 0
    assert its == [0 if A[k, k] == 0.0 else 1 for k in range(len(b))], its
    ref = odirk.dirk_step(P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, A, b, u0, 0.2, rtol=1e-13)
    assert rel(u1, ref["u1"]) <= 1e-11


def test_bad_tableau_is_refused():
    irk = _irk()
    A, b, _ = tableau.dirk33()
    A = A.copy()
    A[0, 2] = 0.1  # not lower triangular
    P = inputs.make_problem(inputs.mesh_1d_chain(5), 3, 1, 0.2, 4.0, seed=1)
    with pytest.raises(irk.IrkError):
        irk.Dirk(A, b, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M)
