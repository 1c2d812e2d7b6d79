"""GPU parity of the reordered / partitioned preconditioners (Sec. 4.5) with
the oracle's ordered stage-uncoupled ILU(0).  Bars as in test_gpu_parity:
FP64 preconditioner 1e-11; FP64 solve +-1 iteration and 1e-10; mixed 1e-6."""
import numpy as np
import pytest

import oracle
from paper_1701_07181_gb300 import inputs

from test_oracle_ordering import greedy_colouring_order, strip_partitions
from _parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def setup(mesh="2d", m=12, s=3, seed=21):
    nb = inputs.mesh_2d_periodic(8, 6) if mesh == "2d" else inputs.mesh_3d_periodic(3, 4, 3)
    P = inputs.make_problem(nb, m, s, 0.3, 4.0, seed)
    return P, oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M)


def solver(P, **kw):
    from paper_1701_07181_gb300 import irk
    return irk.Solver(P.s, P.T, P.m, dev(P.row_ptr), dev(P.col_idx), dev(P.J), dev(P.M), **kw)


@pytest.mark.parametrize("mesh", ["2d", "3d"])
@pytest.mark.parametrize("variant", ["multicolor", "strips4", "jacobi", "user", "multicolor+strips3"])
def test_fp64_ordered_preconditioner(mesh, variant):
    P, ref = setup(mesh)
    perm, part, kw = None, None, {}
    if "multicolor" in variant:
        perm, _ = greedy_colouring_order(P.row_ptr, P.col_idx)
        kw["ordering"] = "multicolor"
    if "strips" in variant:
        n = int(variant.split("strips")[1])
        part = strip_partitions(P.T, n)
        kw["partitions"] = n
    if variant == "jacobi":
        part = np.arange(P.T, dtype=np.int32)
        kw["partitions"] = P.T
    if variant == "user":
        part = (np.arange(P.T) % 3).astype(np.int32)
        kw["partition"] = part
    V = np.random.default_rng(4).standard_normal(P.s * P.n)
    z_ref = ref.precond_apply_ordered(V, 0.3, perm=perm, part=part)
    with solver(P, precond="uncoupled", factor_prec="fp64", krylov="fp64", **kw) as S:
        S.factor(0.3)
        z = S.apply_precond(dev(V))
        lv = S.stats()["levels_lower"]
    assert rel(z, z_ref) <= 1e-11
    if variant == "multicolor" and mesh == "2d":
        assert lv == 2
    if variant == "jacobi":
        assert lv == 1


def test_fp64_multicolor_solve_matches_oracle():
    P, ref = setup("2d")
    perm, _ = greedy_colouring_order(P.row_ptr, P.col_idx)
    out = ref.solve_ordered(P.R, P.dt, perm=perm, rtol=1e-8)
    with solver(P, precond="uncoupled", factor_prec="fp64", krylov="fp64", ordering="multicolor") as S:
        W, iters, relres, rc = S.solve(dev(P.R), P.dt, rtol=1e-8)
    assert rc == 0 and abs(iters - out["iters"]) <= 1
    assert rel(W, out["x"]) <= (1e-10 if iters == out["iters"] else 1e-6)


@pytest.mark.parametrize("pc", ["uncoupled", "coupled"])
@pytest.mark.parametrize("kw", [{"ordering": "multicolor"}, {"partitions": 5}])
def test_mixed_ordered_solve_within_1e6(pc, kw):
    P, ref = setup("3d", m=20)
    W_ref = ref.solve(P.R, P.dt, rtol=1e-12)["x"]
    with solver(P, precond=pc, factor_prec="fp32", krylov="df64", **kw) as S:
        W, iters, relres, rc = S.solve(dev(P.R), P.dt, rtol=1e-8)
    assert rc == 0 and relres <= 1e-8
    assert rel(W, W_ref) <= 1e-6


def test_element_kind_rejects_reordering():
    from paper_1701_07181_gb300 import irk
    P, _ = setup("2d", m=4, s=2)
    with pytest.raises(irk.IrkError):
        solver(P, precond="element", ordering="multicolor")
