"""Parity at the full workload sizes, in the benchmark's launch configuration.

20000 triangles (m = 40, s = 3: the benchmark workload; FP32 factors,
double-float Krylov, two-colour order, shifted uncoupled block ILU(0)) and
48000 tetrahedra (m = 50, s = 3; FP32 and BF16-stored factors):

* the operator product against the oracle's FP64 product on the whole
  vector, <= 1e-13 relative;
* each solve at rtol 1e-8: status OK, and its true residual recomputed by
  the oracle's FP64 operator <= 1e-8 (a property that holds at any size);
  iteration counts on the 20000-element workload equal the oracle's own
  counts (tests/golden/oracle_iters_c1.txt, written by a script that calls
  only the oracle), within one;
* W against the oracle's tightly converged solution for dt = 0.1 on the
  20000-element workload, <= 1e-6 relative (the oracle solve takes tens of
  seconds there, so only this one).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1701_07181_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _irk():
    from paper_1701_07181_gb300 import irk
    return irk


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_iters():
    out = {}
    for line in open(os.path.join(GOLDEN, "oracle_iters_c1.txt")):
        f = line.split()
        if f and not line.startswith("#"):
            out[float(f[0])] = int(f[1])
    return out


@pytest.fixture(scope="module")
def c1():
    return inputs.config("c1", seed=0)


@pytest.fixture(scope="module")
def c1_solver(c1):
    irk = _irk()
    P = c1
    S = irk.Solver(P.s, P.T, P.m, dev(P.row_ptr), dev(P.col_idx), dev(P.J), dev(P.M), precond="uncoupled",
                   factor_prec="fp32", krylov="df64", ordering="multicolor")
    yield S
    S.close()


def test_c1_operator_full_size(c1, c1_solver):
    P = c1
    X = np.random.default_rng(12).standard_normal(P.s * P.T * P.m)
    y = c1_solver.apply_operator(dev(X), 0.1).cpu().numpy()
    y_ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M).apply(X, 0.1)
    assert rel(y, y_ref) <= 1e-13


@pytest.mark.parametrize("dt", [0.01, 0.1, 1.0])
def test_c1_solve_full_size(c1, c1_solver, dt):
    P = c1
    W, it, rr, rc = c1_solver.solve(dev(P.R), dt, rtol=1e-8)
    assert rc == 0 and rr <= 1e-8
    # the second colour level's products ran as staged whole rows
    assert c1_solver.stats()["factor_fused_levels"] == 1
    W = W.cpu().numpy()
    ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M)
    res = np.linalg.norm(P.R - ref.apply(W, dt)) / np.linalg.norm(P.R)
    assert res <= 1e-8, res
    want = oracle_iters().get(dt)
    if want is not None:
        assert abs(it - want) <= 1, (dt, it, want)
    if dt == 0.1:
        W_ref = ref.solve(P.R, dt, rtol=1e-12)["x"]
        assert rel(W, W_ref) <= 1e-6


@pytest.mark.parametrize("fprec", ["fp32", "bf16"])
def test_c2_full_size(fprec):
    irk = _irk()
    P = inputs.config("c2", seed=0)
    ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M)
    with irk.Solver(P.s, P.T, P.m, dev(P.row_ptr), dev(P.col_idx), dev(P.J), dev(P.M), precond="uncoupled",
                    factor_prec=fprec, krylov="df64", ordering="multicolor") as S:
        if fprec == "fp32":
            X = np.random.default_rng(3).standard_normal(P.s * P.T * P.m)
            assert rel(S.apply_operator(dev(X), 0.1).cpu().numpy(), ref.apply(X, 0.1)) <= 1e-13
        W, it, rr, rc = S.solve(dev(P.R), 0.1, rtol=1e-8)
    assert rc == 0 and rr <= 1e-8
    W = W.cpu().numpy()
    res = np.linalg.norm(P.R - ref.apply(W, 0.1)) / np.linalg.norm(P.R)
    assert res <= 1e-8, res
