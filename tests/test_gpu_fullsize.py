"""Parity at the full workload sizes, in the benchmark's launch configuration.

20000 triangles (m = 40, s = 3: the benchmark workload; two-colour order,
shifted uncoupled block ILU(0)) and 48000 tetrahedra (m = 50, s = 3):

* the operator product against the oracle's FP64 product on the whole
  vector, <= 1e-13 relative, norm-wise and element-wise;
* each solve at rtol 1e-8: status OK, and its true residual recomputed by
  the oracle's FP64 operator <= 1e-8 (a property that holds at any size);
  iteration counts of the benchmark configuration equal the oracle's own
  counts (tests/golden/oracle_iters_c1.txt, written by a script that calls
  only the oracle), within one;
* W against the oracle's solution converged to 1e-12, <= 1e-6 relative
  (norm-wise and element-wise) for every dt in {0.01, 0.1, 1} and every
  precision variant: FP32 factors with double-float Krylov (the benchmark),
  FP32 factors with binary64 Krylov, BF16-stored factors with double-float
  Krylov, binary64 factors and Krylov; on the tetrahedra, FP32 and BF16
  factors at dt = 0.1.  The oracle runs in its multi-core build here (the
  same algorithm; its threads split rows, stages and inner products).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1701_07181_gb300 import inputs
from _parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
VARIANTS = [("fp32", "df64"), ("fp32", "fp64"), ("fp32", "fp64-dfop"), ("bf16", "df64"), ("fp64", "fp64")]


def _irk():
    from paper_1701_07181_gb300 import irk
    return irk


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


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
def c1_ref(c1):
    P = c1
    return oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, omp=True)


@pytest.fixture(scope="module")
def c1_tight(c1, c1_ref):
    cache = {}

    def get(dt):
        if dt not in cache:
            cache[dt] = c1_ref.solve(c1.R, dt, rtol=1e-12)["x"]
        return cache[dt]
    return get


@pytest.fixture(scope="module")
def c1_dev(c1):
    P = c1
    return dev(P.row_ptr), dev(P.col_idx), dev(P.J), dev(P.M), dev(P.R)


def test_c1_operator_full_size(c1, c1_ref, c1_dev):
    irk = _irk()
    P = c1
    rp, ci, J, M, _ = c1_dev
    X = np.random.default_rng(12).standard_normal(P.s * P.T * P.m)
    y_ref = c1_ref.apply(X, 0.1)
    for krylov in ("df64", "fp64"):
        with irk.Solver(P.s, P.T, P.m, rp, ci, J, M, precond="uncoupled", factor_prec="fp32", krylov=krylov,
                        ordering="multicolor") as S:
            y = S.apply_operator(dev(X), 0.1)
        assert rel(y, y_ref) <= 1e-13, krylov


@pytest.mark.parametrize("dt", [0.01, 0.1, 1.0])
@pytest.mark.parametrize("fprec,krylov,ortho", [v + ("mgs",) for v in VARIANTS] + [("fp32", "df64", "cgs2")])
def test_c1_solve_full_size(c1, c1_ref, c1_tight, c1_dev, dt, fprec, krylov, ortho):
    irk = _irk()
    P = c1
    rp, ci, J, M, R = c1_dev
    with irk.Solver(P.s, P.T, P.m, rp, ci, J, M, precond="uncoupled", factor_prec=fprec, krylov=krylov,
                    ordering="multicolor", orthogonalization=ortho) as S:
        W, it, rr, rc = S.solve(R, dt, rtol=1e-8)
        fused = S.stats()["factor_fused_levels"]
    assert rc == 0 and rr <= 1e-8
    if fprec == "fp32":
        assert fused == 1  # the second colour level's products ran as staged whole rows
    W = W.cpu().numpy()
    res = np.linalg.norm(P.R - c1_ref.apply(W, dt)) / np.linalg.norm(P.R)
    assert res <= 1e-8, res
    if (fprec, krylov) == ("fp32", "df64"):
        want = oracle_iters().get(dt)
        assert want is None or abs(it - want) <= 1, (dt, it, want)
    assert rel(W, c1_tight(dt)) <= 1e-6, (dt, fprec, krylov, rel(W, c1_tight(dt)))


@pytest.fixture(scope="module")
def c2():
    return inputs.config("c2", seed=0)


@pytest.fixture(scope="module")
def c2_ref(c2):
    P = c2
    return oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, omp=True)


@pytest.fixture(scope="module")
def c2_tight(c2, c2_ref):
    return c2_ref.solve(c2.R, 0.1, rtol=1e-12)["x"]


@pytest.mark.parametrize("fprec,ortho", [("fp32", "mgs"), ("bf16", "mgs"), ("fp32", "cgs2")])
def test_c2_full_size(c2, c2_ref, c2_tight, fprec, ortho):
    irk = _irk()
    P = c2
    with irk.Solver(P.s, P.T, P.m, dev(P.row_ptr), dev(P.col_idx), dev(P.J), dev(P.M), precond="uncoupled",
                    factor_prec=fprec, krylov="df64", ordering="multicolor", orthogonalization=ortho) as S:
        if fprec == "fp32" and ortho == "mgs":
            X = np.random.default_rng(3).standard_normal(P.s * P.T * P.m)
            assert rel(S.apply_operator(dev(X), 0.1), c2_ref.apply(X, 0.1)) <= 1e-13
        W, it, rr, rc = S.solve(dev(P.R), 0.1, rtol=1e-8)
    assert rc == 0 and rr <= 1e-8
    W = W.cpu().numpy()
    res = np.linalg.norm(P.R - c2_ref.apply(W, 0.1)) / np.linalg.norm(P.R)
    assert res <= 1e-8, res
    assert rel(W, c2_tight) <= 1e-6
