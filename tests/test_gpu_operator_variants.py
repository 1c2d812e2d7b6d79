"""Launch variants of the operator product (Sec. 4.1) through the C ABI.

The autotuner picks one of several launches of the same product: the
register-streaming kernel with different chunk widths and CTA sizes, the
bulk-copy pipelined kernel with 2 or 3 shared-memory stages, and the
register-streaming kernel with the block size fixed at compile time, one or
four rows per thread, and the TMA-fed kernel (a producer warp streaming
column chunks and stage values into shared memory).  All of them
accumulate every output in the same order, so each one, pinned with the
kernel option matvec_variant, must give a result bitwise equal to variant 0's, and that
result must match the FP64 oracle (1e-13 relative, the operator bar).
Cases: block sizes that are even (pipelined kernel applies) and odd (it falls
back), s = 1..4, and a mesh large enough that every CTA of the pipelined
kernel takes several rows per group (3200 elements).
"""
import numpy as np
import pytest

import oracle
from paper_1701_07181_gb300 import inputs
from _parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_VARIANTS = 19


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def make(kind, s, m, seed=3):
    nb = {"2d": inputs.mesh_2d_periodic(7, 5), "big2d": inputs.mesh_2d_periodic(40, 40),
          "3d": inputs.mesh_3d_periodic(3, 4, 3), "chain": inputs.mesh_1d_chain(37)}[kind]
    return inputs.make_problem(nb, m, s, 0.2, 4.0, seed)


@pytest.mark.parametrize("krylov", ["fp64", "df64"])
@pytest.mark.parametrize("kind,s,m", [("2d", 3, 40), ("big2d", 3, 40), ("3d", 2, 20), ("chain", 1, 7),
                                      ("2d", 4, 12), ("chain", 2, 100), ("big2d", 2, 12)])
def test_operator_variants_bitwise_equal(krylov, kind, s, m):
    from paper_1701_07181_gb300 import irk
    P = make(kind, s, m)
    X = np.random.default_rng(7).standard_normal(P.s * P.T * P.m)
    outs = []
    for v in range(N_VARIANTS):
        with irk.Solver(P.s, P.T, P.m, dev(P.row_ptr), dev(P.col_idx), dev(P.J), dev(P.M), krylov=krylov,
                        precond="none", kernel_options={"matvec_variant": v}) as S:
            y = S.apply_operator(dev(X), 0.37).cpu().numpy()
            assert S.stats()["matvec_variant"] == v
        outs.append(y)
    for v in range(1, N_VARIANTS):
        np.testing.assert_array_equal(outs[v], outs[0], err_msg="variant %d" % v)
    y_ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M).apply(X, 0.37)
    assert rel(outs[0], y_ref) <= 1e-13


@pytest.mark.parametrize("variant", [4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18])
def test_solve_with_pipelined_product_is_bitwise_equal(variant):
    """The residual form (y = rhs - B x) of the pipelined kernel, inside a
    full preconditioned solve: same W and iteration count as variant 0.
    The compile-time variants (7, 9-18) there also take the kernels that
    skip the zero low words of binary32 preconditioned vectors."""
    from paper_1701_07181_gb300 import irk
    P = make("2d", 3, 40)
    res = []
    for v in (0, variant):
        with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, factor_prec="fp32", krylov="df64",
                        kernel_options={"matvec_variant": v}) as S:
            res.append(S.solve(P.R, P.dt, rtol=1e-8))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1]
