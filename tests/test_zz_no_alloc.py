"""irk_apply_precond_noalloc: the preconditioner application for callers that
cannot allocate device memory when they call it (their device memory held by
another allocator's pool, or a no-allocation rule in a latency-critical
time-stepping loop).  Its working vectors live in a fixed array the library
declares in device memory instead of buffers the context allocated.

Checked through the C ABI against the allocating entry point
irk_apply_precond, on two calls in a row (the array keeps the previous
call's contents, so the second call checks that everything that must start
from zero is cleared), with the bar of the FP64 preconditioner parity test
(1e-11 relative).  Collected last so that a failure here cannot hide the
other tests of a run that stops at the first failure.
"""
import ctypes

import numpy as np
import pytest

from paper_1701_07181_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("fprec,krylov", [("fp32", "df64"), ("fp64", "fp64"), ("bf16", "df64")])
@pytest.mark.parametrize("mesh,s,m", [("2d", 3, 12), ("3d", 2, 20), ("c0", 2, 12)])
def test_noalloc_matches_allocating_entry_point(fprec, krylov, mesh, s, m):
    from paper_1701_07181_gb300 import irk

    if mesh == "c0":
        P = inputs.config("c0", seed=4)
    elif mesh == "2d":
        P = inputs.make_problem(inputs.mesh_2d_periodic(7, 5), m, s, 0.1, 4.0, seed=4)
    else:
        P = inputs.make_problem(inputs.mesh_3d_periodic(3, 4, 3), m, s, 0.1, 4.0, seed=4)
    lib = irk.load()
    with irk.Solver(P.s, P.T, P.m, _dev(P.row_ptr), _dev(P.col_idx), _dev(P.J), _dev(P.M),
                    precond="uncoupled", factor_prec=fprec, krylov=krylov) as S:
        S.factor(0.3)
        rng = np.random.default_rng(8)
        for call in range(2):
            V = _dev(rng.standard_normal(P.s * P.T * P.m))
            ref = S.apply_precond(V)  # the allocating entry point
            Z = torch.full_like(V, float("nan"))
            rc = lib.irk_apply_precond_noalloc(S._h, ctypes.c_void_p(V.data_ptr()),
                                               ctypes.c_void_p(Z.data_ptr()), None)
            assert rc == 0, irk.strerror(rc)
            torch.cuda.synchronize()
            assert _rel(Z, ref) <= 1e-11, (call, _rel(Z, ref))


def test_noalloc_rejects_oversized_and_unfactored():
    from paper_1701_07181_gb300 import irk

    lib = irk.load()
    # 2,105,352 unknowns (171 x 171 split grid, m = 12, s = 3) exceed the
    # array with FP32 factors (limit 2,097,120)
    P = inputs.make_problem(inputs.mesh_2d_periodic(171, 171), 12, 3, 0.1, 4.0, seed=1)
    assert P.s * P.T * P.m > 2097120
    with irk.Solver(P.s, P.T, P.m, _dev(P.row_ptr), _dev(P.col_idx), _dev(P.J), _dev(P.M),
                    precond="uncoupled", factor_prec="fp32", krylov="df64") as S:
        V = _dev(P.R)
        Z = torch.empty_like(V)
        rc = lib.irk_apply_precond_noalloc(S._h, ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(Z.data_ptr()),
                                           None)
        assert rc == -7  # not factored yet
        S.factor(0.1)
        rc = lib.irk_apply_precond_noalloc(S._h, ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(Z.data_ptr()),
                                           None)
        assert rc == -8, irk.strerror(rc)
