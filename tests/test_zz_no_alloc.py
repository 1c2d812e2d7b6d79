"""irk_apply_precond_noalloc: the preconditioner application for callers that
cannot allocate device memory when they call it (their device memory held by
another allocator's pool, or a no-allocation rule in a latency-critical
time-stepping loop).  Its working vectors live in a fixed array the library
declares in device memory instead of buffers the context allocated.

Checked through the C ABI against the allocating entry point
irk_apply_precond, on two calls in a row (the array keeps the previous
call's contents, so the second call checks that everything that must start
from zero is cleared), with the bar of the FP64 preconditioner parity test
(1e-11 relative, norm-wise and element-wise), for the stage-uncoupled and
the stage-coupled (Alg. 3) preconditioners; with FP64 factors also against
the oracle's preconditioner at the same bar.  The error word of the sweep is
reported (a wait given spin limit 1 returns IRK_ERR_TIMEOUT, and the next
call at the default limit is correct), and the array's size limit is
enforced for both factor widths.  Collected last so that a failure here
cannot hide the other tests of a run that stops at the first failure.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1701_07181_gb300 import inputs
from _parity import rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PC = {"uncoupled": oracle.PC_UNCOUPLED, "coupled": oracle.PC_STAGE_MAJOR}


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _noalloc(lib, S, V, Z):
    return lib.irk_apply_precond_noalloc(S._h, ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(Z.data_ptr()), None)


@pytest.mark.parametrize("fprec,krylov", [("fp32", "df64"), ("fp64", "fp64"), ("bf16", "df64")])
@pytest.mark.parametrize("mesh,s,m,pc", [("2d", 3, 12, "uncoupled"), ("3d", 2, 20, "uncoupled"),
                                         ("c0", 2, 12, "uncoupled"), ("2d", 2, 12, "coupled")])
def test_noalloc_matches_allocating_entry_point(fprec, krylov, mesh, s, m, pc):
    from paper_1701_07181_gb300 import irk

    if mesh == "c0":
        P = inputs.config("c0", seed=4)
    elif mesh == "2d":
        P = inputs.make_problem(inputs.mesh_2d_periodic(7, 5), m, s, 0.1, 4.0, seed=4)
    else:
        P = inputs.make_problem(inputs.mesh_3d_periodic(3, 4, 3), m, s, 0.1, 4.0, seed=4)
    lib = irk.load()
    with irk.Solver(P.s, P.T, P.m, _dev(P.row_ptr), _dev(P.col_idx), _dev(P.J), _dev(P.M),
                    precond=pc, factor_prec=fprec, krylov=krylov) as S:
        S.factor(0.3)
        rng = np.random.default_rng(8)
        ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M)
        for call in range(2):
            Vh = rng.standard_normal(P.s * P.T * P.m)
            V = _dev(Vh)
            z_alloc = S.apply_precond(V)  # the allocating entry point
            Z = torch.full_like(V, float("nan"))
            rc = _noalloc(lib, S, V, Z)
            assert rc == 0, irk.strerror(rc)
            torch.cuda.synchronize()
            assert rel(Z, z_alloc) <= 1e-11, (call, rel(Z, z_alloc))
            if fprec == "fp64":
                z_ref = ref.precond_apply(Vh, 0.3, precond=PC[pc])
                assert rel(Z, z_ref) <= 1e-11, (call, rel(Z, z_ref))


def test_noalloc_reports_the_error_word_and_recovers():
    from paper_1701_07181_gb300 import irk

    lib = irk.load()
    P = inputs.make_problem(inputs.mesh_2d_periodic(16, 16), 12, 3, 0.1, 4.0, seed=2)
    with irk.Solver(P.s, P.T, P.m, _dev(P.row_ptr), _dev(P.col_idx), _dev(P.J), _dev(P.M),
                    precond="uncoupled", factor_prec="fp32", krylov="df64", spin_limit=1) as S:
        S.factor(0.2)
        V = _dev(P.R)
        Z = torch.empty_like(V)
        assert _noalloc(lib, S, V, Z) == -5  # a wait on another warp gave up
        S.set_spin_limit(0)
        assert _noalloc(lib, S, V, Z) == 0
        torch.cuda.synchronize()
        assert rel(Z, S.apply_precond(V)) <= 1e-11


@pytest.mark.parametrize("fprec,nx,ok", [("fp32", 171, False), ("fp64", 140, False), ("fp32", 140, True)])
def test_noalloc_size_limit(fprec, nx, ok):
    """FP32 factors: up to 2,097,120 unknowns (16 + 16 bytes each); FP64:
    up to 1,398,080 (16 + 32 bytes each).  171 x 171 and 140 x 140 split
    grids with m = 12, s = 3 hold 2,105,352 and 1,411,200 unknowns."""
    from paper_1701_07181_gb300 import irk

    lib = irk.load()
    P = inputs.make_problem(inputs.mesh_2d_periodic(nx, nx), 12, 3, 0.1, 4.0, seed=1)
    krylov = "fp64" if fprec == "fp64" else "df64"
    with irk.Solver(P.s, P.T, P.m, _dev(P.row_ptr), _dev(P.col_idx), _dev(P.J), _dev(P.M),
                    precond="uncoupled", factor_prec=fprec, krylov=krylov) as S:
        V = _dev(P.R)
        Z = torch.empty_like(V)
        assert _noalloc(lib, S, V, Z) == -7  # not factored yet
        S.factor(0.1)
        rc = _noalloc(lib, S, V, Z)
        if ok:
            assert rc == 0, irk.strerror(rc)
            torch.cuda.synchronize()
            assert rel(Z, S.apply_precond(V)) <= 1e-11
        else:
            assert rc == -8, irk.strerror(rc)
