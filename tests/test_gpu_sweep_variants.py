"""Backward-sweep variants of the uncoupled preconditioner (Sec. 4.3.2).

* Where no factor update reaches an upper block (every generated mesh: no
  element has two mutually adjacent neighbours), each stage's upper blocks
  are -dt J_ij and the backward sweep reads one copy for all stages; the
  application is bitwise equal to the per-stage sweep
  (irk_kernel_options.sweep_shared_upper = 0 forces the latter).
* On a pattern with mutually adjacent elements the factor does modify upper
  blocks; the library keeps the per-stage sweep there, and the FP64
  application still matches the oracle.
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


@pytest.mark.parametrize("fprec,krylov", [("fp32", "df64"), ("fp64", "fp64"), ("bf16", "df64")])
@pytest.mark.parametrize("kind,s,m", [("2d", 3, 40), ("3d", 2, 20), ("2d", 4, 12)])
def test_shared_upper_sweep_is_bitwise_equal(fprec, krylov, kind, s, m):
    irk = _irk()
    nb = inputs.mesh_2d_periodic(9, 7) if kind == "2d" else inputs.mesh_3d_periodic(3, 3, 4)
    P = inputs.make_problem(nb, m, s, 0.3, 4.0, seed=2)
    V = np.random.default_rng(8).standard_normal(P.s * P.T * P.m)
    out = []
    for shared in (1, 0):
        with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, factor_prec=fprec, krylov=krylov,
                        sweep="levels", ordering="multicolor",
                        kernel_options={"sweep_shared_upper": shared}) as S:
            S.factor(0.3)
            out.append(S.apply_precond(V))
    np.testing.assert_array_equal(out[0], out[1])


def test_mutual_neighbours_fall_back_and_match_oracle():
    irk = _irk()
    # 0-1-2 and 1-2-4 are triangles of the element graph
    nbrs = [[1, 2], [0, 2, 3], [0, 1, 4], [1, 4], [2, 3]]
    P = inputs.make_problem(nbrs, 6, 3, 0.4, 4.0, seed=5)
    V = np.random.default_rng(1).standard_normal(P.s * P.T * P.m)
    ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M).precond_apply(V, 0.4)
    for sweep in ("levels", "auto"):
        with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, factor_prec="fp64", krylov="fp64",
                        sweep=sweep) as S:
            S.factor(0.4)
            z = S.apply_precond(V)
        assert rel(z, ref) <= 1e-11


@pytest.mark.parametrize("fprec", ["fp32", "bf16"])
@pytest.mark.parametrize("kind,s,m,shared", [("2d", 3, 40, True), ("3d", 2, 20, True), ("2d", 4, 12, True),
                                             ("3d", 3, 50, True), ("chain", 1, 24, True), ("2d", 3, 40, False)])
def test_two_colour_application_is_bitwise_equal(fprec, kind, s, m, shared):
    """In the two-colour order the first colour's rows have no lower entries
    (y = v there) and the second colour's no upper entries (z = D^{-1} y right
    after the forward row), so the application runs as two launches instead
    of four.  It keeps every dot product's arithmetic: the preconditioned
    vector and a whole FGMRES solve are bitwise equal to the level sweeps'
    (kernel option sweep_two_colour = 0), with two launches fewer per
    application.  Shared upper blocks for all stages, and per-stage upper
    blocks (s = 1, and kernel option sweep_shared_upper = 0).  The Kuhn-tetrahedra meshes need four colours
    in first-fit order: there the level sweeps run either way."""
    irk = _irk()
    nb = {"2d": inputs.mesh_2d_periodic(9, 7), "3d": inputs.mesh_3d_periodic(3, 3, 4),
          "chain": inputs.mesh_1d_chain(38)}[kind]
    P = inputs.make_problem(nb, m, s, 0.3, 4.0, seed=2)
    V = np.random.default_rng(8).standard_normal(P.s * P.T * P.m)
    out, sol, launches = [], [], []
    for off in ("", "1"):
        ko = {"sweep_shared_upper": 1 if shared else 0, "sweep_two_colour": 0 if off else 1}
        with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, factor_prec=fprec, krylov="df64",
                        sweep="levels", ordering="multicolor", timing=True, kernel_options=ko) as S:
            S.factor(0.3)
            out.append(S.apply_precond(V))
            W, it, rr, rc = S.solve(P.R, 0.3, rtol=1e-8)
            assert rc == 0 and rr <= 1e-8
            st = S.stats()
            sol.append((W, it))
            launches.append((st["kernel_launches"], st["n_precond"]))
            assert st["sweep_two_colour"] == (1 if (not off and kind != "3d") else 0)
    np.testing.assert_array_equal(out[0], out[1])
    np.testing.assert_array_equal(sol[0][0], sol[1][0])
    assert sol[0][1] == sol[1][1]
    two_colour = kind != "3d"
    assert launches[1][0] - launches[0][0] == (2 * launches[0][1] if two_colour else 0)


@pytest.mark.parametrize("fprec", ["fp32", "bf16"])
@pytest.mark.parametrize("kind,s,m,shared", [("3d", 3, 50, True), ("3d", 2, 20, True), ("3d", 1, 24, True),
                                             ("2d", 3, 40, True), ("2d", 3, 12, False)])
def test_compiled_level_sweeps_are_bitwise_equal(fprec, kind, s, m, shared):
    """Level sweeps by the kernels compiled for the block size (forward
    levels after the first register-blocked, backward levels with the upper
    blocks read once for all stages) against the generic level kernels
    (kernel option sweep_compiled_levels = 0): the same dot products in the
    same order, so the preconditioned vector and a whole solve agree bit for
    bit.  The Kuhn-tetrahedra meshes take four colours (four levels per
    sweep); the 2D mesh runs its two levels with the two-launch form off."""
    irk = _irk()
    nb = inputs.mesh_3d_periodic(3, 3, 4) if kind == "3d" else inputs.mesh_2d_periodic(9, 7)
    P = inputs.make_problem(nb, m, s, 0.3, 4.0, seed=6)
    V = np.random.default_rng(9).standard_normal(P.s * P.T * P.m)
    out, sol = [], []
    for compiled in (1, 0):
        ko = {"sweep_compiled_levels": compiled, "sweep_two_colour": 0, "sweep_shared_upper": 1 if shared else 0}
        with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, factor_prec=fprec, krylov="df64",
                        sweep="levels", ordering="multicolor", kernel_options=ko) as S:
            S.factor(0.3)
            out.append(S.apply_precond(V))
            W, it, rr, rc = S.solve(P.R, 0.3, rtol=1e-8)
            assert rc == 0 and rr <= 1e-8
            sol.append((W, it))
    np.testing.assert_array_equal(out[0], out[1])
    np.testing.assert_array_equal(sol[0][0], sol[1][0])
    assert sol[0][1] == sol[1][1]
