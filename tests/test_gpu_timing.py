"""Phase timing of the C ABI (irk_options.timing).

timing = 1 reads the events back at the end of every irk_solve; timing = 2
leaves them unread until irk_get_stats, which then reports the phase counts,
phase times and kernel launches summed over every call since the previous
irk_get_stats.  Both time the same kernels: over two solves the counts and
launches of timing 2 equal the sums of the per-solve values of timing 1, a
second irk_get_stats right after reports nothing, and the solutions are
bitwise the same (timing only adds events to the stream).
"""
import numpy as np
import pytest

from paper_1701_07181_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_deferred_timing_totals_match_per_solve_timing():
    from paper_1701_07181_gb300 import irk
    ko = {"matvec_variant": 0}  # no autotuning launches in either context
    P = inputs.make_problem(inputs.mesh_2d_periodic(12, 10), 20, 3, 0.2, 4.0, seed=4)
    dts = (0.05, 0.2)
    per, sols = [], []
    with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, factor_prec="fp32", krylov="df64",
                    ordering="multicolor", timing=1, kernel_options=ko) as S:
        for dt in dts:
            W, it, rr, rc = S.solve(P.R, dt, rtol=1e-8)
            assert rc == 0
            per.append(S.stats())
            sols.append(W)
    with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, factor_prec="fp32", krylov="df64",
                    ordering="multicolor", timing=2, kernel_options=ko) as S:
        S.stats()  # nothing pending yet
        out = [S.solve(P.R, dt, rtol=1e-8)[0] for dt in dts]
        tot = S.stats()
        again = S.stats()
    for a, b in zip(out, sols):
        np.testing.assert_array_equal(a, b)
    for k in ("n_matvec", "n_precond", "n_ortho", "kernel_launches"):
        assert tot[k] == sum(p[k] for p in per), k
    for k in ("matvec_ms", "precond_ms", "ortho_ms", "factor_assemble_ms", "factor_products_ms",
              "factor_inverse_ms", "sweep_fwd_ms", "sweep_bwd_ms"):
        # the same phases are timed (on this small mesh the persistent sweep
        # runs, which has no per-sweep marks: those stay 0 in both modes)
        assert (tot[k] > 0.0) == (sum(p[k] for p in per) > 0.0), k
        assert again[k] == 0.0, k
    assert tot["matvec_ms"] > 0.0 and tot["precond_ms"] > 0.0 and tot["ortho_ms"] > 0.0
    assert again["n_matvec"] == 0 and again["kernel_launches"] == 0


def test_set_timing_samples_calls():
    """irk_set_timing switches the events on and off between calls: marks
    recorded under timing = 2 survive a switch to 0 and are reported by the
    next irk_get_stats under timing = 2; calls made with timing 0 add none."""
    from paper_1701_07181_gb300 import irk
    ko = {"matvec_variant": 0}
    P = inputs.make_problem(inputs.mesh_2d_periodic(12, 10), 20, 3, 0.2, 4.0, seed=4)
    with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, factor_prec="fp32", krylov="df64",
                    ordering="multicolor", timing=1, kernel_options=ko) as S:
        S.solve(P.R, 0.05, rtol=1e-8)
        one = S.stats()
    with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, factor_prec="fp32", krylov="df64",
                    ordering="multicolor", timing=2, kernel_options=ko) as S:
        S.stats()
        S.solve(P.R, 0.05, rtol=1e-8)   # timed
        S.set_timing(0)
        S.solve(P.R, 0.2, rtol=1e-8)    # not timed
        S.set_timing(2)
        tot = S.stats()
        with pytest.raises(irk.IrkError):
            S.set_timing(3)
    assert tot["n_matvec"] == one["n_matvec"] and tot["n_ortho"] == one["n_ortho"]
    assert tot["matvec_ms"] > 0.0
