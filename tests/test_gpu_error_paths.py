"""Error paths of the C ABI on the GPU, each followed by a clean call on the
same context that must match the oracle (the context stays usable).

* Non-finite inputs: a NaN in one J block, an infinity in one M block (at
  irk_update_values) and a NaN / infinity in R (at irk_solve) return
  IRK_ERR_NONFINITE (-4).
* Bounded device waits: with irk_options.spin_limit = 1 the persistent
  sweep's waits for rows published by other warps (input element order, one
  cooperative launch) and the Arnoldi launch's grid barrier give up; the
  kernels record a timeout, let their own bulk copies land and leave, and
  the call returns IRK_ERR_TIMEOUT (-5).  No wait is unbounded and nothing
  faults: this is the status path a wait that runs out takes.
* Double-float range: right-hand sides scaled by 1e-35 and 1e39 (outside
  what a binary32 pair can carry) solve to the oracle's bar through the
  power-of-two scaling; a power-of-two scale gives the unscaled result bit
  for bit; J or dt outside the documented range is refused with
  IRK_ERR_INVALID (-1), while binary64 Krylov arithmetic accepts them.
"""
import numpy as np
import pytest

import oracle
from paper_1701_07181_gb300 import inputs
from _parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NONFINITE, TIMEOUT, INVALID = -4, -5, -1


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _irk():
    from paper_1701_07181_gb300 import irk
    return irk


def problem(s=2, m=12, nx=9, ny=7, seed=21):
    return inputs.make_problem(inputs.mesh_2d_periodic(nx, ny), m, s, 0.1, 4.0, seed)


def ref_solution(P, dt=0.1, R=None):
    ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M)
    return ref.solve(P.R if R is None else R, dt, rtol=1e-12)["x"]


@pytest.mark.parametrize("krylov,fprec", [("df64", "fp32"), ("fp64", "fp64")])
@pytest.mark.parametrize("where", ["J", "M"])
def test_nonfinite_block_reported_then_clean_solve(krylov, fprec, where):
    irk = _irk()
    P = problem()
    W_ref = ref_solution(P)
    bad_J, bad_M = P.J.copy(), P.M.copy()
    if where == "J":
        bad_J[P.row_ptr[5] + 1, 3, 7] = np.nan  # one entry of one off-diagonal J block
    else:
        bad_M[11, 0, 4] = np.inf
    with irk.Solver(P.s, P.T, P.m, dev(P.row_ptr), dev(P.col_idx), dev(P.J), dev(P.M), precond="uncoupled",
                    factor_prec=fprec, krylov=krylov) as S:
        with pytest.raises(irk.IrkError) as e:
            S.update_values(dev(bad_J), dev(bad_M))
        assert e.value.code == NONFINITE
        S.update_values(dev(P.J), dev(P.M))
        W, it, rr, rc = S.solve(dev(P.R), 0.1, rtol=1e-8)
    assert rc == 0 and rr <= 1e-8
    assert rel(W, W_ref) <= 1e-6


def test_nonfinite_block_refused_at_setup():
    irk = _irk()
    P = problem()
    J = P.J.copy()
    J[0, 0, 0] = np.nan
    with pytest.raises(irk.IrkError) as e:
        irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, J, P.M, krylov="df64", factor_prec="fp32")
    assert e.value.code == NONFINITE


@pytest.mark.parametrize("krylov,fprec", [("df64", "fp32"), ("fp64", "fp64")])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_nonfinite_rhs_reported_then_clean_solve(krylov, fprec, bad):
    irk = _irk()
    P = problem()
    W_ref = ref_solution(P)
    R = P.R.copy()
    R[R.size // 3] = bad
    with irk.Solver(P.s, P.T, P.m, dev(P.row_ptr), dev(P.col_idx), dev(P.J), dev(P.M), precond="uncoupled",
                    factor_prec=fprec, krylov=krylov) as S:
        with pytest.raises(irk.IrkError) as e:
            S.solve(dev(R), 0.1, rtol=1e-8)
        assert e.value.code == NONFINITE
        W, it, rr, rc = S.solve(dev(P.R), 0.1, rtol=1e-8)
    assert rc == 0 and rr <= 1e-8
    assert rel(W, W_ref) <= 1e-6


@pytest.mark.parametrize("krylov,fprec", [("df64", "fp32"), ("fp64", "fp64")])
def test_spin_limit_times_out_then_recovers(krylov, fprec):
    irk = _irk()
    P = problem(s=3, m=12, nx=16, ny=16)  # 512 elements, natural order: a long dependency chain
    ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M)
    V = np.random.default_rng(3).standard_normal(P.s * P.T * P.m)
    W_ref = ref.solve(P.R, 0.1, rtol=1e-12)["x"]
    with irk.Solver(P.s, P.T, P.m, dev(P.row_ptr), dev(P.col_idx), dev(P.J), dev(P.M), precond="uncoupled",
                    factor_prec=fprec, krylov=krylov, spin_limit=1) as S:
        S.factor(0.1)
        assert S.stats()["levels_lower"] > 8  # the persistent (published-row) sweep
        with pytest.raises(irk.IrkError) as e:
            S.apply_precond(dev(V))
        assert e.value.code == TIMEOUT
        with pytest.raises(irk.IrkError) as e:
            S.solve(dev(P.R), 0.1, rtol=1e-8)
        assert e.value.code == TIMEOUT
        S.set_spin_limit(0)  # back to the default
        z = S.apply_precond(dev(V))
        W, it, rr, rc = S.solve(dev(P.R), 0.1, rtol=1e-8)
    assert rc == 0 and rr <= 1e-8
    assert rel(W, W_ref) <= 1e-6
    if fprec == "fp64":
        assert rel(z, ref.precond_apply(V, 0.1)) <= 1e-11


def test_spin_limit_rejects_negative():
    irk = _irk()
    P = problem()
    with pytest.raises(irk.IrkError) as e:
        irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, spin_limit=-1)
    assert e.value.code == INVALID
    with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M) as S:
        with pytest.raises(irk.IrkError) as e:
            S.set_spin_limit(-3)
        assert e.value.code == INVALID


@pytest.mark.parametrize("krylov", ["df64", "fp64-dfop"])
@pytest.mark.parametrize("scale", [1e-35, 1e39])
def test_df64_rhs_out_of_binary32_range(scale, krylov):
    """R scaled far outside binary32's range: W within the 1e-6 bar of the
    oracle's solution for the scaled R (binary64 throughout)."""
    irk = _irk()
    P = problem()
    R = P.R * scale
    W_ref = ref_solution(P, R=R)
    with irk.Solver(P.s, P.T, P.m, dev(P.row_ptr), dev(P.col_idx), dev(P.J), dev(P.M), precond="uncoupled",
                    factor_prec="fp32", krylov=krylov) as S:
        W, it, rr, rc = S.solve(dev(R), 0.1, rtol=1e-8)
        y = S.apply_operator(dev(R), 0.1)
    assert rc == 0 and rr <= 1e-8
    assert np.all(np.isfinite(W.cpu().numpy()))
    assert rel(W, W_ref) <= 1e-6
    y_ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M).apply(R, 0.1)
    assert rel(y, y_ref) <= 1e-13


def test_df64_power_of_two_scaling_is_exact():
    irk = _irk()
    P = problem()
    with irk.Solver(P.s, P.T, P.m, dev(P.row_ptr), dev(P.col_idx), dev(P.J), dev(P.M), precond="uncoupled",
                    factor_prec="fp32", krylov="df64") as S:
        W1, it1, *_ = S.solve(dev(P.R), 0.1, rtol=1e-8)
        W2, it2, *_ = S.solve(dev(np.ldexp(P.R, -90)), 0.1, rtol=1e-8)
    assert it1 == it2
    assert torch.equal(torch.ldexp(W2, torch.tensor(90.0, dtype=torch.float64, device=W2.device)), W1)


@pytest.mark.parametrize("krylov", ["df64", "fp64-dfop"])
def test_df64_refuses_out_of_range_values_and_dt(krylov):
    irk = _irk()
    P = problem()
    with pytest.raises(irk.IrkError) as e:
        irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J * 1e35, P.M, krylov=krylov, factor_prec="fp32")
    assert e.value.code == INVALID
    with pytest.raises(irk.IrkError) as e:
        irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M * 1e-35, krylov=krylov, factor_prec="fp32")
    assert e.value.code == INVALID
    # binary64 Krylov arithmetic has binary64's range
    with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J * 1e35, P.M, krylov="fp64") as S:
        S.factor(1e-35)
    with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, krylov=krylov, factor_prec="fp32") as S:
        with pytest.raises(irk.IrkError) as e:
            S.solve(P.R, 1e31, rtol=1e-8)
        assert e.value.code == INVALID
        W, it, rr, rc = S.solve(P.R, 0.1, rtol=1e-8)  # the context is unaffected
        assert rc == 0 and rr <= 1e-8


def test_group_refuses_split_precision():
    """The multi-request engine runs binary64 or double-float Krylov only."""
    irk = _irk()
    import ctypes
    lib = irk.load()
    opt = irk.Options()
    lib.irk_default_options(ctypes.byref(opt))
    opt.krylov_arith = irk.KRYLOV["fp64-dfop"]
    h = ctypes.c_void_p()
    assert lib.irk_group_create(ctypes.byref(h), 2, None, 12, 1000, 4000, 4, ctypes.byref(opt)) == -1
