"""The multi-request engine (irk_group_*) through the C ABI.

* every request's W within 1e-6 of the FP64 oracle (solved tightly) at rtol
  1e-8, with the single-request path's iteration count (+-1);
* a request gives the same result alone and in the mix: alone in a group,
  and submitted while other requests of different sizes are mid-solve
  (continuous admission); its reductions are partitioned by its own size
  only, so the two results are bitwise equal;
* capacity: a request that does not fit is refused (pools full) and
  admitted once another has been collected.
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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def make(nx, ny, m=12, s=3, seed=0, dt=0.2):
    return inputs.make_problem(inputs.mesh_2d_periodic(nx, ny), m, s, dt, 4.0, seed)


def run_all(G, probs, submit_at=None, host=False):
    """Submit problems (at given step numbers), step until all finish."""
    submit_at = submit_at or [0] * len(probs)
    slots, out = {}, {}
    step = 0
    pending = list(range(len(probs)))
    while pending or any(v is not None for v in slots.values()):
        for k in list(pending):
            if submit_at[k] <= step:
                P = probs[k]
                args = (P.row_ptr, P.col_idx, P.J, P.M, P.R) if host else tuple(
                    dev(a) for a in (P.row_ptr, P.col_idx, P.J, P.M, P.R))
                slot = G.submit(P.T, *args, P.dt, 1e-8)
                if slot is not None:
                    slots[k] = slot
                    pending.remove(k)
        G.step()
        step += 1
        for k, slot in list(slots.items()):
            if slot is None:
                continue
            running, iters, relres, status = G.query(slot)
            if not running:
                W = G.collect(slot)
                out[k] = (W, iters, relres, status)
                slots[k] = None
        assert step < 5000
    return out


@pytest.mark.parametrize("fprec,krylov,pc,order", [("fp32", "df64", "uncoupled", "natural"),
                                                   ("fp64", "fp64", "uncoupled", "multicolor"),
                                                   ("fp32", "df64", "none", "natural")])
def test_group_matches_oracle_and_single_path(fprec, krylov, pc, order):
    irk = _irk()
    probs = [make(5, 4, seed=1), make(9, 7, seed=2, dt=0.5), make(3, 3, seed=3, dt=0.05), make(12, 10, seed=4)]
    cap_e = sum(P.T for P in probs)
    cap_b = sum(P.nnzb for P in probs)
    with irk.Group(3, 12, cap_e, cap_b, 8, precond=pc, factor_prec=fprec, krylov=krylov, ordering=order) as G:
        out = run_all(G, probs, host=True)
    for k, P in enumerate(probs):
        W, iters, relres, status = out[k]
        assert status == 0 and relres <= 1e-8
        ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M)
        W_ref = ref.solve(P.R, P.dt, rtol=1e-12)["x"]
        assert rel(W, W_ref) <= 1e-6
        with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, precond=pc, factor_prec=fprec,
                        krylov=krylov, ordering=order) as S:
            W1, it1, rr1, rc1 = S.solve(P.R, P.dt, rtol=1e-8)
        assert abs(iters - it1) <= 1, (iters, it1)
        assert rel(W, W1) <= 1e-6


def test_same_alone_and_in_the_mix():
    irk = _irk()
    target = make(8, 6, seed=11, dt=0.3)
    others = [make(10, 9, seed=12, dt=1.0), make(4, 4, seed=13, dt=0.01), make(7, 5, seed=14, dt=0.1),
              make(11, 3, seed=15, dt=0.6)]
    probs = [target] + others
    cap_e = sum(P.T for P in probs)
    cap_b = sum(P.nnzb for P in probs)
    with irk.Group(3, 12, cap_e, cap_b, 8, factor_prec="fp32", krylov="df64") as G:
        alone = run_all(G, [target])[0]
    with irk.Group(3, 12, cap_e, cap_b, 8, factor_prec="fp32", krylov="df64") as G:
        # others start first; the target arrives while they are mid-solve
        mixed = run_all(G, others + [target], submit_at=[0, 0, 2, 3, 4])[len(others)]
    np.testing.assert_array_equal(alone[0], mixed[0])
    assert alone[1] == mixed[1]


def test_capacity_refusal_and_reuse():
    irk = _irk()
    a, b = make(6, 6, seed=21), make(6, 6, seed=22)
    with irk.Group(3, 12, a.T + 1, a.nnzb, 4, factor_prec="fp32", krylov="df64") as G:
        sa = G.submit(a.T, a.row_ptr, a.col_idx, a.J, a.M, a.R, a.dt)
        assert sa is not None
        assert G.submit(b.T, b.row_ptr, b.col_idx, b.J, b.M, b.R, b.dt) is None  # pools full
        while G.query(sa)[0]:
            G.step()
        G.collect(sa)
        sb = G.submit(b.T, b.row_ptr, b.col_idx, b.J, b.M, b.R, b.dt)
        assert sb is not None
        while G.query(sb)[0]:
            G.step()
        W = G.collect(sb)
        assert G.device_bytes() > 0
    ref = oracle.Problem(b.s, b.T, b.m, b.row_ptr, b.col_idx, b.J, b.M).solve(b.R, b.dt, rtol=1e-12)["x"]
    assert rel(W, ref) <= 1e-6
