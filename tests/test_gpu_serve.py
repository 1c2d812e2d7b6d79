"""Serving loop (paper_1701_07181_gb300.serve): a Poisson stream of requests
of different mesh sizes, dimensions, polynomial degrees and stage counts,
admitted while others are being solved.  Each result is the same alone and
in the mix (bitwise: the request's arithmetic does not depend on the other
requests), within 1e-6 of the FP64 oracle, and latencies are reported."""
import numpy as np
import pytest

import oracle
from paper_1701_07181_gb300 import inputs
from _parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_served_results_equal_alone_and_match_oracle():
    from paper_1701_07181_gb300 import irk, serve
    stream = inputs.serving_stream(12, rate=400.0, seed=5, elements=(150, 1200), degrees=(1, 2), stages=(2, 3))
    probs = serve.prepare(stream, "cuda")
    recs, summ = serve.run_stream(stream, probs, budget_bytes=24 << 30, keep_results=True)
    assert all(r.status == 0 and r.relres <= 1e-8 for r in recs)
    assert summ.n == 12 and summ.p99_ms >= summ.p50_ms > 0 and summ.solves_per_s > 0
    # overlap happened: some request was admitted before an earlier one finished
    assert any(b.admitted < a.finished for a in recs for b in recs if b.idx > a.idx)
    for r in recs:
        P = probs[r.idx]
        with irk.Group(P.s, P.m, P.T + 1, P.nnzb, 2, ordering="multicolor") as G:
            slot = G.submit(P.T, torch.as_tensor(P.row_ptr).cuda(), torch.as_tensor(P.col_idx).cuda(), P.J, P.M,
                            P.R, P.dt, 1e-8)
            while G.query(slot)[0]:
                G.step()
            W = G.collect(slot, device="cuda")
        assert torch.equal(W, r.result), r.idx
    small = sorted(recs, key=lambda r: r.elements * probs[r.idx].m)[:2]
    for r in small:
        P = probs[r.idx]
        ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J.cpu().numpy(), P.M.cpu().numpy())
        W_ref = ref.solve(P.R.cpu().numpy(), P.dt, rtol=1e-12)["x"]
        W = r.result.cpu().numpy()
        assert rel(W, W_ref) <= 1e-6


def test_fifo_plain_path_runs_the_same_stream():
    from paper_1701_07181_gb300 import serve
    stream = inputs.serving_stream(4, rate=400.0, seed=6, elements=(150, 600), degrees=(1,), stages=(2, 3))
    probs = serve.prepare(stream, "cuda")
    recs, summ = serve.run_fifo(stream, probs)
    assert all(r.status == 0 for r in recs) and summ.n == 4
