"""Step outputs of the C ABI (irk_step_outputs, Sec. 4.1) against the oracle.

From a stage solution W (here the library's own solve of a seeded problem,
and a random W), K = (A^-1 (x) I) W and u1 = u0 + dt (b^T A^-1 (x) I) W in
binary64 match oracle.dirk.step_outputs to 1e-14 relative, through host and
device buffers; with b = NULL (Radau IIA, b^T A^-1 = e_s) u1 is u0 + dt w_s
to rounding; a user tableau with its own weights uses b^T A^-1.
"""
import numpy as np
import pytest

from oracle import dirk, tableau
from paper_1701_07181_gb300 import inputs
from _parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("s", [2, 3])
@pytest.mark.parametrize("space", ["host", "device"])
def test_step_outputs_radau(s, space):
    from paper_1701_07181_gb300 import irk
    P = inputs.make_problem(inputs.mesh_2d_periodic(7, 5), 12, s, 0.2, 4.0, seed=s)
    A, b, _ = tableau.radau_iia(s)
    u0 = np.random.default_rng(2).standard_normal(P.T * P.m)
    with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, factor_prec="fp32", krylov="df64") as S:
        W = S.solve(P.R, 0.2, rtol=1e-10)[0]
        Wd = W if space == "host" else torch.as_tensor(W).cuda()
        u0d = u0 if space == "host" else torch.as_tensor(u0).cuda()
        K, u1 = S.step_outputs(Wd, 0.2, u0=u0d)
        if space == "device":
            K, u1 = K.cpu().numpy(), u1.cpu().numpy()
    K_ref, u1_ref = dirk.step_outputs(A, b, W, u0, 0.2)
    assert rel(K, K_ref.reshape(-1)) <= 1e-14
    # b = NULL: the stiffly accurate form u0 + dt w_s (one fused rounding on
    # the device, two in numpy)
    assert rel(u1, u0 + 0.2 * W.reshape(s, -1)[-1]) <= 1e-15
    assert rel(u1, u1_ref) <= 1e-14


def test_step_outputs_user_tableau_weights():
    """A user tableau (here RADAU35's A with DIRK-like weights): u1 uses
    b^T A^-1; K only A^-1."""
    from paper_1701_07181_gb300 import irk
    A, _, _ = tableau.radau_iia(3)
    b = np.array([0.2, 0.5, 0.3])
    P = inputs.make_problem(inputs.mesh_2d_periodic(7, 5), 12, 3, 0.2, 4.0, seed=9)
    W = np.random.default_rng(4).standard_normal(P.s * P.T * P.m)
    u0 = np.random.default_rng(5).standard_normal(P.T * P.m)
    with irk.Solver(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, A=A, factor_prec="fp32",
                    krylov="df64") as S:
        K, u1 = S.step_outputs(W, 0.37, u0=u0, b=b)
        K2, none = S.step_outputs(W, 0.37)
    K_ref, u1_ref = dirk.step_outputs(A, b, W, u0, 0.37)
    assert rel(K, K_ref.reshape(-1)) <= 1e-14
    assert rel(u1, u1_ref) <= 1e-14
    np.testing.assert_array_equal(K, K2)
    assert none is None
