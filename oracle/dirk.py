"""Runge-Kutta steps of the linear(ised) system M u' = J u (oracle side).

TEST INFRASTRUCTURE ONLY: used by the tests and the benchmark's CPU leg; the
library's CUDA path never imports it.

The stage equations of a Runge-Kutta scheme with tableau (A, b) applied to
M u' = J u (Sec. 3) are M k_k = J (u0 + dt sum_j a_kj k_j), and
u1 = u0 + dt sum_k b_k k_k.

* ``dirk_step``: for a lower-triangular A (DIRK, Sec. 3) the stages decouple.
  Stage k solves the single n x n system
      (M - dt a_kk J) k_k = J (u0 + dt sum_{j<k} a_kj k_j)
  with the oracle's FGMRES and the block ILU(0) of that stage matrix (s = 1,
  untransformed form: B = M - dt a_kk J), or, for an explicit stage
  (a_kk = 0, the first stage of ESDIRK65), the block-diagonal solve
  M k_k = J u0 (library dense solves per element).
* ``irk_step``: the fully implicit step for comparison.  With W_k =
  dt sum_j a_kj k_j the stage equations become the transformed system of
  Sec. 4.1, (A^{-1} (x) M) W - dt (I (x) J) W = dt 1 (x) (J u0), and
  u1 = u0 + sum_k (b^T A^{-1})_k W_k (= u0 + W_s for stiffly accurate
  schemes such as Radau IIA).
* ``jacobian_apply``: y_i = sum_j J_ij x_j, the plain block-sparse product.
* ``step_outputs``: from the transformed stage solution W of Sec. 4.1 (W =
  (A (x) I) K), the stage derivatives K = (A^{-1} (x) I) W and the new state
  u1 = u0 + dt (b^T A^{-1} (x) I) W.

The number of n x n matrix-vector products of a step is what Sec. 5 calls
equivalent multiplications: iterations x 1 per DIRK stage, iterations x s for
the coupled system.
"""
from __future__ import annotations

import numpy as np

from . import FORM_TRANSFORMED, FORM_UNTRANSFORMED, PC_STAGE_MAJOR, PC_UNCOUPLED, Problem


def step_outputs(A, b, W, u0, dt):
    """Sec. 4.1: W stacks w_i = sum_j a_ij k_j, so K = (A^{-1} (x) I_n) W, and
    u1 = u0 + dt (b^T A^{-1} (x) I_n) W.  W is s x n (stage-major) or flat;
    returns (K as s x n, u1 or None when u0 is None)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = len(b)
    W = np.asarray(W, dtype=np.float64).reshape(s, -1)
    K = np.linalg.solve(A, W)  # A K = W, row by row
    if u0 is None:
        return K, None
    wts = np.linalg.solve(A.T, b)  # b^T A^{-1}
    return K, np.asarray(u0, dtype=np.float64).reshape(-1) + dt * (wts @ W)


def jacobian_apply(row_ptr, col_idx, J, m, x):
    """y_i = sum over the pattern of row i of J_ij x_j (J row-major blocks)."""
    T = len(row_ptr) - 1
    J = np.asarray(J, dtype=np.float64).reshape(-1, m, m)
    x = np.asarray(x, dtype=np.float64).reshape(T, m)
    y = np.zeros((T, m))
    for i in range(T):
        for p in range(row_ptr[i], row_ptr[i + 1]):
            y[i] += J[p] @ x[col_idx[p]]
    return y.reshape(-1)


def mass_solve(M, m, r):
    """k_i = M_i^{-1} r_i for every element (block-diagonal M)."""
    M = np.asarray(M, dtype=np.float64).reshape(-1, m, m)
    r = np.asarray(r, dtype=np.float64).reshape(-1, m)
    return np.stack([np.linalg.solve(M[i], r[i]) for i in range(M.shape[0])]).reshape(-1)


def dirk_step(T, m, row_ptr, col_idx, J, M, A, b, u0, dt, rtol=1e-10, restart=30, max_iter=3000):
    """One DIRK step; returns dict(u1, K (s x T*m), iters (per stage, 0 for
    an explicit stage), relres (per stage))."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = len(b)
    if np.any(np.triu(A, 1) != 0.0):
        raise ValueError("A must be lower triangular")
    u0 = np.asarray(u0, dtype=np.float64).reshape(-1)
    K = np.zeros((s, T * m))
    iters, relres = [], []
    for k in range(s):
        v = u0 + dt * sum(A[k, j] * K[j] for j in range(k)) if k else u0.copy()
        rhs = jacobian_apply(row_ptr, col_idx, J, m, v)
        if A[k, k] == 0.0:
            K[k] = mass_solve(M, m, rhs)
            iters.append(0)
            relres.append(0.0)
            continue
        prob = Problem(1, T, m, row_ptr, col_idx, J, M, A=[[A[k, k]]])
        out = prob.solve(rhs, dt, rtol=rtol, form=FORM_UNTRANSFORMED, precond=PC_STAGE_MAJOR, restart=restart,
                         max_iter=max_iter)
        K[k] = out["x"]
        iters.append(out["iters"])
        relres.append(out["relres"])
    u1 = u0 + dt * (b @ K)
    return dict(u1=u1, K=K, iters=iters, relres=relres)


def irk_step(T, m, row_ptr, col_idx, J, M, A, b, u0, dt, rtol=1e-10, restart=30, max_iter=3000,
             precond=PC_UNCOUPLED):
    """One fully implicit step through the transformed coupled system;
    returns dict(u1, W (s x T*m, stage-major), iters, relres)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = len(b)
    u0 = np.asarray(u0, dtype=np.float64).reshape(-1)
    Ju0 = jacobian_apply(row_ptr, col_idx, J, m, u0)
    R = np.tile(dt * Ju0, s)
    prob = Problem(s, T, m, row_ptr, col_idx, J, M, A=A)
    out = prob.solve(R, dt, rtol=rtol, form=FORM_TRANSFORMED, precond=precond, restart=restart,
                     max_iter=max_iter)
    W = out["x"].reshape(s, T * m)
    wts = np.linalg.solve(A.T, b)  # b^T A^{-1}
    u1 = u0 + wts @ W
    return dict(u1=u1, W=W, iters=out["iters"], relres=out["relres"])
