"""Pins of the oracle's reordered / partitioned stage-uncoupled block ILU(0)
(Sec. 4.5: partitioned ILU drops the couplings between partitions and, with
one element per partition, reduces to block Jacobi).

* natural order + one partition = the standard preconditioner, bitwise;
* every element its own partition = block Jacobi: z = (d_k M_i - dt J_ii)^{-1} v
  per element and stage (dense LAPACK solves);
* the defining property of ILU(0), in any elimination order and for any kept
  pattern: (L~ U~)_ij = B_ij on every kept block (i, j);
* partitions drop exactly the blocks between different partitions;
* two-colour order on the bipartite split grid: the first colour is never
  eliminated (its pivots are the original blocks), two levels per sweep.
"""
import numpy as np
import pytest

import oracle
from oracle import tableau
from paper_1701_07181_gb300 import inputs


def greedy_colouring_order(row_ptr, col_idx):
    """First-fit colouring in natural order, then elements sorted by
    (colour, index): the documented rule of the multicolour ordering."""
    T = row_ptr.size - 1
    colour = -np.ones(T, int)
    for i in range(T):
        used = {colour[j] for j in col_idx[row_ptr[i]:row_ptr[i + 1]] if j != i and colour[j] >= 0}
        c = 0
        while c in used:
            c += 1
        colour[i] = c
    return np.lexsort((np.arange(T), colour)).astype(np.int32), colour


def strip_partitions(T, P):
    return (np.arange(T) * P // T).astype(np.int32)


def _problem(nbrs, m=4, s=3, seed=5):
    P = inputs.make_problem(nbrs, m, s, 0.2, 4.0, seed)
    return P, oracle.Problem(s, P.T, m, P.row_ptr, P.col_idx, P.J, P.M)


def test_natural_single_partition_is_standard():
    P, pr = _problem(inputs.mesh_2d_periodic(5, 4))
    a = pr.solve(P.R, P.dt, rtol=1e-10, precond=oracle.PC_UNCOUPLED)
    b = pr.solve_ordered(P.R, P.dt, perm=None, part=np.zeros(P.T, np.int32), rtol=1e-10)
    c = pr.solve_ordered(P.R, P.dt, perm=np.arange(P.T, dtype=np.int32), rtol=1e-10)
    np.testing.assert_array_equal(a["x"], b["x"])
    np.testing.assert_array_equal(a["x"], c["x"])
    assert a["iters"] == b["iters"] == c["iters"]


@pytest.mark.parametrize("mesh", ["2d", "3d"])
def test_one_element_per_partition_is_block_jacobi(mesh):
    nbrs = inputs.mesh_2d_periodic(4, 3) if mesh == "2d" else inputs.mesh_3d_periodic(3)
    P, pr = _problem(nbrs)
    alpha = tableau.shift_column_rule(pr.Ainv)
    v = np.random.default_rng(1).standard_normal(P.s * P.n)
    z = pr.precond_apply_ordered(v, P.dt, part=np.arange(P.T, dtype=np.int32))
    diag = P.row_ptr[:-1] + [list(P.col_idx[P.row_ptr[i]:P.row_ptr[i + 1]]).index(i) for i in range(P.T)]
    expect = np.empty_like(v)
    for k in range(P.s):
        d = pr.Ainv[k, k] + alpha[k]
        for i in range(P.T):
            B = d * P.M[i] - P.dt * P.J[diag[i]]
            sl = slice(k * P.n + i * P.m, k * P.n + (i + 1) * P.m)
            expect[sl] = np.linalg.solve(B, v[sl])
    np.testing.assert_allclose(z, expect, rtol=1e-12, atol=1e-14)


def _dense_from_blocks(rp, ci, V, b):
    nb = rp.size - 1
    D = np.zeros((nb * b, nb * b))
    for j in range(nb):
        for p in range(rp[j], rp[j + 1]):
            D[j * b:(j + 1) * b, ci[p] * b:(ci[p] + 1) * b] = V[p]
    return D


@pytest.mark.parametrize("order", ["colour", "random", "reverse"])
@pytest.mark.parametrize("parts", [1, 3])
def test_ilu0_property_in_any_order(order, parts):
    P, pr = _problem(inputs.mesh_2d_periodic(4, 4), m=3)
    if order == "colour":
        perm, _ = greedy_colouring_order(P.row_ptr, P.col_idx)
    elif order == "random":
        perm = np.random.default_rng(3).permutation(P.T).astype(np.int32)
    else:
        perm = np.arange(P.T)[::-1].astype(np.int32)
    part = strip_partitions(P.T, parts)
    rp, ci, V = pr.assemble_ordered(0, 5.0, P.dt, perm=perm, part=part)
    F, _, _ = oracle.bilu0(rp, ci, V)
    b = P.m
    Bd = _dense_from_blocks(rp, ci, V, b)
    L = np.eye(P.T * b)
    U = np.zeros_like(Bd)
    for j in range(P.T):
        for p in range(rp[j], rp[j + 1]):
            i = ci[p]
            blk = (slice(j * b, (j + 1) * b), slice(i * b, (i + 1) * b))
            (L if i < j else U)[blk] = F[p]
    LU = L @ U
    scale = np.abs(Bd).max()
    for j in range(P.T):
        for p in range(rp[j], rp[j + 1]):
            i = ci[p]
            blk = (slice(j * b, (j + 1) * b), slice(i * b, (i + 1) * b))
            assert np.abs(LU[blk] - Bd[blk]).max() <= 1e-12 * scale


def test_partitions_drop_exactly_the_cross_blocks():
    P, pr = _problem(inputs.mesh_2d_periodic(6, 5))
    part = strip_partitions(P.T, 4)
    rp, ci, _ = pr.assemble_ordered(0, 5.0, P.dt, part=part)
    kept = {(j, int(c)) for j in range(P.T) for c in ci[rp[j]:rp[j + 1]]}
    for i in range(P.T):
        for j in P.col_idx[P.row_ptr[i]:P.row_ptr[i + 1]]:
            assert ((i, int(j)) in kept) == (part[i] == part[j])


def test_two_colour_order_on_the_split_grid():
    P, pr = _problem(inputs.mesh_2d_periodic(6, 4))
    perm, colour = greedy_colouring_order(P.row_ptr, P.col_idx)
    assert colour.max() == 1  # bipartite: lower / upper triangles
    nred = int((colour == 0).sum())
    rp, ci, V = pr.assemble_ordered(0, 5.0, P.dt, perm=perm)
    F, _, _ = oracle.bilu0(rp, ci, V)
    for q in range(P.T):
        lower = [c for c in ci[rp[q]:rp[q + 1]] if c < q]
        if q < nred:
            assert not lower  # first colour: nothing to eliminate, pivot = original block
            d = rp[q] + list(ci[rp[q]:rp[q + 1]]).index(q)
            np.testing.assert_array_equal(F[d], V[d])
        else:
            assert all(c < nred for c in lower)  # second colour depends only on the first


def test_ordered_solve_converges_and_reports():
    """Sec. 5.3 / Sec. 4.5 trade-off, reported (not asserted): partitioning the
    ILU raises the iteration count; the two-colour order changes it."""
    P, pr = _problem(inputs.mesh_2d_periodic(10, 10), m=6)
    perm, _ = greedy_colouring_order(P.row_ptr, P.col_idx)
    res = {"natural": pr.solve(P.R, P.dt, rtol=1e-8)["iters"],
           "colour": pr.solve_ordered(P.R, P.dt, perm=perm, rtol=1e-8)["iters"]}
    for parts in (4, 16, P.T):
        out = pr.solve_ordered(P.R, P.dt, part=strip_partitions(P.T, parts), rtol=1e-8)
        assert out["relres"] <= 1e-8
        res["parts=%d" % parts] = out["iters"]
    print("iterations:", res)
