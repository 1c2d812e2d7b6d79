"""Seeded synthetic DG-shaped inputs for the stage-system solve.

This module holds data generation only (meshes, random blocks, right-hand
sides); none of the method's arithmetic.  Both the CUDA path's callers and the
oracle's tests draw their inputs from here, so the two sides see identical
arrays.

Meshes (block structure of Sec. 2.1: one m x m block per element, off-diagonal
blocks for face neighbours):

* ``mesh_2d_periodic(nx, ny)``: nx x ny periodic quads, each split by its
  (0,0)-(1,1) diagonal into a lower triangle (sub-index 0) and an upper one
  (sub-index 1); element id = 2*(y*nx + x) + sub.  r = 3 face neighbours.
* ``mesh_3d_periodic(nx, ny, nz)``: periodic cubes, each split into the 6 Kuhn
  tetrahedra (one per permutation of the axes, in lexicographic order);
  element id = 6*((z*ny + y)*nx + x) + perm.  r = 4 face neighbours.
* ``mesh_1d_chain(T)``: non-periodic chain, neighbours i-1 and i+1.

Blocks (seeded numpy PCG64 stream, drawn in a fixed order: all J blocks in
block-CSR order, then the Q of every mass block, then R):

* J diagonal blocks  N(0,1)/sqrt(m) - sigma*I,
* J face blocks      N(0, 0.25^2)/sqrt(m)   (0.25 is the standard deviation),
* M_i = Q^T Q / m + I with Q ~ N(0,1) (m x m),
* R ~ N(0,1) over s*T*m, stage-major.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np


def mesh_2d_periodic(nx: int, ny: int):
    """Face-neighbour lists of the split periodic quad grid (r = 3)."""
    if nx < 3 or ny < 3:
        raise ValueError("nx, ny >= 3 so that no neighbour repeats")
    nbrs = []
    for y in range(ny):
        for x in range(nx):
            q = y * nx + x
            # lower triangle (0,0)-(1,0)-(1,1): bottom edge, right edge, diagonal
            lo = [2 * (((y - 1) % ny) * nx + x) + 1, 2 * (y * nx + (x + 1) % nx) + 1, 2 * q + 1]
            # upper triangle (0,0)-(1,1)-(0,1): top edge, left edge, diagonal
            up = [2 * (((y + 1) % ny) * nx + x), 2 * (y * nx + (x - 1) % nx), 2 * q]
            nbrs.append(lo)
            nbrs.append(up)
    return nbrs


_PERMS = list(itertools.permutations(range(3)))
_PERM_ID = {p: k for k, p in enumerate(_PERMS)}


def mesh_3d_periodic(nx: int, ny: int | None = None, nz: int | None = None):
    """Face-neighbour lists of the periodic Kuhn-tetrahedra grid (r = 4).

    Tet p = (p0, p1, p2) of a cube has vertices 0, e_p0, e_p0 + e_p1, (1,1,1).
    Its faces: opposite vertex 1 -> tet (p1, p0, p2) of the same cube; opposite
    vertex 2 -> tet (p0, p2, p1) of the same cube; opposite vertex 0 (on the
    plane x_p0 = 1) -> tet (p1, p2, p0) of the cube shifted by +e_p0; opposite
    vertex 3 (on x_p2 = 0) -> tet (p2, p0, p1) of the cube shifted by -e_p2.
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    if min(nx, ny, nz) < 3:
        raise ValueError("grid sizes >= 3 so that no neighbour repeats")
    dims = (nx, ny, nz)

    def cube_id(c):
        return (c[2] * ny + c[1]) * nx + c[0]

    nbrs = []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                c = (x, y, z)
                for p in _PERMS:
                    here = 6 * cube_id(c)
                    lst = [here + _PERM_ID[(p[1], p[0], p[2])], here + _PERM_ID[(p[0], p[2], p[1])]]
                    cp = list(c)
                    cp[p[0]] = (cp[p[0]] + 1) % dims[p[0]]
                    lst.append(6 * cube_id(cp) + _PERM_ID[(p[1], p[2], p[0])])
                    cm = list(c)
                    cm[p[2]] = (cm[p[2]] - 1) % dims[p[2]]
                    lst.append(6 * cube_id(cm) + _PERM_ID[(p[2], p[0], p[1])])
                    nbrs.append(lst)
    return nbrs


def mesh_1d_chain(T: int):
    """Non-periodic chain: element i neighbours i-1 and i+1 (block tridiagonal)."""
    return [[j for j in (i - 1, i + 1) if 0 <= j < T] for i in range(T)]


def bsr_pattern(nbrs):
    """Block-CSR pattern (row_ptr, col_idx) with the diagonal, columns sorted."""
    T = len(nbrs)
    row_ptr = np.zeros(T + 1, np.int32)
    cols = []
    for i, lst in enumerate(nbrs):
        row = sorted(set(lst) | {i})
        if len(row) != len(lst) + 1:
            raise ValueError("element %d has a repeated or self neighbour" % i)
        cols.extend(row)
        row_ptr[i + 1] = len(cols)
    return row_ptr, np.asarray(cols, np.int32)


@dataclass
class StageProblem:
    """One stage-system instance: pattern, J (shared by all stages), M, R, dt."""

    name: str
    s: int
    T: int
    m: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    J: np.ndarray  # (nnzb, m, m)
    M: np.ndarray  # (T, m, m)
    R: np.ndarray  # (s*T*m,) stage-major
    dt: float
    sigma: float
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.T * self.m

    @property
    def nnzb(self):
        return int(self.row_ptr[-1])


def random_blocks(row_ptr, col_idx, m, sigma, rng, scale_face=0.25):
    """J and M per the recipe in the module docstring."""
    T = row_ptr.size - 1
    nnzb = int(row_ptr[-1])
    J = rng.standard_normal((nnzb, m, m))
    rows = np.repeat(np.arange(T), np.diff(row_ptr))
    diag = rows == col_idx
    inv_sqrt_m = 1.0 / math.sqrt(m)
    J[diag] *= inv_sqrt_m
    J[~diag] *= scale_face * inv_sqrt_m
    J[diag] -= sigma * np.eye(m)
    Q = rng.standard_normal((T, m, m))
    M = np.matmul(np.transpose(Q, (0, 2, 1)), Q) / m + np.eye(m)
    return J, M


def make_problem(nbrs, m, s, dt, sigma, seed, name="custom", meta=None):
    rng = np.random.default_rng(seed)
    row_ptr, col_idx = bsr_pattern(nbrs)
    J, M = random_blocks(row_ptr, col_idx, m, sigma, rng)
    T = len(nbrs)
    R = rng.standard_normal(s * T * m)
    return StageProblem(name, s, T, m, row_ptr, col_idx, J, M, R, float(dt), float(sigma), seed,
                        dict(meta or {}))


# Named workloads (the shapes of the paper's DG problems; Sec. 2.1 block
# structure, Sec. 5 problem sizes and polynomial degrees).
def config(name: str, seed: int = 0, dt: float | None = None):
    """Build a named workload.

    c0: 2D periodic 32x32 split grid, T=2048, p=1 (m=12), s=2, dt=0.1, sigma=4.
    c1: 2D periodic 100x100 split grid, T=20000, p=3 (m=40), s=3, dt in
        {0.01, 0.1, 1} (default 0.1), sigma=6.
    c2: 3D periodic 20^3 Kuhn grid, T=48000, p=2 (m=50), s=3, dt=0.1, sigma=6.
    tiny2d / tiny3d / chain: small cases for tests.
    """
    if name == "c0":
        return make_problem(mesh_2d_periodic(32, 32), 12, 2, 0.1 if dt is None else dt, 4.0, seed,
                            name)
    if name == "c1":
        return make_problem(mesh_2d_periodic(100, 100), 40, 3, 0.1 if dt is None else dt, 6.0,
                            seed, name)
    if name == "c2":
        return make_problem(mesh_3d_periodic(20), 50, 3, 0.1 if dt is None else dt, 6.0, seed,
                            name)
    raise KeyError(name)


def mesh_for_elements(T_target: int, dim: int):
    """Periodic grid with about T_target elements (2D: 2 per quad, 3D: 6 per cube)."""
    if dim == 2:
        nx = max(3, round(math.sqrt(T_target / 2)))
        ny = max(3, math.ceil(T_target / (2 * nx)))
        return mesh_2d_periodic(nx, ny)
    n = max(3, round((T_target / 6) ** (1.0 / 3.0)))
    nz = max(3, math.ceil(T_target / (6 * n * n)))
    return mesh_3d_periodic(n, n, nz)


def block_size(dim: int, p: int) -> int:
    """m = (number of P_p basis functions) x (number of conserved variables)."""
    if dim == 2:
        return (p + 1) * (p + 2) // 2 * 4
    return (p + 1) * (p + 2) * (p + 3) // 6 * 5


def _pattern_from_array(nb):
    """bsr_pattern of a (T, r) neighbour array, vectorised: each row's
    neighbours and the element itself, sorted."""
    T, r = nb.shape
    rows = np.sort(np.concatenate([nb, np.arange(T)[:, None]], axis=1), axis=1)
    if np.any(rows[:, 1:] == rows[:, :-1]):
        raise ValueError("an element has a repeated or self neighbour")
    row_ptr = (np.arange(T + 1) * (r + 1)).astype(np.int32)
    return row_ptr, rows.reshape(-1).astype(np.int32)


def pattern_2d_periodic(nx: int, ny: int):
    """bsr_pattern(mesh_2d_periodic(nx, ny)) without Python loops."""
    if nx < 3 or ny < 3:
        raise ValueError("nx, ny >= 3 so that no neighbour repeats")
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    y, x = y.reshape(-1), x.reshape(-1)
    q = y * nx + x
    nb = np.empty((2 * nx * ny, 3), np.int64)
    nb[0::2] = np.stack([2 * (((y - 1) % ny) * nx + x) + 1, 2 * (y * nx + (x + 1) % nx) + 1, 2 * q + 1], axis=1)
    nb[1::2] = np.stack([2 * (((y + 1) % ny) * nx + x), 2 * (y * nx + (x - 1) % nx), 2 * q], axis=1)
    return _pattern_from_array(nb)


def pattern_3d_periodic(nx: int, ny: int | None = None, nz: int | None = None):
    """bsr_pattern(mesh_3d_periodic(nx, ny, nz)) without Python loops (the
    same face rules as mesh_3d_periodic)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    if min(nx, ny, nz) < 3:
        raise ValueError("grid sizes >= 3 so that no neighbour repeats")
    dims = np.array([nx, ny, nz])
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    c = np.stack([x.reshape(-1), y.reshape(-1), z.reshape(-1)], axis=1)  # cube-major order (z, y, x)

    def cube_id(cc):
        return (cc[:, 2] * ny + cc[:, 1]) * nx + cc[:, 0]

    here = 6 * cube_id(c)
    nb = np.empty((c.shape[0], 6, 4), np.int64)
    for k, p in enumerate(_PERMS):
        cp = c.copy()
        cp[:, p[0]] = (cp[:, p[0]] + 1) % dims[p[0]]
        cm = c.copy()
        cm[:, p[2]] = (cm[:, p[2]] - 1) % dims[p[2]]
        nb[:, k, 0] = here + _PERM_ID[(p[1], p[0], p[2])]
        nb[:, k, 1] = here + _PERM_ID[(p[0], p[2], p[1])]
        nb[:, k, 2] = 6 * cube_id(cp) + _PERM_ID[(p[1], p[2], p[0])]
        nb[:, k, 3] = 6 * cube_id(cm) + _PERM_ID[(p[2], p[0], p[1])]
    return _pattern_from_array(nb.reshape(-1, 4))


def pattern_for_elements(T_target: int, dim: int):
    """bsr_pattern(mesh_for_elements(T_target, dim)), vectorised."""
    if dim == 2:
        nx = max(3, round(math.sqrt(T_target / 2)))
        ny = max(3, math.ceil(T_target / (2 * nx)))
        return pattern_2d_periodic(nx, ny)
    n = max(3, round((T_target / 6) ** (1.0 / 3.0)))
    nz = max(3, math.ceil(T_target / (6 * n * n)))
    return pattern_3d_periodic(n, n, nz)


def make_problem_device(nbrs, m, s, dt, sigma, seed, device, name="device", meta=None):
    """The same block recipe drawn on the GPU (torch's seeded device
    generator, so the numbers differ from make_problem's numpy stream): for
    streams of many or large requests whose host generation would dominate.
    J, M, R are CUDA float64 tensors; the pattern stays in numpy.  nbrs is a
    neighbour list or an already built (row_ptr, col_idx) pattern."""
    import torch
    if isinstance(nbrs, tuple) and len(nbrs) == 2 and isinstance(nbrs[0], np.ndarray):
        row_ptr, col_idx = nbrs
    else:
        row_ptr, col_idx = bsr_pattern(nbrs)
    T = int(row_ptr.size - 1)
    nnzb = int(row_ptr[-1])
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    J = torch.randn((nnzb, m, m), generator=gen, device=device, dtype=torch.float64)
    rows = np.repeat(np.arange(T), np.diff(row_ptr))
    diag = torch.as_tensor(rows == col_idx, device=device)
    inv_sqrt_m = 1.0 / math.sqrt(m)
    scale = torch.where(diag, inv_sqrt_m, 0.25 * inv_sqrt_m).to(torch.float64)
    J *= scale[:, None, None]
    eye = torch.eye(m, device=device, dtype=torch.float64)
    J[diag] -= sigma * eye
    Q = torch.randn((T, m, m), generator=gen, device=device, dtype=torch.float64)
    M = torch.matmul(Q.transpose(1, 2), Q) / m + eye
    R = torch.randn((s * T * m,), generator=gen, device=device, dtype=torch.float64)
    return StageProblem(name, s, T, m, row_ptr, col_idx, J, M, R, float(dt), float(sigma), seed,
                        dict(meta or {}))


def serving_stream(n, rate, seed, elements=(1000, 40000), degrees=(1, 2, 3), stages=(2, 3),
                   dims=(2, 3), dt_range=(1e-3, 1.0)):
    """Poisson stream of stage-solve requests: arrival times (s), and per
    request (dim, p, m, s, target elements, dt, seed).  dt is log-uniform."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    out = []
    for k in range(n):
        dim = int(rng.choice(dims))
        p = int(rng.choice(degrees))
        s = int(rng.choice(stages))
        T = int(rng.integers(elements[0], elements[1] + 1))
        dt = float(np.exp(rng.uniform(np.log(dt_range[0]), np.log(dt_range[1]))))
        out.append(dict(arrival=float(t[k]), dim=dim, p=p, m=block_size(dim, p), s=s, elements=T, dt=dt,
                        seed=int(seed) * 100003 + k))
    return out


def batched_uneven(n, seed, elements=(500, 5000), degrees=(1, 2, 3), stages=(2, 3)):
    """Independent 2D meshes with uniform element counts, P1..P3 blocks and
    2 or 3 stages (the batched uneven workload), as request descriptors."""
    return serving_stream(n, 1.0, seed, elements=elements, degrees=degrees, stages=stages, dims=(2,),
                          dt_range=(0.1, 0.1))
