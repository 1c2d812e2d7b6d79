"""Comparison bars of the GPU parity tests.

Every comparison of a GPU result ``a`` with its reference ``b`` (the
oracle's, or the GPU path it must reproduce) is held to one tolerance by two
measures at once:

* norm-wise:     ||a - b||_2 / ||b||_2
* element-wise:  max_i |a_i - b_i| / max_i |b_i|

``rel`` returns the larger of the two, so ``rel(a, b) <= tol`` fails when
either bar is missed: a single wrong entry (a boundary row, the ragged last
thread block) that a global norm would average away still fails the
element-wise bar.
"""
import numpy as np


def _host(a):
    if hasattr(a, "detach"):
        a = a.detach()
    if hasattr(a, "cpu"):
        a = a.cpu().numpy()
    return np.asarray(a, dtype=np.float64).reshape(-1)


def rel_norm(a, b):
    a, b = _host(a), _host(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def rel_max(a, b):
    a, b = _host(a), _host(b)
    mb = np.max(np.abs(b)) if b.size else 0.0
    d = np.max(np.abs(a - b)) if a.size else 0.0
    return float(d / mb) if mb > 0 else float(d)


def rel(a, b):
    """max(norm-wise, element-wise) relative difference of a from b."""
    return max(rel_norm(a, b), rel_max(a, b))
