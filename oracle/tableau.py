"""Butcher tableaux of the Radau IIA schemes (oracle side).

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
benchmark's CPU-baseline leg; the library's CUDA path never imports it.

* ``radau_iia(s)`` builds the s-stage Radau IIA tableau by collocation, the
  construction of App. A: the abscissae c_k are the zeros of
  Q_s(x) = P_s(2x - 1) - P_{s-1}(2x - 1) (P_n the Legendre polynomials), l_k is
  the Lagrange basis polynomial on those abscissae and a_ik is the integral of
  l_k from 0 to c_i; b is the last row of A (c_s = 1).
* ``radau23()`` / ``radau35()`` are the closed forms printed in App. A.
* ``shift_column_rule(Ainv)`` is the shift of Sec. 4.3.2,
  alpha_i = sum_{j != i} |(A^{-1})_{ji}|.
* ``dirk33()`` / ``esdirk65()`` are the comparison DIRK schemes of Sec. 3
  (Table 1) with the coefficients of App. A: DIRK33 from its closed form in
  alpha, ESDIRK65 from the 16-digit values printed there.

All arithmetic is FP64 numpy; root finding, polynomial integration and the
matrix inverse are library primitives.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly


def radau_iia(s: int):
    """(A, b, c) of the s-stage Radau IIA scheme by collocation (App. A)."""
    if s < 1:
        raise ValueError("s must be >= 1")
    # Q_s(y) = P_s(y) - P_{s-1}(y) in the variable y = 2x - 1
    coef = np.zeros(s + 1)
    coef[s] = 1.0
    coef[s - 1] = -1.0
    y = np.sort(np.real(npleg.legroots(coef)))
    c = (y + 1.0) / 2.0
    c[-1] = 1.0  # the right Radau point is exactly 1
    A = np.zeros((s, s))
    for k in range(s):
        others = np.delete(c, k)
        num = nppoly.polyfromroots(others)  # prod_{q != k} (x - c_q)
        den = np.prod(c[k] - others)
        lk = num / den
        Lk = nppoly.polyint(lk)  # antiderivative with Lk(0) = 0
        for i in range(s):
            A[i, k] = nppoly.polyval(c[i], Lk)
    b = A[-1].copy()
    return A, b, c


def radau23():
    """RADAU23, App. A (closed form)."""
    A = np.array([[5.0 / 12.0, -1.0 / 12.0], [3.0 / 4.0, 1.0 / 4.0]])
    b = np.array([3.0 / 4.0, 1.0 / 4.0])
    c = np.array([1.0 / 3.0, 1.0])
    return A, b, c


def radau35():
    """RADAU35, App. A (closed form with sqrt(6))."""
    r6 = math.sqrt(6.0)
    A = np.array([
        [11.0 / 45.0 - 7.0 * r6 / 360.0, 37.0 / 225.0 - 169.0 * r6 / 1800.0, -2.0 / 225.0 + r6 / 75.0],
        [37.0 / 225.0 + 169.0 * r6 / 1800.0, 11.0 / 45.0 + 7.0 * r6 / 360.0, -2.0 / 225.0 - r6 / 75.0],
        [4.0 / 9.0 - r6 / 36.0, 4.0 / 9.0 + r6 / 36.0, 1.0 / 9.0],
    ])
    b = A[2].copy()
    c = np.array([2.0 / 5.0 - r6 / 10.0, 2.0 / 5.0 + r6 / 10.0, 1.0])
    return A, b, c


def inverse(A):
    """A^{-1} (library inverse)."""
    return np.linalg.inv(np.asarray(A, dtype=np.float64))


def shift_column_rule(Ainv):
    """alpha_i = sum_{j != i} |(A^{-1})_{ji}| (Sec. 4.3.2, printed twice)."""
    Ainv = np.asarray(Ainv, dtype=np.float64)
    s = Ainv.shape[0]
    return np.array([sum(abs(Ainv[j, i]) for j in range(s) if j != i) for i in range(s)])


def shift_row_rule(Ainv):
    """alpha_i = sum_{j != i} |(A^{-1})_{ij}| (the row reading, for comparison)."""
    Ainv = np.asarray(Ainv, dtype=np.float64)
    s = Ainv.shape[0]
    return np.array([sum(abs(Ainv[i, j]) for j in range(s) if j != i) for i in range(s)])


def stability_function(A, b, z):
    """R(z) = 1 + z b^T (I - z A)^{-1} 1 (complex z allowed)."""
    A = np.asarray(A, dtype=np.complex128)
    s = A.shape[0]
    one = np.ones(s, dtype=np.complex128)
    return 1.0 + z * (np.asarray(b) @ np.linalg.solve(np.eye(s) - z * A, one))


def dirk33():
    """DIRK33, App. A: three-stage, third-order, L-stable singly diagonally
    implicit scheme (Sec. 3, Table 1), from the closed form of its diagonal
    alpha (tau_2 = (1 + alpha)/2, b_1, b_2 quadratic in alpha)."""
    th = math.atan(math.sqrt(2.0) / 4.0) / 3.0
    al = 1.0 + math.sqrt(6.0) / 2.0 * math.sin(th) - math.sqrt(2.0) / 2.0 * math.cos(th)
    tau2 = (1.0 + al) / 2.0
    b1 = -(6.0 * al * al - 16.0 * al + 1.0) / 4.0
    b2 = (6.0 * al * al - 20.0 * al + 5.0) / 4.0
    A = np.array([[al, 0.0, 0.0], [tau2 - al, al, 0.0], [b1, b2, al]])
    b = np.array([b1, b2, al])
    c = np.array([al, tau2, 1.0])
    return A, b, c


def esdirk65():
    """ESDIRK65, App. A: six stages (explicit first stage, the other five with
    the same diagonal), fifth order, stiffly accurate (b = last row of A)."""
    g = 0.2780538411364465
    A = np.array([
        [0.0, 0.0, 0.0, 0.0, 0.0, 0.0],
        [0.2780538411364465, g, 0.0, 0.0, 0.0, 0.0],
        [0.3137405401502951, 0.4363327154020044, g, 0.0, 0.0, 0.0],
        [0.2741986534107860, -0.0164268277321164, 0.0048197082596452, g, 0.0, 0.0],
        [-0.2441776975175844, -3.3203529439447852, 0.0477747285706825, 3.2974431145814931, g, 0.0],
        [-0.2786732780227907, 1.8929947094010862, -0.1280948204262490, -1.3574693381380240,
         0.5931888860495311, g],
    ])
    b = A[-1].copy()
    c = np.array([0.0, 0.556107682272893, 1.028127096688746, 0.540645375074761, 0.058741042826253, 1.0])
    return A, b, c
