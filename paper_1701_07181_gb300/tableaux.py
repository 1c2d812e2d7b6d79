"""Butcher tableaux of the comparison DIRK schemes (Sec. 3, Table 1, App. A).

For callers of ``irk.Dirk`` / ``irk_dirk_setup``: the library takes any
lower-triangular tableau; these are the two the paper compares with Radau
IIA.  (The Radau IIA tableaux are built inside the library by collocation
when ``irk_setup`` gets A = NULL.)

* ``dirk33()``: three stages, third order, L-stable, all diagonal entries
  equal to alpha, the middle root of x^3 - 3x^2 + 3x/2 - 1/6; App. A gives
  alpha, tau_2 = (1 + alpha)/2 and the weights b_1, b_2 in closed form.
* ``esdirk65()``: six stages, the first explicit, the other five with the
  same diagonal entry, fifth order, stage order 2, stiffly accurate
  (b = last row of A); coefficients to 16 digits as printed in App. A.

Each returns (A, b, c) as numpy arrays.
"""
from __future__ import annotations

import math

import numpy as np


def dirk33():
    th = math.atan(math.sqrt(2.0) / 4.0) / 3.0
    alpha = 1.0 + math.sqrt(6.0) / 2.0 * math.sin(th) - math.sqrt(2.0) / 2.0 * math.cos(th)
    tau2 = 0.5 * (1.0 + alpha)
    b1 = -(6.0 * alpha ** 2 - 16.0 * alpha + 1.0) / 4.0
    b2 = (6.0 * alpha ** 2 - 20.0 * alpha + 5.0) / 4.0
    A = np.zeros((3, 3))
    A[0, 0] = alpha
    A[1, :2] = (tau2 - alpha, alpha)
    A[2, :] = (b1, b2, alpha)
    return A, A[2].copy(), np.array([alpha, tau2, 1.0])


_ESDIRK65_LOWER = (
    (0.2780538411364465,),
    (0.3137405401502951, 0.4363327154020044),
    (0.2741986534107860, -0.0164268277321164, 0.0048197082596452),
    (-0.2441776975175844, -3.3203529439447852, 0.0477747285706825, 3.2974431145814931),
    (-0.2786732780227907, 1.8929947094010862, -0.1280948204262490, -1.3574693381380240, 0.5931888860495311),
)
_ESDIRK65_GAMMA = 0.2780538411364465
_ESDIRK65_C = (0.0, 0.556107682272893, 1.028127096688746, 0.540645375074761, 0.058741042826253, 1.0)


def esdirk65():
    A = np.zeros((6, 6))
    for i, row in enumerate(_ESDIRK65_LOWER, start=1):
        A[i, :len(row)] = row
        A[i, i] = _ESDIRK65_GAMMA
    return A, A[5].copy(), np.array(_ESDIRK65_C)
