"""Pins of the oracle's tableau (App. A, Table 1, Sec. 3, Sec. 4.1, Sec. 4.3.2).

Each check compares the oracle with something other than itself: the closed
forms printed in App. A, the order conditions, the Pade approximant of e^z
(the known stability function of Radau IIA) and the error constants of Table 1.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import tableau

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split(None, 4) if name == "radau_app_a.txt" else line.split())
    return rows


def _eval(expr):
    return eval(expr, {"__builtins__": {}}, {"sqrt": math.sqrt})


def _app_a(scheme):
    s = 2 if scheme == "RADAU23" else 3
    A = np.zeros((s, s))
    b = np.zeros(s)
    c = np.zeros(s)
    for name, what, i, j, expr in _read("radau_app_a.txt"):
        if name != scheme:
            continue
        if what == "A":
            A[int(i), int(j)] = _eval(expr)
        elif what == "b":
            b[int(i)] = _eval(expr)
        else:
            c[int(i)] = _eval(expr)
    return A, b, c


@pytest.mark.parametrize("scheme,s", [("RADAU23", 2), ("RADAU35", 3)])
def test_collocation_matches_app_a_closed_form(scheme, s):
    A, b, c = tableau.radau_iia(s)
    Ag, bg, cg = _app_a(scheme)
    np.testing.assert_allclose(A, Ag, rtol=0, atol=2e-15)
    np.testing.assert_allclose(b, bg, rtol=0, atol=2e-15)
    np.testing.assert_allclose(c, cg, rtol=0, atol=2e-15)


@pytest.mark.parametrize("scheme,s", [("RADAU23", 2), ("RADAU35", 3)])
def test_closed_forms_in_oracle_match_app_a(scheme, s):
    A, b, c = tableau.radau23() if s == 2 else tableau.radau35()
    Ag, bg, cg = _app_a(scheme)
    np.testing.assert_allclose(A, Ag, rtol=0, atol=1e-15)
    np.testing.assert_allclose(b, bg, rtol=0, atol=1e-15)
    np.testing.assert_allclose(c, cg, rtol=0, atol=1e-15)


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5])
def test_order_conditions(s):
    """Radau IIA: B(2s-1) (quadrature order) and C(s) (stage order s, Sec. 3),
    b = last row of A, row sums = c, c_s = 1."""
    A, b, c = tableau.radau_iia(s)
    for k in range(1, 2 * s):
        assert abs(np.dot(b, c ** (k - 1)) - 1.0 / k) < 1e-13, k
    for k in range(1, s + 1):
        np.testing.assert_allclose(A @ c ** (k - 1), c ** k / k, rtol=0, atol=1e-13)
    np.testing.assert_allclose(A.sum(axis=1), c, atol=1e-14)
    np.testing.assert_array_equal(b, A[-1])
    assert c[-1] == 1.0
    assert np.all(np.diff(c) > 0) and c[0] > 0


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5])
def test_bt_ainv_is_last_unit_vector(s):
    """Sec. 4.1: for Radau IIA, b^T A^{-1} = (0, ..., 0, 1)."""
    A, b, _ = tableau.radau_iia(s)
    e = b @ tableau.inverse(A)
    expect = np.zeros(s)
    expect[-1] = 1.0
    np.testing.assert_allclose(e, expect, atol=1e-12)


def _pade_coeffs(k, l):
    """Numerator / denominator of the (k, l) Pade approximant of e^z (exact)."""
    P = [Fraction(math.factorial(k + l - j) * math.factorial(k),
                  math.factorial(k + l) * math.factorial(j) * math.factorial(k - j)) for j in range(k + 1)]
    Q = [Fraction(math.factorial(k + l - j) * math.factorial(l),
                  math.factorial(k + l) * math.factorial(j) * math.factorial(l - j)) * (-1) ** j
         for j in range(l + 1)]
    return P, Q


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5])
def test_stability_function_is_pade(s):
    """Sec. 3: Radau IIA is L-stable; its R(z) is the (s-1, s) Pade approximant of e^z."""
    A, b, _ = tableau.radau_iia(s)
    P, Q = _pade_coeffs(s - 1, s)
    for z in [-1.0, -0.3, 0.5, -7.0, 2.0 + 1.5j, -20.0 - 3.0j]:
        num = sum(float(p) * z ** j for j, p in enumerate(P))
        den = sum(float(q) * z ** j for j, q in enumerate(Q))
        assert abs(tableau.stability_function(A, b, z) - num / den) < 1e-12 * max(1, abs(num / den))
    # L-stability: R(z) -> 0 as z -> -inf, like s/|z|
    big = -1e6
    assert abs(tableau.stability_function(A, b, big)) < 10 * s / 1e6


def test_table1_leading_error_coefficients():
    """Table 1: the leading error coefficient C of each Radau IIA scheme, where
    e^z - R(z) = C z^{2s} + O(z^{2s+1}); R's Taylor coefficients are
    b^T A^{j-1} 1 (Neumann series of (I - zA)^{-1})."""
    for scheme, s, order, stage_order, coef in _read("table1_schemes.txt"):
        s, order = int(s), int(order)
        A, b, _ = tableau.radau_iia(s)
        one = np.ones(s)
        taylor = [1.0] + [b @ np.linalg.matrix_power(A, j - 1) @ one for j in range(1, 2 * s + 1)]
        for j in range(order + 1):
            assert abs(taylor[j] - 1.0 / math.factorial(j)) < 1e-13, (scheme, j)
        C = 1.0 / math.factorial(2 * s) - taylor[2 * s]
        assert float("%.2e" % abs(C)) == float(coef), (scheme, C, coef)


def test_radau23_inverse_and_shift_rule():
    """Hand-derived A^{-1}, shift (Sec. 4.3.2) and d_i for RADAU23."""
    vals = {}
    for what, i, _, expr in _read("radau23_inverse.txt"):
        vals.setdefault(what, {})[int(i)] = Fraction(expr)
    A, _, _ = tableau.radau_iia(2)
    Ainv = tableau.inverse(A)
    rows = [line.split() for line in open(os.path.join(GOLDEN, "radau23_inverse.txt"))
            if line.strip() and not line.startswith("#")]
    for what, i, j, expr in rows:
        if what == "Ainv":
            assert abs(Ainv[int(i), int(j)] - float(Fraction(expr))) < 1e-14
    alpha = oracle.shift_column_rule(Ainv)
    np.testing.assert_allclose(alpha, [float(vals["alpha"][0]), float(vals["alpha"][1])], atol=1e-14)
    np.testing.assert_allclose(tableau.shift_column_rule(Ainv), alpha, atol=0)
    d = np.diag(Ainv) + alpha
    np.testing.assert_allclose(d, [float(vals["d"][0]), float(vals["d"][1])], atol=1e-14)
    # the row reading gives (1/2, 9/2): the two readings differ (kept selectable)
    np.testing.assert_allclose(tableau.shift_row_rule(Ainv), [0.5, 4.5], atol=1e-14)
