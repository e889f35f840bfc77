"""Pins of the oracle's 1-D FR basis (Sec. 3.1) against closed forms and textbook identities."""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as L

from oracle import basis as bs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gauss_legendre.txt")


def _golden():
    rows = {}
    env = {"sqrt": math.sqrt}
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        p, x, w = line.split(None, 2)
        rows.setdefault(int(p), []).append((eval(x, env), eval(w.strip(), env)))
    return rows


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_gauss_points_match_closed_form(p):
    ref = np.array(_golden()[p])
    xs, ws = bs.gauss_points(p)
    np.testing.assert_allclose(xs, ref[:, 0], atol=1e-15)
    np.testing.assert_allclose(ws, ref[:, 1], atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_derivative_matrix_exact_on_polynomials(p):
    b = bs.make_basis(p)
    for m in range(p + 1):
        f = b.xs ** m
        df = m * b.xs ** (m - 1) if m > 0 else 0 * b.xs
        np.testing.assert_allclose(b.D @ f, df, atol=1e-12)
    np.testing.assert_allclose(b.D.sum(axis=1), 0.0, atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_extrapolation_exact_on_polynomials(p):
    b = bs.make_basis(p)
    for m in range(p + 1):
        assert abs(b.lR @ b.xs ** m - 1.0) < 1e-13
        assert abs(b.lL @ b.xs ** m - (-1.0) ** m) < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_radau_corrections_end_values(p):
    gR = bs.radau_right_correction(p)
    gL = bs.radau_left_correction(p)
    assert abs(L.legval(1.0, gR) - 1) < 1e-15 and abs(L.legval(-1.0, gR)) < 1e-15
    assert abs(L.legval(-1.0, gL) - 1) < 1e-15 and abs(L.legval(1.0, gL)) < 1e-15
    b = bs.make_basis(p)
    # g_R'(1) = (p+1)^2/2 and g_L'(-1) = -(p+1)^2/2 (Huynh's g_DG)
    assert abs(b.dgR_end - (p + 1) ** 2 / 2) < 1e-12
    assert abs(b.dgL_end + (p + 1) ** 2 / 2) < 1e-12
    # g_R is orthogonal to all polynomials of degree p-1 (Radau property)
    xs, ws = L.leggauss(p + 3)
    for m in range(p):
        assert abs(np.sum(ws * L.legval(xs, gR) * xs ** m)) < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_radau_fr_equals_nodal_dg_lifting(p):
    """With Gauss solution points the Radau correction reproduces nodal DG (Sec. 3.1):
    g_R'(xi_i) = l_i(1)/w_i and g_L'(xi_i) = -l_i(-1)/w_i (diagonal mass matrix lifting)."""
    b = bs.make_basis(p)
    np.testing.assert_allclose(b.dgR, b.lR / b.ws, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(b.dgL, -b.lL / b.ws, rtol=1e-12, atol=1e-12)
