"""1-D basis of the FR/CPR scheme on [-1, 1] (Sec. 3.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* Solution points: Gauss-Legendre points (the paper does not name its point set;
  Gauss points with the Radau correction functions recover nodal DG, Sec. 3.1).
* Lagrange basis l_k through the solution points; D[i, k] = l_k'(xi_i);
  extrapolation rows l_k(-1), l_k(+1).
* Correction functions: g_L is the right Radau polynomial of degree p+1
  (g_L(-1) = 1, g_L(1) = 0) and g_R the left one (g_R(1) = 1, g_R(-1) = 0),
  g_R = (P_{p+1} + P_p)/2 and g_L(xi) = g_R(-xi), in Legendre polynomials P_k.
"""
from __future__ import annotations

import dataclasses

import numpy as np
from numpy.polynomial import legendre as L


def gauss_points(p: int) -> tuple[np.ndarray, np.ndarray]:
    """Gauss-Legendre points and weights, p+1 of them (library rule)."""
    return L.leggauss(p + 1)


def lagrange_values(xs: np.ndarray, x: float) -> np.ndarray:
    """l_k(x) for the Lagrange basis through xs, from the product definition."""
    n = len(xs)
    out = np.ones(n)
    for k in range(n):
        for m in range(n):
            if m != k:
                out[k] *= (x - xs[m]) / (xs[k] - xs[m])
    return out


def lagrange_derivative_matrix(xs: np.ndarray) -> np.ndarray:
    """D[i, k] = l_k'(xs[i]) from the derivative of the product definition."""
    n = len(xs)
    D = np.zeros((n, n))
    for i in range(n):
        for k in range(n):
            s = 0.0
            for m in range(n):
                if m == k:
                    continue
                term = 1.0 / (xs[k] - xs[m])
                for l in range(n):
                    if l != k and l != m:
                        term *= (xs[i] - xs[l]) / (xs[k] - xs[l])
                s += term
            D[i, k] = s
    return D


def radau_right_correction(p: int) -> np.ndarray:
    """Legendre-series coefficients of g_R = (P_{p+1} + P_p)/2 (left Radau polynomial)."""
    c = np.zeros(p + 2)
    c[p + 1] = 0.5
    c[p] = 0.5
    return c


def radau_left_correction(p: int) -> np.ndarray:
    """Legendre-series coefficients of g_L(xi) = g_R(-xi) = (-1)^(p+1)/2 (P_{p+1} - P_p)."""
    c = np.zeros(p + 2)
    s = (-1.0) ** (p + 1)
    c[p + 1] = 0.5 * s
    c[p] = -0.5 * s
    return c


@dataclasses.dataclass
class Basis:
    p: int
    xs: np.ndarray       # solution points
    ws: np.ndarray       # Gauss weights
    D: np.ndarray        # [n, n]
    lL: np.ndarray       # l_k(-1)
    lR: np.ndarray       # l_k(+1)
    dgL: np.ndarray      # g_L'(xs[i])
    dgR: np.ndarray      # g_R'(xs[i])
    dgL_end: float       # g_L'(-1)  (face end of the left face)
    dgR_end: float       # g_R'(+1)  (face end of the right face)

    @property
    def n(self) -> int:
        return self.p + 1


def make_basis(p: int) -> Basis:
    xs, ws = gauss_points(p)
    gR = radau_right_correction(p)
    gL = radau_left_correction(p)
    dgR = L.legder(gR)
    dgL = L.legder(gL)
    return Basis(
        p=p, xs=xs, ws=ws,
        D=lagrange_derivative_matrix(xs),
        lL=lagrange_values(xs, -1.0),
        lR=lagrange_values(xs, 1.0),
        dgL=L.legval(xs, dgL),
        dgR=L.legval(xs, dgR),
        dgL_end=float(L.legval(-1.0, dgL)),
        dgR_end=float(L.legval(1.0, dgR)),
    )
