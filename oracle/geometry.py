"""Element geometry and grid velocity of Sec. 2.3 on straight-sided (bilinear) quads.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

For the bilinear map x(xi, eta) = sum_a N_a(xi, eta) x_a through the 4 corners:
  |J| = x_xi y_eta - x_eta y_xi,
  S_xi  = |J| grad(xi)  = ( y_eta, -x_eta),
  S_eta = |J| grad(eta) = (-y_xi,   x_xi),
  v_g   = sum_a N_a v_a (corner velocities interpolated with the same map),
  St_xi = |J| xi_t = -v_g . S_xi,   St_eta = |J| eta_t = -v_g . S_eta.
Evaluated at solution points (xi_i, eta_j) and at the flux points of the four faces
L (xi=-1), R (xi=+1), B (eta=-1), T (eta=+1).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .basis import Basis

FACE_L, FACE_R, FACE_B, FACE_T = 0, 1, 2, 3


def _shape(xi, eta):
    N = np.stack([(1 - xi) * (1 - eta), (1 + xi) * (1 - eta),
                  (1 + xi) * (1 + eta), (1 - xi) * (1 + eta)]) / 4.0
    dNx = np.stack([-(1 - eta), (1 - eta), (1 + eta), -(1 + eta)]) / 4.0
    dNe = np.stack([-(1 - xi), -(1 + xi), (1 + xi), (1 - xi)]) / 4.0
    return N, dNx, dNe


@dataclasses.dataclass
class PointGeom:
    x: np.ndarray
    y: np.ndarray
    J: np.ndarray          # |J|
    Sxi: np.ndarray        # [2, ...]
    Seta: np.ndarray       # [2, ...]
    vg: np.ndarray         # [2, ...]
    St_xi: np.ndarray
    St_eta: np.ndarray


def _eval(corners, vel, xi, eta) -> PointGeom:
    N, dNx, dNe = _shape(xi, eta)
    X, Y = corners[..., 0], corners[..., 1]
    VX, VY = vel[..., 0], vel[..., 1]
    # einsum over corner index a: N[a, ...] with X[e, a]
    x = np.einsum("a...,ea->e...", N, X)
    y = np.einsum("a...,ea->e...", N, Y)
    x_xi = np.einsum("a...,ea->e...", dNx, X)
    x_eta = np.einsum("a...,ea->e...", dNe, X)
    y_xi = np.einsum("a...,ea->e...", dNx, Y)
    y_eta = np.einsum("a...,ea->e...", dNe, Y)
    ug = np.einsum("a...,ea->e...", N, VX)
    vg = np.einsum("a...,ea->e...", N, VY)
    J = x_xi * y_eta - x_eta * y_xi
    Sxi = np.stack([y_eta, -x_eta])
    Seta = np.stack([-y_xi, x_xi])
    St_xi = -(ug * Sxi[0] + vg * Sxi[1])
    St_eta = -(ug * Seta[0] + vg * Seta[1])
    return PointGeom(x, y, J, Sxi, Seta, np.stack([ug, vg]), St_xi, St_eta)


@dataclasses.dataclass
class Geometry:
    sol: PointGeom                 # arrays [Ne, n(j), n(i)]
    faces: list                    # 4 PointGeom, arrays [Ne, n] along the face


def element_geometry(corners: np.ndarray, vel: np.ndarray, b: Basis) -> Geometry:
    xs = b.xs
    eta, xi = np.meshgrid(xs, xs, indexing="ij")  # [j, i]
    sol = _eval(corners, vel, xi, eta)
    one = np.ones_like(xs)
    faces = [
        _eval(corners, vel, -one, xs),   # L: xi=-1, along eta_j
        _eval(corners, vel, one, xs),    # R: xi=+1, along eta_j
        _eval(corners, vel, xs, -one),   # B: eta=-1, along xi_i
        _eval(corners, vel, xs, one),    # T: eta=+1, along xi_i
    ]
    return Geometry(sol, faces)
