"""Per-equation magnitude scale of the residual, used to state parity tolerances.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

At low Mach the pressure p ~ 1/(gamma M^2) is large while its fluctuations are
O(1) (Sec. 2.1), so a residual equation sums terms much larger than its result.
The rounding error of any FP64 evaluation of R_k is therefore a small multiple of
unit round-off times the magnitude of those terms, not of R_k itself.  The scale

    sigma_k = max_points (|F_k| + |G_k|) / |J|
            + max_faces |S| |lambda|_max (|Gamma~| |q~|)_k / min |J|

collects the two largest kinds of terms (the computational fluxes of Eq.
computational_flux differentiated along lines, and the preconditioned dissipation
of Eq. Rosanov acting on face states).  Tolerances are stated as multiples of it.

``divergence_scale`` is the smaller, flux-divergence scale
max(||R_k||_inf, max_points max(|d F_k/d xi|, |d G_k/d eta|) / |J|): the size of the
differentiated fluxes themselves rather than of the terms summed into them (a
uniform pressure contributes nothing to it on a static mesh).  Errors are reported in
both scales.
"""
from __future__ import annotations

import numpy as np

from . import physics as ph
from .residual import Mesh, d_eta, d_xi, residual, trace
from .basis import make_basis
from .geometry import FACE_L, FACE_R, FACE_B, FACE_T, element_geometry


def residual_scale(q, mesh: Mesh, p: int, gas: ph.Gas) -> np.ndarray:
    b = make_basis(p)
    geo = element_geometry(mesh.corners, mesh.vel, b)
    P = residual(q, mesh, p, gas, b, geo, parts=True)
    jmin = np.min(geo.sol.J)
    s_flux = np.max((np.abs(P.F) + np.abs(P.G)) / geo.sol.J, axis=(1, 2, 3))
    left, right, bottom, top = mesh.neighbours()
    own = np.arange(mesh.ne)
    top = np.where(top < 0, own, top)       # a boundary face: the element's own trace
    s_diss = np.zeros(4)
    for fm, fp, nb, along in ((FACE_R, FACE_L, right, True), (FACE_T, FACE_B, top, False)):
        qm = trace(b, q, fm)
        qp = trace(b, q, fp)[:, nb]
        fg = geo.faces[fm]
        S = fg.Sxi if along else fg.Seta
        Smag = np.sqrt(S[0] ** 2 + S[1] ** 2)
        nvec = (S[0] / Smag, S[1] / Smag)
        qa = tuple(0.5 * (qm[k] + qp[k]) for k in range(4))
        eps = ph.epsilon(qa, fg.vg, gas)
        lam = ph.eigenvalues(qa, nvec, fg.vg, eps, gas)
        lmax = np.max(np.abs(np.stack(lam)), axis=0)
        G = ph.Gamma_matrix(qa, eps, gas)
        mag = np.einsum("ij...,j...->i...", np.abs(G), np.abs(np.stack(qa)))
        s_diss = np.maximum(s_diss, np.max(Smag * lmax * mag, axis=(1, 2)) / jmin)
    return s_flux + s_diss


def flux_derivative_scale(q, mesh: Mesh, p: int, gas: ph.Gas) -> np.ndarray:
    """Per equation max over solution points of max(|d F_k/d xi|, |d G_k/d eta|) / |J|,
    F and G the computational fluxes at the solution points differentiated along lines
    (interpolant derivatives, element by element)."""
    b = make_basis(p)
    geo = element_geometry(mesh.corners, mesh.vel, b)
    P = residual(q, mesh, p, gas, b, geo, parts=True)
    dF = np.abs(d_xi(b, P.F)) / geo.sol.J
    dG = np.abs(d_eta(b, P.G)) / geo.sol.J
    return np.maximum(dF.max(axis=(1, 2, 3)), dG.max(axis=(1, 2, 3)))


def divergence_scale(q, mesh: Mesh, p: int, gas: ph.Gas) -> np.ndarray:
    """Per equation max(||R_k||_inf, flux_derivative_scale_k)."""
    R = residual(q, mesh, p, gas)
    return np.maximum(np.abs(R).max(axis=(1, 2, 3)), flux_derivative_scale(q, mesh, p, gas))
