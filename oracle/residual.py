"""FR/CPR residual R(q^p) of Sec. 3.1 on structured quad meshes (periodic boxes, O-grids).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Discretised equation (Eq. unsteady_pre_mov_cdomain_GCL divided by |J|, i.e. the
computational-domain form whose physical-domain statement is Eq. cpr_ns):

    R = -(1/|J|) [ dF/dxi + dG/deta - q^c (d(|J| xi_t)/dxi + d(|J| eta_t)/deta) ]

with F = |J|(q^c xi_t + f xi_x + g xi_y), G alike, f = f_inv - f_vis.  FR/CPR:
F = F^loc + F^cor, F^loc the degree-p interpolant of the solution-point fluxes,
F^cor = (F^num_L - F^loc(-1)) g_L + (F^num_R - F^loc(+1)) g_R, and
F^num = |J||grad xi| f_n^com sign(n . grad xi) (Eq. norm_f_2), f_n^com =
f_{n,inv}^com (Eq. Rosanov) - f_{n,vis}^com.

Readings where the paper is silent (used identically by the CUDA library):
* F^loc at a face is the interpolated flux polynomial, not the flux of the
  interpolated state.
* d(|J| xi_t)/dxi is the derivative of the degree-p interpolant of |J| xi_t.
* Local gradients use the chain rule on the interpolant derivatives; the
  corrected gradient adds, for each face f, (q^com - q^loc_f) S_f g_f'(xi) / |J|.
* BR2 (Sec. 3.1): grad q^com = (grad q^+,loc + grad q^-,loc)/2 + eta (r^+ + r^-)/2 with
  r^+- = (q^com - q^+-) S_f g'_f(face end) / |J|^+-_f (face f's own jump only) and the
  face penalty eta = BR2_PENALTY = 2 (the form the paper defers to is not available;
  BR2's face term needs a penalty above one for stability: with eta = 1 the viscous
  vortex on 64 x 64 elements of degree 3 grows unstably, with 2 it does not).  The
  corrected gradient at the solution points keeps eta = 1.
* The common viscous flux is f_vis(q^com, grad q^com) . n.

Mesh: element e = j*nx + i; faces in xi are "owned" by their left element (its
R face, the '-' side), faces in eta by their bottom element (its T face).  The xi
direction is always periodic (a box, or the wrap of an O-grid); eta is periodic,
or bounded by boundary faces below row 0 and above row ny-1 (Sec. 3.3 boundary
conditions), each a far field or an adiabatic no-slip wall moving with the grid.

Boundary faces (readings; the paper states the conditions, not the discrete form):
* A boundary state q_b replaces the missing neighbour: far field q_b = q_inf (all
  four primitive variables imposed); wall q_b = (p^-, v_g, T^-) (pressure and
  temperature from the interior trace, velocity of the moving wall).
* Inviscid flux: the preconditioned Rusanov flux between the interior trace and q_b.
* Viscous terms: q^com = q_b; the lifted jump of the face is the full q_b - q^- (one
  side only), in the corrected gradient and in grad q^com = grad q^-,loc + eta r^- with
  r^- = (q_b - q^-) S_f g'_f(face end) / |J|^-_f; at a wall the normal component of
  grad T^com is removed (adiabatic, dT/dn = 0); f_vis(q_b, grad q^com) . n.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import physics as ph
from .basis import Basis, make_basis
from .geometry import FACE_B, FACE_L, FACE_R, FACE_T, Geometry, element_geometry

BR2_PENALTY = 2.0   # BR2 face penalty eta (reading in the module docstring)


WALL, FARFIELD = "wall", "farfield"


@dataclasses.dataclass
class Mesh:
    nx: int
    ny: int
    corners: np.ndarray        # [Ne, 4, 2]
    vel: np.ndarray            # [Ne, 4, 2]
    periodic: tuple = (True, True)
    # (below row 0, above row ny-1): both None (periodic in eta) or both WALL/FARFIELD
    bc: tuple = (None, None)
    q_inf: tuple | None = None   # far-field primitive state (p, u, v, T)

    def __post_init__(self):
        kinds = (None, WALL, FARFIELD)
        if self.bc[0] not in kinds or self.bc[1] not in kinds or \
                (self.bc[0] is None) != (self.bc[1] is None):
            raise ValueError(f"bc must be (None, None) or two of {kinds[1:]}: {self.bc}")
        if FARFIELD in self.bc and self.q_inf is None:
            raise ValueError("a far-field boundary needs q_inf")
        if self.bounded:
            self.periodic = (True, False)

    @property
    def ne(self) -> int:
        return self.nx * self.ny

    @property
    def bounded(self) -> bool:
        return self.bc[0] is not None

    def neighbours(self):
        """(left, right, bottom, top) element index arrays: periodic wrap, -1 across a
        boundary face."""
        if not self.periodic[0]:
            raise NotImplementedError("xi is periodic")
        e = np.arange(self.ne)
        i, j = e % self.nx, e // self.nx
        left = j * self.nx + (i - 1) % self.nx
        right = j * self.nx + (i + 1) % self.nx
        bottom = ((j - 1) % self.ny) * self.nx + i
        top = ((j + 1) % self.ny) * self.nx + i
        if self.bounded:
            bottom = np.where(j == 0, -1, bottom)
            top = np.where(j == self.ny - 1, -1, top)
        return left, right, bottom, top


def boundary_state(kind: str, qe, vg, q_inf):
    """q_b at the flux points of a boundary face from the interior trace qe ([4, ...])
    and the grid velocity vg ([2, ...])."""
    if kind == FARFIELD:
        return np.stack([np.broadcast_to(np.asarray(q_inf[k]), qe[0].shape) + 0 * qe[0]
                         for k in range(4)])
    return np.stack([qe[0], vg[0] + 0 * qe[0], vg[1] + 0 * qe[0], qe[3]])


# ------------------------------------------------------------------ 1-D operators along lines
# Arrays are [..., Ne, n(j), n(i)]: i is the xi index (last axis), j the eta index.

def d_xi(b: Basis, a):
    return np.einsum("ik,...jk->...ji", b.D, a)


def d_eta(b: Basis, a):
    return np.einsum("jk,...ki->...ji", b.D, a)


def trace(b: Basis, a, face: int):
    """Value of the degree-p interpolant at the flux points of ``face`` ([..., Ne, n])."""
    if face == FACE_L:
        return np.einsum("k,...jk->...j", b.lL, a)
    if face == FACE_R:
        return np.einsum("k,...jk->...j", b.lR, a)
    if face == FACE_B:
        return np.einsum("k,...ki->...i", b.lL, a)
    return np.einsum("k,...ki->...i", b.lR, a)


@dataclasses.dataclass
class Parts:
    """Intermediate quantities of one residual evaluation (for tests)."""
    qc: np.ndarray
    grad_loc: tuple
    grad: tuple
    F: np.ndarray
    G: np.ndarray
    Fnum_xi: np.ndarray     # [4, Ne, n]: common flux on the xi-face owned by e (its R face)
    Fnum_eta: np.ndarray    # [4, Ne, n]: on the eta-face owned by e (its T face)
    div: np.ndarray
    R: np.ndarray
    Fnum_bottom: np.ndarray | None = None   # [4, nx, n]: boundary faces below row 0


def residual(q, mesh: Mesh, p: int, gas: ph.Gas, b: Basis | None = None,
             geo: Geometry | None = None, parts: bool = False):
    """R(q^p) at every solution point, ``[4, Ne, n, n]`` (q^c-equation rows)."""
    b = b or make_basis(p)
    geo = geo or element_geometry(mesh.corners, mesh.vel, b)
    left, right, bottom, top = mesh.neighbours()
    e_all = np.arange(mesh.ne)
    row0 = e_all < mesh.nx                          # elements with a face below row 0
    rowL = e_all >= mesh.ne - mesh.nx               # elements with a face above row ny-1
    if mesh.bounded:   # gathers stay in range; boundary entries are replaced below
        bottom = np.where(bottom < 0, e_all, bottom)
        top = np.where(top < 0, e_all, top)
    g = geo.sol
    qs = tuple(q[k] for k in range(4))

    # Pointwise state, conservative variables and inviscid fluxes (Eq. convection).
    qc = ph.conservative(qs, gas)
    finv, ginv = ph.inviscid_flux(qs, gas)

    # Traces of the primitive state at the flux points of each face.
    qf = [trace(b, q, f) for f in range(4)]           # each [4, Ne, n]

    # Common solution on every face (Sec. 3.1): owned xi-faces (R of e, L of right[e]),
    # owned eta-faces (T of e, B of top[e]).
    qm_xi, qp_xi = qf[FACE_R], qf[FACE_L][:, right]
    qm_eta, qp_eta = qf[FACE_T], qf[FACE_B][:, top]
    qcom_xi = 0.5 * (qm_xi + qp_xi)
    qcom_eta = 0.5 * (qm_eta + qp_eta)
    if mesh.bounded:   # boundary states on the faces below row 0 and above row ny-1
        fB, fT = geo.faces[FACE_B], geo.faces[FACE_T]
        qb_bot = boundary_state(mesh.bc[0], qf[FACE_B][:, row0], fB.vg[:, row0], mesh.q_inf)
        qb_top = boundary_state(mesh.bc[1], qf[FACE_T][:, rowL], fT.vg[:, rowL], mesh.q_inf)
        qcom_eta = qcom_eta.astype(np.result_type(qcom_eta, qb_top))
        qcom_eta[:, rowL] = qb_top
    # q^com seen from each face of each element
    qcom_f = [qcom_xi[:, left], qcom_xi, qcom_eta[:, bottom], qcom_eta]
    if mesh.bounded:
        qcom_f[FACE_B] = qcom_f[FACE_B].astype(np.result_type(qcom_f[FACE_B], qb_bot))
        qcom_f[FACE_B][:, row0] = qb_bot

    if gas.viscous:
        # Local physical gradients by the chain rule.
        q_xi, q_eta = d_xi(b, q), d_eta(b, q)
        qx_loc = (g.Sxi[0] * q_xi + g.Seta[0] * q_eta) / g.J
        qy_loc = (g.Sxi[1] * q_xi + g.Seta[1] * q_eta) / g.J
        # Corrected gradient: add the lifted jumps of all four faces.
        qx, qy = qx_loc.copy(), qy_loc.copy()
        for f, dgv, along_i in ((FACE_L, b.dgL, True), (FACE_R, b.dgR, True),
                                (FACE_B, b.dgL, False), (FACE_T, b.dgR, False)):
            S = geo.faces[f].Sxi if along_i else geo.faces[f].Seta    # [2, Ne, n]
            jump = qcom_f[f] - qf[f]                                   # [4, Ne, n]
            if along_i:   # face value depends on j, correction function on i
                cx = jump[:, :, :, None] * S[0][None, :, :, None] * dgv[None, None, None, :]
                cy = jump[:, :, :, None] * S[1][None, :, :, None] * dgv[None, None, None, :]
            else:         # face value depends on i, correction function on j
                cx = jump[:, :, None, :] * S[0][None, :, None, :] * dgv[None, None, :, None]
                cy = jump[:, :, None, :] * S[1][None, :, None, :] * dgv[None, None, :, None]
            qx = qx + cx / g.J
            qy = qy + cy / g.J
        fv, gv = ph.viscous_flux(qs, tuple(qx), tuple(qy), gas)
        f_all, g_all = finv - fv, ginv - gv
        grad_loc, grad = (qx_loc, qy_loc), (qx, qy)
    else:
        f_all, g_all = finv, ginv
        grad_loc = grad = (None, None)

    # Computational fluxes at solution points (Eq. computational_flux).
    F = g.Sxi[0] * f_all + g.Sxi[1] * g_all + g.St_xi * qc
    G = g.Seta[0] * f_all + g.Seta[1] * g_all + g.St_eta * qc

    # Common normal fluxes on owned faces.
    def common(qm, qp, gf_m, gf_p, Jm, Jp, S, vg, dgm, dgp):
        Smag = np.sqrt(S[0] * S[0] + S[1] * S[1])
        nvec = (S[0] / Smag, S[1] / Smag)
        qmt = tuple(qm[k] for k in range(4))
        qpt = tuple(qp[k] for k in range(4))
        fcom = ph.rusanov(qmt, qpt, nvec, vg, gas)
        if gas.viscous:
            qcom = 0.5 * (qm + qp)
            rmx = (qcom - qm) * S[0] * dgm / Jm
            rmy = (qcom - qm) * S[1] * dgm / Jm
            rpx = (qcom - qp) * S[0] * dgp / Jp
            rpy = (qcom - qp) * S[1] * dgp / Jp
            gx = 0.5 * (gf_m[0] + rmx + gf_p[0] + rpx)
            gy = 0.5 * (gf_m[1] + rmy + gf_p[1] + rpy)
            fv, gv = ph.viscous_flux(tuple(qcom[k] for k in range(4)), tuple(gx), tuple(gy), gas)
            fcom = fcom - (fv * nvec[0] + gv * nvec[1])
        return Smag * fcom

    if gas.viscous:
        gtr = [(trace(b, grad_loc[0], f), trace(b, grad_loc[1], f)) for f in range(4)]
        gm_xi = gtr[FACE_R]
        gp_xi = (gtr[FACE_L][0][:, right], gtr[FACE_L][1][:, right])
        gm_eta = gtr[FACE_T]
        gp_eta = (gtr[FACE_B][0][:, top], gtr[FACE_B][1][:, top])
    else:
        gm_xi = gp_xi = gm_eta = gp_eta = None
    fR, fL_of_right = geo.faces[FACE_R], geo.faces[FACE_L]
    fT, fB_of_top = geo.faces[FACE_T], geo.faces[FACE_B]
    liftR, liftL = BR2_PENALTY * b.dgR_end, BR2_PENALTY * b.dgL_end   # BR2 face liftings
    Fnum_xi = common(qm_xi, qp_xi, gm_xi, gp_xi, fR.J, fL_of_right.J[right], fR.Sxi, fR.vg,
                     liftR, liftL)
    Fnum_eta = common(qm_eta, qp_eta, gm_eta, gp_eta, fT.J, fB_of_top.J[top], fT.Seta, fT.vg,
                      liftR, liftL)
    Fnum_bottom = None
    if mesh.bounded:
        gt_top = gt_bot = None
        if gas.viscous:
            gt_top = (gtr[FACE_T][0][:, rowL], gtr[FACE_T][1][:, rowL])
            gt_bot = (gtr[FACE_B][0][:, row0], gtr[FACE_B][1][:, row0])
        # above row ny-1 the element is on the '-' side of +eta, below row 0 on the '+' side
        top_flux = boundary_flux(mesh.bc[1], qf[FACE_T][:, rowL], qb_top, gt_top,
                                 fT.Seta[:, rowL], fT.J[rowL], fT.vg[:, rowL], liftR, True, gas)
        Fnum_bottom = boundary_flux(mesh.bc[0], qf[FACE_B][:, row0], qb_bot, gt_bot,
                                    fB.Seta[:, row0], fB.J[row0], fB.vg[:, row0], liftL, False, gas)
        Fnum_eta = Fnum_eta.astype(np.result_type(Fnum_eta, top_flux))
        Fnum_eta[:, rowL] = top_flux
    Fnum_f = [Fnum_xi[:, left], Fnum_xi, Fnum_eta[:, bottom], Fnum_eta]
    if mesh.bounded:
        Fnum_f[FACE_B] = Fnum_f[FACE_B].astype(np.result_type(Fnum_f[FACE_B], Fnum_bottom))
        Fnum_f[FACE_B][:, row0] = Fnum_bottom

    # Divergence of F^loc + F^cor, GCL term, and R.
    div = d_xi(b, F) + d_eta(b, G)
    for f, dgv in ((FACE_L, b.dgL), (FACE_R, b.dgR)):
        jump = Fnum_f[f] - trace(b, F, f)                # [4, Ne, n(j)]
        div = div + jump[:, :, :, None] * dgv[None, None, None, :]
    for f, dgv in ((FACE_B, b.dgL), (FACE_T, b.dgR)):
        jump = Fnum_f[f] - trace(b, G, f)                # [4, Ne, n(i)]
        div = div + jump[:, :, None, :] * dgv[None, None, :, None]
    div = div - qc * (d_xi(b, g.St_xi) + d_eta(b, g.St_eta))
    R = -div / g.J
    if parts:
        return Parts(qc, grad_loc, grad, F, G, Fnum_xi, Fnum_eta, div, R, Fnum_bottom)
    return R


def _boundary_gradient(kind, qe, qb, grad_e, S, Je, dg_end, nvec):
    """grad q^com on a boundary face: the interior local gradient plus the lifted full
    jump q_b - q^-; at a wall without the normal component of grad T."""
    gx = grad_e[0] + (qb - qe) * S[0] * dg_end / Je
    gy = grad_e[1] + (qb - qe) * S[1] * dg_end / Je
    if kind == WALL:
        gn = gx[3] * nvec[0] + gy[3] * nvec[1]
        gx = np.concatenate([gx[:3], (gx[3] - gn * nvec[0])[None]])
        gy = np.concatenate([gy[:3], (gy[3] - gn * nvec[1])[None]])
    return gx, gy


def boundary_flux(kind, qe, qb, grad_e, S, Je, vg, dg_end, outward: bool, gas: ph.Gas):
    """|S| f^com on boundary faces, along +xi/+eta like the owned-face fluxes.  The
    element is on the '-' side when S points out of the domain (``outward``), else on
    the '+' side."""
    Smag = np.sqrt(S[0] * S[0] + S[1] * S[1])
    nvec = (S[0] / Smag, S[1] / Smag)
    qet = tuple(qe[k] for k in range(4))
    qbt = tuple(qb[k] for k in range(4))
    fcom = ph.rusanov(qet, qbt, nvec, vg, gas) if outward else ph.rusanov(qbt, qet, nvec, vg, gas)
    if gas.viscous:
        gx, gy = _boundary_gradient(kind, qe, qb, grad_e, S, Je, dg_end, nvec)
        fv, gv = ph.viscous_flux(qbt, tuple(gx), tuple(gy), gas)
        fcom = fcom - (fv * nvec[0] + gv * nvec[1])
    return Smag * fcom


def wall_force(q, mesh: Mesh, p: int, gas: ph.Gas, b: Basis | None = None,
               geo: Geometry | None = None):
    """Force on the walls (the numerator of the force coefficients of Sec. 4):
    F = sum over wall faces of the integral of -(p - p_inf) n + tau . n, n the unit
    normal out of the body (into the fluid), tau from grad q^com of the wall faces,
    p_inf = 1/(gamma M^2).  Gauss quadrature on the flux points: ds = |S| dxi."""
    b = b or make_basis(p)
    geo = geo or element_geometry(mesh.corners, mesh.vel, b)
    e_all = np.arange(mesh.ne)
    Fx = Fy = 0.0
    for side, kind in enumerate(mesh.bc):
        if kind != WALL:
            continue
        face = FACE_B if side == 0 else FACE_T
        rows = e_all < mesh.nx if side == 0 else e_all >= mesh.ne - mesh.nx
        fg = geo.faces[face]
        qe = trace(b, q, face)[:, rows]
        S = fg.Seta[:, rows]
        Smag = np.sqrt(S[0] * S[0] + S[1] * S[1])
        sgn = 1.0 if side == 0 else -1.0       # +eta points into the fluid below row 0
        nb = (sgn * S[0] / Smag, sgn * S[1] / Smag)
        qb = boundary_state(WALL, qe, fg.vg[:, rows], mesh.q_inf)
        tx = -(qb[0] - gas.R) * nb[0]
        ty = -(qb[0] - gas.R) * nb[1]
        if gas.viscous:
            g = geo.sol
            q_xi, q_eta = d_xi(b, q), d_eta(b, q)
            gxl = (g.Sxi[0] * q_xi + g.Seta[0] * q_eta) / g.J
            gyl = (g.Sxi[1] * q_xi + g.Seta[1] * q_eta) / g.J
            ge = (trace(b, gxl, face)[:, rows], trace(b, gyl, face)[:, rows])
            dg = BR2_PENALTY * (b.dgL_end if side == 0 else b.dgR_end)
            nvec = (S[0] / Smag, S[1] / Smag)
            gx, gy = _boundary_gradient(WALL, qe, qb, ge, S, fg.J[rows], dg, nvec)
            fv, gv = ph.viscous_flux(tuple(qb[k] for k in range(4)), tuple(gx), tuple(gy), gas)
            tn = fv * nb[0] + gv * nb[1]            # rows 1, 2: tau . n
            tx = tx + tn[1]
            ty = ty + tn[2]
        w = b.ws[None, :] * Smag
        Fx = Fx + np.sum(w * tx)
        Fy = Fy + np.sum(w * ty)
    return Fx, Fy
