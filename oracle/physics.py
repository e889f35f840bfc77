"""Pointwise physics of Sec. 2: nondimensional gas, fluxes, M, Gamma, eigenvalues, Rusanov.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Arrays: a primitive state is a sequence ``q = (p, u, v, T)`` of equally shaped
arrays; 4x4 matrices are ``[4, 4, ...]`` arrays.  Complex inputs are allowed
(complex-step differentiation): ``cabs``/``cmax``/``cmin`` decide on real parts.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def cabs(x):
    return x * np.where(np.real(x) < 0, -1.0, 1.0)


def cmax(a, b):
    return np.where(np.real(a) >= np.real(b), a, b)


def cmin(a, b):
    return np.where(np.real(a) <= np.real(b), a, b)


@dataclasses.dataclass(frozen=True)
class Gas:
    """Nondimensional gas of Sec. 2.1 (R = 1/(gamma M^2), C_p = 1/((gamma-1) M^2), mu = 1).

    ``re <= 0`` switches the viscous flux off (Euler).  ``kappa`` is the global
    cut-off factor of Eq. eps_nonmove / eps_move; ``eps_floor`` guards U_r = 0 when
    kappa = 0 and the (relative) velocity vanishes.
    """
    mach: float
    re: float = 0.0
    gamma: float = 1.4
    prandtl: float = 0.72
    mu: float = 1.0
    kappa: float = 1.0
    eps_floor: float = 1e-8

    @property
    def R(self) -> float:
        return 1.0 / (self.gamma * self.mach ** 2)

    @property
    def cp(self) -> float:
        return 1.0 / ((self.gamma - 1.0) * self.mach ** 2)

    @property
    def k(self) -> float:
        """Thermal conductivity k = mu C_p / Pr (Sec. 2.1)."""
        return self.mu * self.cp / self.prandtl

    @property
    def viscous(self) -> bool:
        return self.re > 0


# ------------------------------------------------------------------ state relations (Sec. 2.1)

def density(q, gas: Gas):
    p, _, _, T = q
    return p / (gas.R * T)


def conservative(q, gas: Gas):
    """q^c = (rho, rho u, rho v, E), E = p/(gamma-1) + rho (u^2+v^2)/2."""
    p, u, v, T = q
    rho = density(q, gas)
    E = p / (gas.gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E])


def inviscid_flux(q, gas: Gas):
    """Eq. convection: f_inv, g_inv (each [4, ...])."""
    p, u, v, T = q
    rho = density(q, gas)
    E = p / (gas.gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    f = np.stack([rho * u, rho * u * u + p, rho * u * v, (E + p) * u])
    g = np.stack([rho * v, rho * u * v, rho * v * v + p, (E + p) * v])
    return f, g


def viscous_flux(q, qx, qy, gas: Gas):
    """Eqs. diffusion and shear_stress: f_v, g_v (each [4, ...]) from the primitive
    state q and its physical gradients qx = dq/dx, qy = dq/dy (both (p,u,v,T) tuples)."""
    _, u, v, _ = q
    ux, vx, Tx = qx[1], qx[2], qx[3]
    uy, vy, Ty = qy[1], qy[2], qy[3]
    mu = gas.mu
    txx = mu * (4.0 / 3.0 * ux - 2.0 / 3.0 * vy)
    tyy = mu * (4.0 / 3.0 * vy - 2.0 / 3.0 * ux)
    txy = mu * (uy + vx)
    zero = 0.0 * u
    inv_re = 1.0 / gas.re
    fv = inv_re * np.stack([zero, txx, txy, u * txx + v * txy + gas.k * Tx])
    gv = inv_re * np.stack([zero, txy, tyy, u * txy + v * tyy + gas.k * Ty])
    return fv, gv


# ------------------------------------------------------------------ preconditioning (Sec. 2.2-2.3)

def rho_p_rho_T(q, gas: Gas):
    """rho_p = 1/(R T), rho_T = -rho/T."""
    p, u, v, T = q
    rho = density(q, gas)
    return 1.0 / (gas.R * T), -rho / T


def sound_speed(q, gas: Gas):
    return np.sqrt(gas.gamma * gas.R * q[3])


def total_enthalpy(q, gas: Gas):
    """h = C_p T + (u^2 + v^2)/2."""
    return gas.cp * q[3] + 0.5 * (q[1] * q[1] + q[2] * q[2])


def _rows(first_col, q, gas: Gas):
    """Eq. jacobian / Eq. preconditioning share all columns but the first."""
    p, u, v, T = q
    rho = density(q, gas)
    _, rT = rho_p_rho_T(q, gas)
    h = total_enthalpy(q, gas)
    z = 0.0 * p
    a = first_col
    return np.array([
        [a, z, z, rT],
        [a * u, rho, z, rT * u],
        [a * v, z, rho, rT * v],
        [a * h - 1.0, rho * u, rho * v, rT * h + rho * gas.cp],
    ])


def M_matrix(q, gas: Gas):
    """Eq. jacobian: M = d q^c / d q^p."""
    rp, _ = rho_p_rho_T(q, gas)
    return _rows(rp, q, gas)


def epsilon(q, vg, gas: Gas):
    """Eq. eps_move (Eq. eps_nonmove when v_g = 0): eps = min(1, max(kappa M_inf, M_mov)),
    M_mov from v - v_g; floored at eps_floor."""
    _, u, v, _ = q
    wx, wy = u - vg[0], v - vg[1]
    m_mov = np.sqrt(wx * wx + wy * wy) / sound_speed(q, gas)
    e = cmin(1.0 + 0.0 * m_mov, cmax(gas.kappa * gas.mach + 0.0 * m_mov, m_mov))
    return cmax(e, gas.eps_floor + 0.0 * m_mov)


def theta(q, eps, gas: Gas):
    """Eq. theta: Theta = 1/U_r^2 - rho_T/(rho C_p), U_r = eps c."""
    ur = eps * sound_speed(q, gas)
    rho = density(q, gas)
    _, rT = rho_p_rho_T(q, gas)
    return 1.0 / (ur * ur) - rT / (rho * gas.cp)


def Gamma_matrix(q, eps, gas: Gas):
    """Eq. preconditioning: M with rho_p replaced by Theta."""
    return _rows(theta(q, eps, gas), q, gas)


def eigenvalues(q, nvec, vg, eps, gas: Gas):
    """Eqs. eigenvalues, eigenvalues_para with u_n = (v - v_g).n (Sec. 2.3):
    returns (lambda_1, lambda_2, lambda_3, lambda_4)."""
    _, u, v, _ = q
    un = (u - vg[0]) * nvec[0] + (v - vg[1]) * nvec[1]
    rp, rT = rho_p_rho_T(q, gas)
    rho = density(q, gas)
    ur = eps * sound_speed(q, gas)
    beta = rp + rT / (rho * gas.cp)
    alpha = (1.0 - beta * ur * ur) / 2.0
    unp = un * (1.0 - alpha)
    cpr = np.sqrt(alpha * alpha * un * un + ur * ur)
    return un, un, unp + cpr, unp - cpr


def normal_inviscid_flux(q, nvec, vg, gas: Gas):
    """f_{n,inv} = f n_x + g n_y - (v_g . n) q^c (Sec. 3.1)."""
    f, g = inviscid_flux(q, gas)
    qc = conservative(q, gas)
    vgn = vg[0] * nvec[0] + vg[1] * nvec[1]
    return f * nvec[0] + g * nvec[1] - vgn * qc


def rusanov(qm, qp, nvec, vg, gas: Gas):
    """Eq. Rosanov: preconditioned Rusanov flux along unit normal n (pointing from the
    '-' side to the '+' side).  Gamma~, |lambda|_max, eps and U_r all use the
    averaged primitive state; eps uses v - v_g."""
    qa = tuple(0.5 * (a + b) for a, b in zip(qm, qp))
    eps = epsilon(qa, vg, gas)
    lam = eigenvalues(qa, nvec, vg, eps, gas)
    lmax = cabs(lam[0])
    for l in lam[1:]:
        lmax = cmax(lmax, cabs(l))
    G = Gamma_matrix(qa, eps, gas)
    dq = np.stack([b - a for a, b in zip(qm, qp)])
    diss = np.einsum("ij...,j...->i...", G, dq)
    fm = normal_inviscid_flux(qm, nvec, vg, gas)
    fp = normal_inviscid_flux(qp, nvec, vg, gas)
    return 0.5 * (fp + fm) - 0.5 * lmax * diss
