"""Discrete adjoint of the BDF2 march (Sec. 3.2) for the sensitivities of the mean thrust
coefficient of a plunging airfoil (Secs. 4, 4.4) to the plunge amplitude h and the
free-stream Mach number M.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Dense Jacobians by complex steps and
dense solves: small meshes only.  The paper computes no sensitivities; this is the exact
discrete adjoint of its BDF2 march, the target of the GPU adjoint sweep.

March.  q^0 is given and held fixed; for n = 1 .. K, at t^n = t0 + n dt,

    G^n(q^n, q^{n-1}, q^{n-2}; h, M) = R(q^n; mesh(t^n, h), M)
                                       - (a0 qc(q^n) + a1 qc(q^{n-1}) + a2 qc(q^{n-2})) / dt = 0

(Eq. unsteady_pre_discretized_3 at convergence of the pseudo-time loop), with the BDF1
coefficients at n = 1 and BDF2 after (reading r12).  The mesh is the reference O-grid
translated by the rigid plunge y = h sin(2 pi f t), k = 2 pi f (Sec. 4.4); M enters R, the
conservative map qc and the far-field state.

Objective.  J = (1/K) sum_n C_t(q^n), C_t = -C_d = -F_x / (rho_inf U_inf^2 c / 2) =
-2 F_x (rho_inf = U_inf = c = 1, reading r25), F the wall force.

Adjoint.  With A^n = dG^n/dq^n and dG^m/dq^{m-k} = -(a_k^m / dt) Mq(q^{m-k}) (Mq = dqc/dq,
pointwise 4 x 4), for n = K .. 1:

    (A^n)^T lam^n = -dJ/dq^n + (a_1^{n+1}/dt) Mq(q^n)^T lam^{n+1} + (a_2^{n+2}/dt) Mq(q^n)^T lam^{n+2}

and dJ/dtheta = dJ/dtheta|_q + sum_n lam^n . dG^n/dtheta|_q (theta = h, M; partial
derivatives at fixed states by complex steps).  ``tangent_gradient`` computes the same
derivatives forward (dq^n/dtheta by the linearised march) for the pins.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from paper_1903_06304_gb300 import inputs as inp

from . import physics as ph
from . import residual as rs
from . import solver as sv

EPS = 1e-30   # complex step


@dataclasses.dataclass
class PlungeCase:
    ref: np.ndarray        # reference corners [Ne, 4, 2] of the O-grid
    ni: int
    nj: int
    p: int
    re: float
    kappa: float
    k: float               # reduced frequency
    t0: float
    dt: float
    nsteps: int
    q0: np.ndarray         # initial state, independent of (h, M)

    def time(self, n: int) -> float:
        return self.t0 + n * self.dt

    def coeffs(self, n: int):
        return sv.BDF1 if n == 1 else sv.BDF2


def problem(case: PlungeCase, t: float, h, mach) -> sv.Problem:
    """The bounded problem (wall below row 0, far field above) at time t; h and mach may be
    complex (the mesh is linear in h: reference plus h times the unit-amplitude motion)."""
    c1, v1 = inp.plunge(case.ref, t, 1.0, case.k)
    corners = case.ref + h * (c1 - case.ref)
    vel = h * v1
    gas = ph.Gas(mach=mach, re=case.re, kappa=case.kappa)
    mesh = rs.Mesh(case.ni, case.nj, corners, vel, bc=(rs.WALL, rs.FARFIELD),
                   q_inf=inp.far_field_state(mach))
    return sv.Problem(mesh, case.p, gas)


def step_residual(case: PlungeCase, n: int, qs, h, mach):
    """G^n of the states qs[n], qs[n-1], qs[n-2] (qs[m] for m < 0 unused)."""
    prob = problem(case, case.time(n), h, mach)
    a0, a1, a2 = case.coeffs(n)
    G = prob.R(qs[n]) - (a0 * prob.qc(qs[n]) + a1 * prob.qc(qs[n - 1])) / case.dt
    if a2 != 0.0:
        G = G - a2 * prob.qc(qs[n - 2]) / case.dt
    return G


def step_jacobian(case: PlungeCase, n: int, q, h, mach):
    """A^n = dG^n/dq^n, dense: -(Newton operator with inv_dtau = 0, a0_dt = a0/dt)."""
    prob = problem(case, case.time(n), h, mach)
    return -sv.dense_operator(prob, q, 0.0, case.coeffs(n)[0] / case.dt)


def march(case: PlungeCase, h, mach, tol: float = 1e-12, maxit: int = 30):
    """States q^0 .. q^K by Newton's method on each G^n with exact (dense) solves, the
    Jacobian taken at the step's initial guess and refreshed if the iteration stalls."""
    qs = [case.q0.copy()]
    for n in range(1, case.nsteps + 1):
        qs.append(qs[-1].copy())
        A = step_jacobian(case, n, qs[n], h, mach)
        G = step_residual(case, n, qs, h, mach)
        g0 = np.linalg.norm(G)
        for it in range(maxit):
            if np.linalg.norm(G) <= tol * g0:
                break
            qs[n] = qs[n] - np.linalg.solve(A, G.ravel()).reshape(G.shape)
            Gn = step_residual(case, n, qs, h, mach)
            if np.linalg.norm(Gn) > 0.5 * np.linalg.norm(G):
                A = step_jacobian(case, n, qs[n], h, mach)
            G = Gn
        else:
            raise RuntimeError(f"Newton did not converge at step {n}")
    return qs


def thrust(case: PlungeCase, n: int, q, h, mach):
    """C_t = -2 F_x at step n."""
    prob = problem(case, case.time(n), h, mach)
    Fx, _ = rs.wall_force(q, prob.mesh, case.p, prob.gas, prob.basis, prob.geo)
    return -2.0 * Fx


def objective(case: PlungeCase, qs, h, mach):
    return sum(thrust(case, n, qs[n], h, mach) for n in range(1, case.nsteps + 1)) / case.nsteps


def _dJ_dq(case: PlungeCase, n: int, q, h, mach):
    """dJ/dq^n by complex steps, one unknown at a time."""
    prob = problem(case, case.time(n), h, mach)
    g = np.zeros(q.size)
    for k in range(q.size):
        e = np.zeros(q.size, dtype=complex)
        e[k] = 1j * EPS
        Fx, _ = rs.wall_force(q + e.reshape(q.shape), prob.mesh, case.p, prob.gas, prob.basis,
                              prob.geo)
        g[k] = -2.0 * np.imag(Fx) / EPS
    return g.reshape(q.shape) / case.nsteps


def _partials(case: PlungeCase, qs, h, mach):
    """dG^n/dtheta and dJ/dtheta at fixed states, theta = (h, M), by complex steps."""
    dG = []
    dJ = np.zeros(2)
    for n in range(1, case.nsteps + 1):
        cols = []
        for th in range(2):
            hh = h + 1j * EPS if th == 0 else h
            mm = mach + 1j * EPS if th == 1 else mach
            cols.append(np.imag(step_residual(case, n, qs, hh, mm)) / EPS)
            dJ[th] += np.imag(thrust(case, n, qs[n], hh, mm)) / EPS / case.nsteps
        dG.append(cols)
    return dG, dJ


def _Mq(case: PlungeCase, n: int, q, h, mach):
    """Pointwise dqc/dq at step n's gas, [4, 4, Ne, n, n]."""
    return problem(case, case.time(n), h, mach).point_matrices(q)[1]


def adjoint_gradient(case: PlungeCase, h: float, mach: float):
    """(J, dJ/dh, dJ/dM) by the reverse sweep."""
    qs = march(case, h, mach)
    J = objective(case, qs, h, mach)
    K, dt = case.nsteps, case.dt
    dG, dJ = _partials(case, qs, h, mach)
    lam = [None] * (K + 3)
    for n in range(K, 0, -1):
        rhs = -_dJ_dq(case, n, qs[n], h, mach)
        Mq = _Mq(case, n, qs[n], h, mach)
        for m, kk in ((n + 1, 1), (n + 2, 2)):
            if m <= K:
                a = case.coeffs(m)[kk]
                if a != 0.0:
                    rhs = rhs + (a / dt) * np.einsum("ij...,i...->j...", Mq, lam[m])
        A = step_jacobian(case, n, qs[n], h, mach)
        lam[n] = np.linalg.solve(A.T, rhs.ravel()).reshape(rhs.shape)
    grad = dJ.copy()
    for n in range(1, K + 1):
        for th in range(2):
            grad[th] += np.sum(lam[n] * dG[n - 1][th])
    return J, grad[0], grad[1]


def tangent_gradient(case: PlungeCase, h: float, mach: float):
    """(dJ/dh, dJ/dM) by the forward linearised march (dq^0 = 0)."""
    qs = march(case, h, mach)
    K, dt = case.nsteps, case.dt
    dG, dJ = _partials(case, qs, h, mach)
    grad = dJ.copy()
    for th in range(2):
        dq = [np.zeros_like(case.q0)]
        for n in range(1, K + 1):
            a0, a1, a2 = case.coeffs(n)
            rhs = -dG[n - 1][th]
            Mq1 = _Mq(case, n, qs[n - 1], h, mach)
            rhs = rhs + (a1 / dt) * np.einsum("ij...,j...->i...", Mq1, dq[n - 1])
            if a2 != 0.0:
                Mq2 = _Mq(case, n, qs[n - 2], h, mach)
                rhs = rhs + (a2 / dt) * np.einsum("ij...,j...->i...", Mq2, dq[n - 2])
            A = step_jacobian(case, n, qs[n], h, mach)
            dq.append(np.linalg.solve(A, rhs.ravel()).reshape(rhs.shape))
            grad[th] += np.sum(_dJ_dq(case, n, qs[n], h, mach) * dq[n])
    return grad[0], grad[1]
