"""Implicit time marching of Sec. 3.2: JVP, element block Jacobian, restarted GMRES,
BDF2 dual-time Newton (Eq. unsteady_pre_discretized_3) and steady PTC with SER
(Eqs. steady_pre_discretized_1, SER).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Linear operator of one pseudo-time step (Eq. unsteady_pre_discretized_3; the steady
Eq. steady_pre_discretized_1 is the case a0/dt = 0):

    A = Gamma / dtau + (a0/dt) M - dR/dq^p

where a0 = 3/2 for BDF2 and 1 for a first BDF1 step.  Right-hand side:

    r(q) = -(a0 q^c(q) + a1 q^c,n + a2 q^c,n-1)/dt + R(q)      (BDF2: a = 3/2, -2, 1/2)

Readings where the paper is silent:
* dR/dq^p . v is exact (complex step), not a first-order finite difference.
* The preconditioner is element block-Jacobi: B_e = Gamma_e/dtau + (a0/dt) M_e -
  dR_e/dq_e (neighbours frozen), inverted exactly.  It is rebuilt every ``lag``
  pseudo-iterations (2 for unsteady runs, 1 for steady runs, Sec. 4).
* GMRES: the paper solves with PETSc's restarted GMRES, whose default is left
  preconditioning with the preconditioned residual norm: the Krylov space of
  B^-1 A is built, ||B^-1 (b - A x)|| is minimised and convergence is tol_res
  relative to ||B^-1 b|| (zero initial guess).  Classical Gram-Schmidt with one
  re-orthogonalisation (CGS2); the residual is recomputed at every restart.  Right
  preconditioning is kept as an option (side="right").
* Res_m, "the relative residual of pressure", is the 2-norm of the first
  (continuity) row of r over all solution points.
* SER: the step q^m -> q^m+1 uses dtau_m; dtau_0 = dtau0 and
  dtau_m = clip(dtau_m-1 (Res_m-1/Res_m)^r_ser, dtau_min, dtau_max).
* Gamma and M at solution points use eps from the point's own v - v_g.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import physics as ph
from .basis import make_basis
from .geometry import element_geometry
from .residual import Mesh, residual

BDF2 = (1.5, -2.0, 0.5)
BDF1 = (1.0, -1.0, 0.0)
COMPLEX_STEP = 1e-30


@dataclasses.dataclass
class Problem:
    mesh: Mesh
    p: int
    gas: ph.Gas

    def __post_init__(self):
        self.basis = make_basis(self.p)
        self.geo = element_geometry(self.mesh.corners, self.mesh.vel, self.basis)

    @property
    def shape(self):
        n = self.p + 1
        return (4, self.mesh.ne, n, n)

    def R(self, q):
        return residual(q, self.mesh, self.p, self.gas, self.basis, self.geo)

    def qc(self, q):
        return ph.conservative(tuple(q[k] for k in range(4)), self.gas)

    def point_matrices(self, q):
        """(Gamma, M) at solution points, each [4, 4, Ne, n, n]."""
        qs = tuple(q[k] for k in range(4))
        eps = ph.epsilon(qs, self.geo.sol.vg, self.gas)
        return ph.Gamma_matrix(qs, eps, self.gas), ph.M_matrix(qs, self.gas)


# ------------------------------------------------------------------ operators

def jacobian_vector(prob: Problem, q, v):
    """dR/dq^p . v by the complex step (exact to rounding)."""
    h = COMPLEX_STEP
    return np.imag(prob.R(q + 1j * h * v)) / h


def apply_A(prob: Problem, q, v, inv_dtau: float, a0_dt: float):
    """A v = Gamma v / dtau + (a0/dt) M v - dR/dq . v."""
    G, M = prob.point_matrices(q)
    Gv = np.einsum("ab...,b...->a...", G, v)
    Mv = np.einsum("ab...,b...->a...", M, v)
    return inv_dtau * Gv + a0_dt * Mv - jacobian_vector(prob, q, v)


def time_rhs(prob: Problem, q, qc_n, qc_nm1, dt: float, coeffs=BDF2, steady=False):
    """Pseudo-step right-hand side: R (steady) or -(BDF q^c)/dt + R (unsteady)."""
    R = prob.R(q)
    if steady:
        return R
    a0, a1, a2 = coeffs
    return -(a0 * prob.qc(q) + a1 * qc_n + a2 * qc_nm1) / dt + R


def element_colouring(mesh: Mesh) -> np.ndarray:
    """Greedy colouring so that no two elements of one colour share a face."""
    left, right, bottom, top = mesh.neighbours()
    colour = -np.ones(mesh.ne, dtype=int)
    for e in range(mesh.ne):
        used = {colour[nb] for nb in (left[e], right[e], bottom[e], top[e]) if nb >= 0}
        c = 0
        while c in used:
            c += 1
        colour[e] = c
    return colour


def block_jacobian(prob: Problem, q, inv_dtau: float, a0_dt: float):
    """Element blocks B_e = Gamma_e/dtau + (a0/dt) M_e - dR_e/dq_e, [Ne, b, b] with the
    local index d = var * n^2 + j * n + i.  dR_e/dq_e by complex steps seeded on one
    local unknown of every element of one colour at a time (no two of them neighbours,
    and R_e depends only on e and its face neighbours)."""
    ne = prob.mesh.ne
    n = prob.p + 1
    np2 = n * n
    bsz = 4 * np2
    colour = element_colouring(prob.mesh)
    B = np.zeros((ne, bsz, bsz))
    h = COMPLEX_STEP
    for c in range(colour.max() + 1):
        sel = colour == c
        for d in range(bsz):
            var, rem = divmod(d, np2)
            j, i = divmod(rem, n)
            dq = np.zeros(prob.shape)
            dq[var, sel, j, i] = 1.0
            col = np.imag(prob.R(q + 1j * h * dq)) / h       # [4, Ne, n, n]
            B[sel, :, d] = -col[:, sel].transpose(1, 0, 2, 3).reshape(-1, bsz)
    G, M = prob.point_matrices(q)
    P = inv_dtau * G + a0_dt * M                              # [4, 4, Ne, n, n]
    for a in range(4):
        for bb in range(4):
            vals = P[a, bb].reshape(ne, np2)
            idx = np.arange(np2)
            B[:, a * np2 + idx, bb * np2 + idx] += vals
    return B


def dense_operator(prob: Problem, q, inv_dtau: float, a0_dt: float):
    """The Newton operator A = Gamma/dtau + (a0/dt) M - dR/dq as a dense matrix, one column
    per unknown (complex steps); small meshes only."""
    nd = q.size
    A = np.zeros((nd, nd))
    for k in range(nd):
        e = np.zeros(nd)
        e[k] = 1.0
        A[:, k] = apply_A(prob, q, e.reshape(q.shape), inv_dtau, a0_dt).ravel()
    return A


def vjp(prob: Problem, q, w, inv_dtau: float, a0_dt: float):
    """A^T w by its definition: the transpose of the dense operator (small meshes)."""
    A = dense_operator(prob, q, inv_dtau, a0_dt)
    return (A.T @ w.ravel()).reshape(q.shape)


def block_apply(Binv, r):
    """z_e = B_e^{-1} r_e for [4, Ne, n, n] vectors."""
    ne, bsz, _ = Binv.shape
    re = r.transpose(1, 0, 2, 3).reshape(ne, bsz)
    z = np.einsum("eab,eb->ea", Binv, re)
    return z.reshape(ne, 4, *r.shape[2:]).transpose(1, 0, 2, 3)


# ------------------------------------------------------------------ GMRES

@dataclasses.dataclass
class GmresResult:
    x: np.ndarray
    iterations: int
    converged: bool
    res_history: list


def gmres(Aop, b, Minv, restart: int, tol: float, maxit: int, side: str = "left",
          passes: int = 2) -> GmresResult:
    """Restarted preconditioned GMRES(m) with CGS2 Arnoldi (see module notes); passes=1
    is classical Gram-Schmidt without re-orthogonalisation (PETSc's default refinement
    setting, "never").

    side="left" (the default of PETSc, whose solver the paper uses): Krylov space of
    M^-1 A, the preconditioned residual M^-1 (b - A x) is minimised and tested against
    tol * ||M^-1 b||.  side="right": Krylov space of A M^-1, x = M^-1 V y, the true
    residual b - A x is minimised and tested against tol * ||b||."""
    shape = b.shape
    left = side == "left"
    bv = (Minv(b) if left else b).ravel()
    bnorm = np.linalg.norm(bv)
    x = np.zeros_like(bv)
    hist = [bnorm]
    if bnorm == 0.0:
        return GmresResult(x.reshape(shape), 0, True, hist)
    total = 0
    r = bv.copy()
    beta = bnorm
    converged = False
    while True:
        if beta <= tol * bnorm:
            converged = True
            break
        if total >= maxit:
            break
        m = restart
        V = np.zeros((m + 1, bv.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            if left:
                w = Minv(Aop(V[j].reshape(shape))).ravel()
            else:
                w = Aop(Minv(V[j].reshape(shape))).ravel()
            h1 = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h1
            if passes == 2:
                h2 = V[: j + 1] @ w
                w = w - V[: j + 1].T @ h2
                H[: j + 1, j] = h1 + h2
            else:
                H[: j + 1, j] = h1
            hn = np.linalg.norm(w)
            H[j + 1, j] = hn
            if hn > 0:
                V[j + 1] = w / hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            k = j + 1
            hist.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= tol * bnorm or total >= maxit or hn == 0:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1: k] @ y[i + 1: k]) / H[i, i]
        if left:
            x = x + V[:k].T @ y
            r = Minv((b.ravel() - Aop(x.reshape(shape)).ravel()).reshape(shape)).ravel()
        else:
            x = x + Minv((V[:k].T @ y).reshape(shape)).ravel()
            r = bv - Aop(x.reshape(shape)).ravel()
        beta = np.linalg.norm(r)
    return GmresResult(x.reshape(shape), total, converged, hist)


# ------------------------------------------------------------------ Newton loops

@dataclasses.dataclass
class StepStats:
    newton_iterations: int
    gmres_iterations: list
    res_history: list            # Res_m (continuity row 2-norm), m = 0..
    dtau_history: list
    converged: bool


def newton_solve(prob: Problem, q, rhs, a0_dt: float, dtau0: float, restart: int,
                 tol_res: float, maxit_lin: int, tol_pseudo: float, maxit_newton: int,
                 lag: int, ser=None, side: str = "left", line_search: int = 0,
                 precond: str = "block"):
    """Pseudo-time Newton loop shared by BDF2 and PTC; ``ser`` = (dtau_min, dtau_max, r).
    line_search = k > 0: backtracking on the full residual 2-norm, lambda = 1, 1/2, ...,
    2^-k (the paper takes plain Newton updates, k = 0).  precond: "block" (element
    block Jacobi) or "twolevel" (``oracle.twolevel``: the blocks as smoother plus the
    P1 coarse correction, its smoothing step with the Newton operator of the build),
    either rebuilt every ``lag`` iterations."""
    from . import twolevel as tl
    q = q.copy()
    r = rhs(q)
    res = [float(np.linalg.norm(r[0]))]
    dtau = dtau0
    dtaus = [dtau]
    its = []
    Binv = None
    converged = False
    for m in range(maxit_newton):
        if res[-1] <= tol_pseudo * res[0]:
            converged = True
            break
        inv_dtau = 1.0 / dtau
        if m % lag == 0 or Binv is None or ser is not None:
            if precond == "twolevel":
                Binv = tl.build(prob, q, inv_dtau, a0_dt)
                # the smoothing step applies the operator of the build
                Abuild = lambda v, qb=q, ib=inv_dtau: apply_A(prob, qb, v, ib, a0_dt)
            else:
                Binv = np.linalg.inv(block_jacobian(prob, q, inv_dtau, a0_dt))
        qm = q
        Aop = lambda v: apply_A(prob, qm, v, inv_dtau, a0_dt)
        if precond == "twolevel":
            Minv = lambda v, pc=Binv, Ab=Abuild: pc.apply(v, Ab)
        else:
            Minv = lambda v, B=Binv: block_apply(B, v)
        out = gmres(Aop, r, Minv, restart, tol_res, maxit_lin, side)
        its.append(out.iterations)
        prev_all = np.linalg.norm(r)
        lam = 1.0
        q = qm + lam * out.x
        r = rhs(q)
        for _ in range(line_search):
            if np.linalg.norm(r) < prev_all:
                break
            lam *= 0.5
            q = qm + lam * out.x
            r = rhs(q)
        res.append(float(np.linalg.norm(r[0])))
        if ser is not None:
            dmin, dmax, rser = ser
            dtau = max(dmin, min(dmax, dtau * (res[-2] / res[-1]) ** rser))
            dtaus.append(dtau)
    else:
        converged = res[-1] <= tol_pseudo * res[0]
    return q, StepStats(len(its), its, res, dtaus, converged)


def bdf2_step(prob: Problem, q, qc_n, qc_nm1, dt: float, coeffs=BDF2, dtau: float = 1e20,
              restart: int = 30, tol_res: float = 1e-6, maxit_lin: int = 100,
              tol_pseudo: float = 1e-8, maxit_newton: int = 20, lag: int = 2,
              side: str = "left", ser=None, line_search: int = 0, precond: str = "block"):
    """One physical BDF2 step (Eq. unsteady_pre_discretized_3) from q^n = q (initial guess).
    ser = (dtau_min, dtau_max, r_ser): adapt the pseudo step from dtau by the SER law
    (pseudo-transient continuation, the steady strategy of Sec. 3.2) instead of the fixed
    dtau of the paper's unsteady runs."""
    rhs = lambda s: time_rhs(prob, s, qc_n, qc_nm1, dt, coeffs)
    return newton_solve(prob, q, rhs, coeffs[0] / dt, dtau, restart, tol_res, maxit_lin,
                        tol_pseudo, maxit_newton, lag, ser=ser, side=side, line_search=line_search,
                        precond=precond)


def ptc_solve(prob: Problem, q, dtau0: float = 0.01, dtau_min: float = 0.01,
              dtau_max: float = 1e20, r_ser: float = 2.0, restart: int = 20,
              tol_res: float = 1e-6, maxit_lin: int = 100, tol_pseudo: float = 1e-8,
              maxit_newton: int = 10, side: str = "left"):
    """Steady pseudo-transient continuation with SER (Eqs. steady_pre_discretized_1, SER)."""
    rhs = lambda s: prob.R(s)
    return newton_solve(prob, q, rhs, 0.0, dtau0, restart, tol_res, maxit_lin, tol_pseudo,
                        maxit_newton, 1, ser=(dtau_min, dtau_max, r_ser), side=side)


# ------------------------------------------------------------------ norms (Sec. 4)

def l2_error(prob: Problem, phi, phi_exact):
    """E_phi = sqrt(int (phi - phi_exact)^2 dV / int dV) by Gauss quadrature."""
    b = prob.basis
    w = np.outer(b.ws, b.ws) * prob.geo.sol.J
    return float(np.sqrt(np.sum(w * (phi - phi_exact) ** 2) / np.sum(w)))


def entropy_error(prob: Problem, q):
    """E_s of Sec. 4 with p_inf/rho_inf^gamma of the free stream (rho = T = 1)."""
    b = prob.basis
    g = prob.gas
    w = np.outer(b.ws, b.ws) * prob.geo.sol.J
    rho = ph.density(tuple(q[k] for k in range(4)), g)
    s_inf = g.R  # p_inf / rho_inf^gamma with rho_inf = T_inf = 1
    s = q[0] / rho ** g.gamma
    return float(np.sqrt(np.sum(w * (s - s_inf) ** 2) / np.sum(w * s_inf ** 2)))


# ------------------------------------------------------------------ parameter sensitivities

def param_vjp(prob: Problem, q, w):
    """Sensitivities of w . R to the parameters, by the complex step (brute force: one
    complex residual per parameter):

        dmach          = w . dR/dM_inf     (R, C_p, k and kappa M_inf move with M_inf, Sec. 2.1)
        dcorners[e,a,c] = w . dR/d(corner a of element e, coordinate c)
        dvel[e,a,c]     = w . dR/d(velocity of corner a of element e, component c)
    """
    h = COMPLEX_STEP
    gas_c = dataclasses.replace(prob.gas, mach=prob.gas.mach + 1j * h)
    dmach = float(np.sum(w * np.imag(Problem(prob.mesh, prob.p, gas_c).R(q))) / h)
    m = prob.mesh
    out = []
    for which in ("corners", "vel"):
        base = getattr(m, which)
        d = np.zeros(base.shape)
        for e in range(base.shape[0]):
            for a in range(4):
                for c in range(2):
                    pert = base.astype(complex)
                    pert[e, a, c] += 1j * h
                    corners = pert if which == "corners" else m.corners
                    vel = pert if which == "vel" else m.vel
                    Rc = Problem(Mesh(m.nx, m.ny, corners, vel), prob.p, prob.gas).R(q)
                    d[e, a, c] = np.sum(w * np.imag(Rc)) / h
        out.append(d)
    return dmach, out[0], out[1]
