"""Two-level preconditioner for the Newton operator of Sec. 3.2: element block-Jacobi
smoothing with a coarse correction on the discontinuous linear (P1) space, the coarse
operator formed by Galerkin projection and solved by an agglomeration multigrid V-cycle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper preconditions restarted GMRES with block Jacobi over processes and ILU(0)
inside each (Sec. 4, parallel setting).  The element block-Jacobi preconditioner that
replaces it here stalls once the preconditioned dissipation's pressure coupling
dominates the BDF2 term (it grows as p^2/h against rho_p a0/dt = gamma M^2 a0/dt): the
smooth, domain-wide pressure modes are not reached by element-local solves.  This
preconditioner adds them back.  Definition (every step plain linear algebra):

* Coarse space P1: for element e and variable v three coefficients (c0, c1, c2), the
  function c0 + c1 xi + c2 eta of the element's reference coordinates.  P maps them to
  the solution points: q[v, e, j, i] = c0 + c1 xi_i + c2 eta_j.  Coarse vectors are
  [Ne, 12] with index 3 v + m.
* A1 = P^T A P (Galerkin), A the Newton operator Gamma/dtau + (a0/dt) M - dR/dq.  Its
  12x12 blocks couple an element with itself and its face neighbours.
* Agglomeration: the cells of level l form an nx_l x ny_l grid per case (periodic in xi;
  periodic or bounded in eta like the mesh); the parent of cell (i, j) is
  (i // 2, j // 2) on an ceil(nx_l/2) x ceil(ny_l/2) grid.  Q maps the parent's P1
  function, written in the parent's reference coordinates X, Y in [-1, 1], to each
  child's P1 coefficients: with X = (xi + s_a)/2 along a direction the parent splits in
  two (s_a = -1 for the first child, +1 for the second) and X = xi along a direction it
  does not split (a leftover single cell), c0 + c1 X + c2 Y becomes
  (c0 + c1 s_a f_x + c2 s_b f_y) + (c1 f_x) xi + (c2 f_y) eta, f = 1/2 or 1.
  A_{l+1} = Q^T A_l Q.  Coarsening stops when a level has at most ``coarsest`` cells.
* Smoother on level l: damped block Jacobi x <- x + omega D_l^-1 (b - A_l x), D_l the
  12x12 diagonal blocks of A_l.
* V-cycle(l, b): the coarsest level solves A_L x = b exactly; otherwise x = 0, nu
  smoothing sweeps, e = V-cycle(l+1, Q^T (b - A_l x)), x = x + Q e, nu sweeps.
* Preconditioner ("coarse, then smooth"): z0 = P V-cycle(1, P^T r),
  M^-1 r = z0 + B^-1 (r - A z0), B^-1 the element block-Jacobi inverse of the fine
  operator (``solver.block_jacobian``) and A the Newton operator of the build.  The
  blocks, the coarse operators and this A are built at one linearisation and kept for
  ``lag`` Newton iterations like the blocks alone (on the device, the products of A with
  the P1 functions that form A_0 are kept, so A z0 needs no operator product).

It is one fixed linear map between builds, as GMRES requires.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from . import solver as sv


def p1_prolongation(ne: int, p: int, xs: np.ndarray) -> sp.csr_matrix:
    """P: [Ne*12] coarse coefficients -> fine vector in the solver's [4, Ne, n, n] order."""
    n = p + 1
    rows, cols, vals = [], [], []
    for v in range(4):
        for e in range(ne):
            for j in range(n):
                for i in range(n):
                    row = ((v * ne + e) * n + j) * n + i
                    base = e * 12 + 3 * v
                    rows += [row, row, row]
                    cols += [base, base + 1, base + 2]
                    vals += [1.0, xs[i], xs[j]]
    return sp.csr_matrix((vals, (rows, cols)), shape=(4 * ne * n * n, 12 * ne))


def stencils(mesh) -> list:
    """Each element's distinct stencil members: itself and its face neighbours."""
    left, right, bottom, top = mesh.neighbours()
    out = []
    for e in range(mesh.ne):
        s = [e]
        for nb in (left[e], right[e], bottom[e], top[e]):
            if nb >= 0 and nb not in s:
                s.append(int(nb))
        out.append(s)
    return out


def distance2_colouring(st: list) -> np.ndarray:
    """Greedy colouring in which no stencil holds two elements of one colour."""
    ne = len(st)
    members_of = [[] for _ in range(ne)]        # stencils that contain element f
    for e, s in enumerate(st):
        for f in s:
            members_of[f].append(e)
    colour = -np.ones(ne, dtype=int)
    for f in range(ne):
        used = set()
        for e in members_of[f]:
            used.update(colour[g] for g in st[e] if colour[g] >= 0)
        c = 0
        while c in used:
            c += 1
        colour[f] = c
    return colour


def galerkin_p1(prob: sv.Problem, q, inv_dtau: float, a0_dt: float, P: sp.csr_matrix):
    """A1 = P^T A P, column by column: A applied (exactly, by the complex step) to the P1
    basis function k of every element of one colour at a time; the response on element e
    comes from the single member of e's stencil that has the colour."""
    ne = prob.mesh.ne
    st = stencils(prob.mesh)
    colour = distance2_colouring(st)
    rows, cols, vals = [], [], []
    PT = P.T.tocsr()
    for c in range(colour.max() + 1):
        sel = np.where(colour == c)[0]
        for k in range(12):
            coarse = np.zeros(12 * ne)
            coarse[sel * 12 + k] = 1.0
            x = (P @ coarse).reshape(prob.shape)
            y = sv.apply_A(prob, q, x, inv_dtau, a0_dt).ravel()
            yc = (PT @ y).reshape(ne, 12)
            for e in range(ne):
                src = [f for f in st[e] if colour[f] == c]
                if src:
                    rows += list(e * 12 + np.arange(12))
                    cols += [src[0] * 12 + k] * 12
                    vals += list(yc[e])
    return sp.csr_matrix((vals, (rows, cols)), shape=(12 * ne, 12 * ne))


def agglomerate(nx: int, ny: int):
    """Q (children x parents, P1 coefficients) and the parent grid size."""
    NX, NY = (nx + 1) // 2, (ny + 1) // 2
    rows, cols, vals = [], [], []
    for j in range(ny):
        for i in range(nx):
            I, J = i // 2, j // 2
            split_x = 2 * I + 1 < nx
            split_y = 2 * J + 1 < ny
            sa = (2 * (i - 2 * I) - 1) if split_x else 0
            sb = (2 * (j - 2 * J) - 1) if split_y else 0
            fx = 0.5 if split_x else 1.0
            fy = 0.5 if split_y else 1.0
            ch, pa = j * nx + i, J * NX + I
            for v in range(4):
                r, c = ch * 12 + 3 * v, pa * 12 + 3 * v
                rows += [r, r, r, r + 1, r + 2]
                cols += [c, c + 1, c + 2, c + 1, c + 2]
                vals += [1.0, sa * fx, sb * fy, fx, fy]
    Q = sp.csr_matrix((vals, (rows, cols)), shape=(12 * nx * ny, 12 * NX * NY))
    return Q, NX, NY


def block_diagonal(A: sp.csr_matrix, bs: int) -> np.ndarray:
    nb = A.shape[0] // bs
    D = np.zeros((nb, bs, bs))
    for e in range(nb):
        D[e] = A[e * bs:(e + 1) * bs, e * bs:(e + 1) * bs].toarray()
    return D


@dataclasses.dataclass
class Hierarchy:
    A: list            # coarse operators A_1 .. A_L (scipy CSR, 12x12 blocks)
    Q: list            # Q_l: level l+1 -> level l
    Dinv: list         # inverses of the diagonal blocks of A_1 .. A_{L-1}
    Ainv_coarsest: np.ndarray
    omega: float
    nu: int


def build_hierarchy(A1: sp.csr_matrix, nx: int, ny: int, omega: float = 0.7,
                    nu: int = 2, coarsest: int = 4) -> Hierarchy:
    A, Q, Dinv = [A1.tocsr()], [], []
    while nx * ny > coarsest:
        Dinv.append(np.linalg.inv(block_diagonal(A[-1], 12)))
        Ql, nx, ny = agglomerate(nx, ny)
        Q.append(Ql)
        A.append((Ql.T @ A[-1] @ Ql).tocsr())
    return Hierarchy(A, Q, Dinv, np.linalg.inv(A[-1].toarray()), omega, nu)


def vcycle(h: Hierarchy, level: int, b: np.ndarray) -> np.ndarray:
    if level == len(h.A) - 1:
        return h.Ainv_coarsest @ b
    A, Dinv = h.A[level], h.Dinv[level]
    nb = Dinv.shape[0]

    def sweep(x):
        r = (b - A @ x).reshape(nb, 12)
        return x + h.omega * np.einsum("eab,eb->ea", Dinv, r).ravel()

    x = np.zeros_like(b)
    for _ in range(h.nu):
        x = sweep(x)
    e = vcycle(h, level + 1, h.Q[level].T @ (b - A @ x))
    x = x + h.Q[level] @ e
    for _ in range(h.nu):
        x = sweep(x)
    return x


@dataclasses.dataclass
class TwoLevel:
    """The preconditioner at one linearisation: apply(r) = M^-1 r."""
    Binv: np.ndarray
    P: sp.csr_matrix
    h: Hierarchy

    def coarse(self, r):
        return (self.P @ vcycle(self.h, 0, self.P.T @ r.ravel())).reshape(r.shape)

    def apply(self, r, Aop):
        """M^-1 r with Aop the Newton operator of the build (a function of a state-shaped
        vector): the preconditioner is one fixed linear map between builds."""
        z0 = self.coarse(r)
        return z0 + sv.block_apply(self.Binv, r - Aop(z0))


def build(prob: sv.Problem, q, inv_dtau: float, a0_dt: float, omega: float = 0.7, nu: int = 2,
          coarsest: int = 4) -> TwoLevel:
    mesh = prob.mesh
    Binv = np.linalg.inv(sv.block_jacobian(prob, q, inv_dtau, a0_dt))
    P = p1_prolongation(mesh.ne, prob.p, prob.basis.xs)
    A1 = galerkin_p1(prob, q, inv_dtau, a0_dt, P)
    h = build_hierarchy(A1, mesh.nx, mesh.ny, omega, nu, coarsest)
    return TwoLevel(Binv, P, h)
