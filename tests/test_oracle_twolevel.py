"""Pins of the oracle's two-level preconditioner (oracle.twolevel): the P1 prolongation and
the agglomeration reproduce linear functions, the coloured Galerkin operator equals
P^T A P of the dense operator, the multigrid cycle converges as an iteration, the
preconditioner is exact where its definition says it must be, and it removes the
stagnation of element block Jacobi on a stiff low-Mach case."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import physics as ph
from oracle import residual as rs
from oracle import solver as sv
from oracle import twolevel as tl
from paper_1903_06304_gb300 import inputs as inp


def _problem(nx, ny, p, mach=0.05, re=10.0, deforming=True, bounded=False, seed=3):
    ref = inp.box_mesh(nx, ny, 0, 10, 0, 10)
    c, v = inp.deform(ref, 0.13, inp.Motion()) if deforming else (ref, np.zeros_like(ref))
    gas = ph.Gas(mach=mach, re=re, kappa=1.0)
    if bounded:
        mesh = rs.Mesh(nx, ny, c, v, bc=(rs.WALL, rs.FARFIELD), q_inf=inp.far_field_state(mach))
    else:
        mesh = rs.Mesh(nx, ny, c, v)
    q = inp.random_perturbation(inp.uniform_state(nx * ny, p, mach, 0.8, 0.3), seed, 0.1, mach)
    return sv.Problem(mesh, p, gas), q


def test_p1_prolongation_reproduces_a_linear_field():
    """On a Cartesian mesh f = a + b x + c y has, per element, mean f(centre) and reference
    slopes b hx/2 along xi and c hy/2 along eta; P of those coefficients is f at every
    solution point (variable v scaled by v + 1)."""
    nx, ny, p = 4, 3, 2
    hx, hy = 10 / nx, 10 / ny
    corners = inp.box_mesh(nx, ny, 0, 10, 0, 10)
    x, y = inp.sample_points(corners, p)
    a, b, c = 0.3, -1.7, 2.2
    coef = np.zeros((nx * ny, 12))
    for e in range(nx * ny):
        xc, yc = corners[e, :, 0].mean(), corners[e, :, 1].mean()
        for v in range(4):
            coef[e, 3 * v:3 * v + 3] = (v + 1) * np.array([a + b * xc + c * yc, b * hx / 2, c * hy / 2])
    P = tl.p1_prolongation(nx * ny, p, np.polynomial.legendre.leggauss(p + 1)[0])
    got = (P @ coef.ravel()).reshape(4, nx * ny, p + 1, p + 1)
    for v in range(4):
        np.testing.assert_allclose(got[v], (v + 1) * (a + b * x + c * y), rtol=0, atol=1e-12)


@pytest.mark.parametrize("nx,ny", [(4, 4), (5, 3), (1, 2), (3, 1)])
def test_agglomeration_keeps_each_linear_function(nx, ny):
    """A parent's function c0 + c1 X + c2 Y (X, Y its reference coordinates) evaluated at a
    point of a child equals the child's coefficients evaluated there: the children tile
    the parent, a split direction halving it."""
    Q, NX, NY = tl.agglomerate(nx, ny)
    rng = np.random.default_rng(1)
    parent = rng.standard_normal(12 * NX * NY)
    child = (Q @ parent).reshape(nx * ny, 4, 3)
    parent = parent.reshape(NX * NY, 4, 3)
    for j in range(ny):
        for i in range(nx):
            I, J = i // 2, j // 2
            wx = 2 if 2 * I + 1 < nx else 1
            wy = 2 if 2 * J + 1 < ny else 1
            for xi, eta in rng.uniform(-1, 1, size=(3, 2)):
                # the child's point in the parent's reference coordinates
                X = -1 + (2 * (i - 2 * I) + xi + 1) / wx
                Y = -1 + (2 * (j - 2 * J) + eta + 1) / wy
                cc = child[j * nx + i]
                pc = parent[J * NX + I]
                np.testing.assert_allclose(cc[:, 0] + cc[:, 1] * xi + cc[:, 2] * eta,
                                           pc[:, 0] + pc[:, 1] * X + pc[:, 2] * Y, atol=1e-12)


@pytest.mark.parametrize("nx,ny,p,bounded", [(3, 3, 1, False), (2, 3, 1, False), (4, 2, 1, True)])
def test_coloured_galerkin_operator_equals_dense_product(nx, ny, p, bounded):
    """A1 from coloured exact products equals P^T A P with A the dense operator (one
    column per unknown), including 2-wide periodic meshes where the left and right
    neighbour coincide and bounded meshes."""
    prob, q = _problem(nx, ny, p, bounded=bounded)
    inv_dtau, a0_dt = 0.7, 150.0
    P = tl.p1_prolongation(prob.mesh.ne, p, prob.basis.xs)
    A1 = tl.galerkin_p1(prob, q, inv_dtau, a0_dt, P).toarray()
    A = sv.dense_operator(prob, q, inv_dtau, a0_dt)
    ref = P.T @ A @ P
    assert np.abs(A1 - ref).max() <= 1e-11 * np.abs(ref).max()


def test_multigrid_cycle_converges_as_an_iteration():
    """x <- x + V(b - A1 x) on the coarse operator of a stiff low-Mach problem contracts the
    error (spectral radius of I - V A1 below one), so the hierarchy, its transfers and its
    smoother fit together."""
    prob, q = _problem(8, 8, 1, mach=0.01)
    P = tl.p1_prolongation(prob.mesh.ne, 1, prob.basis.xs)
    A1 = tl.galerkin_p1(prob, q, 0.0, 150.0, P)
    h = tl.build_hierarchy(A1, 8, 8, coarsest=4)
    assert len(h.A) == 3
    n = A1.shape[0]
    V = np.stack([tl.vcycle(h, 0, e) for e in np.eye(n)], axis=1)
    rho = np.max(np.abs(np.linalg.eigvals(np.eye(n) - V @ A1.toarray())))
    assert rho < 0.99, rho


def test_two_grid_correction_is_exact_on_the_coarse_range():
    """Without smoothing and with an exact solve on the next level, one cycle returns Q c
    for a right-hand side A_l Q c: restriction, Galerkin operator and prolongation are
    consistent (Q^T A Q is the operator of the coarse unknowns)."""
    prob, q = _problem(4, 4, 1, mach=0.01)
    P = tl.p1_prolongation(prob.mesh.ne, 1, prob.basis.xs)
    A1 = tl.galerkin_p1(prob, q, 0.0, 150.0, P)
    h = tl.build_hierarchy(A1, 4, 4, nu=0, coarsest=4)
    assert len(h.A) == 2
    c = inp.random_vector(48, 6)
    x = h.Q[0] @ c
    np.testing.assert_allclose(tl.vcycle(h, 0, A1 @ x), x, rtol=0, atol=1e-10 * np.abs(x).max())


def test_preconditioner_is_exact_for_block_diagonal_operators():
    """For an element-block-diagonal operator B, z0 + B^-1 (r - B z0) = B^-1 r whatever the
    coarse correction z0."""
    prob, q = _problem(3, 3, 1)
    pc = tl.build(prob, q, 0.5, 150.0)
    B = np.linalg.inv(pc.Binv)
    Bop = lambda v: sv.block_apply(B, v)
    r = inp.random_vector(prob.shape, 4)
    np.testing.assert_allclose(pc.apply(r, Bop), sv.block_apply(pc.Binv, r), rtol=0,
                               atol=1e-12 * np.abs(sv.block_apply(pc.Binv, r)).max())


def test_preconditioner_is_exact_on_the_coarse_space():
    """With an exact coarse solve (a single-level hierarchy), a right-hand side A P c is
    solved exactly: z0 = P c and the smoothing step adds nothing."""
    prob, q = _problem(3, 3, 2, mach=0.01)
    inv_dtau, a0_dt = 0.0, 150.0
    pc = tl.build(prob, q, inv_dtau, a0_dt, coarsest=9)
    assert len(pc.h.A) == 1
    Aop = lambda v: sv.apply_A(prob, q, v, inv_dtau, a0_dt)
    c = inp.random_vector(12 * prob.mesh.ne, 5)
    x = (pc.P @ c).reshape(prob.shape)
    got = pc.apply(Aop(x), Aop)
    np.testing.assert_allclose(got, x, rtol=0, atol=1e-9 * np.abs(x).max())


def test_two_level_gmres_beats_block_jacobi_on_a_stiff_case():
    """M = 0.01 on a 16 x 16 deforming mesh at p = 2 (the low-Mach pressure coupling):
    GMRES(30) with element block Jacobi needs well over twice the iterations to 1e-6 that
    it needs with the coarse correction (108 against 41; the gap widens with the mesh)."""
    prob, q = _problem(16, 16, 2, mach=0.01)
    inv_dtau, a0_dt = 0.0, 150.0
    Aop = lambda v: sv.apply_A(prob, q, v, inv_dtau, a0_dt)
    b = prob.R(q)
    Binv = np.linalg.inv(sv.block_jacobian(prob, q, inv_dtau, a0_dt))
    bj = sv.gmres(Aop, b, lambda v: sv.block_apply(Binv, v), 30, 1e-6, 400)
    pc = tl.build(prob, q, inv_dtau, a0_dt)
    two = sv.gmres(Aop, b, lambda v: pc.apply(v, Aop), 30, 1e-6, 300)
    assert two.converged
    assert two.iterations * 2 <= bj.iterations, (two.iterations, bj.iterations)
    # both solve the same system
    x_bj = bj.x if bj.converged else None
    res = np.linalg.norm((Aop(two.x) - b).ravel()) / np.linalg.norm(b.ravel())
    assert res < 1e-3
    if x_bj is not None:
        assert np.abs(two.x - x_bj).max() <= 1e-3 * np.abs(x_bj).max()


def test_bdf_step_with_two_level_preconditioner_converges():
    """A BDF1 step of a stiff case reaches Res_m/Res_0 <= 1e-8 with the two-level
    preconditioner and lands on the same state as the block-Jacobi Newton loop given
    enough GMRES iterations."""
    prob, q = _problem(6, 6, 2, mach=0.01)
    qc = prob.qc(q)
    q2, st2 = sv.bdf2_step(prob, q, qc, qc, 0.01, coeffs=sv.BDF1, precond="twolevel", maxit_lin=60)
    q1, st1 = sv.bdf2_step(prob, q, qc, qc, 0.01, coeffs=sv.BDF1, maxit_lin=400, restart=60)
    assert st2.converged and st1.converged
    dq = np.abs(q1 - q).max(axis=(1, 2, 3))
    assert np.all(np.abs(q2 - q1).max(axis=(1, 2, 3)) <= 1e-6 * dq)
