"""Pins of the oracle's implicit machinery (Sec. 3.2): exact JVP vs finite differences,
element blocks vs the dense finite-difference Jacobian, GMRES vs a direct solve and
the Krylov minimal-residual property, BDF2 second-order convergence in time, Newton
convergence, and steady PTC with SER."""
import numpy as np
import pytest

from oracle import physics as ph
from oracle import residual as rs
from oracle import solver as sv
from paper_1903_06304_gb300 import inputs as inp


def _small_problem(p=2, nx=3, ny=3, re=10.0, mach=0.05, deforming=True, seed=3):
    ref = inp.box_mesh(nx, ny, 0, 10, 0, 10)
    c, v = inp.deform(ref, 0.13, inp.Motion()) if deforming else (ref, np.zeros_like(ref))
    gas = ph.Gas(mach=mach, re=re, kappa=1.0)
    prob = sv.Problem(rs.Mesh(nx, ny, c, v), p, gas)
    q = inp.random_perturbation(inp.uniform_state(nx * ny, p, mach, 0.8, 0.3), seed, 0.1, mach)
    return prob, q


def _dense_fd_jacobian(prob, q, h_rel=1e-6):
    """Central finite differences of R, one unknown at a time (independent of the
    complex-step path)."""
    N = q.size
    Jd = np.zeros((N, N))
    scale = np.abs(q).reshape(4, -1).max(axis=1)
    for k in range(N):
        var = k // (N // 4)
        h = h_rel * scale[var]
        e = np.zeros(N)
        e[k] = h
        Jd[:, k] = ((prob.R(q + e.reshape(q.shape)) - prob.R(q - e.reshape(q.shape))) / (2 * h)).ravel()
    return Jd


@pytest.mark.parametrize("re", [0.0, 10.0])
def test_jvp_matches_central_differences(re):
    prob, q = _small_problem(re=re)
    v = inp.random_vector(q.shape, 5)
    v[0] *= prob.gas.R * 1e-3
    jv = sv.jacobian_vector(prob, q, v)
    h = 1e-4
    fd = (prob.R(q + h * v) - prob.R(q - h * v)) / (2 * h)
    assert np.abs(fd - jv).max() <= 1e-6 * np.abs(jv).max()


@pytest.mark.parametrize("re", [0.0, 10.0])
def test_blocks_are_diagonal_blocks_of_dense_fd_jacobian(re):
    prob, q = _small_problem(p=1, re=re)
    inv_dtau, a0_dt = 1.0 / 0.3, 1.5 / 0.01
    B = sv.block_jacobian(prob, q, inv_dtau, a0_dt)
    Jd = _dense_fd_jacobian(prob, q)
    G, M = prob.point_matrices(q)
    ne, n = prob.mesh.ne, prob.p + 1
    np2 = n * n

    def gidx(e, d):
        var, rem = divmod(d, np2)
        j, i = divmod(rem, n)
        return ((var * ne + e) * n + j) * n + i

    bs = 4 * np2
    for e in range(ne):
        ids = [gidx(e, d) for d in range(bs)]
        ref = -Jd[np.ix_(ids, ids)]
        for a in range(4):
            for b in range(4):
                for pt in range(np2):
                    j, i = divmod(pt, n)
                    ref[a * np2 + pt, b * np2 + pt] += (inv_dtau * G[a, b, e, j, i]
                                                        + a0_dt * M[a, b, e, j, i])
        scale = np.abs(ref).max()
        assert np.abs(B[e] - ref).max() <= 2e-6 * scale


def test_residual_stencil_is_face_neighbours_only():
    """Seeding one element changes R only on it and its four face neighbours, which the
    colouring of block_jacobian relies on."""
    prob, q = _small_problem(p=2, nx=5, ny=5)
    v = np.zeros(q.shape)
    v[:, 12] = inp.random_vector(v[:, 12].shape, 1)
    jv = sv.jacobian_vector(prob, q, v)
    touched = set(np.nonzero(np.abs(jv).max(axis=(0, 2, 3)) > 0)[0].tolist())
    assert touched == {12, 11, 13, 7, 17}


@pytest.mark.parametrize("passes", [2, 1])
def test_gmres_matches_direct_solve_with_restarts(passes):
    rng = np.random.default_rng(0)
    N = 60
    A = np.eye(N) * 4 + rng.standard_normal((N, N)) * 0.3
    b = rng.standard_normal(N)
    P = np.diag(1 / np.diag(A))
    for side in ("left", "right"):
        out = sv.gmres(lambda v: A @ v, b, lambda v: P @ v, 10, 1e-12, 500, side=side,
                       passes=passes)
        assert out.converged
        np.testing.assert_allclose(out.x, np.linalg.solve(A, b), atol=1e-10)
    np.testing.assert_allclose(out.x, np.linalg.solve(A, b), atol=1e-10)


@pytest.mark.parametrize("passes", [2, 1])
@pytest.mark.parametrize("side", ["left", "right"])
def test_gmres_minimal_residual_property(side, passes):
    """Without restart, after k steps GMRES attains the least-squares minimum over its
    Krylov space (library lstsq on an explicit basis): right preconditioning minimises
    ||b - A x|| over x in P K_k(A P, b); left preconditioning minimises ||P (b - A x)||
    over x in K_k(P A, P b)."""
    rng = np.random.default_rng(1)
    N, k = 40, 7
    A = np.eye(N) * 3 + rng.standard_normal((N, N)) * 0.5
    P = np.diag(1.0 + rng.uniform(0, 1, N))
    b = rng.standard_normal(N)
    out = sv.gmres(lambda v: A @ v, b, lambda v: P @ v, 50, 0.0, k, side=side, passes=passes)
    if side == "right":
        K = np.stack([np.linalg.matrix_power(A @ P, i) @ b for i in range(k)], axis=1)
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(A @ P @ Q, b, rcond=None)
        best = np.linalg.norm(b - A @ P @ Q @ y)
        got = np.linalg.norm(b - A @ out.x)
    else:
        K = np.stack([np.linalg.matrix_power(P @ A, i) @ (P @ b) for i in range(k)], axis=1)
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(P @ A @ Q, P @ b, rcond=None)
        best = np.linalg.norm(P @ b - P @ A @ Q @ y)
        got = np.linalg.norm(P @ (b - A @ out.x))
    assert out.iterations == k
    assert abs(got - best) <= 1e-10 * np.linalg.norm(b)


def test_block_inverse_is_exact_solver_for_block_diagonal_operator():
    """If the operator has no coupling (single element, periodic onto itself is not
    block diagonal, so use the blocks themselves) block-Jacobi GMRES converges in 1."""
    prob, q = _small_problem(p=1)
    B = sv.block_jacobian(prob, q, 0.0, 150.0)
    Binv = np.linalg.inv(B)
    r = inp.random_vector(q.shape, 2)

    def A(v):
        ne, bs, _ = B.shape
        ve = v.transpose(1, 0, 2, 3).reshape(ne, bs)
        return np.einsum("eab,eb->ea", B, ve).reshape(ne, 4, *v.shape[2:]).transpose(1, 0, 2, 3)

    out = sv.gmres(A, r, lambda v: sv.block_apply(Binv, v), 5, 1e-12, 5)
    assert out.iterations == 1
    np.testing.assert_allclose(A(out.x), r, atol=1e-10 * np.abs(r).max())


def _vortex_problem(N=4, p=2, mach=0.05, half=5.0, kappa=0.0):
    ref = inp.box_mesh(N, N, -half, half, -half, half)
    gas = ph.Gas(mach=mach, re=0.0, kappa=kappa)
    prob = sv.Problem(rs.Mesh(N, N, ref, np.zeros_like(ref)), p, gas)
    vx = inp.Vortex(mach=mach, period_x=2 * half, period_y=2 * half)
    X = inp.sample_points(ref, p)
    return prob, (lambda t: inp.vortex_state(*X, t, vx))


def _march(prob, exact, dt, nsteps, tol_pseudo=1e-8):
    """BDF1 first step from the interpolated exact state, BDF2 afterwards (an exact
    q^{n-1} would be inconsistent with the semi-discrete trajectory by O(dt h^p))."""
    q = exact(0.0)
    q_nm1 = q
    for s in range(nsteps):
        qc_n, qc_nm1 = prob.qc(q), prob.qc(q_nm1)
        q_new, st = sv.bdf2_step(prob, q, qc_n, qc_nm1, dt, coeffs=sv.BDF1 if s == 0 else sv.BDF2,
                                 tol_res=1e-10, tol_pseudo=tol_pseudo, maxit_lin=200,
                                 maxit_newton=12)
        assert st.converged
        q_nm1, q = q, q_new
    return q


@pytest.mark.slow
def test_bdf2_second_order_in_time():
    """Eq. unsteady_pre_discretized_2: BDF2 self-convergence ratio ~4 per halving of dt
    at fixed space (Sec. 4.3 study).  Time steps resolve the acoustic time h/c (at
    larger steps the stiff acoustic modes excited by the start are outside the
    asymptotic range)."""
    prob, exact = _vortex_problem(mach=0.1, kappa=1.0)
    T = 0.05
    ref = _march(prob, exact, T / 32, 32)
    errs = []
    for nst in (4, 8):
        q = _march(prob, exact, T / nst, nst)
        errs.append(sv.l2_error(prob, q[1], ref[1]))
    ratio = errs[0] / errs[1]
    # self-convergence against dt/8: e(dt)/e(dt/2) = (1 - 1/64)/(1/4 - 1/64) ~ 4.2
    assert 3.3 < ratio < 5.0, (errs, ratio)


def test_newton_converges_fast_with_exact_jvp():
    prob, exact = _vortex_problem(N=4, p=2)
    q0 = exact(0.0)
    qc = prob.qc(q0)
    _, st = sv.bdf2_step(prob, q0, qc, prob.qc(exact(-0.02)), 0.02, tol_res=1e-12,
                         tol_pseudo=1e-11, maxit_lin=300, maxit_newton=8)
    assert st.converged
    r = np.array(st.res_history) / st.res_history[0]
    # superlinear: each contraction factor is smaller than the previous one
    factors = r[1:] / r[:-1]
    assert factors[-1] < 1e-2 and np.all(np.diff(factors[:3]) < 0) or len(factors) <= 2


def test_ptc_ser_on_gaussian_bump():
    """Steady PTC with SER (Eqs. steady_pre_discretized_1, SER) on the Euler bump:
    after the pseudo-transient the residual collapses (Newton limit) while dtau grows
    from dtau_0 = 0.01 by orders of magnitude."""
    w = inp.EULER_BUMP_8
    w = inp.Workload(w.name, 4, 4, 2, w.mach, 0.0, 1.0, w.box, ic="bump", restart=20)
    c, v, q = inp.make_case(w)
    prob = sv.Problem(rs.Mesh(w.nx, w.ny, c, v), w.p, ph.Gas(mach=w.mach, kappa=1.0))
    _, st = sv.ptc_solve(prob, q, maxit_newton=26, restart=20, tol_res=1e-6, tol_pseudo=1e-8)
    res = np.array(st.res_history)
    assert st.converged and res[-1] <= 1e-8 * res[0]
    assert st.dtau_history[-1] > 1e6 * st.dtau_history[0]
    # SER law: dtau_m follows the last residual ratio squared, clipped to [dtau_min, dtau_max]
    for m in range(1, len(st.dtau_history)):
        want = min(1e20, max(0.01, st.dtau_history[m - 1] * (res[m - 1] / res[m]) ** 2))
        assert abs(st.dtau_history[m] - want) <= 1e-12 * want


def test_dense_operator_columns_match_jvp_and_fd():
    """The dense operator used for the transpose product agrees with the JVP on random
    vectors and with central differences of the residual (independent of complex steps)."""
    prob, q = _small_problem(p=1, nx=2, ny=2)
    A = sv.dense_operator(prob, q, 0.3, 150.0)
    v = inp.random_vector(q.shape, 3)
    np.testing.assert_allclose(A @ v.ravel(), sv.apply_A(prob, q, v, 0.3, 150.0).ravel(),
                               rtol=1e-12, atol=1e-12 * np.abs(A).max())
    G, M = prob.point_matrices(q)
    h = 1e-5
    fd = -(prob.R(q + h * v) - prob.R(q - h * v)) / (2 * h)
    fd = fd + np.einsum("ab...,b...->a...", 0.3 * G + 150.0 * M, v)
    assert np.abs(fd.ravel() - A @ v.ravel()).max() <= 1e-6 * np.abs(A @ v.ravel()).max()
    w = inp.random_vector(q.shape, 4)
    assert abs(w.ravel() @ (A @ v.ravel()) - sv.vjp(prob, q, w, 0.3, 150.0).ravel() @ v.ravel()) \
        <= 1e-12 * np.linalg.norm(w) * np.linalg.norm(A @ v.ravel())
