"""Bounded meshes (fr_set_mesh_bounded): the residual, the dual-number and linearised
JVP, the transposed operator (VJP), the element blocks of both build modes, GMRES and a
BDF step with wall and far-field faces (Sec. 3.3) against the oracle, on plunging
NACA 0012 O-grids (Secs. 4.2, 4.4) from a few elements up to the full 256 x 96 grid."""
import numpy as np
import pytest

from oracle import physics as ph
from oracle import residual as rs
from oracle import scale as sc
from oracle import solver as sv
from paper_1903_06304_gb300 import inputs as inp

from gpu_helpers import (BLK_TOL, JVP_TOL, RES_TOL, block_errors, jvp_errors, residual_errors,
                         to_dev, to_host)

pytestmark = pytest.mark.gpu

KIND = {"wall": rs.WALL, "farfield": rs.FARFIELD}


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def bounded_case(ni, nj, p, mach, re, kappa, bc, t=0.3, seed=7, rel=0.05, first=1e-3, **kw):
    from paper_1903_06304_gb300 import fr
    c, v = inp.plunge(inp.naca_ogrid(ni, nj, first=first), t)
    qi = inp.far_field_state(mach)
    gas = ph.Gas(mach=mach, re=re, kappa=kappa)
    mesh = rs.Mesh(ni, nj, c, v, bc=(KIND[bc[0]], KIND[bc[1]]), q_inf=qi)
    q = inp.random_perturbation(inp.uniform_state(ni * nj, p, mach), seed, rel, mach)
    S = fr.Solver(fr.Config(p=p, mach=mach, re=re, kappa=kappa, **kw), ni, nj, bc=bc, q_inf=qi)
    S.update_mesh(to_dev(c), to_dev(v))
    return S, sv.Problem(mesh, p, gas), q


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("re", [0.0, 200.0])
@pytest.mark.parametrize("bc", [("wall", "farfield"), ("farfield", "farfield"), ("wall", "wall")])
def test_bounded_residual_parity(torch, p, re, bc):
    # 13 x 5 elements: a ragged count against every tile of elements per block
    S, prob, q = bounded_case(13, 5, p, 0.1, re, 1.0, bc)
    R = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    S.residual(to_dev(q), R)
    err = residual_errors(to_host(R), prob.R(q), q, prob.mesh, p, prob.gas)
    assert np.all(err <= RES_TOL), err


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("re", [0.0, 200.0])
@pytest.mark.parametrize("bc", [("wall", "farfield"), ("farfield", "wall")])
def test_bounded_jvp_parity(torch, p, re, bc):
    """A v = inv_dtau Gamma v + a0_dt M v - dR/dq v through the boundary faces (the wall
    state depends on the trace, the far-field state does not)."""
    S, prob, q = bounded_case(11, 4, p, 0.1, re, 1.0, bc)
    x = inp.random_vector(q.shape, 21) * np.array([inp.p_inf(0.1) * 1e-2, 1, 1, 1])[:, None, None, None]
    inv_dtau, a0_dt = 0.3, 150.0
    out = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    S.jvp(to_dev(q), to_dev(x), out, inv_dtau, a0_dt)
    err = jvp_errors(to_host(out), sv.apply_A(prob, q, x, inv_dtau, a0_dt))
    assert np.all(err <= JVP_TOL), err


@pytest.mark.parametrize("re", [0.0, 100.0])
def test_bounded_free_stream_preserved(torch, re):
    """The free stream with far-field faces on both sides of a plunging O-grid."""
    from paper_1903_06304_gb300 import fr
    ni, nj, p, mach = 24, 6, 3, 0.1
    c, v = inp.plunge(inp.naca_ogrid(ni, nj), 0.3)
    qi = inp.far_field_state(mach)
    S = fr.Solver(fr.Config(p=p, mach=mach, re=re, kappa=1.0), ni, nj, bc=("farfield", "farfield"),
                  q_inf=qi)
    S.update_mesh(to_dev(c), to_dev(v))
    q = inp.uniform_state(ni * nj, p, mach)
    R = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    S.residual(to_dev(q), R)
    gas = ph.Gas(mach=mach, re=re, kappa=1.0)
    s = sc.residual_scale(q, rs.Mesh(ni, nj, c, v, bc=(rs.FARFIELD, rs.FARFIELD), q_inf=qi), p, gas)
    assert np.all(np.abs(to_host(R)).max(axis=(1, 2, 3)) <= RES_TOL * s)


def test_bounded_residual_full_naca_ogrid(torch):
    """The plunging NACA 0012 workload's grid at full size: 256 x 96 elements, p = 3,
    Re = 1e4, kappa = sqrt(5), wall below row 0 and far field above the last row; every
    point against the oracle, and the pseudo-step right-hand side with BDF2 terms."""
    from paper_1903_06304_gb300 import fr
    ni, nj, p, mach = 256, 96, 3, 0.1
    S, prob, q = bounded_case(ni, nj, p, mach, 1e4, 5 ** 0.5, ("wall", "farfield"), t=0.9)
    qd = to_dev(q)
    R = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    S.residual(qd, R)
    Ro = prob.R(q)
    err = residual_errors(to_host(R), Ro, q, prob.mesh, p, prob.gas)
    assert np.all(err <= RES_TOL), err
    # r = R - (a0 q^c + a1 qc_n + a2 qc_nm1)/dt
    qn = inp.random_perturbation(q, 8, 1e-3, mach)
    qnm = inp.random_perturbation(q, 9, 1e-3, mach)
    qcn, qcnm = prob.qc(qn), prob.qc(qnm)
    dt = 0.05
    r = torch.empty_like(R)
    S.bdf_rhs(qd, to_dev(qcn), to_dev(qcnm), fr.BDF2, dt, r)
    want = sv.time_rhs(prob, q, qcn, qcnm, dt, coeffs=fr.BDF2)
    err = residual_errors(to_host(r), want, q, prob.mesh, p, prob.gas)
    assert np.all(err <= RES_TOL), err


@pytest.mark.parametrize("mode", ["linearized", "dual"])
@pytest.mark.parametrize("re", [0.0, 200.0])
@pytest.mark.parametrize("bc", [("wall", "farfield"), ("farfield", "wall")])
def test_bounded_blocks_parity(torch, mode, re, bc):
    """Element blocks with wall and far-field faces (the boundary flux depends on the
    element's own trace), from the stored local Jacobians or by dual numbers, against the
    oracle's complex-step blocks."""
    S, prob, q = bounded_case(10, 4, 2, 0.1, re, 1.0, bc, first=0.05, block_mode=mode)
    inv_dtau, a0_dt = 0.2, 150.0
    S.precond_build(to_dev(q), inv_dtau, a0_dt)
    B = torch.empty((prob.mesh.ne, S.block_size, S.block_size), dtype=torch.float64, device="cuda:0")
    S.precond_blocks(B)
    err = block_errors(to_host(B), sv.block_jacobian(prob, q, inv_dtau, a0_dt), 9)
    assert np.all(err <= BLK_TOL), err


@pytest.mark.parametrize("side", ["left", "right"])
def test_bounded_gmres_parity(torch, side):
    S, prob, q = bounded_case(10, 4, 2, 0.1, 200.0, 1.0, ("wall", "farfield"), first=0.05,
                              restart=20, maxit_lin=200, tol_res=1e-8, gmres_side=side)
    inv_dtau, a0_dt = 1e-20, 100.0
    b = inp.random_vector(q.shape, 13)
    Binv = np.linalg.inv(sv.block_jacobian(prob, q, inv_dtau, a0_dt))
    P = lambda x: sv.block_apply(Binv, x)
    want = sv.gmres(lambda x: sv.apply_A(prob, q, x, inv_dtau, a0_dt), b, P, 20, 1e-8, 200, side=side)
    qd = to_dev(q)
    S.precond_build(qd, inv_dtau, a0_dt)
    x = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    its = S.gmres(qd, to_dev(b), x, inv_dtau, a0_dt)
    assert its == want.iterations
    assert np.abs(to_host(x) - want.x).max() <= 1e-9 * np.abs(want.x).max()


@pytest.mark.parametrize("mode", ["linearized", "dual"])
def test_bounded_bdf_step_parity(torch, mode):
    """One BDF1 step on a plunging O-grid with a wall and a far field: the Newton loop with
    the stored (or dual-number) operator and blocks takes the oracle's Newton and GMRES
    iterations."""
    from paper_1903_06304_gb300 import fr
    kw = dict(restart=30, tol_res=1e-6, maxit_lin=100, tol_pseudo=1e-8, maxit_newton=10, lag=2)
    S, prob, q = bounded_case(10, 4, 2, 0.1, 200.0, 1.0, ("wall", "farfield"), first=0.05, rel=0.02,
                              jvp_mode=mode, block_mode=mode, **kw)
    qc = prob.qc(q)
    q1, st = sv.bdf2_step(prob, q, qc, qc, 0.01, coeffs=sv.BDF1, **kw)
    qd, qcd = to_dev(q), to_dev(qc)
    sg = S.bdf2_step(qd, qcd, qcd, 0.01, coeffs=fr.BDF1).summary()
    assert sg["converged"] and st.converged
    assert sg["newton_iterations"] == st.newton_iterations
    assert sg["gmres_iterations"] == st.gmres_iterations
    np.testing.assert_allclose(sg["res_history"], st.res_history, rtol=1e-6,
                               atol=1e-12 * st.res_history[0])
    scale = np.abs(q1 - q).max(axis=(1, 2, 3))
    assert np.all(np.abs(to_host(qd) - q1).max(axis=(1, 2, 3)) <= 1e-6 * scale)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("re", [0.0, 200.0])
@pytest.mark.parametrize("bc", [("wall", "farfield"), ("farfield", "wall"), ("wall", "wall")])
def test_wall_force_parity(torch, p, re, bc):
    """The device wall force against the oracle's (pressure and viscous traction of the
    wall's common gradient, Gauss quadrature over the wall faces)."""
    S, prob, q = bounded_case(13, 5, p, 0.1, re, 1.0, bc)
    got = np.array(S.wall_force(to_dev(q)))
    want = np.array(rs.wall_force(q, prob.mesh, p, prob.gas))
    # the integrand sums terms of the size of p - p_inf and of the stress over the wall
    scale = max(np.abs(want).max(), 1e-3)
    assert np.all(np.abs(got - want) <= 1e-11 * scale), (got, want)


def test_wall_force_of_linear_pressure_is_exact(torch):
    """No flow, p = p_inf + a x + b y: F = -(a, b) x the area enclosed by the wall polygon."""
    from paper_1903_06304_gb300 import fr
    ni, nj, p, mach = 48, 4, 3, 0.05
    c = inp.naca_ogrid(ni, nj)
    qi = inp.far_field_state(mach)
    S = fr.Solver(fr.Config(p=p, mach=mach, re=50.0, kappa=1.0), ni, nj, bc=("wall", "farfield"),
                  q_inf=qi)
    S.update_mesh(to_dev(c), to_dev(np.zeros_like(c)))
    a, b = 0.3, -0.7
    X, Y = inp.sample_points(c, p)
    q = np.stack([inp.p_inf(mach) + a * X + b * Y, 0 * X, 0 * X, 1 + 0 * X])
    Fx, Fy = S.wall_force(to_dev(q))
    w = c[:ni, 0]
    A = abs(0.5 * np.sum(w[:, 0] * np.roll(w[:, 1], -1) - np.roll(w[:, 0], -1) * w[:, 1]))
    assert abs(Fx + a * A) <= 1e-11 and abs(Fy + b * A) <= 1e-11, (Fx, Fy, -a * A, -b * A)


def test_wall_force_needs_a_wall(torch):
    from paper_1903_06304_gb300 import fr
    S, prob, q = bounded_case(8, 3, 2, 0.1, 50.0, 1.0, ("farfield", "farfield"))
    with pytest.raises(fr.FrError, match="wall"):
        S.wall_force(to_dev(q))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("re", [0.0, 200.0])
@pytest.mark.parametrize("bc", [("wall", "farfield"), ("farfield", "wall"), ("wall", "wall")])
def test_bounded_linearized_jvp_parity(torch, p, re, bc):
    """The stored linearisation with boundary faces (the boundary map's Jacobian in the
    trace and its gradient, q^com = D_b q^-) against the oracle's complex step and the
    dual-number product."""
    S, prob, q = bounded_case(11, 4, p, 0.1, re, 1.0, bc)
    x = inp.random_vector(q.shape, 22) * np.array([inp.p_inf(0.1) * 1e-2, 1, 1, 1])[:, None, None, None]
    qd, xd = to_dev(q), to_dev(x)
    lin = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    dual = torch.empty_like(lin)
    for inv_dtau, a0_dt in ((0.0, 0.0), (0.3, 150.0)):
        S.linearize(qd, inv_dtau, a0_dt)
        S.apply_linear(xd, lin)
        S.jvp(qd, xd, dual, inv_dtau, a0_dt)
        want = sv.apply_A(prob, q, x, inv_dtau, a0_dt)
        assert np.all(jvp_errors(to_host(lin), want) <= JVP_TOL)
        assert np.all(jvp_errors(to_host(lin), to_host(dual)) <= JVP_TOL)


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("re", [0.0, 200.0])
@pytest.mark.parametrize("bc", [("wall", "farfield"), ("farfield", "wall"), ("wall", "wall")])
def test_bounded_vjp_parity_dense_oracle(torch, p, re, bc):
    """fr_vjp on a bounded mesh against the transpose of the oracle's dense operator."""
    ni, nj = (6, 3) if p == 1 else (5, 2)
    S, prob, q = bounded_case(ni, nj, p, 0.1, re, 1.0, bc, first=0.05)
    w = inp.random_vector(q.shape, 14)
    out = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    for inv_dtau, a0_dt in ((0.0, 0.0), (0.3, 150.0)):
        S.vjp(to_dev(q), to_dev(w), out, inv_dtau, a0_dt)
        want = sv.vjp(prob, q, w, inv_dtau, a0_dt)
        err = np.abs(to_host(out) - want).max(axis=(1, 2, 3)) / np.abs(want).max(axis=(1, 2, 3))
        assert np.all(err <= 1e-11), err


@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("re", [0.0, 200.0])
def test_bounded_vjp_dot_product_identity(torch, p, re):
    """<y, A x> = <A^T y, x> for the stored forward and reverse products with wall and
    far-field faces (13 x 5: a ragged count of elements per block)."""
    S, prob, q = bounded_case(13, 5, p, 0.1, re, 1.0, ("wall", "farfield"))
    qd = to_dev(q)
    rng = np.random.default_rng(33)
    for inv_dtau, a0_dt in ((0.0, 0.0), (0.3, 150.0)):
        S.linearize(qd, inv_dtau, a0_dt)
        for _ in range(3):
            x = to_dev(rng.standard_normal(q.shape))
            y = to_dev(rng.standard_normal(q.shape))
            Ax = torch.empty_like(x)
            ATy = torch.empty_like(x)
            S.apply_linear(x, Ax)
            S.apply_linear(y, ATy, transpose=True)
            lhs, rhs = float((y * Ax).sum()), float((ATy * x).sum())
            assert abs(lhs - rhs) <= 1e-12 * float(y.norm() * Ax.norm()), (lhs, rhs)


def test_bounded_vjp_full_naca_ogrid_sampled(torch):
    """The transposed operator on the full 256 x 96 O-grid (p = 3, Re = 1e4), sampled: w
    lives on mutually distant elements, including the wall row and the far-field row, so
    for every x the identity sum over the stencil of e of (A^T w)_g . x_g = w_e . (A x)_e
    holds per pick, with A x from the oracle's complex step."""
    ni, nj, p, mach = 256, 96, 3, 0.1
    S, prob, q = bounded_case(ni, nj, p, mach, 1e4, 5 ** 0.5, ("wall", "farfield"), t=0.9)
    a0_dt = 1.5 / 0.0314
    rng = np.random.default_rng(37)
    rows = [0, 1, 40, 94, 95]
    picks = [j * ni + i for j in rows for i in range(3 * (j % 3), ni, 41)]
    wv = np.zeros(q.shape)
    for e in picks:
        wv[:, e] = rng.standard_normal(wv[:, e].shape)
    out = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    S.vjp(to_dev(q), to_dev(wv), out, 1e-20, a0_dt)
    ATw = to_host(out)
    left, right, bottom, top = prob.mesh.neighbours()
    for trial in range(2):
        x = rng.standard_normal(q.shape)
        x[0] *= prob.gas.R * 1e-2
        Ax = sv.apply_A(prob, q, x, 1e-20, a0_dt)
        for e in picks:
            st = {int(g) for g in (e, left[e], right[e], bottom[e], top[e]) if g >= 0}
            lhs = sum(float(np.sum(ATw[:, g] * x[:, g])) for g in st)
            rhs = float(np.sum(wv[:, e] * Ax[:, e]))
            scale = sum(float(np.sum(np.abs(ATw[:, g] * x[:, g]))) for g in st)
            assert abs(lhs - rhs) <= 1e-11 * scale, (trial, e, lhs, rhs)


def test_bad_boundaries_rejected(torch):
    from paper_1903_06304_gb300 import fr
    cfg = fr.Config(p=2, mach=0.1)
    with pytest.raises(fr.FrError):
        fr.Solver(cfg, 8, 3, bc=("farfield", "wall"), q_inf=None)       # far field without q_inf
    with pytest.raises(fr.FrError):
        fr.Solver(cfg, 8, 3, bc=("wall", "farfield"), q_inf=(-1.0, 1.0, 0.0, 1.0))
    with pytest.raises(fr.FrError):
        fr.Solver(cfg, 1, 3, bc=("wall", "wall"))


@pytest.mark.parametrize("precond", ["block", "twolevel"])
def test_steady_ptc_on_a_cylinder_matches_oracle(torch, precond):
    """Steady pseudo-transient continuation with SER (Eqs. steady_pre_discretized_1, SER)
    on a small cylinder O-grid (no-slip adiabatic wall, far field at 20 diameters,
    Re = 20, M = 0.1) from the impulsively started free stream: the GPU takes the
    oracle's pseudo steps and GMRES iterations and follows its Res_m history, with the
    element blocks or with the coarse correction."""
    from paper_1903_06304_gb300 import fr
    ni, nj, p, mach, re = 12, 4, 1, 0.1, 20.0
    c = inp.cylinder_ogrid(ni, nj, 20.0, 0.05)
    v = np.zeros_like(c)
    qi = inp.far_field_state(mach)
    q = inp.uniform_state(ni * nj, p, mach)
    mesh = rs.Mesh(ni, nj, c, v, bc=(rs.WALL, rs.FARFIELD), q_inf=qi)
    prob = sv.Problem(mesh, p, ph.Gas(mach=mach, re=re, kappa=1.0))
    rhs = lambda s: prob.R(s)
    _, sto = sv.newton_solve(prob, q, rhs, 0.0, 0.01, 20, 1e-6, 100, 1e-6, 12, 1,
                             ser=(0.01, 1e20, 2.0), precond=precond)
    S = fr.Solver(fr.Config(p=p, mach=mach, re=re, kappa=1.0, restart=20, tol_pseudo=1e-6,
                            maxit_newton=12, precond=precond, mg_prec="fp64"), ni, nj,
                  bc=("wall", "farfield"), q_inf=qi)
    S.update_mesh(to_dev(c), to_dev(v))
    st = S.ptc_solve(to_dev(q), allow_unconverged=True).summary()
    assert st["newton_iterations"] == sto.newton_iterations
    if precond == "block":
        assert st["gmres_iterations"] == sto.gmres_iterations
        # the last entries sit seven orders below Res_0, where the Newton updates carry
        # the GMRES round-off (summation order) of the tolerance-limited solves: compare
        # those on the scale of Res_0
        np.testing.assert_allclose(st["res_history"], sto.res_history, rtol=1e-6,
                                   atol=1e-12 * sto.res_history[0])
    else:
        # the coarse solve sums in another order than the oracle's dense one: a GMRES
        # solve whose residual lands within rounding of tol_res may take one iteration
        # more or less, and the next pseudo step then starts from a state that differs
        # by up to tol_res of the update
        assert np.all(np.abs(np.subtract(st["gmres_iterations"], sto.gmres_iterations)) <= 1)
        np.testing.assert_allclose(st["res_history"], sto.res_history, rtol=1e-3,
                                   atol=1e-9 * sto.res_history[0])
    S.close()
