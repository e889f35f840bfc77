"""Bounded meshes (fr_set_mesh_bounded): the residual, the dual-number JVP, the element
blocks, GMRES and a BDF step with wall and far-field faces (Sec. 3.3) against the oracle,
on plunging NACA 0012 O-grids (Secs. 4.2, 4.4) from a few elements up to the full
256 x 96 grid; and the stored-Jacobian calls, which do not treat boundary faces yet,
refuse a bounded mesh."""
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


@pytest.mark.parametrize("re", [0.0, 200.0])
def test_bounded_blocks_parity(torch, re):
    """Element blocks by dual numbers with wall and far-field faces (the boundary flux
    depends on the element's own trace) against the oracle's complex-step blocks."""
    S, prob, q = bounded_case(10, 4, 2, 0.1, re, 1.0, ("wall", "farfield"), first=0.05)
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


def test_bounded_bdf_step_parity(torch):
    """One BDF1 step on a plunging O-grid with a wall and a far field: the Newton loop with
    the dual-number operator and blocks takes the oracle's Newton and GMRES iterations."""
    from paper_1903_06304_gb300 import fr
    kw = dict(restart=30, tol_res=1e-6, maxit_lin=100, tol_pseudo=1e-8, maxit_newton=10, lag=2)
    S, prob, q = bounded_case(10, 4, 2, 0.1, 200.0, 1.0, ("wall", "farfield"), first=0.05, rel=0.02,
                              **kw)
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


def test_bounded_mesh_refuses_stored_jacobian_paths(torch):
    from paper_1903_06304_gb300 import fr
    S, prob, q = bounded_case(8, 3, 2, 0.1, 50.0, 1.0, ("wall", "farfield"))
    qd = to_dev(q)
    with pytest.raises(fr.FrError, match="bounded"):
        S.linearize(qd, 0.0, 150.0)
    out = torch.empty_like(qd)
    with pytest.raises(fr.FrError, match="bounded"):
        S.vjp(qd, qd, out, 0.0, 150.0)
    # the available calls still work after a refusal
    R = torch.empty_like(qd)
    S.residual(qd, R)
    err = residual_errors(to_host(R), prob.R(q), q, prob.mesh, 2, prob.gas)
    assert np.all(err <= RES_TOL), err


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
    assert st["gmres_iterations"] == sto.gmres_iterations
    np.testing.assert_allclose(st["res_history"], sto.res_history, rtol=1e-6)
    S.close()
