"""Bounded meshes (fr_set_mesh_bounded): the residual and the dual-number JVP with wall and
far-field faces (Sec. 3.3) against the oracle, on plunging NACA 0012 O-grids (Secs. 4.2,
4.4) from a few elements up to the full 256 x 96 grid; and the calls that do not treat
boundary faces yet refuse a bounded mesh."""
import numpy as np
import pytest

from oracle import physics as ph
from oracle import residual as rs
from oracle import scale as sc
from oracle import solver as sv
from paper_1903_06304_gb300 import inputs as inp

from gpu_helpers import JVP_TOL, RES_TOL, jvp_errors, residual_errors, to_dev, to_host

pytestmark = pytest.mark.gpu

KIND = {"wall": rs.WALL, "farfield": rs.FARFIELD}


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def bounded_case(ni, nj, p, mach, re, kappa, bc, t=0.3, seed=7, rel=0.05):
    from paper_1903_06304_gb300 import fr
    c, v = inp.plunge(inp.naca_ogrid(ni, nj), t)
    qi = inp.far_field_state(mach)
    gas = ph.Gas(mach=mach, re=re, kappa=kappa)
    mesh = rs.Mesh(ni, nj, c, v, bc=(KIND[bc[0]], KIND[bc[1]]), q_inf=qi)
    q = inp.random_perturbation(inp.uniform_state(ni * nj, p, mach), seed, rel, mach)
    S = fr.Solver(fr.Config(p=p, mach=mach, re=re, kappa=kappa), ni, nj, bc=bc, q_inf=qi)
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


def test_bounded_mesh_refuses_solver_paths(torch):
    from paper_1903_06304_gb300 import fr
    S, prob, q = bounded_case(8, 3, 2, 0.1, 50.0, 1.0, ("wall", "farfield"))
    qd = to_dev(q)
    with pytest.raises(fr.FrError, match="bounded"):
        S.precond_build(qd, 0.0, 150.0)
    with pytest.raises(fr.FrError, match="bounded"):
        S.linearize(qd, 0.0, 150.0)
    qc = torch.empty_like(qd)
    S.conservative(qd, qc)
    with pytest.raises(fr.FrError, match="bounded"):
        S.bdf2_step(qd, qc, qc, 0.01, coeffs=fr.BDF1)
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
