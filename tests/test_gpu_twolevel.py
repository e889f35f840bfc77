"""GPU parity of the two-level preconditioner (element block-Jacobi smoothing plus the
Galerkin P1 coarse correction solved by an agglomeration V-cycle) against the oracle's
definition (oracle.twolevel): the preconditioner applied to a vector, GMRES iteration
counts and BDF steps on stiff low-Mach cases, bounded meshes, batches against single
contexts, and convergence of the deforming 128 x 128 M = 0.01 workload."""
import numpy as np
import pytest

from gpu_helpers import case, oracle_problem, solver_for, to_dev, to_host
from oracle import physics as ph
from oracle import residual as rs
from oracle import solver as sv
from oracle import twolevel as tl
from paper_1903_06304_gb300 import inputs as inp

pytestmark = pytest.mark.gpu

# Relative tolerance of M^-1 r: both sides apply the same linear map in FP64, but through
# inverses of the coarse operators (condition numbers up to ~1e6 at M = 0.01), so rounding
# of the operands is amplified by up to that factor.  The FP32 coarse levels (the default)
# round the coarse correction to single precision: against the FP64 coarse levels the
# preconditioned vector differs by a few times 2^-24 amplified by the same conditioning.
APPLY_TOL = 1e-9
FP32_COARSE_TOL = 1e-3


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


# (nx, ny, p, mach, re, kappa, deforming): ragged element counts, the 2-wide periodic
# mesh whose left and right neighbours coincide, odd sizes that agglomerate with a
# leftover column, M from 0.01 to 0.1
APPLY_CASES = [
    (9, 7, 2, 0.05, 10.0, 1.0, True),
    (6, 5, 3, 0.01, 10.0, 1.0, True),
    (2, 3, 1, 0.1, 0.0, 1.0, False),
    (13, 4, 1, 0.01, 10.0, 1.0, True),
    (5, 5, 4, 0.05, 10.0, 1.0, False),
]


@pytest.mark.parametrize("cfg", APPLY_CASES)
def test_two_level_apply_matches_oracle(torch, cfg):
    nx, ny, p, mach, re, kappa, deforming = cfg
    c, v, q = case(nx, ny, p, mach, re, kappa, deforming)
    prob = oracle_problem(c, v, nx, ny, p, mach, re, kappa)
    inv_dtau, a0_dt = 0.0, 150.0
    S = solver_for(c, v, nx, ny, p, mach, re, kappa, precond="twolevel", mg_prec="fp64")
    qd = to_dev(q)
    S.precond_build(qd, inv_dtau, a0_dt)
    pc = tl.build(prob, q, inv_dtau, a0_dt)
    Aop = lambda x: sv.apply_A(prob, q, x, inv_dtau, a0_dt)
    for seed in (7, 8):
        r = inp.random_vector(prob.shape, seed)
        want = pc.apply(r, Aop)
        out = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
        S.precond_apply(to_dev(r), out)
        got = to_host(out)
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err <= APPLY_TOL, err
    S.close()


def test_two_level_apply_on_a_bounded_mesh(torch):
    """Plunging O-grid with a wall below row 0 and a far field above the last row: the
    coarse levels do not wrap across the boundaries (dual-number operator)."""
    ni, nj, p, mach, re = 12, 4, 2, 0.1, 200.0
    c, v = inp.plunge(inp.naca_ogrid(ni, nj), 0.3)
    qi = inp.far_field_state(mach)
    q = inp.random_perturbation(inp.uniform_state(ni * nj, p, mach), 3, 0.02, mach)
    from paper_1903_06304_gb300 import fr
    S = fr.Solver(fr.Config(p=p, mach=mach, re=re, kappa=5 ** 0.5, precond="twolevel",
                            mg_prec="fp64"), ni, nj,
                  bc=("wall", "farfield"), q_inf=qi)
    S.update_mesh(to_dev(c), to_dev(v))
    mesh = rs.Mesh(ni, nj, c, v, bc=(rs.WALL, rs.FARFIELD), q_inf=qi)
    prob = sv.Problem(mesh, p, ph.Gas(mach=mach, re=re, kappa=5 ** 0.5))
    inv_dtau, a0_dt = 0.0, 1.5 / 0.05
    qd = to_dev(q)
    S.precond_build(qd, inv_dtau, a0_dt)
    pc = tl.build(prob, q, inv_dtau, a0_dt)
    r = inp.random_vector(prob.shape, 9)
    want = pc.apply(r, lambda x: sv.apply_A(prob, q, x, inv_dtau, a0_dt))
    out = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    S.precond_apply(to_dev(r), out)
    err = np.abs(to_host(out) - want).max() / np.abs(want).max()
    assert err <= APPLY_TOL, err
    S.close()


@pytest.mark.parametrize("side", ["left", "right"])
def test_two_level_gmres_iterations_match_oracle(torch, side):
    nx = ny = 12
    p, mach, re = 2, 0.01, 10.0
    c, v, q = case(nx, ny, p, mach, re, 1.0, True)
    prob = oracle_problem(c, v, nx, ny, p, mach, re, 1.0)
    inv_dtau, a0_dt = 0.0, 150.0
    b = prob.R(q)
    pc = tl.build(prob, q, inv_dtau, a0_dt)
    Aop = lambda x: sv.apply_A(prob, q, x, inv_dtau, a0_dt)
    want = sv.gmres(Aop, b, lambda x: pc.apply(x, Aop), 30, 1e-6, 200, side=side)
    S = solver_for(c, v, nx, ny, p, mach, re, 1.0, precond="twolevel", gmres_side=side,
                   maxit_lin=200, mg_prec="fp64")
    qd = to_dev(q)
    S.precond_build(qd, inv_dtau, a0_dt)
    x = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    its = S.gmres(qd, to_dev(b), x, inv_dtau, a0_dt)
    assert its == want.iterations
    got = to_host(x)
    assert np.abs(got - want.x).max() <= 1e-7 * np.abs(want.x).max()
    S.close()


def test_two_level_bdf_step_matches_oracle(torch):
    nx = ny = 6
    p, mach, re, dt = 2, 0.01, 10.0, 0.01
    c, v, q = case(nx, ny, p, mach, re, 1.0, True)
    prob = oracle_problem(c, v, nx, ny, p, mach, re, 1.0)
    qc = prob.qc(q)
    qo, sto = sv.bdf2_step(prob, q, qc, qc, dt, coeffs=sv.BDF1, precond="twolevel")
    from paper_1903_06304_gb300 import fr
    S = solver_for(c, v, nx, ny, p, mach, re, 1.0, precond="twolevel", mg_prec="fp64")
    qd = to_dev(q)
    qcd = to_dev(qc)
    st = S.bdf2_step(qd, qcd, qcd, dt, coeffs=fr.BDF1).summary()
    assert st["converged"] and sto.converged
    assert st["newton_iterations"] == sto.newton_iterations
    assert st["gmres_iterations"] == sto.gmres_iterations
    # the last entries sit near the round-off floor of the pseudo-step residual (about
    # 1e-11 of Res_0 here), where the two evaluation orders legitimately differ
    np.testing.assert_allclose(st["res_history"], sto.res_history, rtol=1e-6, atol=1e-11 * sto.res_history[0])
    dq = np.abs(qo - q).max(axis=(1, 2, 3))
    assert np.all(np.abs(to_host(qd) - qo).max(axis=(1, 2, 3)) <= 1e-6 * dq)
    S.close()


def test_two_level_batch_equals_single_contexts(torch):
    """Cases of different sizes agglomerate to different depths; each case of a batch
    follows its single-case context (same Newton and GMRES counts, same state)."""
    from paper_1903_06304_gb300 import fr
    specs = [(8, 6, 0.02, "vortex"), (5, 9, 0.05, "vortex"), (12, 12, 0.01, "vortex")]
    p, dt = 2, 0.01
    cases, states, corners = [], [], []
    for k, (nx, ny, m, _ic) in enumerate(specs):
        ref = inp.box_mesh(nx, ny, 0.0, 10.0, 0.0, 10.0)
        x, y = inp.sample_points(ref, p)
        vx = inp.Vortex(mach=m, alpha=2.0, x0=3.0 + k, y0=4.0, period_x=10.0, period_y=10.0)
        qk = inp.vortex_state(x, y, 0.0, vx)
        cases.append(fr.Case(p, nx, ny, m, 10.0, 1.0))
        states.append(qk)
        corners.append(ref)
    cfg = fr.Config(precond="twolevel", maxit_newton=20)
    B = fr.Batch(cfg, cases)
    cor = np.zeros((B.ne, 4, 2))
    qb = np.zeros(B.ndof)
    for k in range(len(cases)):
        cor[B.elem_slice(k)] = corners[k]
        qb[B.case_slice(k)] = states[k].ravel()
    B.update_mesh(to_dev(cor), to_dev(np.zeros_like(cor)))
    qd = to_dev(qb)
    qc = torch.empty_like(qd)
    B.conservative(qd, qc)
    sts = B.bdf2_step(qd, qc, qc, [(1.0, -1.0, 0.0, dt)] * len(cases))
    got = to_host(qd)
    for k, (nx, ny, m, _ic) in enumerate(specs):
        S = solver_for(corners[k], np.zeros_like(corners[k]), nx, ny, p, m, 10.0, 1.0,
                       precond="twolevel", maxit_newton=20)
        q1 = to_dev(states[k])
        qc1 = torch.empty_like(q1)
        S.conservative(q1, qc1)
        st = S.bdf2_step(q1, qc1, qc1, dt, coeffs=fr.BDF1).summary()
        assert sts[k].converged and st["converged"]
        assert sts[k].newton_iterations == st["newton_iterations"]
        assert list(sts[k].gmres_iterations[:st["newton_iterations"]]) == st["gmres_iterations"]
        dq = np.abs(to_host(q1) - states[k]).max()
        assert np.abs(got[B.case_slice(k)] - to_host(q1).ravel()).max() <= 1e-9 * dq
        S.close()
    B.close()


def test_low_mach_deforming_step_reaches_the_rounding_floor(torch):
    """The deforming vortex at M = 0.01, p = 3 on 48 x 48 elements (the element size at which
    element block Jacobi already stalls): with the coarse correction the first BDF1 step
    drives Res_m/Res_0 to 1e-7 within 6 Newton iterations (the FP64 rounding floor of the
    continuity residual sits near 2e-8 of Res_0 here) with well under half the GMRES
    iterations that block Jacobi alone spends (its GMRES runs to the cap every step)."""
    from paper_1903_06304_gb300 import fr
    w = inp.Workload("deform_48", 48, 48, 3, 0.01, 10.0, 1.0, ic="vortex", deforming=True)
    c0, v0, q0 = inp.make_case(w, t=0.0)
    c1, v1, _ = inp.make_case(w, t=w.dt)
    res = {}
    for precond in ("twolevel", "block"):
        S = fr.Solver(fr.Config(p=w.p, mach=w.mach, re=w.re, kappa=w.kappa, precond=precond,
                                maxit_newton=6, tol_pseudo=1e-7), w.nx, w.ny)
        S.update_mesh(to_dev(c1), to_dev(v1))
        q = to_dev(q0)
        qc = torch.empty_like(q)
        S.conservative(q, qc)
        res[precond] = S.bdf2_step(q, qc, qc, w.dt, coeffs=fr.BDF1, allow_unconverged=True).summary()
        S.close()
    assert res["twolevel"]["converged"], res["twolevel"]
    # block Jacobi needs GMRES at its cap on every Newton step; the coarse correction a
    # fraction of it
    tot = {k: sum(v["gmres_iterations"]) for k, v in res.items()}
    assert 2 * tot["twolevel"] <= tot["block"], tot


@pytest.mark.parametrize("cfg", APPLY_CASES[:3])
def test_fp32_coarse_levels_against_fp64(torch, cfg):
    """The FP32 coarse levels (storage and sweeps; FP64 builds and fine transfers) apply
    the same preconditioner to single-precision rounding, and GMRES with them takes about
    the same iterations to a true residual of the same size."""
    nx, ny, p, mach, re, kappa, deforming = cfg
    c, v, q = case(nx, ny, p, mach, re, kappa, deforming)
    inv_dtau, a0_dt = 0.0, 150.0
    qd = to_dev(q)
    r = to_dev(inp.random_vector(q.shape, 7))
    b = to_dev(inp.random_vector(q.shape, 8))
    out, its, xs = {}, {}, {}
    for prec in ("fp64", "fp32"):
        S = solver_for(c, v, nx, ny, p, mach, re, kappa, precond="twolevel", mg_prec=prec,
                       maxit_lin=300, restart=60)
        S.precond_build(qd, inv_dtau, a0_dt)
        o = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
        S.precond_apply(r, o)
        out[prec] = to_host(o)
        x = torch.empty_like(o)
        its[prec] = S.gmres(qd, b, x, inv_dtau, a0_dt)
        Ax = torch.empty_like(o)
        S.jvp(qd, x, Ax, inv_dtau, a0_dt)
        xs[prec] = float(torch.linalg.norm(b - Ax) / torch.linalg.norm(b))
        S.close()
    err = np.abs(out["fp32"] - out["fp64"]).max() / np.abs(out["fp64"]).max()
    assert err <= FP32_COARSE_TOL, err
    assert abs(its["fp32"] - its["fp64"]) <= max(2, 0.15 * its["fp64"]), its
    # both true residuals at the level GMRES was asked for
    assert xs["fp32"] <= 10 * max(xs["fp64"], 1e-7), xs


@pytest.mark.parametrize("cfg", APPLY_CASES)
@pytest.mark.parametrize("bounded", [False, True])
def test_local_galerkin_build_equals_operator_products(torch, cfg, bounded):
    """The level-0 operators and A P columns formed from the stored local Jacobians (face
    couplings and the element blocks: the build of the linearised operator mode) against
    those formed by coloured products of the dual-number operator: the same preconditioner
    to the rounding of the two evaluation orders."""
    from paper_1903_06304_gb300 import fr
    nx, ny, p, mach, re, kappa, deforming = cfg
    inv_dtau, a0_dt = 0.3, 150.0
    if bounded:
        nx, ny = max(nx, 4), max(ny, 3)
        c, v = inp.plunge(inp.naca_ogrid(nx, ny, first=0.05), 0.3)
        qi = inp.far_field_state(mach)
        q = inp.random_perturbation(inp.uniform_state(nx * ny, p, mach), 5, 0.02, mach)
    else:
        c, v, q = case(nx, ny, p, mach, re, kappa, deforming)
    r = to_dev(inp.random_vector(q.shape, 19))
    outs = []
    for mode in ("dual", "linearized"):
        kw = dict(p=p, mach=mach, re=re, kappa=kappa, precond="twolevel", mg_prec="fp64",
                  jvp_mode=mode, block_mode=mode)
        if bounded:
            S = fr.Solver(fr.Config(**kw), nx, ny, bc=("wall", "farfield"), q_inf=qi)
        else:
            S = fr.Solver(fr.Config(**kw), nx, ny)
        S.update_mesh(to_dev(c), to_dev(v))
        S.precond_build(to_dev(q), inv_dtau, a0_dt)
        out = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
        S.precond_apply(r, out)
        outs.append(to_host(out))
        S.close()
    err = np.abs(outs[1] - outs[0]).max() / np.abs(outs[0]).max()
    assert err <= APPLY_TOL, err


@pytest.mark.parametrize("cfg", APPLY_CASES)
@pytest.mark.parametrize("bounded", [False, True])
def test_transposed_two_level_is_the_transpose(torch, cfg, bounded):
    """<y, M^-1 x> = <M^-T y, x>: the transposed map (transposed blocks, the transposed
    coarse hierarchy and the transposed smoothing step) against the forward one, FP64
    blocks and coarse levels."""
    from paper_1903_06304_gb300 import fr
    nx, ny, p, mach, re, kappa, deforming = cfg
    inv_dtau, a0_dt = 0.3, 150.0
    kw = dict(p=p, mach=mach, re=re, kappa=kappa, precond="twolevel", mg_prec="fp64", prec="fp64")
    if bounded:
        nx, ny = max(nx, 4), max(ny, 3)
        c, v = inp.plunge(inp.naca_ogrid(nx, ny, first=0.05), 0.3)
        q = inp.random_perturbation(inp.uniform_state(nx * ny, p, mach), 5, 0.02, mach)
        S = fr.Solver(fr.Config(**kw), nx, ny, bc=("wall", "farfield"), q_inf=inp.far_field_state(mach))
    else:
        c, v, q = case(nx, ny, p, mach, re, kappa, deforming)
        S = fr.Solver(fr.Config(**kw), nx, ny)
    S.update_mesh(to_dev(c), to_dev(v))
    S.precond_build(to_dev(q), inv_dtau, a0_dt)
    rng = np.random.default_rng(41)
    for _ in range(2):
        x = to_dev(rng.standard_normal(q.shape))
        y = to_dev(rng.standard_normal(q.shape))
        Mx = torch.empty_like(x)
        MTy = torch.empty_like(x)
        S.precond_apply(x, Mx)
        S.precond_apply_transposed(y, MTy)
        lhs, rhs = float((y * Mx).sum()), float((MTy * x).sum())
        scale = float((y.abs() * Mx.abs()).sum())
        assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs, scale)
    S.close()
