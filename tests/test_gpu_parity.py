"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle on the same
seeded inputs: geometry-dependent residual, BDF right-hand side, exact JVP, element
blocks, block apply, GMRES and whole BDF2 / PTC Newton steps.  Sizes span several
thread blocks with ragged tails; full workload sizes are checked too."""
import numpy as np
import pytest

from gpu_helpers import (BLK_TOL, JVP_TOL, RES_TOL, block_errors, case, jvp_errors,
                         oracle_problem, residual_errors, solver_for, to_dev, to_host)
from oracle import solver as sv
from paper_1903_06304_gb300 import inputs as inp

pytestmark = pytest.mark.gpu

# (nx, ny, p, mach, re, kappa, deforming): ragged tails (Ne not a multiple of the
# elements per block: 14 at p=2, 8 at p=3, 5 at p=4), Euler and Navier-Stokes, static and
# deforming, M from 0.01 to 0.3, kappa = 0 (vortex reading) and 1.
CASES = [
    (4, 3, 1, 0.1, 0.0, 1.0, False),
    (5, 3, 2, 0.05, 10.0, 1.0, True),
    (6, 5, 3, 0.01, 10.0, 1.0, True),
    (3, 4, 4, 0.05, 10.0, 0.0, True),
    (7, 5, 3, 0.3, 0.0, 1.0, False),
    (9, 7, 2, 0.1, 100.0, 1.0, True),
    (2, 2, 3, 0.05, 10.0, 1.0, True),
]


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.mark.parametrize("cfg", CASES)
def test_residual_parity(torch, cfg):
    nx, ny, p, mach, re, kappa, deforming = cfg
    c, v, q = case(nx, ny, p, mach, re, kappa, deforming)
    prob = oracle_problem(c, v, nx, ny, p, mach, re, kappa)
    S = solver_for(c, v, nx, ny, p, mach, re, kappa)
    out = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    S.residual(to_dev(q), out)
    err = residual_errors(to_host(out), prob.R(q), q, prob.mesh, p, prob.gas)
    assert np.all(err <= RES_TOL), err


@pytest.mark.parametrize("cfg", CASES[:4])
def test_bdf_rhs_parity(torch, cfg):
    nx, ny, p, mach, re, kappa, deforming = cfg
    c, v, q = case(nx, ny, p, mach, re, kappa, deforming)
    prob = oracle_problem(c, v, nx, ny, p, mach, re, kappa)
    qn = inp.random_perturbation(q, 21, 0.05, mach)
    qnm1 = inp.random_perturbation(q, 22, 0.05, mach)
    qcn, qcnm1 = prob.qc(qn), prob.qc(qnm1)
    dt = 0.01
    want = sv.time_rhs(prob, q, qcn, qcnm1, dt, sv.BDF2)
    S = solver_for(c, v, nx, ny, p, mach, re, kappa)
    out = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    S.bdf_rhs(to_dev(q), to_dev(qcn), to_dev(qcnm1), (1.5, -2.0, 0.5), dt, out)
    got = to_host(out)
    # the time term adds terms of size |a_i q^c_i| / dt to each equation's scale
    from oracle import scale as sc
    s = sc.residual_scale(q, prob.mesh, p, prob.gas)
    tscale = (1.5 * np.abs(prob.qc(q)) + 2.0 * np.abs(qcn) + 0.5 * np.abs(qcnm1)).max(axis=(1, 2, 3)) / dt
    err = np.abs(got - want).max(axis=(1, 2, 3))
    assert np.all(err <= RES_TOL * (s + tscale)), (err, s, tscale)
    qc = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    S.conservative(to_dev(q), qc)
    np.testing.assert_allclose(to_host(qc), prob.qc(q), rtol=1e-14, atol=0)


@pytest.mark.parametrize("cfg", CASES)
def test_jvp_parity(torch, cfg):
    nx, ny, p, mach, re, kappa, deforming = cfg
    c, v, q = case(nx, ny, p, mach, re, kappa, deforming)
    prob = oracle_problem(c, v, nx, ny, p, mach, re, kappa)
    w = inp.random_vector(q.shape, 9)
    w[0] *= prob.gas.R * 1e-2
    S = solver_for(c, v, nx, ny, p, mach, re, kappa)
    out = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    for inv_dtau, a0_dt in ((0.0, 0.0), (0.5, 150.0), (1e-20, 150.0)):
        want = sv.apply_A(prob, q, w, inv_dtau, a0_dt)
        S.jvp(to_dev(q), to_dev(w), out, inv_dtau, a0_dt)
        err = jvp_errors(to_host(out), want)
        assert np.all(err <= JVP_TOL), (inv_dtau, a0_dt, err)


@pytest.mark.parametrize("cfg", CASES)
def test_linearized_operator_matches_dual_jvp_and_oracle(torch, cfg):
    """fr_linearize + fr_apply_linear (stored local Jacobians) equals the dual-number JVP
    and the oracle's complex-step operator."""
    nx, ny, p, mach, re, kappa, deforming = cfg
    c, v, q = case(nx, ny, p, mach, re, kappa, deforming)
    prob = oracle_problem(c, v, nx, ny, p, mach, re, kappa)
    w = inp.random_vector(q.shape, 9)
    w[0] *= prob.gas.R * 1e-2
    S = solver_for(c, v, nx, ny, p, mach, re, kappa)
    qd, wd = to_dev(q), to_dev(w)
    lin = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    dual = torch.empty_like(lin)
    for inv_dtau, a0_dt in ((0.0, 0.0), (0.5, 150.0)):
        S.linearize(qd, inv_dtau, a0_dt)
        S.apply_linear(wd, lin)
        S.jvp(qd, wd, dual, inv_dtau, a0_dt)
        want = sv.apply_A(prob, q, w, inv_dtau, a0_dt)
        assert np.all(jvp_errors(to_host(lin), want) <= JVP_TOL)
        assert np.all(jvp_errors(to_host(lin), to_host(dual)) <= JVP_TOL)


@pytest.mark.parametrize("cfg", CASES)
def test_vjp_dot_product_identity(torch, cfg):
    """<w, A v> = <A^T w, v> for the GPU forward and reverse products at the same state."""
    nx, ny, p, mach, re, kappa, deforming = cfg
    c, v, q = case(nx, ny, p, mach, re, kappa, deforming)
    S = solver_for(c, v, nx, ny, p, mach, re, kappa)
    qd = to_dev(q)
    rng = np.random.default_rng(31)
    for inv_dtau, a0_dt in ((0.0, 0.0), (0.5, 150.0)):
        S.linearize(qd, inv_dtau, a0_dt)
        for _ in range(3):
            x = to_dev(rng.standard_normal(q.shape))
            y = to_dev(rng.standard_normal(q.shape))
            Ax = torch.empty_like(x)
            ATy = torch.empty_like(x)
            S.apply_linear(x, Ax)
            S.apply_linear(y, ATy, transpose=True)
            lhs = float((y * Ax).sum())
            rhs = float((ATy * x).sum())
            scale = float(y.norm() * Ax.norm())
            assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs, scale)


@pytest.mark.parametrize("cfg", [CASES[i] for i in (0, 1, 3, 6)])
def test_vjp_parity_dense_oracle(torch, cfg):
    """fr_vjp against the transpose of the oracle's dense operator (small meshes)."""
    nx, ny, p, mach, re, kappa, deforming = cfg
    if nx * ny * (p + 1) ** 2 > 200:
        nx, ny = 2, 2
    c, v, q = case(nx, ny, p, mach, re, kappa, deforming)
    prob = oracle_problem(c, v, nx, ny, p, mach, re, kappa)
    w = inp.random_vector(q.shape, 12)
    S = solver_for(c, v, nx, ny, p, mach, re, kappa)
    out = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    for inv_dtau, a0_dt in ((0.0, 0.0), (0.5, 150.0)):
        S.vjp(to_dev(q), to_dev(w), out, inv_dtau, a0_dt)
        want = sv.vjp(prob, q, w, inv_dtau, a0_dt)
        err = np.abs(to_host(out) - want).max(axis=(1, 2, 3)) / np.abs(want).max(axis=(1, 2, 3))
        assert np.all(err <= 1e-11), err


def test_autograd_residual_gradient(torch):
    """torch.autograd through the library: d<c, R(q)>/dq equals the oracle's transpose
    product, and matches the forward-mode directional derivative."""
    from paper_1903_06304_gb300 import fr
    nx, ny, p, mach, re, kappa, deforming = 3, 2, 2, 0.05, 10.0, 1.0, True
    c, v, q = case(nx, ny, p, mach, re, kappa, deforming)
    prob = oracle_problem(c, v, nx, ny, p, mach, re, kappa)
    S = solver_for(c, v, nx, ny, p, mach, re, kappa)
    cvec = inp.random_vector(q.shape, 41)
    qd = to_dev(q).requires_grad_(True)
    R = fr.residual_function().apply(qd, S)
    (R * to_dev(cvec)).sum().backward()
    got = to_host(qd.grad)
    want = -sv.vjp(prob, q, cvec, 0.0, 0.0)
    assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max()
    d = inp.random_vector(q.shape, 42)
    jv = -sv.apply_A(prob, q, d, 0.0, 0.0)
    assert abs(float((got * d).sum()) - float((cvec * jv).sum())) <= 1e-11 * np.linalg.norm(got) * np.linalg.norm(d)


def test_jvp_of_zero_vector_is_zero(torch):
    c, v, q = case(5, 4, 3, 0.05, 10.0, 1.0, True)
    S = solver_for(c, v, 5, 4, 3, 0.05, 10.0, 1.0)
    out = torch.full(S.shape, 7.0, dtype=torch.float64, device="cuda:0")
    S.jvp(to_dev(q), torch.zeros(S.shape, dtype=torch.float64, device="cuda:0"), out, 0.3, 150.0)
    assert np.all(to_host(out) == 0.0)


@pytest.mark.parametrize("cfg", [CASES[i] for i in (0, 1, 2, 3, 6)])
def test_block_parity(torch, cfg):
    """Element blocks from the stored local Jacobians (default) and by dual numbers, both
    against the oracle's coloured complex-step blocks."""
    nx, ny, p, mach, re, kappa, deforming = cfg
    c, v, q = case(nx, ny, p, mach, re, kappa, deforming)
    prob = oracle_problem(c, v, nx, ny, p, mach, re, kappa)
    inv_dtau, a0_dt = 0.5, 150.0
    want = sv.block_jacobian(prob, q, inv_dtau, a0_dt)
    got = {}
    for mode in ("linearized", "dual"):
        S = solver_for(c, v, nx, ny, p, mach, re, kappa, block_mode=mode)
        S.precond_build(to_dev(q), inv_dtau, a0_dt)
        B = torch.empty((nx * ny, S.block_size, S.block_size), dtype=torch.float64, device="cuda:0")
        S.precond_blocks(B)
        got[mode] = to_host(B)
        err = block_errors(got[mode], want, (p + 1) ** 2)
        assert np.all(err <= BLK_TOL), (mode, err)
    # the two constructions agree to rounding
    assert np.all(block_errors(got["linearized"], got["dual"], (p + 1) ** 2) <= 1e-12)


@pytest.mark.parametrize("prec,tol,accum", [("fp64", 1e-11, "df64"), ("fp32", 2e-4, "df64"),
                                            ("bf16", 1e-1, "df64"), ("fp32", 2e-4, "fp32"),
                                            ("bf16", 1e-1, "fp32")])
def test_block_apply(torch, prec, tol, accum):
    """z_e = B_e^-1 r_e against numpy's inverse of the oracle blocks; FP32/BF16 storage
    within their unit round-off times the block condition (equilibrated)."""
    nx, ny, p, mach, re, kappa, deforming = 5, 3, 2, 0.05, 10.0, 1.0, True
    c, v, q = case(nx, ny, p, mach, re, kappa, deforming)
    prob = oracle_problem(c, v, nx, ny, p, mach, re, kappa)
    Bo = sv.block_jacobian(prob, q, 0.0, 150.0)
    r = inp.random_vector(q.shape, 11)
    want = sv.block_apply(np.linalg.inv(Bo), r)
    S = solver_for(c, v, nx, ny, p, mach, re, kappa, prec=prec, apply_accum=accum)
    S.precond_build(to_dev(q), 0.0, 150.0)
    z = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    S.precond_apply(to_dev(r), z)
    got = to_host(z)
    # residual of the block system in the oracle's FP64 blocks, per element
    ne, bs = Bo.shape[0], Bo.shape[1]
    ge = got.transpose(1, 0, 2, 3).reshape(ne, bs)
    re_ = r.transpose(1, 0, 2, 3).reshape(ne, bs)
    rel = np.linalg.norm(np.einsum("eab,eb->ea", Bo, ge) - re_, axis=1) / np.linalg.norm(re_, axis=1)
    assert rel.max() <= tol, rel.max()
    if prec == "fp64":
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-3)])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_block_inverse_every_degree(torch, p, prec, tol):
    """The factorisation is compiled per degree: at every degree B_e z_e = r_e in the
    oracle's FP64 blocks, and the FP64 inverse equals numpy's."""
    nx, ny, mach, re, kappa = 3, 3, 0.05, 10.0, 1.0
    c, v, q = case(nx, ny, p, mach, re, kappa, True)
    prob = oracle_problem(c, v, nx, ny, p, mach, re, kappa)
    Bo = sv.block_jacobian(prob, q, 0.0, 150.0)
    r = inp.random_vector(q.shape, 5 + p)
    S = solver_for(c, v, nx, ny, p, mach, re, kappa, prec=prec)
    S.precond_build(to_dev(q), 0.0, 150.0)
    z = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    S.precond_apply(to_dev(r), z)
    got = to_host(z)
    ne, bs = Bo.shape[0], Bo.shape[1]
    ge = got.transpose(1, 0, 2, 3).reshape(ne, bs)
    re_ = r.transpose(1, 0, 2, 3).reshape(ne, bs)
    rel = np.linalg.norm(np.einsum("eab,eb->ea", Bo, ge) - re_, axis=1) / np.linalg.norm(re_, axis=1)
    assert rel.max() <= tol, rel.max()
    if prec == "fp64":
        want = sv.block_apply(np.linalg.inv(Bo), r)
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_block_apply_double_float_is_linear(torch, prec):
    """With FP32/BF16-stored inverses and double-float accumulation the preconditioner is a
    linear map to near FP64 rounding: z(a r1 + b r2) = a z(r1) + b z(r2) within 1e-11;
    plain FP32 accumulation is not (its deviation is of the order of FP32 round-off)."""
    nx, ny, p, mach, re, kappa, deforming = 5, 3, 3, 0.05, 10.0, 1.0, True
    c, v, q = case(nx, ny, p, mach, re, kappa, deforming)
    r1 = to_dev(inp.random_vector(q.shape, 21))
    r2 = to_dev(inp.random_vector(q.shape, 22)) * 1e-3
    dev = {}
    for accum in ("df64", "fp32"):
        S = solver_for(c, v, nx, ny, p, mach, re, kappa, prec=prec, apply_accum=accum)
        S.precond_build(to_dev(q), 0.0, 150.0)
        z1, z2, z12 = (torch.empty(S.shape, dtype=torch.float64, device="cuda:0") for _ in range(3))
        S.precond_apply(r1, z1)
        S.precond_apply(r2, z2)
        S.precond_apply(0.7 * r1 + 1.3 * r2, z12)
        lin = 0.7 * z1 + 1.3 * z2
        dev[accum] = float((z12 - lin).abs().max() / lin.abs().max())
    assert dev["df64"] <= 1e-11, dev
    assert dev["fp32"] > 100 * dev["df64"], dev


# restart <= 128: device-resident Arnoldi; restart 140: the host-Givens path; CGS2 (the
# default) and one classical pass; FP64 or double-float basis (the latter only on the
# device-resident cycle; restart 140 ignores it)
@pytest.mark.parametrize("side,restart,orthog,arith", [
    ("left", 10, "cgs2", "fp64"), ("right", 10, "cgs2", "fp64"), ("left", 40, "cgs2", "fp64"),
    ("right", 40, "cgs2", "fp64"), ("left", 140, "cgs2", "fp64"), ("left", 10, "cgs", "fp64"),
    ("right", 40, "cgs", "fp64"), ("left", 140, "cgs", "fp64"), ("left", 10, "cgs2", "df64"),
    ("right", 40, "cgs2", "df64"), ("left", 40, "cgs", "df64"), ("left", 140, "cgs2", "df64")])
def test_gmres_parity(torch, side, restart, orthog, arith):
    nx, ny, p, mach, re, kappa, deforming = 4, 4, 2, 0.05, 10.0, 1.0, True
    c, v, q = case(nx, ny, p, mach, re, kappa, deforming)
    prob = oracle_problem(c, v, nx, ny, p, mach, re, kappa)
    inv_dtau, a0_dt = 1e-20, 150.0
    b = inp.random_vector(q.shape, 13)
    Binv = np.linalg.inv(sv.block_jacobian(prob, q, inv_dtau, a0_dt))
    P = lambda x: sv.block_apply(Binv, x)
    want = sv.gmres(lambda x: sv.apply_A(prob, q, x, inv_dtau, a0_dt), b, P, restart, 1e-8, 200,
                    side=side, passes=2 if orthog == "cgs2" else 1)
    S = solver_for(c, v, nx, ny, p, mach, re, kappa, restart=restart, maxit_lin=200,
                   tol_res=1e-8, gmres_side=side, orthog=orthog, krylov_arith=arith)
    qd = to_dev(q)
    S.precond_build(qd, inv_dtau, a0_dt)
    x = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    its = S.gmres(qd, to_dev(b), x, inv_dtau, a0_dt)
    assert its == want.iterations
    got = to_host(x)
    assert np.abs(got - want.x).max() <= 1e-9 * np.abs(want.x).max()
    # and it solves the system to the tolerance, in the norm the side minimises
    res = b - sv.apply_A(prob, q, got, inv_dtau, a0_dt)
    if side == "left":
        assert np.linalg.norm(P(res)) <= 1.01e-8 * np.linalg.norm(P(b))
    else:
        assert np.linalg.norm(res) <= 1.01e-8 * np.linalg.norm(b)


def test_gmres_zero_rhs(torch):
    c, v, q = case(3, 3, 2, 0.05, 10.0, 1.0, False)
    S = solver_for(c, v, 3, 3, 2, 0.05, 10.0, 1.0)
    qd = to_dev(q)
    S.precond_build(qd, 0.0, 150.0)
    x = torch.full(S.shape, 3.0, dtype=torch.float64, device="cuda:0")
    assert S.gmres(qd, torch.zeros_like(x), x, 0.0, 150.0) == 0
    assert np.all(to_host(x) == 0.0)


@pytest.mark.parametrize("prec,arith", [("fp64", "fp64"), ("fp32", "fp64"), ("fp64", "df64")])
def test_bdf2_step_parity(torch, prec, arith):
    """One BDF2 step (BDF1 start) of the vortex: same Newton/GMRES iteration counts and
    Res_m history as the oracle, final states equal to the Newton tolerance."""
    w = inp.Workload("t", 4, 4, 2, 0.05, 10.0, 0.0, (0.0, 10.0, 0.0, 10.0), dt=0.01)
    c, v, q = inp.make_case(w)
    prob = oracle_problem(c, v, w.nx, w.ny, w.p, w.mach, w.re, w.kappa)
    qc = prob.qc(q)
    q1, st = sv.bdf2_step(prob, q, qc, qc, w.dt, coeffs=sv.BDF1, restart=30, tol_res=1e-6,
                          maxit_lin=100, tol_pseudo=1e-8, maxit_newton=10, lag=2)
    S = solver_for(c, v, w.nx, w.ny, w.p, w.mach, w.re, w.kappa, prec=prec, restart=30,
                   tol_res=1e-6, maxit_lin=100, tol_pseudo=1e-8, maxit_newton=10, lag=2,
                   krylov_arith=arith)
    qd = to_dev(q)
    qcd = to_dev(qc)
    sg = S.bdf2_step(qd, qcd, qcd, w.dt, coeffs=(1.0, -1.0, 0.0)).summary()
    assert sg["converged"] and st.converged
    res_o = np.array(st.res_history)
    res_g = np.array(sg["res_history"])
    if prec == "fp64":
        assert sg["newton_iterations"] == st.newton_iterations
        assert sg["gmres_iterations"] == st.gmres_iterations
        np.testing.assert_allclose(res_g[:2], res_o[:2], rtol=1e-9)
    else:
        assert abs(sg["newton_iterations"] - st.newton_iterations) <= 1
    got = to_host(qd)
    scale = np.abs(q1 - q).max(axis=(1, 2, 3))
    assert np.all(np.abs(got - q1).max(axis=(1, 2, 3)) <= 1e-5 * scale)


def test_ptc_parity(torch):
    """Steady PTC with SER on the Gaussian bump: Res_m and dtau histories follow the oracle."""
    w = inp.Workload("b", 4, 4, 2, 0.1, 0.0, 1.0, (0.0, 1.0, 0.0, 1.0), ic="bump", restart=20)
    c, v, q = inp.make_case(w)
    prob = oracle_problem(c, v, w.nx, w.ny, w.p, w.mach, w.re, w.kappa)
    _, st = sv.ptc_solve(prob, q, maxit_newton=12, restart=20, tol_res=1e-6, tol_pseudo=1e-8)
    S = solver_for(c, v, w.nx, w.ny, w.p, w.mach, w.re, w.kappa, restart=20, tol_res=1e-6,
                   maxit_newton=12, tol_pseudo=1e-8, lag=1)
    sg = S.ptc_solve(to_dev(q), allow_unconverged=True).summary()
    n = min(len(sg["res_history"]), len(st.res_history))
    np.testing.assert_allclose(sg["res_history"][:n], st.res_history[:n], rtol=1e-6)
    np.testing.assert_allclose(sg["dtau_history"][:n], st.dtau_history[:n], rtol=1e-5)
    assert sg["gmres_iterations"][:n - 1] == st.gmres_iterations[:n - 1]


# ------------------------------------------------------------------ full workload sizes

@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_free_stream_preserved_on_deforming_mesh(torch, p):
    """The GCL invariant at the deforming benchmark's size (128x128, M = 0.01): a uniform
    state on the moving mesh has zero residual to rounding, on the GPU as in the oracle."""
    w = inp.NS_DEFORM_128
    ref = inp.box_mesh(w.nx, w.ny, *w.box)
    c, v = inp.deform(ref, 0.13, w.motion)
    q = inp.uniform_state(w.nx * w.ny, p, w.mach, 0.8, 0.3)
    S = solver_for(c, v, w.nx, w.ny, p, w.mach, w.re, w.kappa)
    out = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    S.residual(to_dev(q), out)
    prob = oracle_problem(c, v, w.nx, w.ny, p, w.mach, w.re, w.kappa)
    from oracle import scale as sc
    sigma = sc.residual_scale(q, prob.mesh, p, prob.gas)
    err = np.abs(to_host(out)).max(axis=(1, 2, 3)) / sigma
    # the residual tolerance (rounding of the summed terms); measured <= 1.2e-13 at p = 4
    assert np.all(err <= RES_TOL), err


@pytest.mark.parametrize("w", [inp.NS_VORTEX_64, inp.NS_DEFORM_128], ids=lambda w: w.name)
def test_full_size_residual_and_jvp(torch, w):
    """At the benchmark's full sizes, in the bench's launch configuration: every residual
    and JVP entry against the oracle (vectorised, so it finishes in seconds)."""
    c, v, q = inp.make_case(w, t=0.13)
    prob = oracle_problem(c, v, w.nx, w.ny, w.p, w.mach, w.re, w.kappa)
    S = solver_for(c, v, w.nx, w.ny, w.p, w.mach, w.re, w.kappa)
    qd = to_dev(q)
    out = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    S.residual(qd, out)
    err = residual_errors(to_host(out), prob.R(q), q, prob.mesh, w.p, prob.gas)
    assert np.all(err <= RES_TOL), err
    x = inp.random_vector(q.shape, 5)
    x[0] *= prob.gas.R * 1e-2
    S.jvp(qd, to_dev(x), out, 1e-20, 1.5 / w.dt)
    err = jvp_errors(to_host(out), sv.apply_A(prob, q, x, 1e-20, 1.5 / w.dt))
    assert np.all(err <= JVP_TOL), err


@pytest.mark.parametrize("w", [inp.NS_VORTEX_64, inp.NS_DEFORM_128], ids=lambda w: w.name)
def test_full_size_blocks_sampled(torch, w):
    """Blocks at full size, sampled: for a vector supported on a set of mutually distant
    elements, the oracle's operator rows on those elements equal B_e w_e."""
    c, v, q = inp.make_case(w, t=0.13)
    prob = oracle_problem(c, v, w.nx, w.ny, w.p, w.mach, w.re, w.kappa)
    S = solver_for(c, v, w.nx, w.ny, w.p, w.mach, w.re, w.kappa)
    a0_dt = 1.5 / w.dt
    S.precond_build(to_dev(q), 1e-20, a0_dt)
    B = torch.empty((w.ne, S.block_size, S.block_size), dtype=torch.float64, device="cuda:0")
    S.precond_blocks(B)
    B = to_host(B)
    rng = np.random.default_rng(17)
    picks = [j * w.nx + i for j in range(1, w.ny, 7) for i in range(3 * (j % 2) + 1, w.nx, 7)]
    picks = rng.choice(picks, size=min(24, len(picks)), replace=False)
    x = np.zeros(q.shape)
    for e in picks:
        x[:, e] = rng.standard_normal(x[:, e].shape)
    Ax = sv.apply_A(prob, q, x, 1e-20, a0_dt)
    bs = S.block_size
    for e in picks:
        xe = x[:, e].reshape(bs)
        want = Ax[:, e].reshape(bs)
        got = B[e] @ xe
        assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max()


def test_full_size_gmres_double_float_basis(torch):
    """The benchmark's linear systems at full size (64x64 p=3 vortex, GMRES(30) capped at
    60 iterations, the regime of the BDF2 steps): with the double-float basis the solver
    takes the same iterations and returns the FP64-basis solution to 1e-8, and its true
    preconditioned residual (operator and block apply on the device) is the same."""
    w = inp.NS_VORTEX_64
    c, v, q = inp.make_case(w, t=0.13)
    inv_dtau, a0_dt = 1e-20, 1.5 / w.dt
    b = to_dev(inp.random_vector(q.shape, 23))
    qd = to_dev(q)
    out = {}
    for arith in ("fp64", "df64"):
        S = solver_for(c, v, w.nx, w.ny, w.p, w.mach, w.re, w.kappa, prec="fp32", restart=30,
                       maxit_lin=60, tol_res=1e-12, krylov_arith=arith)
        S.precond_build(qd, inv_dtau, a0_dt)
        x = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
        its = S.gmres(qd, b, x, inv_dtau, a0_dt)
        Ax = torch.empty_like(x)
        S.jvp(qd, x, Ax, inv_dtau, a0_dt)
        Pr, Pb = torch.empty_like(x), torch.empty_like(x)
        S.precond_apply(b - Ax, Pr)
        S.precond_apply(b, Pb)
        out[arith] = (its, to_host(x), float(torch.linalg.norm(Pr) / torch.linalg.norm(Pb)))
    (i64, x64, r64), (idf, xdf, rdf) = out["fp64"], out["df64"]
    assert i64 == idf == 60
    assert np.abs(xdf - x64).max() <= 1e-8 * np.abs(x64).max()
    assert abs(rdf - r64) <= 1e-6 * r64


def test_invalid_mesh_rejected(torch):
    from paper_1903_06304_gb300 import fr
    with pytest.raises(fr.FrError):
        fr.Solver(fr.Config(p=3), 1, 4)


@pytest.mark.parametrize("w", [inp.NS_VORTEX_64], ids=lambda w: w.name)
def test_full_size_vjp_sampled(torch, w):
    """The transposed operator at full size (all of the adjoint kernels' blocks), sampled:
    w is supported on mutually distant elements e_k (cyclic distance >= 5 in i or j), so the
    stencils of different e_k do not meet and, for every x, the identity
    sum over g in stencil(e_k) of (A^T w)_g . x_g = w_e_k . (A x)_e_k holds per pick, with A x
    from the oracle's complex step."""
    c, v, q = inp.make_case(w, t=0.13)
    prob = oracle_problem(c, v, w.nx, w.ny, w.p, w.mach, w.re, w.kappa)
    S = solver_for(c, v, w.nx, w.ny, w.p, w.mach, w.re, w.kappa)
    a0_dt = 1.5 / w.dt
    rng = np.random.default_rng(29)
    picks = [j * w.nx + i for j in range(2, w.ny, 9) for i in range(4 * (j % 2) + 2, w.nx, 9)]
    picks = rng.choice(picks, size=min(24, len(picks)), replace=False)
    wv = np.zeros(q.shape)
    for e in picks:
        wv[:, e] = rng.standard_normal(wv[:, e].shape)
    qd = to_dev(q)
    out = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    S.vjp(qd, to_dev(wv), out, 1e-20, a0_dt)
    ATw = to_host(out)
    left, right, bottom, top = prob.mesh.neighbours()
    for trial in range(6):
        x = rng.standard_normal(q.shape)
        x[0] *= prob.gas.R * 1e-2
        Ax = sv.apply_A(prob, q, x, 1e-20, a0_dt)
        for e in picks:
            st = {int(e), int(left[e]), int(right[e]), int(bottom[e]), int(top[e])}
            lhs = sum(float(np.sum(ATw[:, g] * x[:, g])) for g in st)
            rhs = float(np.sum(wv[:, e] * Ax[:, e]))
            scale = sum(float(np.sum(np.abs(ATw[:, g] * x[:, g]))) for g in st)
            assert abs(lhs - rhs) <= 1e-11 * scale, (trial, e, lhs, rhs)
