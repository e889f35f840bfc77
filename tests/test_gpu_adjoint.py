"""The discrete adjoint of the BDF2 march on the device (Sec. 3.2 march; Sec. 4 forces;
Sec. 4.4 plunge): its building blocks against the oracle (the wall force's state
gradient, the transposed conservative map and its Mach derivative, the parameter
directional derivatives of R and F, the transposed GMRES solve), then the whole reverse
sweep for d(mean thrust)/d(plunge amplitude, Mach) against the oracle's adjoint on the
oracle's states, and against central differences of the device's own march."""
import math

import numpy as np
import pytest

from oracle import adjoint as ad
from oracle import physics as ph
from oracle import residual as rs
from oracle import solver as sv
from paper_1903_06304_gb300 import inputs as inp

from gpu_helpers import to_dev, to_host

pytestmark = pytest.mark.gpu

NI, NJ, P, MACH, H, RE, K_RED = 6, 2, 1, 0.2, 0.25, 50.0, 2.0
EPS = 1e-30


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def plunge_case(q0, nsteps=3):
    ref = inp.naca_ogrid(NI, NJ, first=0.05)
    return ad.PlungeCase(ref, NI, NJ, P, re=RE, kappa=1.0, k=K_RED, t0=0.3, dt=0.05, nsteps=nsteps, q0=q0)


def solver(mach=MACH, **kw):
    from paper_1903_06304_gb300 import fr
    cfg = dict(p=P, mach=mach, re=RE, kappa=1.0, restart=40, maxit_lin=400, tol_res=1e-13,
               tol_pseudo=1e-13, maxit_newton=30)
    cfg.update(kw)
    return fr.Solver(fr.Config(**cfg), NI, NJ, bc=("wall", "farfield"), q_inf=inp.far_field_state(mach))


def mesh_at(case, t, h):
    """Corners and velocities of the plunging grid at t for amplitude h, and their
    derivatives in h (the unit-amplitude motion)."""
    c1, v1 = inp.plunge(case.ref, t, 1.0, case.k)
    return case.ref + h * (c1 - case.ref), h * v1, c1 - case.ref, v1


def dqinf_dmach(mach):
    return (-2.0 / (inp.GAMMA * mach ** 3), 0.0, 0.0, 0.0)


def perturbed_state(seed=5, rel=0.02, mach=MACH):
    return inp.random_perturbation(inp.uniform_state(NI * NJ, P, mach), seed, rel, mach)


def test_wall_force_vjp_matches_complex_step(torch):
    case = plunge_case(None)
    q = perturbed_state()
    prob = ad.problem(case, 0.4, H, MACH)
    S = solver()
    c, v, _, _ = mesh_at(case, 0.4, H)
    S.update_mesh(to_dev(c), to_dev(v))
    wx, wy = -0.7, 1.3
    want = np.zeros(q.size)
    for k in range(q.size):
        e = np.zeros(q.size, dtype=complex)
        e[k] = 1j * EPS
        Fx, Fy = rs.wall_force(q + e.reshape(q.shape), prob.mesh, P, prob.gas, prob.basis, prob.geo)
        want[k] = (wx * np.imag(Fx) + wy * np.imag(Fy)) / EPS
    want = want.reshape(q.shape)
    qd = to_dev(q)
    out = torch.empty_like(qd)
    S.wall_force_vjp(qd, wx, wy, out)
    assert np.abs(to_host(out) - want).max() <= 1e-12 * np.abs(want).max()
    # accumulate form: out = beta out + alpha g
    prev = to_dev(inp.random_vector(q.shape, 3))
    acc = prev.clone()
    S.wall_force_vjp(qd, wx, wy, acc, alpha=-2.0, beta=0.5)
    ref = 0.5 * to_host(prev) - 2.0 * want
    assert np.abs(to_host(acc) - ref).max() <= 1e-12 * np.abs(ref).max()


def test_conservative_vjp_and_mach_derivative(torch):
    q = perturbed_state(rel=0.05)
    case = plunge_case(None)
    prob = ad.problem(case, 0.4, H, MACH)
    S = solver()
    w = inp.random_vector(q.shape, 8)
    Mq = prob.point_matrices(q)[1]
    want = np.einsum("ij...,i...->j...", Mq, w)
    qd, wd = to_dev(q), to_dev(w)
    out = torch.empty_like(qd)
    S.conservative_vjp(qd, wd, out)
    assert np.abs(to_host(out) - want).max() <= 1e-13 * np.abs(want).max()
    prev = to_dev(inp.random_vector(q.shape, 4))
    acc = prev.clone()
    S.conservative_vjp(qd, wd, acc, alpha=3.0, beta=-1.0)
    ref = -to_host(prev) + 3.0 * want
    assert np.abs(to_host(acc) - ref).max() <= 1e-13 * np.abs(ref).max()
    # w . dq^c/dM at fixed q by a complex step of the gas
    gas_c = ph.Gas(mach=MACH + 1j * EPS, re=RE, kappa=1.0)
    dqc = np.imag(np.stack(ph.conservative(tuple(q[k] for k in range(4)), gas_c))) / EPS
    got = S.conservative_dmach(qd, wd)
    assert abs(got - np.sum(w * dqc)) <= 1e-12 * np.sum(np.abs(w * dqc))


@pytest.mark.parametrize("which", ["h", "mach"])
def test_param_jvp_matches_complex_step(torch, which):
    """w . R' and F' along the plunge amplitude (corners and corner velocities move with h)
    and along the Mach number (gas constants and the far-field pressure) at a fixed state."""
    case = plunge_case(None)
    q = perturbed_state(rel=0.05)
    t = 0.45
    dh = 1j * EPS if which == "h" else 0.0
    dm = 1j * EPS if which == "mach" else 0.0
    prob_c = ad.problem(case, t, H + dh, MACH + dm)
    w = inp.random_vector(q.shape, 9)
    Rc = prob_c.R(q)
    want_wR = float(np.sum(w * np.imag(Rc))) / EPS
    Fc = rs.wall_force(q, prob_c.mesh, P, prob_c.gas, prob_c.basis, prob_c.geo)
    want_F = np.array([np.imag(Fc[0]), np.imag(Fc[1])]) / EPS
    S = solver()
    c, v, dc, dv = mesh_at(case, t, H)
    cd, vd = to_dev(c), to_dev(v)
    S.update_mesh(cd, vd)
    if which == "h":
        wR, F = S.param_jvp(to_dev(q), cd, vd, dcorners=to_dev(dc), dvel=to_dev(dv), w=to_dev(w), force=True)
    else:
        wR, F = S.param_jvp(to_dev(q), cd, vd, dmach=1.0, dqinf=dqinf_dmach(MACH), w=to_dev(w), force=True)
    scale = float(np.sum(np.abs(w * np.real(Rc))))
    assert abs(wR - want_wR) <= 1e-11 * max(abs(want_wR), 1e-3 * scale), (wR, want_wR)
    # the far-field pressure's share of the force, p_inf times the closed wall's sum of
    # n ds, vanishes up to rounding: its tangent along M is rounding on the scale of
    # |dp_inf/dM| times the perimeter (about 2 chords)
    fscale = max(np.abs(want_F).max(), 2.0 * inp.p_inf(MACH) / MACH * 2.0 * 1e-3)
    assert np.all(np.abs(np.array(F) - want_F) <= 1e-11 * fscale), (F, want_F)


@pytest.mark.parametrize("precond", ["block", "twolevel"])
@pytest.mark.parametrize("side", ["left", "right"])
def test_adjoint_solve_matches_dense_transpose(torch, side, precond):
    case = plunge_case(None)
    q = perturbed_state(rel=0.05)
    prob = ad.problem(case, 0.4, H, MACH)
    a0_dt = 1.5 / 0.05
    A = sv.dense_operator(prob, q, 0.0, a0_dt)
    g = inp.random_vector(q.shape, 10)
    want = np.linalg.solve(A.T, g.ravel()).reshape(q.shape)
    S = solver(gmres_side=side, precond=precond, mg_prec="fp64")
    c, v, _, _ = mesh_at(case, 0.4, H)
    S.update_mesh(to_dev(c), to_dev(v))
    lam = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    its = S.adjoint_solve(to_dev(q), to_dev(g), lam, 0.0, a0_dt)
    assert 0 < its < 400
    assert np.abs(to_host(lam) - want).max() <= 1e-9 * np.abs(want).max()


def gpu_reverse_sweep(torch, S, case, qs, h, mach):
    """dJ/dh, dJ/dM of J = (1/K) sum_n -2 F_x(q^n) by the device adjoint, given the states
    q^0 .. q^K (device tensors): the sweep of the adjoint's header in include/fr.h."""
    K, dt = case.nsteps, case.dt
    wx = -2.0 / K
    lam = [None] * (K + 3)
    grad = np.zeros(2)
    dq_inf = dqinf_dmach(mach)
    its = []
    for n in range(K, 0, -1):
        t = case.time(n)
        c, v, dc, dv = mesh_at(case, t, h)
        cd, vd = to_dev(c), to_dev(v)
        S.update_mesh(cd, vd)
        a0 = case.coeffs(n)[0]
        # A^T lam = dJ/dq - sum_k (a_k^{n+k}/dt) Mq(q^n)^T lam^{n+k}   (dG/dq = -A)
        g = torch.empty_like(qs[n])
        S.wall_force_vjp(qs[n], wx, 0.0, g)
        for m, kk in ((n + 1, 1), (n + 2, 2)):
            if m <= K:
                a = case.coeffs(m)[kk]
                if a != 0.0:
                    S.conservative_vjp(qs[n], lam[m], g, alpha=-a / dt, beta=1.0)
        lam[n] = torch.empty_like(g)
        its.append(S.adjoint_solve(qs[n], g, lam[n], 0.0, a0 / dt))
        # lam . dG/dtheta + dJ/dtheta at fixed states
        wRh, Fh = S.param_jvp(qs[n], cd, vd, dcorners=to_dev(dc), dvel=to_dev(dv), w=lam[n], force=True)
        wRm, Fm = S.param_jvp(qs[n], cd, vd, dmach=1.0, dqinf=dq_inf, w=lam[n], force=True)
        grad[0] += wRh + wx * Fh[0]
        grad[1] += wRm + wx * Fm[0]
        coeffs = case.coeffs(n)
        for k, a in enumerate(coeffs):
            if a != 0.0:
                grad[1] -= a / dt * S.conservative_dmach(qs[n - k], lam[n])
    return grad, its


@pytest.mark.parametrize("precond", ["block", "twolevel"])
def test_adjoint_sweep_matches_oracle_adjoint(torch, precond):
    """On the oracle's converged states, the device sweep reproduces the oracle's
    d(mean C_t)/dh and d(mean C_t)/dM, with the transposed element blocks or the
    transposed two-level preconditioner in the adjoint solves."""
    q0 = inp.random_perturbation(inp.uniform_state(NI * NJ, P, MACH), 3, 0.01, MACH)
    case = plunge_case(q0)
    J, gh, gm = ad.adjoint_gradient(case, H, MACH)
    qs = [to_dev(x) for x in ad.march(case, H, MACH)]
    S = solver(precond=precond, mg_prec="fp64")
    grad, its = gpu_reverse_sweep(torch, S, case, qs, H, MACH)
    assert all(i > 0 for i in its)
    assert abs(grad[0] - gh) <= 1e-9 * abs(gh), (grad[0], gh)
    assert abs(grad[1] - gm) <= 1e-9 * abs(gm), (grad[1], gm)


def gpu_march(torch, S, case, h, mach):
    """States q^0 .. q^K of the device's BDF1-then-BDF2 march and J."""
    from paper_1903_06304_gb300 import fr
    q = to_dev(case.q0)
    qc0 = torch.empty_like(q)
    S.update_mesh(*[to_dev(a) for a in mesh_at(case, case.time(0), h)[:2]])
    S.conservative(q, qc0)
    qn, qm = qc0.clone(), qc0.clone()
    qs, J = [q.clone()], 0.0
    for n in range(1, case.nsteps + 1):
        c, v, _, _ = mesh_at(case, case.time(n), h)
        S.update_mesh(to_dev(c), to_dev(v))
        S.bdf2_step(q, qn, qm, case.dt, coeffs=fr.BDF1 if n == 1 else fr.BDF2, allow_unconverged=True)
        qm.copy_(qn)
        S.conservative(q, qn)
        qs.append(q.clone())
        J += -2.0 * S.wall_force(q)[0] / case.nsteps
    return qs, J


def test_adjoint_sweep_matches_finite_differences_of_the_device_march(torch):
    q0 = inp.random_perturbation(inp.uniform_state(NI * NJ, P, MACH), 3, 0.01, MACH)
    case = plunge_case(q0)
    S = solver()
    qs, J = gpu_march(torch, S, case, H, MACH)
    grad, _ = gpu_reverse_sweep(torch, S, case, qs, H, MACH)
    eh, em = 1e-5, 1e-6
    jh = [gpu_march(torch, S, case, H + s * eh, MACH)[1] for s in (1, -1)]
    jm = []
    for s in (1, -1):
        Sm = solver(mach=MACH + s * em)
        jm.append(gpu_march(torch, Sm, case, H, MACH + s * em)[1])
        Sm.close()
    fh = (jh[0] - jh[1]) / (2 * eh)
    fm = (jm[0] - jm[1]) / (2 * em)
    assert abs(grad[0] - fh) <= 1e-6 * abs(fh), (grad[0], fh)
    assert abs(grad[1] - fm) <= 1e-6 * abs(fm), (grad[1], fm)
