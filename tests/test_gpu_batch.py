"""Batched cases (fr_batch_*): every case of a batch must give what a single-case context
gives for it, and what the oracle gives, although the batch runs each kernel once over
all cases of a group with per-case parameters and per-case reductions."""
import numpy as np
import pytest

from oracle import physics as ph
from oracle import solver as sv
from paper_1903_06304_gb300 import inputs as inp

from gpu_helpers import (RES_TOL, oracle_problem, residual_errors, solver_for, to_dev,
                         to_host)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


# (p, nx, ny, mach, re, kappa, ic): two cases share the (p=2, viscous) group, the others
# each form their own group (degree 1..3, Euler and Navier-Stokes)
MIXED = [
    (2, 6, 5, 0.1, 0.0, 1.0, "bump"),
    (3, 4, 4, 0.05, 10.0, 1.0, "vortex"),
    (2, 5, 5, 0.2, 10.0, 1.0, "vortex"),
    (1, 7, 4, 0.3, 0.0, 1.0, "bump"),
    (2, 4, 6, 0.05, 10.0, 0.0, "vortex"),
]


def case_state(spec, seed):
    p, nx, ny, mach, re, kappa, ic = spec
    w = inp.Workload("b", nx, ny, p, mach, re, kappa, (0.0, 10.0, 0.0, 10.0), ic=ic)
    c, v, q = inp.make_case(w)
    if ic == "bump":   # the bump of make_case is narrow on a coarse mesh: widen it
        x, y = inp.sample_points(c, p)
        q = inp.gaussian_bump(x, y, mach, amp=3e-3, width=2.0, xc=4.0, yc=6.0, period=10.0)
    q = inp.random_perturbation(q, seed, 1e-3, mach)
    return c, v, q


def make_batch(specs, **kw):
    from paper_1903_06304_gb300 import fr
    cases = [fr.Case(p, nx, ny, mach, re, kappa) for (p, nx, ny, mach, re, kappa, _) in specs]
    B = fr.Batch(fr.Config(**kw), cases)
    states = [case_state(s, 11 + k) for k, s in enumerate(specs)]
    corners = np.zeros((B.ne, 4, 2))
    vel = np.zeros((B.ne, 4, 2))
    q = np.zeros(B.ndof)
    for k, (c, v, qk) in enumerate(states):
        corners[B.elem_slice(k)] = c
        vel[B.elem_slice(k)] = v
        q[B.case_slice(k)] = qk.ravel()
    B.update_mesh(to_dev(corners), to_dev(vel))
    return B, states, to_dev(q)


def test_batch_layout_groups_and_offsets(torch):
    B, states, _ = make_batch(MIXED)
    assert B.num_groups == 4
    assert B.ndof == sum(qk.size for (_, _, qk) in states)
    # cases of one group are adjacent; slices tile the batch vector
    spans = sorted((B.dof_off[k], B.case_ndof[k]) for k in range(len(MIXED)))
    pos = 0
    for off, n in spans:
        assert off == pos
        pos += n
    assert pos == B.ndof
    assert abs(B.dof_off[2] + B.case_ndof[2] - B.dof_off[4]) == 0 or \
        abs(B.dof_off[4] + B.case_ndof[4] - B.dof_off[2]) == 0


def test_batch_residual_matches_single_contexts_and_oracle(torch):
    B, states, qd = make_batch(MIXED)
    R = torch.empty_like(qd)
    B.residual(qd, R)
    Rh = to_host(R)
    for k, (p, nx, ny, mach, re, kappa, _) in enumerate(MIXED):
        c, v, qk = states[k]
        S = solver_for(c, v, nx, ny, p, mach, re, kappa)
        Rs = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
        S.residual(to_dev(qk), Rs)
        got = Rh[B.case_slice(k)].reshape(qk.shape)
        # the same kernels on the same element data: identical values
        np.testing.assert_array_equal(got, to_host(Rs))
        prob = oracle_problem(c, v, nx, ny, p, mach, re, kappa)
        err = residual_errors(got, prob.R(qk), qk, prob.mesh, p, prob.gas)
        assert np.all(err <= RES_TOL), (k, err)


def test_batch_conservative_matches_single(torch):
    B, states, qd = make_batch(MIXED)
    qc = torch.empty_like(qd)
    B.conservative(qd, qc)
    qch = to_host(qc)
    for k, (p, nx, ny, mach, re, kappa, _) in enumerate(MIXED):
        c, v, qk = states[k]
        gas = ph.Gas(mach=mach, re=re, kappa=kappa)
        want = ph.conservative(qk, gas)
        got = qch[B.case_slice(k)].reshape(qk.shape)
        assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


SOLVE = dict(restart=30, tol_res=1e-6, maxit_lin=100, tol_pseudo=1e-8, maxit_newton=12, lag=2)


@pytest.mark.parametrize("prec,side,arith", [("fp64", "left", "fp64"), ("fp32", "left", "fp64"),
                                             ("fp64", "right", "fp64"), ("fp32", "left", "df64"),
                                             ("fp64", "right", "df64")])
def test_batch_bdf_step_matches_single_contexts(torch, prec, side, arith):
    """BDF1 and BDF2 steps of different dt per case: per case the same Newton and GMRES
    iteration counts and the same state as a single-case context, to rounding."""
    specs = [MIXED[1], MIXED[2], MIXED[4]]
    # GMRES capped at 8 iterations: inexact Newton steps whose convergence rate depends on
    # the case, so the cases converge after different numbers of Newton iterations and
    # converged cases sit out the remaining ones
    kw = dict(SOLVE, maxit_lin=8, maxit_newton=40, gmres_side=side, krylov_arith=arith)
    B, states, qd = make_batch(specs, prec=prec, **kw)
    qc = torch.empty_like(qd)
    B.conservative(qd, qc)
    dts = [0.01, 0.05, 0.001]
    coef = [(1.0, -1.0, 0.0, dts[0]), (1.5, -2.0, 0.5, dts[1]), (1.0, -1.0, 0.0, dts[2])]
    q0 = to_host(qd).copy()
    stats = B.bdf2_step(qd, qc, qc, coef)
    qh = to_host(qd)
    for k, (p, nx, ny, mach, re, kappa, _) in enumerate(specs):
        c, v, qk = states[k]
        S = solver_for(c, v, nx, ny, p, mach, re, kappa, prec=prec, **kw)
        qs = to_dev(qk)
        qcs = torch.empty_like(qs)
        S.conservative(qs, qcs)
        st = S.bdf2_step(qs, qcs, qcs, coef[k][3], coeffs=coef[k][:3]).summary()
        sb = stats[k].summary()
        assert sb["converged"] and st["converged"]
        assert sb["newton_iterations"] == st["newton_iterations"]
        assert sb["gmres_iterations"] == st["gmres_iterations"]
        # the per-case reductions sum in another order than the single-case ones: the
        # histories agree to rounding relative to Res_0
        np.testing.assert_allclose(sb["res_history"], st["res_history"], rtol=1e-6,
                                   atol=1e-12 * st["res_history"][0])
        got = qh[B.case_slice(k)].reshape(qk.shape)
        want = to_host(qs)
        step = np.abs(want - q0[B.case_slice(k)].reshape(qk.shape)).max(axis=(1, 2, 3))
        assert np.all(np.abs(got - want).max(axis=(1, 2, 3)) <= 1e-6 * step + 1e-300)
    counts = [s.newton_iterations for s in stats]
    assert len(set(counts)) > 1, counts


def test_batch_bdf1_step_matches_oracle(torch):
    """A batch case against the oracle's Newton loop directly."""
    specs = [MIXED[1], MIXED[2]]
    B, states, qd = make_batch(specs, **SOLVE)
    qc = torch.empty_like(qd)
    B.conservative(qd, qc)
    dt = 0.01
    stats = B.bdf2_step(qd, qc, None, [(1.0, -1.0, 0.0, dt)] * 2)
    qh = to_host(qd)
    for k, (p, nx, ny, mach, re, kappa, _) in enumerate(specs):
        c, v, qk = states[k]
        prob = oracle_problem(c, v, nx, ny, p, mach, re, kappa)
        qck = prob.qc(qk)
        q1, st = sv.bdf2_step(prob, qk, qck, qck, dt, coeffs=sv.BDF1, restart=30, tol_res=1e-6,
                              maxit_lin=100, tol_pseudo=1e-8, maxit_newton=12, lag=2)
        sb = stats[k].summary()
        assert sb["converged"] and st.converged
        assert sb["newton_iterations"] == st.newton_iterations
        assert sb["gmres_iterations"] == st.gmres_iterations
        got = qh[B.case_slice(k)].reshape(qk.shape)
        scale = np.abs(q1 - qk).max(axis=(1, 2, 3))
        assert np.all(np.abs(got - q1).max(axis=(1, 2, 3)) <= 1e-5 * scale)


def test_batch_ptc_matches_single_contexts(torch):
    specs = [MIXED[0], (2, 4, 4, 0.1, 0.0, 1.0, "bump")]
    kw = dict(restart=20, tol_res=1e-6, maxit_newton=10, tol_pseudo=1e-8, lag=1)
    B, states, qd = make_batch(specs, **kw)
    stats = B.ptc_solve(qd, allow_unconverged=True)
    for k, (p, nx, ny, mach, re, kappa, _) in enumerate(specs):
        c, v, qk = states[k]
        S = solver_for(c, v, nx, ny, p, mach, re, kappa, **kw)
        st = S.ptc_solve(to_dev(qk), allow_unconverged=True).summary()
        sb = stats[k].summary()
        assert sb["newton_iterations"] == st["newton_iterations"]
        assert sb["gmres_iterations"] == st["gmres_iterations"]
        np.testing.assert_allclose(sb["res_history"], st["res_history"], rtol=1e-6)
        np.testing.assert_allclose(sb["dtau_history"], st["dtau_history"], rtol=1e-6)


def test_batch_of_one_case_matches_single_context(torch):
    spec = MIXED[1]
    B, states, qd = make_batch([spec], **SOLVE)
    qc = torch.empty_like(qd)
    B.conservative(qd, qc)
    stats = B.bdf2_step(qd, qc, None, [(1.0, -1.0, 0.0, 0.01)])
    p, nx, ny, mach, re, kappa, _ = spec
    c, v, qk = states[0]
    S = solver_for(c, v, nx, ny, p, mach, re, kappa, **SOLVE)
    qs = to_dev(qk)
    qcs = torch.empty_like(qs)
    S.conservative(qs, qcs)
    st = S.bdf2_step(qs, qcs, qcs, 0.01, coeffs=(1.0, -1.0, 0.0)).summary()
    assert stats[0].summary()["gmres_iterations"] == st["gmres_iterations"]
