"""The fused Arnoldi step (arnoldi_fused): one launch per CGS2 (or CGS) step whose blocks
keep their part of w in shared memory and meet at bounded barriers of their case for the
step's reductions (Sec. 3.2, restarted GMRES).  It must reproduce the oracle's GMRES
(iteration counts and solution), the split passes at full size for every part size,
per case in a batch, and report a barrier wait that runs out as FR_ERR_TIMEOUT with the
context intact."""
import numpy as np
import pytest

from gpu_helpers import case, oracle_problem, solver_for, to_dev, to_host
from oracle import solver as sv
from paper_1903_06304_gb300 import inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


# 8x5 elements of p = 3: 2,560 entries = 1,280 pairs: three blocks of one pair per
# thread; forced 2 pairs per thread: two blocks
@pytest.mark.parametrize("side,restart,orthog,fused", [
    ("left", 10, "cgs2", 1), ("right", 40, "cgs2", 1), ("left", 40, "cgs", 1),
    ("right", 10, "cgs", 1), ("left", 10, "cgs2", 2)])
def test_fused_gmres_matches_oracle(torch, side, restart, orthog, fused):
    nx, ny, p, mach, re, kappa, deforming = 8, 5, 3, 0.05, 10.0, 1.0, True
    c, v, q = case(nx, ny, p, mach, re, kappa, deforming)
    prob = oracle_problem(c, v, nx, ny, p, mach, re, kappa)
    inv_dtau, a0_dt = 1e-20, 150.0
    b = inp.random_vector(q.shape, 13)
    Binv = np.linalg.inv(sv.block_jacobian(prob, q, inv_dtau, a0_dt))
    P = lambda x: sv.block_apply(Binv, x)
    want = sv.gmres(lambda x: sv.apply_A(prob, q, x, inv_dtau, a0_dt), b, P, restart, 1e-8, 200,
                    side=side, passes=2 if orthog == "cgs2" else 1)
    S = solver_for(c, v, nx, ny, p, mach, re, kappa, restart=restart, maxit_lin=200,
                   tol_res=1e-8, gmres_side=side, orthog=orthog, arnoldi_fused=fused)
    qd = to_dev(q)
    S.precond_build(qd, inv_dtau, a0_dt)
    x = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    its = S.gmres(qd, to_dev(b), x, inv_dtau, a0_dt)
    assert its == want.iterations
    got = to_host(x)
    assert np.abs(got - want.x).max() <= 1e-9 * np.abs(want.x).max()
    res = b - sv.apply_A(prob, q, got, inv_dtau, a0_dt)
    if side == "left":
        assert np.linalg.norm(P(res)) <= 1.01e-8 * np.linalg.norm(P(b))
    else:
        assert np.linalg.norm(res) <= 1.01e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("fused", [1, 2, 4])
@pytest.mark.parametrize("precond", ["block", "twolevel"])
def test_fused_full_size_equals_split_passes(torch, fused, precond):
    """The benchmark's linear systems (64x64 p = 3 vortex, GMRES(30) capped at 60
    iterations): 128 / 128 / 64 blocks of 512 threads, 2 / 2 / 4 pairs each.  The fused
    step sums in another order than the split passes: the same iterations, the solution
    to 1e-9 and the same true preconditioned residual.  The two-level preconditioner runs
    with FP64 coarse levels here: FP32 coarse sums round inputs that differ in their last
    FP64 bits to values one FP32 unit apart, which moves the solution by ~1e-8 whichever
    pass structure runs."""
    w = inp.NS_VORTEX_64
    c, v, q = inp.make_case(w, t=0.13)
    inv_dtau, a0_dt = 1e-20, 1.5 / w.dt
    b = to_dev(inp.random_vector(q.shape, 23))
    qd = to_dev(q)
    out = {}
    for mode in (0, fused):
        S = solver_for(c, v, w.nx, w.ny, w.p, w.mach, w.re, w.kappa, prec="fp32", restart=30,
                       maxit_lin=60, tol_res=1e-12, precond=precond, mg_prec="fp64",
                       arnoldi_fused=mode)
        S.precond_build(qd, inv_dtau, a0_dt)
        x = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
        its = S.gmres(qd, b, x, inv_dtau, a0_dt)
        Ax = torch.empty_like(x)
        S.jvp(qd, x, Ax, inv_dtau, a0_dt)
        Pr, Pb = torch.empty_like(x), torch.empty_like(x)
        S.precond_apply(b - Ax, Pr)
        S.precond_apply(b, Pb)
        out[mode] = (its, to_host(x), float(torch.linalg.norm(Pr) / torch.linalg.norm(Pb)))
        S.close()
    (i0, x0, r0), (i1, x1, r1) = out[0], out[fused]
    assert i0 == i1 == 60
    assert np.abs(x1 - x0).max() <= 1e-9 * np.abs(x0).max()
    assert abs(r1 - r0) <= 1e-6 * r0


def test_fused_is_deterministic(torch):
    """Fixed block table, fixed summation order: two solves give the same bits."""
    w = inp.NS_VORTEX_64
    c, v, q = inp.make_case(w, t=0.13)
    b = to_dev(inp.random_vector(q.shape, 29))
    qd = to_dev(q)
    S = solver_for(c, v, w.nx, w.ny, w.p, w.mach, w.re, w.kappa, prec="fp32", restart=30,
                   maxit_lin=40, tol_res=1e-12, arnoldi_fused=1)
    S.precond_build(qd, 1e-20, 1.5 / w.dt)
    xs = []
    for _ in range(2):
        x = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
        S.gmres(qd, b, x, 1e-20, 1.5 / w.dt)
        xs.append(to_host(x))
    assert np.array_equal(xs[0], xs[1])


def test_fused_batch_matches_single_contexts(torch):
    """Cases of different sizes and degrees in one batch: per case the fused step gives the
    Newton and GMRES counts and the state of a single-case context with the split passes."""
    from test_gpu_batch import MIXED, make_batch
    specs = [MIXED[1], MIXED[2], MIXED[4]]
    kw = dict(restart=30, tol_res=1e-6, tol_pseudo=1e-8, lag=2, maxit_lin=8, maxit_newton=40)
    B, states, qd = make_batch(specs, arnoldi_fused=1, **kw)
    qc = torch.empty_like(qd)
    B.conservative(qd, qc)
    coef = [(1.0, -1.0, 0.0, 0.01), (1.5, -2.0, 0.5, 0.05), (1.0, -1.0, 0.0, 0.001)]
    q0 = to_host(qd).copy()
    stats = B.bdf2_step(qd, qc, qc, coef)
    qh = to_host(qd)
    for k, (p, nx, ny, mach, re, kappa, _) in enumerate(specs):
        c, v, qk = states[k]
        S = solver_for(c, v, nx, ny, p, mach, re, kappa, **kw)
        qs = to_dev(qk)
        qcs = torch.empty_like(qs)
        S.conservative(qs, qcs)
        st = S.bdf2_step(qs, qcs, qcs, coef[k][3], coeffs=coef[k][:3]).summary()
        sb = stats[k].summary()
        assert sb["converged"] and st["converged"]
        assert sb["newton_iterations"] == st["newton_iterations"]
        assert sb["gmres_iterations"] == st["gmres_iterations"]
        got = qh[B.case_slice(k)].reshape(qk.shape)
        want = to_host(qs)
        step = np.abs(want - q0[B.case_slice(k)].reshape(qk.shape)).max(axis=(1, 2, 3))
        assert np.all(np.abs(got - want).max(axis=(1, 2, 3)) <= 1e-6 * step + 1e-300)
        S.close()
    B.close()


def test_a_barrier_wait_that_runs_out_returns_timeout(torch):
    """A barrier of the fused step that cannot complete (one arrival injected on the host,
    so that one block of the 16x12 p = 3 case's 12 waits for an arrival that never comes):
    its wait runs out of its budget, the solve returns FR_ERR_TIMEOUT at the end of its
    first chunk, the counters are reset and the same context then solves the system as
    a fresh context with the split passes does."""
    from paper_1903_06304_gb300 import fr
    nx, ny, p, mach = 16, 12, 3, 0.05
    ref = inp.box_mesh(nx, ny, 0.0, 10.0, 0.0, 10.0)
    x, y = inp.sample_points(ref, p)
    vx = inp.Vortex(mach=mach, alpha=2.0, x0=4.0, y0=5.0, period_x=10.0, period_y=10.0)
    q = inp.vortex_state(x, y, 0.0, vx)
    b = to_dev(inp.random_vector(q.shape, 31))
    qd = to_dev(q)
    S = solver_for(ref, np.zeros_like(ref), nx, ny, p, mach, 10.0, 1.0, arnoldi_fused=1,
                   wait_spins=200000, tol_res=1e-10, maxit_lin=30)
    S.precond_build(qd, 1e-20, 150.0)
    xs = torch.empty_like(qd)
    S.inject_barrier_offset(1)
    with pytest.raises(fr.FrError) as ex:
        S.gmres(qd, b, xs, 1e-20, 150.0)
    assert ex.value.code == -5   # FR_ERR_TIMEOUT
    R = torch.empty_like(qd)
    S.residual(qd, R)
    assert bool(torch.isfinite(R).all())
    its = {1: S.gmres(qd, b, xs, 1e-20, 150.0)}
    x1 = to_host(xs)
    S2 = solver_for(ref, np.zeros_like(ref), nx, ny, p, mach, 10.0, 1.0, arnoldi_fused=0,
                    tol_res=1e-10, maxit_lin=30)
    S2.precond_build(qd, 1e-20, 150.0)
    x2 = torch.empty_like(qd)
    its[0] = S2.gmres(qd, b, x2, 1e-20, 150.0)
    assert its[0] == its[1]
    assert np.abs(x1 - to_host(x2)).max() <= 1e-9 * np.abs(to_host(x2)).max()
    S2.close()
    S.close()
