"""Failure detection without a GPU fault: non-finite values written into a state on the
host are reported by the Newton loops as FR_ERR_NONFINITE (single cases), and a batch
reports the failing case while every other case still advances exactly as it would
alone."""
import numpy as np
import pytest

from gpu_helpers import solver_for, to_dev, to_host
from paper_1903_06304_gb300 import inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _vortex(nx, ny, p, mach, alpha=2.0):
    ref = inp.box_mesh(nx, ny, 0.0, 10.0, 0.0, 10.0)
    x, y = inp.sample_points(ref, p)
    vx = inp.Vortex(mach=mach, alpha=alpha, x0=4.0, y0=5.0, period_x=10.0, period_y=10.0)
    return ref, inp.vortex_state(x, y, 0.0, vx)


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_single_case_reports_a_non_finite_state(torch, bad):
    from paper_1903_06304_gb300 import fr
    nx, ny, p, mach = 6, 5, 2, 0.1
    c, q = _vortex(nx, ny, p, mach)
    S = solver_for(c, np.zeros_like(c), nx, ny, p, mach, 10.0, 1.0)
    q = q.copy()
    q[1, 7, 1, 2] = bad
    qd = to_dev(q)
    qc = torch.empty_like(qd)
    S.conservative(to_dev(np.nan_to_num(q, nan=1.0, posinf=1.0)), qc)
    with pytest.raises(fr.FrError) as ex:
        S.bdf2_step(qd, qc, qc, 0.01, coeffs=fr.BDF1)
    assert ex.value.code == -3
    S.close()


def test_batch_isolates_the_non_finite_case(torch):
    from paper_1903_06304_gb300 import fr
    p, dt = 2, 0.01
    specs = [(6, 5, 0.1), (7, 4, 0.05), (5, 5, 0.2)]
    cases, states, corners = [], [], []
    for nx, ny, m in specs:
        c, q = _vortex(nx, ny, p, m)
        cases.append(fr.Case(p, nx, ny, m, 10.0, 1.0))
        states.append(q)
        corners.append(c)
    B = fr.Batch(fr.Config(), cases)
    cor = np.zeros((B.ne, 4, 2))
    qb = np.zeros(B.ndof)
    for k in range(len(cases)):
        cor[B.elem_slice(k)] = corners[k]
        qb[B.case_slice(k)] = states[k].ravel()
    B.update_mesh(to_dev(cor), to_dev(np.zeros_like(cor)))
    qd = to_dev(qb)
    qc = torch.empty_like(qd)
    B.conservative(qd, qc)
    # a NaN written on the host into case 1's state after its history was formed
    bad = qb.copy()
    bad[B.case_slice(1).start + 11] = float("nan")
    qd.copy_(to_dev(bad))
    sts = B.bdf2_step(qd, qc, qc, [(1.0, -1.0, 0.0, dt)] * 3, allow_nonfinite=True)
    assert B.last_rc == -3
    assert not sts[1].converged
    got = to_host(qd)
    for k in (0, 2):
        nx, ny, m = specs[k]
        S = solver_for(corners[k], np.zeros_like(corners[k]), nx, ny, p, m, 10.0, 1.0)
        q1 = to_dev(states[k])
        qc1 = torch.empty_like(q1)
        S.conservative(q1, qc1)
        st = S.bdf2_step(q1, qc1, qc1, dt, coeffs=fr.BDF1).summary()
        assert sts[k].converged and st["converged"]
        assert sts[k].newton_iterations == st["newton_iterations"]
        assert np.all(np.isfinite(got[B.case_slice(k)]))
        dq = np.abs(to_host(q1) - states[k]).max()
        assert np.abs(got[B.case_slice(k)] - to_host(q1).ravel()).max() <= 1e-9 * dq
        S.close()
    B.close()


@pytest.mark.parametrize("precond", ["block", "twolevel"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_bulk_copy_apply_equals_one_block_per_element(torch, precond, prec):
    """The persistent block apply fed by bulk copies (apply_bulk = 3) computes the same
    arithmetic as the one-block-per-element kernel: equal bit for bit."""
    nx, ny, p, mach = 9, 7, 3, 0.05
    c, q = _vortex(nx, ny, p, mach)
    r = inp.random_vector(q.shape, 17)
    out = []
    for bulk in (3, 0):
        S = solver_for(c, np.zeros_like(c), nx, ny, p, mach, 10.0, 1.0, precond=precond,
                       prec=prec, apply_bulk=bulk)
        qd = to_dev(q)
        S.precond_build(qd, 1e-20, 150.0)
        z = torch.empty_like(qd)
        S.precond_apply(to_dev(r), z)
        out.append(to_host(z))
        S.close()
    assert np.array_equal(out[0], out[1])


def test_a_device_wait_that_runs_out_returns_timeout(torch):
    """A bounded device wait (the bulk copies of the block apply) given no budget: the
    call returns FR_ERR_TIMEOUT after the blocks have waited for their copies, and the
    context keeps working."""
    from paper_1903_06304_gb300 import fr
    nx, ny, p, mach = 16, 12, 3, 0.05
    c, q = _vortex(nx, ny, p, mach)
    S = solver_for(c, np.zeros_like(c), nx, ny, p, mach, 10.0, 1.0, apply_bulk=2, wait_spins=-1)
    qd = to_dev(q)
    S.precond_build(qd, 1e-20, 150.0)
    r = to_dev(inp.random_vector(q.shape, 18))
    z = torch.empty_like(qd)
    with pytest.raises(fr.FrError) as ex:
        S.precond_apply(r, z)
    assert ex.value.code == -5   # FR_ERR_TIMEOUT
    # the context is intact: the residual, and the same apply with a budget, still run
    R = torch.empty_like(qd)
    S.residual(qd, R)
    assert bool(torch.isfinite(R).all())
    S2 = solver_for(c, np.zeros_like(c), nx, ny, p, mach, 10.0, 1.0)
    S2.precond_build(qd, 1e-20, 150.0)
    z2 = torch.empty_like(qd)
    S2.precond_apply(r, z2)
    assert bool(torch.isfinite(z2).all())
