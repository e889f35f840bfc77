"""GMRES chunks replayed from CUDA graphs give bit-identical results, and the same launch
counts, as the same chunks launched one kernel at a time."""
import numpy as np
import pytest

from paper_1903_06304_gb300 import inputs as inp

from gpu_helpers import solver_for, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


KW = dict(restart=30, tol_res=1e-6, maxit_lin=100, tol_pseudo=1e-8, maxit_newton=10, lag=2)


def two_steps(torch, graphs, jvp_mode, side):
    w = inp.Workload("g", 6, 6, 2, 0.05, 10.0, 0.0, (0.0, 10.0, 0.0, 10.0), dt=0.01)
    c, v, q = inp.make_case(w)
    S = solver_for(c, v, w.nx, w.ny, w.p, w.mach, w.re, w.kappa, graphs=graphs,
                   jvp_mode=jvp_mode, gmres_side=side, **KW)
    qd = to_dev(q)
    qc0 = torch.empty_like(qd)
    S.conservative(qd, qc0)
    s1 = S.bdf2_step(qd, qc0, qc0, w.dt, coeffs=(1.0, -1.0, 0.0)).summary()
    qc1 = torch.empty_like(qd)
    S.conservative(qd, qc1)
    # second step: every chunk of the first is replayed from its graph
    s2 = S.bdf2_step(qd, qc1, qc0, w.dt).summary()
    return to_host(qd), s1, s2, S.kernel_launches


@pytest.mark.parametrize("jvp_mode,side", [("linearized", "left"), ("dual", "left"),
                                           ("linearized", "right")])
def test_graph_replay_is_bit_identical(torch, jvp_mode, side):
    qa, a1, a2, la = two_steps(torch, 1, jvp_mode, side)
    qb, b1, b2, lb = two_steps(torch, 0, jvp_mode, side)
    assert a1 == b1 and a2 == b2
    np.testing.assert_array_equal(qa, qb)
    assert la == lb
