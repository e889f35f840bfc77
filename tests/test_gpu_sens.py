"""Parameter sensitivities on the GPU (fr_param_vjp) against the oracle's complex step:
w . dR/dM_inf, w . dR/d(corner coordinates), w . dR/d(corner velocities)."""
import dataclasses

import numpy as np
import pytest

from oracle import solver as sv
from paper_1903_06304_gb300 import inputs as inp

from gpu_helpers import case, oracle_problem, solver_for, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


# (nx, ny, p, mach, re, kappa, deforming): colour classes 3x3 (multiples of 3), 4x5
# (remainder columns and rows), 2x4 (left and right neighbour are the same element)
CASES = [
    (3, 3, 2, 0.2, 0.0, 1.0, True),
    (4, 5, 3, 0.1, 10.0, 1.0, True),
    (2, 4, 1, 0.3, 10.0, 1.0, True),
    (6, 3, 2, 0.05, 10.0, 1.0, False),
]


@pytest.mark.parametrize("cfg", CASES, ids=lambda c: f"{c[0]}x{c[1]}p{c[2]}")
def test_param_vjp_matches_oracle(torch, cfg):
    nx, ny, p, mach, re, kappa, deforming = cfg
    c, v, q = case(nx, ny, p, mach, re, kappa, deforming, rel=0.05)
    w = inp.random_vector(q.shape, 9)
    prob = oracle_problem(c, v, nx, ny, p, mach, re, kappa)
    dm_o, dc_o, dv_o = sv.param_vjp(prob, q, w)
    S = solver_for(c, v, nx, ny, p, mach, re, kappa)
    dc = torch.full((nx * ny, 4, 2), np.nan, dtype=torch.float64, device="cuda:0")
    dv = torch.full_like(dc, np.nan)
    dm = S.param_vjp(to_dev(q), to_dev(w), to_dev(c), to_dev(v), dc, dv)
    # scale of the Mach sum: sum |w_i dR_i/dM| (the terms that may cancel)
    h = sv.COMPLEX_STEP
    gas_c = dataclasses.replace(prob.gas, mach=mach + 1j * h)
    dRdM = np.imag(sv.Problem(prob.mesh, p, gas_c).R(q)) / h
    assert abs(dm - dm_o) <= 1e-11 * np.abs(w * dRdM).sum()
    for got, want in ((to_host(dc), dc_o), (to_host(dv), dv_o)):
        assert np.isfinite(got).all()
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max(), np.abs(got - want).max()


def test_autograd_parameter_gradients(torch):
    """torch.autograd through the residual: gradients w.r.t. q, corners, velocities and
    Mach equal the library's VJP and parameter sensitivities."""
    from paper_1903_06304_gb300 import fr
    nx, ny, p, mach, re, kappa, deforming = CASES[1]
    c, v, q = case(nx, ny, p, mach, re, kappa, deforming, rel=0.05)
    w = to_dev(inp.random_vector(q.shape, 9))
    S = solver_for(c, v, nx, ny, p, mach, re, kappa)
    qd = to_dev(q).requires_grad_(True)
    cd = to_dev(c).requires_grad_(True)
    vd = to_dev(v).requires_grad_(True)
    md = torch.tensor(mach, dtype=torch.float64, device="cuda:0", requires_grad=True)
    R = fr.residual_function().apply(qd, S, cd, vd, md)
    (R * w).sum().backward()
    prob = oracle_problem(c, v, nx, ny, p, mach, re, kappa)
    dm_o, dc_o, dv_o = sv.param_vjp(prob, q, to_host(w))
    assert np.abs(to_host(cd.grad) - dc_o).max() <= 1e-10 * np.abs(dc_o).max()
    assert np.abs(to_host(vd.grad) - dv_o).max() <= 1e-10 * np.abs(dv_o).max()
    gas_c = dataclasses.replace(prob.gas, mach=mach + 1j * sv.COMPLEX_STEP)
    dRdM = np.imag(sv.Problem(prob.mesh, p, gas_c).R(q)) / sv.COMPLEX_STEP
    assert abs(float(md.grad) - dm_o) <= 1e-11 * np.abs(to_host(w) * dRdM).sum()
    # dR/dq^T w against the transpose of the oracle's complex-step operator (A = -dR/dq
    # with no pseudo-time or BDF terms)
    want = -sv.vjp(prob, q, to_host(w), 0.0, 0.0)
    got = to_host(qd.grad)
    assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max()
