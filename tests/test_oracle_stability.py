"""Linear stability of the oracle's semi-discrete viscous operator (Sec. 3.1's FR/CPR
discretisation with BR2 viscous terms): about a uniform stream on a periodic box of 4 x 4
elements of the 64 x 64 vortex workload's size (h = 10/64, M = 0.05, Re 10 per unit
length), every eigenvalue of M^-1 dR/dq^p (M = dq^c/dq^p) has a real part <= 0 at p = 3
and 4, so no discrete mode grows.  The same operator with the BR2 face penalty 1 has a
mode growing at about 135 (p = 3) and 580 (p = 4) per unit time, the rate at which the
vortex was seen to leave its advected solution with that penalty: the pin fails for the
penalty that fails."""
import numpy as np
import pytest

from gpu_helpers import oracle_problem
from oracle import physics as ph
from oracle import residual as rs
from oracle import solver as sv
from paper_1903_06304_gb300 import inputs as inp


def _growth_rate(n_el: int = 4, p: int = 3, mach: float = 0.05) -> tuple[float, float]:
    """(max Re, min Re) of the eigenvalues of M^-1 dR/dq^p at a uniform stream."""
    L = 10.0 / 64 * n_el
    c = inp.box_mesh(n_el, n_el, 0.0, L, 0.0, L)
    prob = oracle_problem(c, np.zeros_like(c), n_el, n_el, p, mach, 10.0, 0.0)
    q = inp.uniform_state(n_el * n_el, p, mach, u=0.5 ** 0.5, v=0.5 ** 0.5)
    n = q.size
    J = np.empty((n, n))
    for k in range(n):
        x = np.zeros(n)
        x[k] = 1.0
        # A x = -dR/dq x with no pseudo-time and no physical-time term
        J[:, k] = -sv.apply_A(prob, q, x.reshape(q.shape), 0.0, 0.0).ravel()
    Mp = ph.M_matrix(tuple(q[k] for k in range(4)), prob.gas)
    npts = n // 4
    Mb = np.array([[np.broadcast_to(Mp[a][b], q[0].shape).ravel() for b in range(4)] for a in range(4)])
    Minv = np.zeros((n, n))
    for i in range(npts):
        Mi = np.linalg.inv(Mb[:, :, i])
        Minv[np.ix_(np.arange(4) * npts + i, np.arange(4) * npts + i)] = Mi
    lam = np.linalg.eigvals(Minv @ J)
    return float(lam.real.max()), float(lam.real.min())


@pytest.mark.parametrize("p", [3, 4])
def test_viscous_operator_has_no_growing_mode(p):
    hi, lo = _growth_rate(p=p)
    # the spectrum spans |Re| up to ~1.5e5; rounding leaves the conserved modes near 0
    assert hi <= 1e-8 * abs(lo), (hi, lo)


@pytest.mark.parametrize("p", [3, 4])
def test_penalty_one_has_a_growing_mode(monkeypatch, p):
    monkeypatch.setattr(rs, "BR2_PENALTY", 1.0)
    hi, lo = _growth_rate(p=p)
    assert hi > 50.0, (hi, lo)
