"""Pins of the oracle's error norms (Sec. 4) and of the scales the parity tolerances are
stated in, against closed forms worked out by hand and an independent quadrature."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import physics as ph
from oracle import residual as rs
from oracle import scale as sc
from oracle import solver as sv
from paper_1903_06304_gb300 import inputs as inp

GAMMA = 1.4


def _problem(nx, ny, p, mach, box=(0.0, 10.0, 0.0, 10.0), deforming=False, re=0.0, kappa=1.0):
    ref = inp.box_mesh(nx, ny, *box)
    c, v = inp.deform(ref, 0.2, inp.Motion()) if deforming else (ref, np.zeros_like(ref))
    return sv.Problem(rs.Mesh(nx, ny, c, v), p, ph.Gas(mach=mach, re=re, kappa=kappa)), c


@pytest.mark.parametrize("deforming", [False, True])
def test_entropy_error_vanishes_for_the_isentropic_vortex(deforming):
    """The vortex of Eq. VP_Solution is isentropic: p / rho^gamma equals the free stream's
    at every point, so E_s is zero up to rounding."""
    w = inp.Workload("v", 6, 6, 3, 0.05, 0.0, 0.0, ic="vortex", deforming=deforming)
    c, v, q = inp.make_case(w, t=0.2)
    prob = sv.Problem(rs.Mesh(6, 6, c, v), 3, ph.Gas(mach=0.05, re=0.0, kappa=0.0))
    assert sv.entropy_error(prob, q) <= 1e-14


@pytest.mark.parametrize("delta", [1e-3, -0.02, 0.3])
def test_entropy_error_of_a_uniform_pressure_offset(delta):
    """T = 1 and p = p_inf (1 + delta) everywhere: rho = 1 + delta, so
    p / rho^gamma = p_inf (1 + delta)^(1 - gamma) at every point and
    E_s = |(1 + delta)^(1 - gamma) - 1| whatever the quadrature."""
    mach = 0.1
    prob, _ = _problem(3, 2, 2, mach, deforming=True)
    q = inp.uniform_state(6, 2, mach)
    q[0] *= 1.0 + delta
    want = abs((1.0 + delta) ** (1.0 - GAMMA) - 1.0)
    assert sv.entropy_error(prob, q) == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("deforming", [False, True])
def test_entropy_error_of_a_linear_pressure_field_matches_quadrature(deforming):
    """p = p_inf (1 + 0.4 x / 10), T = 1 on [0,10]^2 (the deformation keeps the boundary
    fixed): E_s^2 = (1/10) int_0^10 ((1 + 0.04 x)^(1 - gamma) - 1)^2 dx, evaluated by
    adaptive quadrature; the oracle's Gauss rule with |J| weights agrees to its accuracy."""
    mach, p = 0.05, 4
    prob, c = _problem(6, 5, p, mach, deforming=deforming)
    x, _y = inp.sample_points(c, p)
    q = inp.uniform_state(30, p, mach)
    q[0] = inp.p_inf(mach) * (1.0 + 0.04 * x)
    f = lambda t: ((1.0 + 0.04 * t) ** (1.0 - GAMMA) - 1.0) ** 2
    want = math.sqrt(integrate.quad(f, 0.0, 10.0, epsabs=0, epsrel=1e-13)[0] / 10.0)
    assert sv.entropy_error(prob, q) == pytest.approx(want, rel=1e-8)


def test_residual_scale_of_a_uniform_stream_by_hand():
    """Uniform Euler stream (p_inf, 1, 0, 1) on a static Cartesian mesh with hx = 2, hy = 1
    and kappa = 1/M (so eps = 1 and Gamma = M).  By hand:
    flux part 2|f_k|/hx + 2|g_k|/hy with f = (rho u, rho u^2 + p, 0, u (E + p)),
    g = (0, 0, p, 0), rho = 1, E = p/(gamma-1) + 1/2;
    dissipation part max(|S_xi| (|u| + c), |S_eta| c) (|M| |q|)_k / |J| with
    |S_xi| = hy/2, |S_eta| = hx/2, |J| = hx hy/4, c = 1/M and
    |M||q| = (2 rho, 3 rho |u|, 0, p/(gamma-1) + 2 rho) from the Jacobian of
    (rho, rho u, rho v, E) with respect to (p, u, v, T)."""
    mach = 0.2
    hx, hy = 2.0, 1.0
    prob, _ = _problem(4, 3, 2, mach, box=(0.0, 8.0, 0.0, 3.0), kappa=1.0 / mach)
    q = inp.uniform_state(12, 2, mach)
    pinf = inp.p_inf(mach)
    E = pinf / (GAMMA - 1.0) + 0.5
    f = np.array([1.0, 1.0 + pinf, 0.0, E + pinf])
    g = np.array([0.0, 0.0, pinf, 0.0])
    flux = 2.0 * np.abs(f) / hx + 2.0 * np.abs(g) / hy
    c = 1.0 / mach
    mq = np.array([2.0, 3.0, 0.0, pinf / (GAMMA - 1.0) + 2.0])
    diss = max(hy / 2 * (1.0 + c), hx / 2 * c) * mq / (hx * hy / 4)
    got = sc.residual_scale(q, prob.mesh, 2, prob.gas)
    np.testing.assert_allclose(got, flux + diss, rtol=1e-13)


def test_flux_derivative_scale_of_a_linear_pressure_field():
    """At rest (u = v = 0, T = 1) with p = p_inf + a x on a static Cartesian mesh, the only
    non-zero flux is the x-momentum flux F = (hy/2) p, so (d F/d xi) / |J| = dp/dx = a
    exactly in every element (the interpolant derivative is exact on linear data and acts
    within the element), and every other equation's flux derivatives vanish."""
    mach, a = 0.1, 0.37
    prob, c = _problem(3, 3, 3, mach, box=(0.0, 6.0, 0.0, 3.0))
    x, _y = inp.sample_points(c, 3)
    q = inp.uniform_state(9, 3, mach, u=0.0)
    q[0] = inp.p_inf(mach) + a * x
    s = sc.flux_derivative_scale(q, prob.mesh, 3, prob.gas)
    np.testing.assert_allclose(s, [0.0, a, 0.0, 0.0], rtol=1e-12, atol=1e-12 * a)
    d = sc.divergence_scale(q, prob.mesh, 3, prob.gas)
    np.testing.assert_array_equal(d, np.maximum(s, np.abs(prob.R(q)).max(axis=(1, 2, 3))))
