"""Pins of the oracle's pointwise physics (Secs. 2.1-2.3, 3.1) against closed forms,
numerically computed Jacobians/eigenvalues and special cases."""
import numpy as np
import pytest

from oracle import physics as ph

H = 1e-30


def _state(seed, mach):
    rng = np.random.default_rng(seed)
    p = ph.Gas(mach=mach).R * (1 + 0.1 * rng.uniform(-1, 1))
    u, v = rng.uniform(-1, 1, 2)
    T = 1 + 0.2 * rng.uniform(-1, 1)
    rho = p / (ph.Gas(mach=mach).R * T)
    return np.array([rho * ph.Gas(mach=mach).R * T, u, v, T])


def _cs_jac(fun, x):
    """Jacobian by complex steps (independent of any closed form)."""
    n = len(x)
    cols = []
    for k in range(n):
        e = np.zeros(n, dtype=complex)
        e[k] = 1j * H
        cols.append(np.imag(np.asarray(fun(x + e))) / H)
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("mach", [0.01, 0.1, 0.5])
@pytest.mark.parametrize("seed", range(4))
def test_M_is_jacobian_of_conservative_map(mach, seed):
    gas = ph.Gas(mach=mach)
    q = _state(seed, mach)
    J = _cs_jac(lambda s: ph.conservative(tuple(s), gas), q)
    M = ph.M_matrix(tuple(q), gas)
    # entry (4,4) = rho_T h + rho C_p cancels terms of size rho C_p ~ 1/M^2: the
    # absolute tolerance is relative to that term size.
    term = ph.density(tuple(q), gas) * gas.cp
    np.testing.assert_allclose(M, J, rtol=1e-13, atol=1e-14 * term)


@pytest.mark.parametrize("mach", [0.01, 0.05, 0.3])
@pytest.mark.parametrize("seed", range(4))
def test_preconditioned_eigenvalues(mach, seed):
    """eig(Gamma^-1 A_n,mov) = {u_n, u_n, u'_n + c', u'_n - c'} (Eqs. eigenvalues(_para), A_n,mov)."""
    rng = np.random.default_rng(100 + seed)
    gas = ph.Gas(mach=mach, kappa=1.0)
    q = _state(seed, mach)
    ang = rng.uniform(0, 2 * np.pi)
    n = np.array([np.cos(ang), np.sin(ang)])
    vg = rng.uniform(-0.5, 0.5, 2)
    An = _cs_jac(lambda s: ph.normal_inviscid_flux(tuple(s), n, vg, gas), q)
    eps = ph.epsilon(tuple(q), vg, gas)
    G = ph.Gamma_matrix(tuple(q), eps, gas)
    ev = np.sort(np.linalg.eigvals(np.linalg.solve(G, An)).real)
    ref = np.sort(np.array(ph.eigenvalues(tuple(q), n, vg, eps, gas)))
    np.testing.assert_allclose(ev, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("mach", [0.01, 0.2])
def test_beta_is_inverse_sound_speed_squared(mach):
    gas = ph.Gas(mach=mach)
    q = _state(1, mach)
    rp, rT = ph.rho_p_rho_T(tuple(q), gas)
    rho = ph.density(tuple(q), gas)
    beta = rp + rT / (rho * gas.cp)
    c = ph.sound_speed(tuple(q), gas)
    assert abs(beta * c * c - 1) < 1e-13


def test_eps_one_recovers_unpreconditioned_system():
    """eps = 1: Gamma = M, alpha = 0, c' = c, eigenvalues u_n, u_n, u_n +- c."""
    gas = ph.Gas(mach=0.3)
    q = _state(2, 0.3)
    G = ph.Gamma_matrix(tuple(q), 1.0, gas)
    M = ph.M_matrix(tuple(q), gas)
    np.testing.assert_allclose(G, M, rtol=1e-13, atol=1e-13)
    n = np.array([0.6, 0.8])
    lam = ph.eigenvalues(tuple(q), n, np.zeros(2), 1.0, gas)
    un = q[1] * n[0] + q[2] * n[1]
    c = ph.sound_speed(tuple(q), gas)
    np.testing.assert_allclose(lam, [un, un, un + c, un - c], rtol=1e-13, atol=1e-13)


def test_epsilon_cutoffs():
    gas = ph.Gas(mach=0.05, kappa=1.0)
    c = 1 / 0.05
    T = 1.0
    p = gas.R
    # slow flow: eps = kappa M_inf
    assert abs(ph.epsilon((p, 0.1, 0.0, T), np.zeros(2), gas) - 0.05) < 1e-15
    # fast flow: eps = M
    assert abs(ph.epsilon((p, 3.0, 4.0, T), np.zeros(2), gas) - 5.0 / c) < 1e-15
    # supersonic: eps = 1
    assert ph.epsilon((p, 30.0, 0.0, T), np.zeros(2), gas) == 1.0
    # moving grid: M_mov from v - v_g
    assert abs(ph.epsilon((p, 3.0, 4.0, T), np.array([3.0, 4.0 - 2.0]), gas) - 0.1) < 1e-15


@pytest.mark.parametrize("mach", [0.01, 0.1])
def test_rusanov_consistency_and_conservation(mach):
    gas = ph.Gas(mach=mach, kappa=1.0)
    a, b = _state(3, mach), _state(4, mach)
    n = np.array([0.28, 0.96])
    vg = np.array([0.1, -0.3])
    f_same = ph.rusanov(tuple(a), tuple(a), n, vg, gas)
    np.testing.assert_allclose(f_same, ph.normal_inviscid_flux(tuple(a), n, vg, gas), rtol=1e-14)
    f1 = ph.rusanov(tuple(a), tuple(b), n, vg, gas)
    f2 = ph.rusanov(tuple(b), tuple(a), -n, vg, gas)
    np.testing.assert_allclose(f1, -f2, rtol=1e-13, atol=1e-10)


def test_rusanov_scalar_like_upwinding_at_eps_one():
    """At eps = 1 (Gamma = M) the dissipation is |lambda|max (q^c+ - q^c-) to first order."""
    gas = ph.Gas(mach=0.5, kappa=10.0)   # kappa*M >= 1 -> eps = 1
    a = _state(5, 0.5)
    da = np.array([1e-7 * gas.R, 1e-7, -2e-7, 1e-7])
    n = np.array([1.0, 0.0])
    f = ph.rusanov(tuple(a), tuple(a + da), n, np.zeros(2), gas)
    fm = ph.normal_inviscid_flux(tuple(a), n, np.zeros(2), gas)
    fp = ph.normal_inviscid_flux(tuple(a + da), n, np.zeros(2), gas)
    qm = ph.conservative(tuple(a), gas)
    qp = ph.conservative(tuple(a + da), gas)
    c = ph.sound_speed(tuple(a + 0.5 * da), gas)
    lmax = abs(a[1] + 0.5 * da[1]) + c
    ref = 0.5 * (fm + fp) - 0.5 * lmax * (qp - qm)
    np.testing.assert_allclose(f, ref, rtol=1e-9, atol=1e-12 * np.abs(fm).max())


def test_viscous_flux_special_fields():
    gas = ph.Gas(mach=0.1, re=50.0)
    q = (gas.R, 0.3, -0.2, 1.0)
    zero = (0.0, 0.0, 0.0, 0.0)
    # rigid rotation u = -y, v = x: no stress, no heat flux
    fv, gv = ph.viscous_flux(q, (0.0, 0.0, 1.0, 0.0), (0.0, -1.0, 0.0, 0.0), gas)
    np.testing.assert_allclose(fv, 0.0, atol=1e-15)
    np.testing.assert_allclose(gv, 0.0, atol=1e-15)
    # simple shear u = y: tau_xy = mu, energy flux u tau_xy in g, v tau_xy in f
    fv, gv = ph.viscous_flux(q, zero, (0.0, 1.0, 0.0, 0.0), gas)
    np.testing.assert_allclose(fv, np.array([0, 0, 1, -0.2]) / 50.0, atol=1e-15)
    np.testing.assert_allclose(gv, np.array([0, 1, 0, 0.3]) / 50.0, atol=1e-15)
    # pure heat conduction: k dT/dx with k = mu C_p / Pr
    fv, gv = ph.viscous_flux(q, (0.0, 0.0, 0.0, 2.0), zero, gas)
    k = 1.0 / ((1.4 - 1) * 0.01) / 0.72
    np.testing.assert_allclose(fv, np.array([0, 0, 0, 2 * k]) / 50.0, rtol=1e-14)
    # uniaxial strain u = x: tau_xx = 4/3 mu, tau_yy = -2/3 mu
    fv, gv = ph.viscous_flux(q, (0.0, 1.0, 0.0, 0.0), zero, gas)
    np.testing.assert_allclose(fv[1], 4 / 3 / 50.0, rtol=1e-14)
    np.testing.assert_allclose(gv[2], -2 / 3 / 50.0, rtol=1e-14)
