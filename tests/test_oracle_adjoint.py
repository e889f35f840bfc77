"""Pins of the oracle's discrete adjoint of the BDF2 march (Sec. 3.2) for the mean thrust
coefficient of a plunging NACA 0012 (Secs. 4, 4.4): the reverse sweep equals the forward
linearised march (the same Jacobians applied in the opposite order, so a wrong
transposition, coefficient or time index breaks the equality), both equal central finite
differences of the whole nonlinear march, and the plunge's mirror symmetry holds: for a
symmetric body and a symmetric initial stream J(h) = J(-h), so dJ/dh is odd in h and
dJ/dM even."""
import numpy as np
import pytest

from oracle import adjoint as ad
from paper_1903_06304_gb300 import inputs as inp

NI, NJ, P, MACH, H = 6, 2, 1, 0.2, 0.25


def _case(q0):
    ref = inp.naca_ogrid(NI, NJ, first=0.05)
    return ad.PlungeCase(ref, NI, NJ, P, re=50.0, kappa=1.0, k=2.0, t0=0.3, dt=0.05, nsteps=3, q0=q0)


@pytest.fixture(scope="module")
def perturbed():
    q0 = inp.random_perturbation(inp.uniform_state(NI * NJ, P, MACH), 3, 0.01, MACH)
    case = _case(q0)
    return case, ad.adjoint_gradient(case, H, MACH)


def test_adjoint_equals_tangent_march(perturbed):
    case, (J, gh, gm) = perturbed
    th, tm = ad.tangent_gradient(case, H, MACH)
    assert abs(gh - th) <= 1e-9 * abs(th) and abs(gm - tm) <= 1e-9 * abs(tm), (gh, th, gm, tm)


def test_adjoint_matches_finite_differences_of_the_march(perturbed):
    case, (J, gh, gm) = perturbed
    eh, em = 1e-5, 1e-6
    jh = [ad.objective(case, ad.march(case, H + s * eh, MACH), H + s * eh, MACH) for s in (1, -1)]
    jm = [ad.objective(case, ad.march(case, H, MACH + s * em), H, MACH + s * em) for s in (1, -1)]
    fh = (jh[0] - jh[1]) / (2 * eh)
    fm = (jm[0] - jm[1]) / (2 * em)
    assert abs(gh - fh) <= 1e-6 * abs(fh) and abs(gm - fm) <= 1e-6 * abs(fm), (gh, fh, gm, fm)
    assert abs(J - ad.objective(case, ad.march(case, H, MACH), H, MACH)) <= 1e-12 * abs(J)


def test_mirror_symmetry_of_the_plunge_sensitivities():
    case = _case(inp.uniform_state(NI * NJ, P, MACH))
    J1, h1, m1 = ad.adjoint_gradient(case, H, MACH)
    J2, h2, m2 = ad.adjoint_gradient(case, -H, MACH)
    assert abs(J1 - J2) <= 1e-12 * abs(J1)
    assert abs(h1 + h2) <= 1e-10 * abs(h1) and abs(h1) > 1e-4
    assert abs(m1 - m2) <= 1e-10 * abs(m1)
