"""Pins of the oracle's parameter sensitivities (w . dR/dM_inf, w . dR/dcorners,
w . dR/dvel): central finite differences of the real residual, translation invariance of
R, and free-stream preservation (R = 0 for a uniform state on any moving mesh, so every
sensitivity vanishes there)."""
import dataclasses

import numpy as np
import pytest

from oracle import physics as ph
from oracle import residual as rs
from oracle import solver as sv
from paper_1903_06304_gb300 import inputs as inp


def problem(nx, ny, p, mach, re, kappa, seed=5, deforming=True, uniform=False):
    ref = inp.box_mesh(nx, ny, 0, 10, 0, 10)
    c, v = inp.deform(ref, 0.13, inp.Motion()) if deforming else (ref, np.zeros_like(ref))
    q = inp.uniform_state(nx * ny, p, mach, 0.8, 0.3)
    if not uniform:
        q = inp.random_perturbation(q, seed, 0.05, mach)
    prob = sv.Problem(rs.Mesh(nx, ny, c, v), p, ph.Gas(mach=mach, re=re, kappa=kappa))
    w = inp.random_vector(q.shape, seed + 1)
    return prob, q, w


def wR(prob, q, w, mach=None, corners=None, vel=None):
    m = prob.mesh
    gas = prob.gas if mach is None else dataclasses.replace(prob.gas, mach=mach)
    mesh = rs.Mesh(m.nx, m.ny, m.corners if corners is None else corners,
                   m.vel if vel is None else vel)
    return float(np.sum(w * sv.Problem(mesh, prob.p, gas).R(q)))


@pytest.mark.parametrize("re", [0.0, 10.0])
def test_param_vjp_matches_central_differences(re):
    prob, q, w = problem(3, 3, 2, 0.2, re, 1.0)
    dm, dc, dv = sv.param_vjp(prob, q, w)
    M = prob.gas.mach
    h = 1e-6 * M
    fd = (wR(prob, q, w, mach=M + h) - wR(prob, q, w, mach=M - h)) / (2 * h)
    assert abs(dm - fd) <= 1e-6 * abs(dm)
    rng = np.random.default_rng(0)
    for _ in range(4):
        e, a, c = int(rng.integers(9)), int(rng.integers(4)), int(rng.integers(2))
        for which, d in (("corners", dc), ("vel", dv)):
            base = getattr(prob.mesh, which)
            hp = 1e-6
            up, dn = base.copy(), base.copy()
            up[e, a, c] += hp
            dn[e, a, c] -= hp
            fd = (wR(prob, q, w, **{which: up}) - wR(prob, q, w, **{which: dn})) / (2 * hp)
            assert abs(d[e, a, c] - fd) <= 1e-6 * np.abs(d).max(), (which, e, a, c)


def test_corner_sensitivities_sum_to_zero_under_translation():
    """Translating every corner by the same vector leaves R unchanged, so the corner
    sensitivities of each coordinate sum to zero."""
    prob, q, w = problem(3, 4, 2, 0.1, 10.0, 1.0)
    _, dc, _ = sv.param_vjp(prob, q, w)
    scale = np.abs(dc).max()
    assert abs(dc[:, :, 0].sum()) <= 1e-11 * scale * dc[:, :, 0].size
    assert abs(dc[:, :, 1].sum()) <= 1e-11 * scale * dc[:, :, 1].size


def node_sums(d, nx, ny):
    """Sum the per-element corner copies of each mesh node (periodic box numbering:
    element (i, j) = j nx + i, corners counter-clockwise from (i, j))."""
    out = np.zeros((ny, nx, 2))
    for e in range(nx * ny):
        i, j = e % nx, e // nx
        for a, (di, dj) in enumerate(((0, 0), (1, 0), (1, 1), (0, 1))):
            out[(j + dj) % ny, (i + di) % nx] += d[e, a]
    return out


def test_free_stream_sensitivities_vanish():
    """A uniform state is an exact discrete steady solution on any conforming moving mesh
    (GCL term), for any Mach number: the Mach sensitivity and every node sensitivity (all
    element copies of a node moved together) vanish.  Moving one element's copy alone
    makes the mesh non-conforming, so single copies need not vanish."""
    nx, ny = 3, 3
    prob, q, w = problem(nx, ny, 2, 0.1, 10.0, 1.0, uniform=True)
    dm, dc, dv = sv.param_vjp(prob, q, w)
    prob2, q2, _ = problem(nx, ny, 2, 0.1, 10.0, 1.0)
    _, dc2, dv2 = sv.param_vjp(prob2, q2, w)
    for d, d2 in ((dc, dc2), (dv, dv2)):
        ref = np.abs(node_sums(d2, nx, ny)).max()
        assert np.abs(node_sums(d, nx, ny)).max() <= 1e-10 * ref
        assert np.abs(d).max() > 1e-3 * np.abs(d2).max()   # the copies themselves do not
    assert abs(dm) <= 1e-10 * np.abs(w).sum()
