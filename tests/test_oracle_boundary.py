"""Pins of the oracle's boundary faces (Sec. 3.3: far field q_b = q_inf through the
approximate Riemann solver, adiabatic no-slip wall moving with the grid), the NACA 0012
O-grid of Sec. 4.2 and the rigid plunge of Sec. 4.4, and the wall force of Sec. 4's
force coefficients, against what the mathematics fixes: free-stream preservation with
far-field faces on a moving O-grid, consistency with the exact flux divergence of a
manufactured field that satisfies the wall and far-field conditions, discrete
conservation up to the boundary fluxes, exact forces for linear pressure and shear
fields, and exact complex-step derivatives through the boundary code."""
import math

import numpy as np
import pytest

from oracle import physics as ph
from oracle import residual as rs
from oracle import scale as sc
from oracle import solver as sv
from oracle.basis import make_basis
from oracle.geometry import element_geometry
from paper_1903_06304_gb300 import inputs as inp


# ------------------------------------------------------------------ the O-grid

def _polygon_area(x, y):
    """Enclosed area of a closed polygon (shoelace; the wall runs clockwise)."""
    return abs(0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


def test_naca_ogrid_geometry():
    ni, nj, r_far, first = 128, 32, 20.0, 1e-3
    c = inp.naca_ogrid(ni, nj, r_far, first)
    wall = c[:ni, 0]                                   # corner 0 of row 0: the wall nodes
    # closed trailing edge at (1, 0); wall nodes on the thickness law, lower side first
    assert np.allclose(wall[0], (1.0, 0.0), atol=1e-15)
    yt = inp.naca0012_half_thickness(wall[:, 0])
    assert np.allclose(np.abs(wall[:, 1]), yt, atol=1e-15)
    assert np.all(wall[1:ni // 2, 1] < 0) and np.all(wall[ni // 2 + 1:, 1] > 0)
    # the far-field nodes lie on the circle of r_far chords about the mid-chord
    far = c[(nj - 1) * ni:, 3]
    assert np.allclose(np.hypot(far[:, 0] - 0.5, far[:, 1]), r_far, rtol=1e-14)
    # first cell: `first` of the wall-to-far-field distance at the mid-chord column
    col = ni // 4
    d0 = np.hypot(*(c[col, 3] - c[col, 0]))
    dall = np.hypot(*(c[(nj - 1) * ni + col, 3] - c[col, 0]))
    assert abs(d0 / dall * r_far - first) <= 1e-6 * first
    # the blended chordwise distribution: every wall spacing in x is at least the uniform
    # part's 2 blend / ni (cosine clustering alone gives (pi/ni)^2 at the edges)
    blend = 0.5
    dx = np.abs(np.diff(np.append(wall[:, 0], wall[0, 0])))
    assert dx.min() >= 2 * blend / ni * (1 - 1e-12) and dx.min() < 1.1 * 2 * blend / ni
    cc = inp.naca_ogrid(ni, nj, r_far, first, blend=0.0)[:ni, 0]
    assert np.abs(np.diff(cc[:, 0])).min() < (math.pi / ni) ** 2 * 1.01
    # positive Jacobian at every solution and flux point (p = 3)
    geo = element_geometry(c, np.zeros_like(c), make_basis(3))
    assert geo.sol.J.min() > 0 and min(f.J.min() for f in geo.faces) > 0
    # the wall polygon's area converges to the closed-form area of the profile,
    # 2 * 0.6 * (0.2969 * 2/3 - 0.1260/2 - 0.3516/3 + 0.2843/4 - 0.1036/5)
    exact = 1.2 * (0.2969 * 2 / 3 - 0.1260 / 2 - 0.3516 / 3 + 0.2843 / 4 - 0.1036 / 5)
    errs = []
    for n in (64, 128, 256):
        w = inp.naca_ogrid(n, 4, blend=0.0)[:n, 0]
        errs.append(abs(_polygon_area(w[:, 0], w[:, 1]) - exact) / exact)
    assert errs[-1] < 2e-4 and errs[0] / errs[-1] > 12, errs   # second order in 1/ni


def test_plunge_is_rigid_translation():
    ref = inp.naca_ogrid(16, 4)
    h, k, t = 0.25, 1.0, 0.7
    c, v = inp.plunge(ref, t, h, k)
    f = k / (2 * math.pi)
    assert np.allclose(c[..., 0], ref[..., 0]) and np.allclose(c[..., 1] - ref[..., 1],
                                                                 h * math.sin(2 * math.pi * f * t))
    assert np.all(v[..., 0] == 0.0)
    # the velocity is the time derivative of the position
    dt = 1e-6
    cp, _ = inp.plunge(ref, t + dt, h, k)
    cm, _ = inp.plunge(ref, t - dt, h, k)
    assert np.allclose((cp - cm) / (2 * dt), v, atol=1e-9)


# ------------------------------------------------------------------ free stream

@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("re", [0.0, 100.0])
def test_free_stream_preserved_with_far_field_on_plunging_ogrid(p, re):
    """q = q_inf everywhere is a discrete steady state of the moving O-grid with far-field
    faces on both sides: uniform flux (GCL) and boundary states equal to the trace."""
    ref = inp.naca_ogrid(24, 6)
    c, v = inp.plunge(ref, 0.3)
    mach = 0.1
    gas = ph.Gas(mach=mach, re=re, kappa=1.0)
    m = rs.Mesh(24, 6, c, v, bc=(rs.FARFIELD, rs.FARFIELD), q_inf=inp.far_field_state(mach))
    q = inp.uniform_state(m.ne, p, mach)
    R = rs.residual(q, m, p, gas)
    s = sc.residual_scale(q, m, p, gas)
    assert np.all(np.abs(R).max(axis=(1, 2, 3)) <= 1e-12 * s)


def test_far_field_state_differing_from_trace_is_felt():
    """A far-field state other than the interior state changes only the boundary row."""
    mach = 0.1
    gas = ph.Gas(mach=mach, re=100.0, kappa=1.0)
    c = inp.naca_ogrid(16, 5)
    q = inp.uniform_state(16 * 5, 2, mach)
    qi = (inp.p_inf(mach), 1.0, 0.05, 1.0)
    m = rs.Mesh(16, 5, c, np.zeros_like(c), bc=(rs.FARFIELD, rs.FARFIELD), q_inf=qi)
    R = rs.residual(q, m, 2, gas)
    row = np.arange(m.ne) // 16
    inner = (row > 0) & (row < 4)
    s = sc.residual_scale(q, m, 2, gas)
    assert np.all(np.abs(R[:, inner]).max(axis=(1, 2, 3)) <= 1e-12 * s)
    assert np.abs(R[:, row == 0]).max() > 1e-6 * s.max()


# ------------------------------------------------------------------ manufactured consistency

sp = pytest.importorskip("sympy")
L_BOX = 10.0
U_INF = 0.8


def _channel_manufactured(gas_v, wall_heat=0.0):
    """Smooth field on the channel [0,10] x [0,10] (periodic in x) with u = v = 0 and
    dT/dy = wall_heat * pi/10 on the wall y = 0 (adiabatic when 0) and
    q = (p_inf, U_INF, 0, 1) on the far field y = 10."""
    x, y = sp.symbols("x y", real=True)
    k = 2 * sp.pi / L_BOX
    a = sp.pi / L_BOX
    P = gas_v.R * (1 + 0.02 * sp.sin(k * x + 0.3) * (1 + sp.cos(a * y)))
    U = U_INF * sp.sin(a * y / 2) + 0.05 * sp.sin(a * y) * sp.cos(k * x)
    V = 0.1 * sp.sin(a * y) * sp.sin(k * x)
    T = 1 + 0.02 * sp.cos(k * x) * (1 + sp.cos(a * y)) + wall_heat * sp.sin(a * y)
    q = (P, U, V, T)
    qx = tuple(sp.diff(e, x) for e in q)
    qy = tuple(sp.diff(e, y) for e in q)
    fi, gi = ph.inviscid_flux(q, gas_v)
    fv, gv = ph.viscous_flux(q, qx, qy, gas_v)
    qc = ph.conservative(q, gas_v)
    lam = lambda e: sp.lambdify((x, y), e, "numpy")
    return dict(q=[lam(e) for e in q],
                div_inv=[lam(sp.diff(fi[i], x) + sp.diff(gi[i], y)) for i in range(4)],
                div_vis=[lam(sp.diff(fv[i], x) + sp.diff(gv[i], y)) for i in range(4)],
                qcx=[lam(sp.diff(qc[i], x)) for i in range(4)],
                qcy=[lam(sp.diff(qc[i], y)) for i in range(4)])


def _ev(f, X):
    return np.broadcast_to(f(*X), X[0].shape)


def _channel(N, t):
    ref = inp.box_mesh(N, N, 0.0, L_BOX, 0.0, L_BOX)
    return inp.deform(ref, t, inp.Motion())     # boundary nodes stay on y = 0 and y = 10


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("part", ["inviscid", "viscous", "grid"])
def test_wall_and_far_field_consistency_order(p, part):
    """With a wall below row 0 and a far field above the last row, the residual minus its
    exact continuous counterpart converges everywhere, boundary elements included, at the
    orders of the periodic case: inviscid ~p, viscous ~p-1, grid-velocity ~p."""
    gas_v = ph.Gas(mach=0.2, re=20.0, kappa=1.0)
    gas_i = ph.Gas(mach=0.2, re=0.0, kappa=1.0)
    ex = _channel_manufactured(gas_v)
    qi = (gas_v.R, U_INF, 0.0, 1.0)
    bc = dict(bc=(rs.WALL, rs.FARFIELD), q_inf=qi)
    errs = []
    for N in (8, 16, 32):
        c, v = _channel(N, 0.13)
        X = inp.sample_points(c, p)
        Vg = inp.sample_points(v, p)
        qh = np.stack([_ev(f, X) for f in ex["q"]])
        if part == "inviscid":
            got = rs.residual(qh, rs.Mesh(N, N, c, np.zeros_like(v), **bc), p, gas_i)
            want = np.stack([-_ev(f, X) for f in ex["div_inv"]])
        elif part == "viscous":
            m = rs.Mesh(N, N, c, v, **bc)
            got = rs.residual(qh, m, p, gas_v) - rs.residual(qh, m, p, gas_i)
            want = np.stack([_ev(f, X) for f in ex["div_vis"]])
        else:
            got = (rs.residual(qh, rs.Mesh(N, N, c, v, **bc), p, gas_i)
                   - rs.residual(qh, rs.Mesh(N, N, c, np.zeros_like(v), **bc), p, gas_i))
            want = np.stack([Vg[0] * ex["qcx"][i](*X) + Vg[1] * ex["qcy"][i](*X) for i in range(4)])
        scale = np.abs(want).max(axis=(1, 2, 3))
        keep = scale > 0
        errs.append(np.abs(got - want).max(axis=(1, 2, 3))[keep] / scale[keep])
    errs = np.array(errs)
    order = np.log2(errs[-2] / errs[-1])
    need = {"inviscid": p - 0.5, "viscous": p - 1.5, "grid": p - 0.5}[part]
    assert np.all(order >= need), (order, errs)
    assert np.all(errs[-1] < 0.25)


@pytest.mark.parametrize("part", ["inviscid", "viscous"])
def test_wrong_wall_state_is_inconsistent(part):
    """The consistency above depends on the wall: the same field with the wall replaced by
    a far field at q_inf (a wrong boundary state below row 0) does not converge there."""
    gas = ph.Gas(mach=0.2, re=20.0 if part == "viscous" else 0.0, kappa=1.0)
    gas_v = ph.Gas(mach=0.2, re=20.0, kappa=1.0)
    ex = _channel_manufactured(gas_v)
    qi = (gas_v.R, U_INF, 0.0, 1.0)
    errs = []
    for N in (8, 16):
        c, _ = _channel(N, 0.13)
        X = inp.sample_points(c, 2)
        qh = np.stack([_ev(f, X) for f in ex["q"]])
        m = rs.Mesh(N, N, c, np.zeros_like(c), bc=(rs.FARFIELD, rs.FARFIELD), q_inf=qi)
        got = rs.residual(qh, m, 2, gas)
        want = np.stack([-_ev(f, X) for f in ex["div_inv"]])
        if part == "viscous":
            want = want + np.stack([_ev(f, X) for f in ex["div_vis"]])
        scale = np.abs(want).max(axis=(1, 2, 3))
        errs.append(np.abs(got - want)[1:3].max() / scale[1:3].max())
    assert errs[-1] > 0.5 * errs[0], errs


def test_adiabatic_wall_rejects_wall_heat_flux():
    """A field with dT/dn != 0 at the wall is not consistent with the adiabatic wall: the
    energy row of the wall elements keeps an O(1) error under refinement, while the same
    field is consistent in the interior rows."""
    gas_v = ph.Gas(mach=0.2, re=20.0, kappa=1.0)
    gas_i = ph.Gas(mach=0.2, re=0.0, kappa=1.0)
    ex = _channel_manufactured(gas_v, wall_heat=0.05)
    qi = (gas_v.R, U_INF, 0.0, 1.0)
    wall_err, inner_err = [], []
    for N in (8, 16, 32):
        c, _ = _channel(N, 0.13)
        m = rs.Mesh(N, N, c, np.zeros_like(c), bc=(rs.WALL, rs.FARFIELD), q_inf=qi)
        X = inp.sample_points(c, 2)
        qh = np.stack([_ev(f, X) for f in ex["q"]])
        got = rs.residual(qh, m, 2, gas_v) - rs.residual(qh, m, 2, gas_i)
        want = _ev(ex["div_vis"][3], X)
        err = np.abs(got[3] - want) / np.abs(want).max()
        row = np.arange(m.ne) // N
        wall_err.append(err[row == 0].max())
        inner_err.append(err[(row >= N // 4) & (row < 3 * N // 4)].max())
    assert wall_err[-1] > 0.5 * wall_err[0], wall_err
    assert inner_err[-1] < 0.3 * inner_err[0], inner_err     # viscous part: order p - 1


@pytest.mark.parametrize("re", [0.0, 30.0])
def test_stream_along_walls_moving_with_it_is_preserved(re):
    """u = (0.6, 0) everywhere, with the whole channel (walls included) sliding at the same
    velocity: the wall state (p^-, v_g, T^-) equals the trace, so R = 0 to rounding."""
    N, p, mach = 5, 3, 0.1
    c, _ = _channel(N, 0.21)
    vel = np.zeros_like(c)
    vel[..., 0] = 0.6
    gas = ph.Gas(mach=mach, re=re, kappa=1.0)
    m = rs.Mesh(N, N, c, vel, bc=(rs.WALL, rs.WALL))
    q = inp.uniform_state(m.ne, p, mach, 0.6, 0.0)
    R = rs.residual(q, m, p, gas)
    s = sc.residual_scale(q, m, p, gas)
    assert np.all(np.abs(R).max(axis=(1, 2, 3)) <= 1e-12 * s)
    # a stream that does not move with the walls is not a steady state at the walls
    m2 = rs.Mesh(N, N, c, np.zeros_like(c), bc=(rs.WALL, rs.WALL))
    R2 = rs.residual(q, m2, p, gas)
    assert np.abs(R2[:, :N]).max() > 1e-6 * s.max()


# ------------------------------------------------------------------ conservation

@pytest.mark.parametrize("re", [0.0, 10.0])
def test_discrete_conservation_up_to_boundary_fluxes(re):
    """On a static mesh, sum_e sum_ij w_i w_j |J| R = -(sum of the fluxes leaving through
    the far-field faces - the fluxes entering through the wall faces): interior and
    periodic faces telescope, boundary faces do not."""
    c, _ = _channel(6, 0.21)
    mach = 0.05
    gas = ph.Gas(mach=mach, re=re, kappa=1.0)
    qi = inp.far_field_state(mach, 0.8, 0.1)
    m = rs.Mesh(6, 6, c, np.zeros_like(c), bc=(rs.WALL, rs.FARFIELD), q_inf=qi)
    p = 3
    q = inp.random_perturbation(inp.uniform_state(m.ne, p, mach, 0.8, 0.3), 5, 0.1, mach)
    prob = sv.Problem(m, p, gas)
    P = rs.residual(q, m, p, gas, prob.basis, prob.geo, parts=True)
    w = np.outer(prob.basis.ws, prob.basis.ws)[None] * prob.geo.sol.J
    total = np.einsum("veji,eji->v", P.R, w)
    ws = prob.basis.ws
    top = np.einsum("vei,i->v", P.Fnum_eta[:, -6:], ws)
    bot = np.einsum("vei,i->v", P.Fnum_bottom, ws)
    s = sc.residual_scale(q, m, p, gas) * np.sum(w)
    assert np.all(np.abs(total + (top - bot)) <= 1e-13 * s), (total, top - bot, s)
    assert np.all(np.abs(total) > 1e-8 * s)


# ------------------------------------------------------------------ wall force

@pytest.mark.parametrize("p", [1, 2, 3])
def test_wall_force_of_linear_pressure_is_exact(p):
    """No flow and p = p_inf + a x + b y: the force on the body is -(a, b) times the
    area enclosed by its (straight-sided) wall polygon (divergence theorem), exactly."""
    ni, nj, mach = 48, 4, 0.05
    c = inp.naca_ogrid(ni, nj)
    gas = ph.Gas(mach=mach, re=50.0, kappa=1.0)
    m = rs.Mesh(ni, nj, c, np.zeros_like(c), bc=(rs.WALL, rs.FARFIELD),
                q_inf=inp.far_field_state(mach))
    a, b = 0.3, -0.7
    X, Y = inp.sample_points(c, p)
    q = np.stack([gas.R + a * X + b * Y, 0 * X, 0 * X, 1 + 0 * X])
    Fx, Fy = rs.wall_force(q, m, p, gas)
    wall = c[:ni, 0]
    A = _polygon_area(wall[:, 0], wall[:, 1])
    assert abs(Fx + a * A) <= 1e-12 and abs(Fy + b * A) <= 1e-12, (Fx, Fy, -a * A, -b * A)


def test_wall_force_of_linear_shear_is_exact():
    """u = g y, v = 0, p = p_inf, T = 1 over a flat static wall y = 0 of length 10: the
    fluid pulls the body below along +x with mu g / Re per unit length."""
    N, p, g = 6, 2, 0.4
    c, _ = _channel(N, 0.21)
    gas = ph.Gas(mach=0.1, re=25.0, kappa=1.0)
    m = rs.Mesh(N, N, c, np.zeros_like(c), bc=(rs.WALL, rs.FARFIELD), q_inf=(gas.R, 1.0, 0.0, 1.0))
    X, Y = inp.sample_points(c, p)
    q = np.stack([gas.R + 0 * X, g * Y, 0 * X, 1 + 0 * X])
    Fx, Fy = rs.wall_force(q, m, p, gas)
    assert abs(Fx - gas.mu * g / gas.re * L_BOX) <= 1e-13 and abs(Fy) <= 1e-12, (Fx, Fy)


def test_wall_force_uses_wall_velocity():
    """The same shear field seen from a wall moving with u = g y at the wall (here 0) is
    unchanged, and a uniform stream past a wall moving with it exerts no force."""
    N, p = 5, 2
    c, _ = _channel(N, 0.21)
    gas = ph.Gas(mach=0.1, re=25.0, kappa=1.0)
    vel = np.zeros_like(c)
    vel[..., 0] = 0.6                                   # the whole mesh slides along x
    m = rs.Mesh(N, N, c, vel, bc=(rs.WALL, rs.FARFIELD), q_inf=(gas.R, 0.6, 0.0, 1.0))
    X, _ = inp.sample_points(c, p)
    q = np.stack([gas.R + 0 * X, 0.6 + 0 * X, 0 * X, 1 + 0 * X])
    Fx, Fy = rs.wall_force(q, m, p, gas)
    assert abs(Fx) <= 1e-13 and abs(Fy) <= 1e-12


# ------------------------------------------------------------------ derivatives

def test_complex_step_through_boundary_faces_matches_central_differences():
    """The complex-step JVP that the oracle's Newton solver uses stays exact with wall and
    far-field faces (every boundary operation is complex-safe)."""
    ni, nj, p, mach = 8, 3, 2, 0.1
    c, v = inp.plunge(inp.naca_ogrid(ni, nj), 0.2)
    gas = ph.Gas(mach=mach, re=50.0, kappa=1.0)
    m = rs.Mesh(ni, nj, c, v, bc=(rs.WALL, rs.FARFIELD), q_inf=inp.far_field_state(mach))
    prob = sv.Problem(m, p, gas)
    q = inp.random_perturbation(inp.uniform_state(m.ne, p, mach), 3, 0.05, mach)
    d = inp.random_vector(q.shape, 4) * np.array([inp.p_inf(mach) * 1e-2, 1, 1, 1])[:, None, None, None]
    jv = sv.jacobian_vector(prob, q, d)
    h = 1e-6
    fd = (prob.R(q + h * d) - prob.R(q - h * d)) / (2 * h)
    s = np.abs(jv).max(axis=(1, 2, 3))
    assert np.all(np.abs(jv - fd).max(axis=(1, 2, 3)) <= 1e-5 * s), np.abs(jv - fd).max(axis=(1, 2, 3)) / s


def test_cylinder_ogrid_geometry():
    """The cylinder O-grid input: wall nodes on the circle of diameter 1, outer nodes on the
    far-field circle, the first radial cell of the requested size, every element with
    positive area (right-handed), and the wrap closing the grid around the body."""
    ni, nj, rf, first = 24, 10, 20.0, 1e-2
    c = inp.cylinder_ogrid(ni, nj, rf, first)
    r_wall = np.hypot(c[:ni, 0, 0], c[:ni, 0, 1])
    r_far = np.hypot(c[-ni:, 3, 0], c[-ni:, 3, 1])
    np.testing.assert_allclose(r_wall, 0.5, rtol=1e-14)
    np.testing.assert_allclose(r_far, rf, rtol=1e-12)
    r1 = np.hypot(c[:ni, 3, 0], c[:ni, 3, 1])
    np.testing.assert_allclose(r1 - 0.5, first, rtol=1e-6)
    a = c[:, 2] - c[:, 0]
    b = c[:, 3] - c[:, 1]
    assert np.all(a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0] > 0)
    # element ni-1's right edge is element 0's left edge
    np.testing.assert_allclose(c[ni - 1, 1], c[0, 0], atol=1e-15)
