"""Pins of the oracle's FR/CPR residual (Sec. 3.1) against what the paper and the
mathematics fix: free-stream preservation on deforming meshes (GCL, Sec. 2.3),
discrete conservation on static periodic meshes (Radau FR = nodal DG), consistency
with the exact flux divergence of a manufactured field (inviscid, viscous and
grid-velocity parts separately), and the k+1/2 spatial order on the translating
isentropic vortex (Sec. 4.3)."""
import numpy as np
import pytest

from oracle import physics as ph
from oracle import residual as rs
from oracle import scale as sc
from oracle import solver as sv
from paper_1903_06304_gb300 import inputs as inp


def _deformed(nx, ny, t, box=(0.0, 10.0, 0.0, 10.0), motion=inp.Motion()):
    ref = inp.box_mesh(nx, ny, *box)
    return inp.deform(ref, t, motion)


@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("t", [0.05, 0.13, 0.4])
@pytest.mark.parametrize("re", [0.0, 10.0])
def test_free_stream_preserved_on_deforming_mesh(p, t, re):
    """Uniform flow stays a solution on a moving mesh (implicit GCL, Eqs. gcl_eqs,
    unsteady_pre_mov_cdomain_GCL): R = 0 to rounding at M = 0.01."""
    c, v = _deformed(6, 5, t)
    mesh = rs.Mesh(6, 5, c, v)
    gas = ph.Gas(mach=0.01, re=re, kappa=1.0)
    q = inp.uniform_state(mesh.ne, p, 0.01, 0.8, 0.3)
    R = rs.residual(q, mesh, p, gas)
    s = sc.residual_scale(q, mesh, p, gas)
    assert np.all(np.abs(R).max(axis=(1, 2, 3)) <= 1e-13 * s)


def test_free_stream_violated_without_gcl_term():
    """Control: the same flow on a moving mesh WITHOUT the grid-velocity terms is not
    preserved, so the previous test is sensitive to them."""
    c, v = _deformed(6, 5, 0.13)
    gas = ph.Gas(mach=0.01, re=0.0, kappa=1.0)
    q = inp.uniform_state(30, 3, 0.01, 0.8, 0.3)
    s = sc.residual_scale(q, rs.Mesh(6, 5, c, v), 3, gas)
    # wrong: pretend the mesh is static while the metrics are those of the moving mesh,
    # and keep the grid velocity only in the face fluxes
    from oracle.basis import make_basis
    from oracle.geometry import element_geometry
    b = make_basis(3)
    geo = element_geometry(c, v, b)
    geo.sol.St_xi = 0 * geo.sol.St_xi
    geo.sol.St_eta = 0 * geo.sol.St_eta
    R = rs.residual(q, rs.Mesh(6, 5, c, v), 3, gas, b, geo)
    assert np.abs(R).max(axis=(1, 2, 3))[0] > 1e-6 * s[0]


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("re", [0.0, 5.0])
def test_discrete_conservation_on_static_periodic_mesh(p, re):
    """sum_e sum_ij w_i w_j |J| R = 0: the Radau FR scheme with Gauss points is nodal
    DG and the common fluxes telescope over periodic faces."""
    c, _ = _deformed(5, 4, 0.21)   # distorted but static
    mesh = rs.Mesh(5, 4, c, np.zeros_like(c))
    gas = ph.Gas(mach=0.05, re=re, kappa=1.0)
    q = inp.random_perturbation(inp.uniform_state(mesh.ne, p, 0.05, 0.8, 0.3), 7, 0.1, 0.05)
    prob = sv.Problem(mesh, p, gas)
    R = prob.R(q)
    w = np.outer(prob.basis.ws, prob.basis.ws)[None] * prob.geo.sol.J
    total = np.einsum("veji,eji->v", R, w)
    s = sc.residual_scale(q, mesh, p, gas) * np.sum(w)
    assert np.all(np.abs(total) <= 1e-13 * s), (total, s)
    assert np.all(np.abs(R).max(axis=(1, 2, 3)) > 1e-6 * s / np.sum(w))


# ------------------------------------------------------------------ manufactured consistency

sp = pytest.importorskip("sympy")
L_BOX = 10.0


def _manufactured(gas_v):
    x, y = sp.symbols("x y", real=True)
    k = 2 * sp.pi / L_BOX
    P = gas_v.R * (1 + 0.02 * sp.sin(k * x + 0.3) * sp.cos(k * y))
    U = 0.8 + 0.1 * sp.sin(k * y + 0.3) * sp.cos(k * x)
    V = 0.3 + 0.1 * sp.cos(k * x + 0.7) * sp.sin(2 * k * y)
    T = 1 + 0.02 * sp.cos(k * x) * sp.sin(k * y + 0.1)
    q = (P, U, V, T)
    qx = tuple(sp.diff(a, x) for a in q)
    qy = tuple(sp.diff(a, y) for a in q)
    fi, gi = ph.inviscid_flux(q, gas_v)
    fv, gv = ph.viscous_flux(q, qx, qy, gas_v)
    qc = ph.conservative(q, gas_v)
    lam = lambda e: sp.lambdify((x, y), e, "numpy")
    return dict(
        q=[lam(a) for a in q],
        div_inv=[lam(sp.diff(fi[i], x) + sp.diff(gi[i], y)) for i in range(4)],
        div_vis=[lam(sp.diff(fv[i], x) + sp.diff(gv[i], y)) for i in range(4)],
        qcx=[lam(sp.diff(qc[i], x)) for i in range(4)],
        qcy=[lam(sp.diff(qc[i], y)) for i in range(4)],
    )


def _ev(f, X):
    return np.broadcast_to(f(*X), X[0].shape)


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("part", ["inviscid", "viscous", "grid"])
def test_manufactured_consistency_order(p, part):
    """Residual minus its exact continuous counterpart converges under refinement:
    inviscid R -> -div f_inv (order ~p), viscous part -> +div f_vis (order ~p-1),
    grid-velocity part -> v_g . grad q^c (order ~p)."""
    gas_v = ph.Gas(mach=0.2, re=20.0, kappa=1.0)
    gas_i = ph.Gas(mach=0.2, re=0.0, kappa=1.0)
    ex = _manufactured(gas_v)
    errs = []
    for N in (8, 16, 32):
        c, v = _deformed(N, N, 0.13)
        X = inp.sample_points(c, p)
        Vg = inp.sample_points(v, p)
        qh = np.stack([_ev(f, X) for f in ex["q"]])
        if part == "inviscid":
            m = rs.Mesh(N, N, c, np.zeros_like(v))
            got = rs.residual(qh, m, p, gas_i)
            want = np.stack([-_ev(f, X) for f in ex["div_inv"]])
        elif part == "viscous":
            m = rs.Mesh(N, N, c, v)
            got = rs.residual(qh, m, p, gas_v) - rs.residual(qh, m, p, gas_i)
            want = np.stack([_ev(f, X) for f in ex["div_vis"]])
        else:
            got = (rs.residual(qh, rs.Mesh(N, N, c, v), p, gas_i)
                   - rs.residual(qh, rs.Mesh(N, N, c, np.zeros_like(v)), p, gas_i))
            want = np.stack([Vg[0] * ex["qcx"][i](*X) + Vg[1] * ex["qcy"][i](*X) for i in range(4)])
        scale = np.abs(want).max(axis=(1, 2, 3))
        keep = scale > 0
        errs.append((np.abs(got - want).max(axis=(1, 2, 3))[keep] / scale[keep]))
    errs = np.array(errs)
    order = np.log2(errs[-2] / errs[-1])
    need = {"inviscid": p - 0.5, "viscous": p - 1.5, "grid": p - 0.5}[part]
    assert np.all(order >= need), (order, errs)
    assert np.all(errs[-1] < 0.25)


# ------------------------------------------------------------------ vortex accuracy

def _q_from_qc(qc, gas):
    rho = qc[0]
    u = qc[1] / rho
    v = qc[2] / rho
    p = (gas.gamma - 1) * (qc[3] - 0.5 * rho * (u * u + v * v))
    return np.stack([p, u, v, p / (rho * gas.R)])


def _vortex_error(N, p, deforming, mach=0.5, half=6.0, t_end=0.3):
    ref = inp.box_mesh(N, N, -half, half, -half, half)
    vx = inp.Vortex(mach=mach, period_x=2 * half, period_y=2 * half)
    gas = ph.Gas(mach=mach, re=0.0, kappa=1.0)
    mot = inp.Motion(ax=0.2, ay=0.2, fx=1 / (2 * half), fy=1 / (2 * half), fn=1.0)

    def mesh_at(t):
        if deforming:
            c, v = inp.deform(ref + half, t, mot)
            return c - half, v
        return ref, np.zeros_like(ref)

    c, _ = mesh_at(0.0)
    q = inp.vortex_state(*inp.sample_points(c, p), 0.0, vx)
    qc = ph.conservative(tuple(q), gas)
    h = 2 * half / N
    dt = 0.3 * h / ((2 * p + 1) * (2.0 + 1 / mach) / mach ** 2)
    nst = int(np.ceil(t_end / dt))
    dt = t_end / nst

    def rhs(s, t):
        cc, vv = mesh_at(t)
        return rs.residual(_q_from_qc(s, gas), rs.Mesh(N, N, cc, vv), p, gas)

    t = 0.0
    for _ in range(nst):   # classical RK4 on dq^c/dt = R (test-local integrator)
        k1 = rhs(qc, t)
        k2 = rhs(qc + 0.5 * dt * k1, t + 0.5 * dt)
        k3 = rhs(qc + 0.5 * dt * k2, t + 0.5 * dt)
        k4 = rhs(qc + dt * k3, t + dt)
        qc = qc + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        t += dt
    c, v = mesh_at(t_end)
    qe = inp.vortex_state(*inp.sample_points(c, p), t_end, vx)
    prob = sv.Problem(rs.Mesh(N, N, c, v), p, gas)
    qn = _q_from_qc(qc, gas)
    return np.array([sv.l2_error(prob, qn[k], qe[k]) for k in (0, 1)])


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("deforming", [False, True])
def test_vortex_spatial_order(p, deforming):
    """Sec. 4.3: L2 errors of p and u converge at about k+1/2 with the Rusanov flux,
    with and without the deforming mesh."""
    e1 = _vortex_error(12, p, deforming)
    e2 = _vortex_error(24, p, deforming)
    order = np.log2(e1 / e2)
    assert np.all(order >= p - 0.3), (order, e1, e2)


def test_batch_recipe_is_seeded_and_in_range():
    """The batch workload recipe: deterministic for a seed, every case inside the stated
    ranges (mesh side 32..128, p in {2,3,4}, M in [0.01, 0.3], alpha in [1, 5], vortex
    or bump), and an initial state of the right shape for each case."""
    from paper_1903_06304_gb300 import inputs as inp
    a, b = inp.batch_cases(seed=0, ncases=64), inp.batch_cases(seed=0, ncases=64)
    assert a == b and inp.batch_cases(seed=1, ncases=64) != a
    for c in a:
        assert 32 <= c.n <= 128 and c.p in (2, 3, 4) and 0.01 <= c.mach <= 0.3
        assert 1.0 <= c.alpha <= 5.0 and c.ic in ("vortex", "bump")
        assert 0.0 <= c.xc <= 10.0 and 0.0 <= c.yc <= 10.0
    assert {c.ic for c in a} == {"vortex", "bump"} and {c.p for c in a} == {2, 3, 4}
    small = inp.BatchCase(2, 4, 0.1, "bump", 9.5, 0.2, 2.0)
    corners, vel, q = inp.make_batch_case(small)
    assert corners.shape == (16, 4, 2) and q.shape == (4, 16, 3, 3) and not vel.any()
    # the bump is periodic: equal pressure at points mirrored across the periodic seam
    assert np.isfinite(q).all()
