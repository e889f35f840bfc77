"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds NO arithmetic of the method (no metrics, fluxes, residuals or
solvers).  It only builds inputs: element corner coordinates and corner
velocities of structured quadrilateral meshes (Sec. 4.3 prescribed grid motion),
and primitive states (p, u, v, T) sampled at physical points (uniform flow, a
Gaussian pressure bump, the isentropic vortex of Eq. VP_Solution).  Sampling
points are produced with numpy's Gauss-Legendre rule and bilinear shape
functions purely to decide WHERE an initial condition is sampled; both the
oracle and the CUDA library compute their own points and metrics independently.

Conventions
-----------
* Element ``e = j * nx + i`` (``i`` along xi, ``j`` along eta).
* Corner order per element: (xi, eta) = (-1,-1), (+1,-1), (+1,+1), (-1,+1).
* Primitive state arrays are ``[4][Ne][n][n]`` float64 (var, elem, eta-index j,
  xi-index i) with ``n = p + 1``; variables are (p, u, v, T).
* Nondimensionalisation of Sec. 2.1: free stream rho = T = 1, |v| = 1,
  R = 1/(gamma M^2), so p_inf = 1/(gamma M^2).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAMMA = 1.4
PRANDTL = 0.72


# ----------------------------------------------------------------------------- meshes

def box_mesh(nx: int, ny: int, x0: float, x1: float, y0: float, y1: float) -> np.ndarray:
    """Corners ``[Ne, 4, 2]`` of a uniform nx-by-ny quad mesh of [x0,x1]x[y0,y1]."""
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    c = np.empty((ny, nx, 4, 2))
    X, Y = np.meshgrid(xs, ys)  # [ny+1, nx+1]
    c[:, :, 0, 0], c[:, :, 0, 1] = X[:-1, :-1], Y[:-1, :-1]
    c[:, :, 1, 0], c[:, :, 1, 1] = X[:-1, 1:], Y[:-1, 1:]
    c[:, :, 2, 0], c[:, :, 2, 1] = X[1:, 1:], Y[1:, 1:]
    c[:, :, 3, 0], c[:, :, 3, 1] = X[1:, :-1], Y[1:, :-1]
    return c.reshape(nx * ny, 4, 2)


@dataclasses.dataclass(frozen=True)
class Motion:
    """Prescribed deforming-grid motion of Sec. 4.3:
    x = x_r + a_x sin(2 pi f_n t) sin(2 pi f_x x_r) sin(2 pi f_y y_r), and y alike."""
    ax: float = 0.2
    ay: float = 0.2
    fx: float = 0.1
    fy: float = 0.1
    fn: float = 1.0


def deform(ref_corners: np.ndarray, t: float, m: Motion) -> tuple[np.ndarray, np.ndarray]:
    """Moved corners and their analytic velocities at time ``t`` (both ``[Ne,4,2]``)."""
    xr, yr = ref_corners[..., 0], ref_corners[..., 1]
    shape = np.sin(2 * math.pi * m.fx * xr) * np.sin(2 * math.pi * m.fy * yr)
    s = math.sin(2 * math.pi * m.fn * t)
    ds = 2 * math.pi * m.fn * math.cos(2 * math.pi * m.fn * t)
    pos = np.empty_like(ref_corners)
    vel = np.empty_like(ref_corners)
    pos[..., 0] = xr + m.ax * s * shape
    pos[..., 1] = yr + m.ay * s * shape
    vel[..., 0] = m.ax * ds * shape
    vel[..., 1] = m.ay * ds * shape
    return pos, vel


# ----------------------------------------------------------------------------- O-grids

def naca0012_half_thickness(x: np.ndarray) -> np.ndarray:
    """Half thickness of the NACA 0012 profile of Sec. 4.2, chord 1, with the closed
    trailing edge (last coefficient -0.1036, so that it vanishes at x = 1)."""
    return 0.6 * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x ** 2 + 0.2843 * x ** 3
                  - 0.1036 * x ** 4)


def _stretch_ratio(nj: int, first: float, span: float) -> float:
    """Ratio r of a geometric distribution of nj cells over ``span`` whose first cell is
    ``first`` long: first = span (r - 1) / (r^nj - 1), by bisection."""
    lo, hi = 1.0 + 1e-12, 2.0
    while (hi - 1.0) / (hi ** nj - 1.0) * span > first:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if (mid - 1.0) / (mid ** nj - 1.0) * span > first:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def naca_ogrid(ni: int = 256, nj: int = 96, r_far: float = 20.0, first: float = 1e-3,
               blend: float = 0.5) -> np.ndarray:
    """Corners ``[ni*nj, 4, 2]`` of an algebraic O-grid around the NACA 0012 (chord 1,
    leading edge at the origin): element e = j*ni + i, i around the body (periodic:
    the wrap closes at the trailing edge), j from the wall (row 0) to the far field
    (row nj-1), a circle of radius ``r_far`` chords about the mid-chord.

    Around the body, x = (1 - blend) (1 + cos s)/2 + blend |1 - s/pi| for s = 2 pi i/ni:
    cosine clustering at both edges (smallest chordwise spacing about (pi/ni)^2 at
    ``blend`` = 0) blended with a uniform distribution (about 2 ``blend``/ni at the edges
    when ``blend`` > 0), the lower surface first so that (i, j) is right-handed; the
    far-field node of column i sits at the angle -s.  Along each column the nodes follow a geometric
    distribution from the wall node to the far-field node whose first cell is ``first``
    of the wall-to-far-field distance at the mid-chord."""
    s = 2.0 * math.pi * np.arange(ni) / ni
    xw = (1.0 - blend) * 0.5 * (1.0 + np.cos(s)) + blend * np.abs(1.0 - s / math.pi)
    yt = naca0012_half_thickness(xw)
    yw = np.where(s <= math.pi, -yt, yt)
    xf = 0.5 + r_far * np.cos(-s)
    yf = r_far * np.sin(-s)
    r = _stretch_ratio(nj, first, r_far)
    frac = (r ** np.arange(nj + 1) - 1.0) / (r ** nj - 1.0)           # [nj+1], 0 .. 1
    X = xw[None, :] + frac[:, None] * (xf - xw)[None, :]             # [nj+1, ni]
    Y = yw[None, :] + frac[:, None] * (yf - yw)[None, :]
    ip = (np.arange(ni) + 1) % ni
    c = np.empty((nj, ni, 4, 2))
    c[:, :, 0, 0], c[:, :, 0, 1] = X[:-1, :], Y[:-1, :]
    c[:, :, 1, 0], c[:, :, 1, 1] = X[:-1, ip], Y[:-1, ip]
    c[:, :, 2, 0], c[:, :, 2, 1] = X[1:, ip], Y[1:, ip]
    c[:, :, 3, 0], c[:, :, 3, 1] = X[1:, :], Y[1:, :]
    return c.reshape(ni * nj, 4, 2)


def cylinder_ogrid(ni: int = 64, nj: int = 32, r_far: float = 20.0, first: float = 1e-2) -> np.ndarray:
    """Corners ``[ni*nj, 4, 2]`` of an O-grid around a circular cylinder of diameter 1
    centred at the origin (the body of Sec. 4.1): element e = j*ni + i, i around the body
    clockwise (periodic), j from the wall (row 0) to a circle of radius ``r_far`` diameters;
    straight radial lines with a geometric distribution whose first cell is ``first``
    diameters, equal angles around the body."""
    ang = -2.0 * math.pi * np.arange(ni) / ni
    r = _stretch_ratio(nj, first, r_far - 0.5)
    rad = 0.5 + (r_far - 0.5) * (r ** np.arange(nj + 1) - 1.0) / (r ** nj - 1.0)   # [nj+1]
    X = rad[:, None] * np.cos(ang)[None, :]
    Y = rad[:, None] * np.sin(ang)[None, :]
    ip = (np.arange(ni) + 1) % ni
    c = np.empty((nj, ni, 4, 2))
    c[:, :, 0, 0], c[:, :, 0, 1] = X[:-1, :], Y[:-1, :]
    c[:, :, 1, 0], c[:, :, 1, 1] = X[:-1, ip], Y[:-1, ip]
    c[:, :, 2, 0], c[:, :, 2, 1] = X[1:, ip], Y[1:, ip]
    c[:, :, 3, 0], c[:, :, 3, 1] = X[1:, :], Y[1:, :]
    return c.reshape(ni * nj, 4, 2)


def plunge(ref_corners: np.ndarray, t: float, h: float = 0.25, k: float = 1.0):
    """Rigid plunge of Sec. 4.4 (chord 1, U_inf = 1): y = y_r + h sin(2 pi f t) with the
    reduced frequency k = 2 pi f; the whole mesh moves.  Corners and velocities."""
    f = k / (2.0 * math.pi)
    pos = ref_corners.copy()
    vel = np.zeros_like(ref_corners)
    pos[..., 1] += h * math.sin(2.0 * math.pi * f * t)
    vel[..., 1] = 2.0 * math.pi * f * h * math.cos(2.0 * math.pi * f * t)
    return pos, vel


def far_field_state(mach: float, u: float = 1.0, v: float = 0.0) -> tuple:
    """Primitive free stream (p_inf, u, v, T_inf = 1) of the nondimensional gas."""
    return (p_inf(mach), u, v, 1.0)


def sample_points(corners: np.ndarray, p: int) -> tuple[np.ndarray, np.ndarray]:
    """Physical (x, y) ``[Ne, n, n]`` where initial conditions are sampled (Gauss points)."""
    g, _ = np.polynomial.legendre.leggauss(p + 1)
    eta, xi = np.meshgrid(g, g, indexing="ij")  # [j, i]
    N = np.stack([(1 - xi) * (1 - eta), (1 + xi) * (1 - eta),
                  (1 + xi) * (1 + eta), (1 - xi) * (1 + eta)]) / 4.0  # [4, n, n]
    x = np.einsum("ajk,ea->ejk", N, corners[..., 0])
    y = np.einsum("ajk,ea->ejk", N, corners[..., 1])
    return x, y


# ----------------------------------------------------------------------------- states

def p_inf(mach: float) -> float:
    return 1.0 / (GAMMA * mach * mach)


def uniform_state(ne: int, p: int, mach: float, u: float = 1.0, v: float = 0.0) -> np.ndarray:
    n = p + 1
    q = np.empty((4, ne, n, n))
    q[0], q[1], q[2], q[3] = p_inf(mach), u, v, 1.0
    return q


def gaussian_bump(x: np.ndarray, y: np.ndarray, mach: float, amp: float = 1e-3,
                  width: float = 0.1, xc: float = 0.5, yc: float = 0.5,
                  period: float = 0.0) -> np.ndarray:
    """Uniform flow u=1, v=0, T=1 plus a Gaussian pressure bump
    p = p_inf (1 + amp exp(-|x - x_c|^2 / width^2)); period > 0 measures the distance
    to the nearest periodic image of the centre."""
    dx, dy = x - xc, y - yc
    if period > 0:
        dx = dx - period * np.round(dx / period)
        dy = dy - period * np.round(dy / period)
    r2 = dx ** 2 + dy ** 2
    q = np.empty((4,) + x.shape)
    q[0] = p_inf(mach) * (1.0 + amp * np.exp(-r2 / width ** 2))
    q[1], q[2], q[3] = 1.0, 0.0, 1.0
    return q


@dataclasses.dataclass(frozen=True)
class Vortex:
    """Isentropic vortex of Eq. VP_Solution, translating with the free stream."""
    mach: float = 0.05
    alpha: float = 5.0
    phi: float = 0.5
    x0: float = 0.0
    y0: float = 0.0
    u_inf: float = math.sqrt(0.5)
    v_inf: float = math.sqrt(0.5)
    period_x: float = 0.0   # > 0: periodic domain length in x (images summed over nearest copies)
    period_y: float = 0.0


def vortex_state(x: np.ndarray, y: np.ndarray, t: float, vx: Vortex) -> np.ndarray:
    """Primitive (p,u,v,T) of the vortex at time t.

    The perturbation of Eq. VP_Solution is stated for a gas constant of one; in the
    Sec. 2.1 scaling (T_inf = 1, R = 1/(gamma M^2)) the temperature perturbation is
    multiplied by gamma M^2, which leaves rho, u, v and p unchanged.  ``r^2`` is the
    squared distance to the centre (the printed ``r`` is read as ``r^2``).
    """
    cx = vx.x0 + vx.u_inf * t
    cy = vx.y0 + vx.v_inf * t
    dx = x - cx
    dy = y - cy
    if vx.period_x > 0:
        dx = dx - vx.period_x * np.round(dx / vx.period_x)
    if vx.period_y > 0:
        dy = dy - vx.period_y * np.round(dy / vx.period_y)
    r2 = dx * dx + dy * dy
    ex = np.exp(vx.phi * (1.0 - r2))
    du = -vx.alpha / (2 * math.pi) * dy * ex
    dv = vx.alpha / (2 * math.pi) * dx * ex
    dT = -(vx.alpha ** 2) * (GAMMA - 1) * vx.mach ** 2 / (16 * vx.phi * math.pi ** 2) * ex * ex
    T = 1.0 + dT
    rho = T ** (1.0 / (GAMMA - 1))
    q = np.empty((4,) + x.shape)
    q[0] = rho * T / (GAMMA * vx.mach ** 2)
    q[1] = vx.u_inf + du
    q[2] = vx.v_inf + dv
    q[3] = T
    return q


def random_perturbation(q: np.ndarray, seed: int, rel: float = 1e-2, mach: float = 0.1) -> np.ndarray:
    """q plus seeded uniform noise, scaled per variable to its natural fluctuation size
    at Mach ``mach``: p and (u, v) by ``rel`` (pressure fluctuations ~ rho |v|^2 ~ 1),
    T by ``rel * mach^2``."""
    rng = np.random.default_rng(seed)
    scale = np.array([rel, rel, rel, rel * mach * mach])
    return q + scale[:, None, None, None] * rng.uniform(-1.0, 1.0, size=q.shape)


def random_vector(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=shape)


# ----------------------------------------------------------------------------- workloads

@dataclasses.dataclass(frozen=True)
class Workload:
    """A named synthetic workload (mesh, order, flow parameters, solver knobs)."""
    name: str
    nx: int
    ny: int
    p: int
    mach: float
    re: float            # <= 0: inviscid (Euler)
    kappa: float
    box: tuple = (0.0, 10.0, 0.0, 10.0)
    ic: str = "vortex"   # "vortex" | "bump" | "uniform"
    deforming: bool = False
    dt: float = 0.01
    restart: int = 30
    tol_res: float = 1e-6
    tol_pseudo: float = 1e-8
    maxit_lin: int = 100
    maxit_newton: int = 20
    motion: Motion = Motion()

    @property
    def ne(self) -> int:
        return self.nx * self.ny

    @property
    def dof(self) -> int:
        return 4 * self.ne * (self.p + 1) ** 2


# Gaussian bump, 8x8 periodic unit square, p=2, M=0.1, Euler, steady PTC with GMRES(20).
EULER_BUMP_8 = Workload("euler_bump_8x8_p2", 8, 8, 2, 0.1, 0.0, 1.0, (0.0, 1.0, 0.0, 1.0),
                        ic="bump", restart=20, tol_res=1e-6, maxit_newton=10)
# Isentropic vortex, periodic [0,10]^2, 64x64, p=3, M=0.05, Re=100 on the box length
# (Re_ref = 10 per unit length), BDF2 dt = 0.01, GMRES(30).
NS_VORTEX_64 = Workload("ns_vortex_64x64_p3", 64, 64, 3, 0.05, 10.0, 0.0, (0.0, 10.0, 0.0, 10.0),
                        ic="vortex", dt=0.01, restart=30)
# Deforming [0,10]^2, 128x128, p=3, M=0.01 (kappa=1, see the kappa reading), Re_ref = 10.
NS_DEFORM_128 = Workload("ns_deform_128x128_p3", 128, 128, 3, 0.01, 10.0, 1.0, (0.0, 10.0, 0.0, 10.0),
                         ic="vortex", deforming=True, dt=0.01, restart=30)

WORKLOADS = {w.name: w for w in (EULER_BUMP_8, NS_VORTEX_64, NS_DEFORM_128)}


def make_case(w: Workload, t: float = 0.0):
    """Corners, corner velocities and initial primitive state of workload ``w`` at time t."""
    x0, x1, y0, y1 = w.box
    ref = box_mesh(w.nx, w.ny, x0, x1, y0, y1)
    if w.deforming:
        corners, vel = deform(ref, t, w.motion)
    else:
        corners, vel = ref, np.zeros_like(ref)
    x, y = sample_points(corners, w.p)
    if w.ic == "bump":
        q = gaussian_bump(x, y, w.mach, xc=0.5 * (x0 + x1), yc=0.5 * (y0 + y1))
    elif w.ic == "vortex":
        vx = Vortex(mach=w.mach, x0=0.5 * (x0 + x1), y0=0.5 * (y0 + y1),
                    period_x=x1 - x0, period_y=y1 - y0)
        q = vortex_state(x, y, t, vx)
    else:
        q = uniform_state(w.ne, w.p, w.mach)
    return corners, vel, q


# ------------------------------------------------------------------ batches of cases
@dataclasses.dataclass(frozen=True)
class BatchCase:
    """One case of a batch workload: a periodic n x n box [0, box]^2 at degree p."""
    p: int
    n: int
    mach: float
    ic: str              # "vortex" | "bump"
    xc: float
    yc: float
    alpha: float         # vortex strength, or bump amplitude in units of 1e-3 p_inf
    re: float = 10.0     # Re = 100 on the box length 10
    kappa: float = 1.0
    box: float = 10.0


def batch_cases(seed: int = 0, ncases: int = 64, side=(32, 128), degrees=(2, 3, 4),
                mach=(0.01, 0.3)) -> list:
    """Seeded batch recipe: mesh side uniform in [side[0], side[1]], degree uniform over
    ``degrees``, Mach uniform in ``mach``, vortex or bump with probability 1/2, centre
    uniform in the box, strength alpha uniform in [1, 5]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(ncases):
        n = int(rng.integers(side[0], side[1] + 1))
        p = int(rng.choice(degrees))
        m = float(rng.uniform(mach[0], mach[1]))
        ic = "vortex" if rng.uniform() < 0.5 else "bump"
        xc, yc = (float(v) for v in rng.uniform(0.0, 10.0, size=2))
        alpha = float(rng.uniform(1.0, 5.0))
        out.append(BatchCase(p, n, m, ic, xc, yc, alpha))
    return out


def make_batch_case(bc: BatchCase):
    """Corners, corner velocities (static mesh) and initial state of one batch case.  The
    bump has width box/10 (C1's width relative to its box) and amplitude alpha 1e-3 p_inf."""
    corners = box_mesh(bc.n, bc.n, 0.0, bc.box, 0.0, bc.box)
    vel = np.zeros_like(corners)
    x, y = sample_points(corners, bc.p)
    if bc.ic == "vortex":
        vx = Vortex(mach=bc.mach, alpha=bc.alpha, x0=bc.xc, y0=bc.yc,
                    period_x=bc.box, period_y=bc.box)
        q = vortex_state(x, y, 0.0, vx)
    else:
        q = gaussian_bump(x, y, bc.mach, amp=1e-3 * bc.alpha, width=0.1 * bc.box, xc=bc.xc,
                          yc=bc.yc, period=bc.box)
    return corners, vel, q
