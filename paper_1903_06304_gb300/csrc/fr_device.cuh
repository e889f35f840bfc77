// fr_device.cuh -- device building blocks of the preconditioned FR/CPR residual
// (Wang & Yu, arXiv 1903.06304, Secs. 2-3) for sm_103a.
//
// Every arithmetic routine is a template on the scalar T: double for the residual,
// Dual (value + one tangent) for the exact forward-mode Jacobian action.  The FP64
// pipe is the binding resource on GB300, so the formulas are arranged to minimise
// FP64 instructions: no unit normals (|S| f_n = f . S), the FR correction folded into
// a corrected derivative matrix, BR2 liftings in closed form, one reciprocal per
// temperature.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fr {

constexpr int MAXN = 5;  // p <= 4

// ---------------------------------------------------------------- constants
// 1-D FR basis on [-1,1] with Gauss solution points (Sec. 3.1).
// Penalty of the BR2 face lifting (the face gradient's lifted jumps are scaled by it; the
// corrected gradient at the solution points keeps the plain liftings).  With 1 the viscous
// vortex on 64 x 64 elements of degree 3 grows unstably; 2 keeps it stable (as do 4 and 6,
// with the same solution), and larger values stiffen the thin wall cells of an O-grid
// (with 4 the first step of the M = 0.3 plunge breaks down).
constexpr double BR2_PENALTY = 2.0;

struct Basis {
  double D[MAXN][MAXN];   // D[i][k] = l_k'(x_i)
  double Dc[MAXN][MAXN];  // D[i][k] - g_L'(x_i) l_k(-1) - g_R'(x_i) l_k(1)
  double lL[MAXN], lR[MAXN];
  double dgL[MAXN], dgR[MAXN];
  double lift_end;        // BR2 face lifting factor eta g_R'(1), g_R'(1) = (p+1)^2/2 = -g_L'(-1)
  double xs[MAXN];        // solution points
  double ws[MAXN];        // Gauss weights of the solution points
};

// Nondimensional gas of Sec. 2.1 and preconditioning cut-off (Eqs. eps_nonmove/move).
struct Gas {
  double gamma, R, inv_R, cp, inv_cp, inv_gm1;
  double mu, inv_re, k_cond;     // k_cond = mu C_p / Pr
  double kappa_minf, eps_floor;
  int viscous;
};

// Geometry at solution points: arrays gs[k][Ne*np2].
enum { GS_SXX, GS_SXY, GS_SEX, GS_SEY, GS_STX, GS_STE, GS_INVJ, GS_DIVST, GS_UG, GS_VG, GS_J,
       GS_COUNT };
// Geometry at flux points: arrays gf[k][Ne][4 faces][n].  S is |J| grad(xi) on the
// L/R faces and |J| grad(eta) on the B/T faces.
enum { GF_SX, GF_SY, GF_J, GF_UG, GF_VG, GF_COUNT };
enum { FACE_L = 0, FACE_R = 1, FACE_B = 2, FACE_T = 3 };
// Boundary faces (Sec. 3.3): a face without a neighbour stores -kind in the neighbour
// table.
enum { BC_WALL = 1, BC_FARFIELD = 2 };

// Parameters of one independent case (a batch holds several): its gas, the time terms of
// the pseudo-step right-hand side r = R - (a0 q^c + a1 qc_n + a2 qc_nm1)/dt (per dt) and
// the coefficients of the Newton operator A = inv_dtau Gamma + a0_dt M - dR/dq.
struct CaseParams {
  Gas gas;
  double a0dt, a1dt, a2dt;
  double inv_dtau, a0_dt;
  // layout of the case in the state vectors the kernels read and write: the case's
  // values are contiguous, [variable][element of the case][point], from DOF offset off;
  // e0 is its first element in the launch's element numbering, sn = elements x points.
  long long off;
  int e0, sn;
  int nx, ny;   // the case's box: element e0 + j nx + i is at column i, row j
  int active;   // 0: the Newton loop of this case has stopped; its elements are skipped
  double qinf[4];   // far-field primitive state (p, u, v, T) of far-field boundary faces
};

// Element topology of one launch: face neighbours (L, R, B, T) by global element index,
// the case of each element and the case parameters.  All cases of a launch share the
// polynomial degree (a template parameter of the kernels) and the viscous switch.
struct Mesh {
  const int* nbr;          // [ne][4]
  const int* ecase;        // [ne]
  const CaseParams* cp;    // [ncases]
  int ne;
  int viscous;
  __device__ __forceinline__ int left(int e) const { return nbr[4 * e + FACE_L]; }
  __device__ __forceinline__ int right(int e) const { return nbr[4 * e + FACE_R]; }
  __device__ __forceinline__ int bottom(int e) const { return nbr[4 * e + FACE_B]; }
  __device__ __forceinline__ int top(int e) const { return nbr[4 * e + FACE_T]; }
  __device__ __forceinline__ const CaseParams& par(int e) const { return cp[ecase[e]]; }
  __device__ __forceinline__ bool on(int e) const { return cp[ecase[e]].active != 0; }
  // index of variable 0 at point 0 of element e in a state vector, and the stride
  // between the variables of e's case
  __device__ __forceinline__ size_t qbase(int e, int np) const {
    const CaseParams& c = par(e);
    return (size_t)c.off + (size_t)(e - c.e0) * np;
  }
  __device__ __forceinline__ size_t qstride(int e) const { return (size_t)par(e).sn; }
};

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v, d;
};
__device__ __forceinline__ Dual mk(double v, double d) { Dual r; r.v = v; r.d = d; return r; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return mk(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return mk(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator-(Dual a) { return mk(-a.v, -a.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return mk(a.v * b.v, fma(a.v, b.d, a.d * b.v)); }
__device__ __forceinline__ Dual operator+(Dual a, double b) { return mk(a.v + b, a.d); }
__device__ __forceinline__ Dual operator+(double a, Dual b) { return mk(a + b.v, b.d); }
__device__ __forceinline__ Dual operator-(Dual a, double b) { return mk(a.v - b, a.d); }
__device__ __forceinline__ Dual operator-(double a, Dual b) { return mk(a - b.v, -b.d); }
__device__ __forceinline__ Dual operator*(Dual a, double b) { return mk(a.v * b, a.d * b); }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return mk(a * b.v, a * b.d); }
__device__ __forceinline__ Dual inv(Dual a) {
  double r = 1.0 / a.v;
  return mk(r, -a.d * r * r);
}
__device__ __forceinline__ double inv(double a) { return 1.0 / a; }
__device__ __forceinline__ Dual sqrt_(Dual a) {
  double s = sqrt(a.v);
  return mk(s, a.d * (0.5 / s));
}
__device__ __forceinline__ double sqrt_(double a) { return sqrt(a); }
__device__ __forceinline__ double val(double a) { return a; }
__device__ __forceinline__ double val(Dual a) { return a.v; }
__device__ __forceinline__ double tan_(double) { return 0.0; }
__device__ __forceinline__ double tan_(Dual a) { return a.d; }
template <class T> __device__ __forceinline__ T abs_(T a) { return val(a) < 0 ? -a : a; }
// max/min deciding on values; ties keep the first argument (same rule as the oracle).
template <class T> __device__ __forceinline__ T vmax(T a, T b) { return val(a) >= val(b) ? a : b; }
template <class T> __device__ __forceinline__ T vmin(T a, T b) { return val(a) <= val(b) ? a : b; }
template <class T> __device__ __forceinline__ T fmadd(T a, T b, T c) { return a * b + c; }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }

template <class T> __device__ __forceinline__ T from_parts(double v, double d);
template <> __device__ __forceinline__ double from_parts<double>(double v, double) { return v; }
template <> __device__ __forceinline__ Dual from_parts<Dual>(double v, double d) { return mk(v, d); }

// A constant (double) or a parameter-dependent value (Dual) as a T.
template <class T> __device__ __forceinline__ T as_T(double x) { return from_parts<T>(x, 0.0); }
template <class T> __device__ __forceinline__ T as_T(Dual x);
template <> __device__ __forceinline__ Dual as_T<Dual>(Dual x) { return x; }

// Gas with the tangent of its Mach-dependent constants (R = 1/(gamma M^2), C_p =
// 1/((gamma-1) M^2), k = mu C_p / Pr, kappa M_inf) for a Mach tangent dM; the others have
// zero tangent.
struct GasD {
  Dual gamma, R, inv_R, cp, inv_cp, inv_gm1, mu, inv_re, k_cond, kappa_minf, eps_floor;
  int viscous;
};
__device__ __forceinline__ GasD gas_tangent(const Gas& g, double dM) {
  const double M = sqrt(g.inv_R / g.gamma);   // inv_R = gamma M^2
  const double s = dM / M;                    // d(M^k)/M^k = k dM / M
  GasD o;
  o.gamma = mk(g.gamma, 0.0);
  o.R = mk(g.R, -2.0 * g.R * s);
  o.inv_R = mk(g.inv_R, 2.0 * g.inv_R * s);
  o.cp = mk(g.cp, -2.0 * g.cp * s);
  o.inv_cp = mk(g.inv_cp, 2.0 * g.inv_cp * s);
  o.inv_gm1 = mk(g.inv_gm1, 0.0);
  o.mu = mk(g.mu, 0.0);
  o.inv_re = mk(g.inv_re, 0.0);
  o.k_cond = mk(g.k_cond, -2.0 * g.k_cond * s);
  o.kappa_minf = mk(g.kappa_minf, g.kappa_minf * s);
  o.eps_floor = mk(g.eps_floor, 0.0);
  o.viscous = g.viscous;
  return o;
}
// The gas a kernel instantiation computes with: plain for G = double, with the Mach
// tangent for G = Dual (the parameter-sensitivity path).
template <class G> struct GasOf { using type = const Gas&; };
template <> struct GasOf<Dual> { using type = GasD; };
template <class G> __device__ __forceinline__ typename GasOf<G>::type gas_for(const Gas& g, double dM);
template <> __device__ __forceinline__ const Gas& gas_for<double>(const Gas& g, double) { return g; }
template <> __device__ __forceinline__ GasD gas_for<Dual>(const Gas& g, double dM) { return gas_tangent(g, dM); }

// Geometry read as G: plain values, or values with tangents from a second array.
template <class G> __device__ __forceinline__ G geo(const double* v, const double* d, size_t i);
template <> __device__ __forceinline__ double geo<double>(const double* v, const double*, size_t i) { return v[i]; }
template <> __device__ __forceinline__ Dual geo<Dual>(const double* v, const double* d, size_t i) { return mk(v[i], d[i]); }

// A device buffer of T stored as separate value / tangent FP64 arrays.
template <class T> struct Buf;
template <> struct Buf<double> {
  double* v;
  __device__ __forceinline__ double ld(size_t i) const { return v[i]; }
  __device__ __forceinline__ void st(size_t i, double x) const { v[i] = x; }
};
template <> struct Buf<Dual> {
  double* v;
  double* d;
  __device__ __forceinline__ Dual ld(size_t i) const { return mk(v[i], d[i]); }
  __device__ __forceinline__ void st(size_t i, Dual x) const { v[i] = x.v; d[i] = x.d; }
};

// ---------------------------------------------------------------- pointwise physics
// State relations (Sec. 2.1): rho = p/(R T), q^c, inviscid fluxes (Eq. convection).
template <class T>
struct Thermo {
  T rho, qc[4], f[4], g[4];
};

template <class T, class GS>
__device__ __forceinline__ void thermo(const T q[4], const GS& gs, Thermo<T>& o) {
  const T invT = inv(q[3]);
  o.rho = q[0] * invT * gs.inv_R;
  const T ru = o.rho * q[1], rv = o.rho * q[2];
  const T ke = 0.5 * (ru * q[1] + rv * q[2]);
  const T E = q[0] * gs.inv_gm1 + ke;
  const T H = E + q[0];
  o.qc[0] = o.rho; o.qc[1] = ru; o.qc[2] = rv; o.qc[3] = E;
  o.f[0] = ru; o.f[1] = ru * q[1] + q[0]; o.f[2] = ru * q[2]; o.f[3] = H * q[1];
  o.g[0] = rv; o.g[1] = o.f[2];          o.g[2] = rv * q[2] + q[0]; o.g[3] = H * q[2];
}

// Viscous fluxes (Eqs. diffusion, shear_stress), added with the FR sign: the total
// flux is f_inv - f_vis, so fv/gv here are returned as -f_vis, -g_vis.
template <class T, class GS>
__device__ __forceinline__ void neg_viscous_flux(const T q[4], const T qx[4], const T qy[4],
                                                 const GS& gs, T fv[4], T gv[4]) {
  const auto m43 = 4.0 / 3.0 * gs.mu * gs.inv_re, m23 = 2.0 / 3.0 * gs.mu * gs.inv_re;
  const auto m1 = gs.mu * gs.inv_re, kr = gs.k_cond * gs.inv_re;
  const T txx = m43 * qx[1] - m23 * qy[2];
  const T tyy = m43 * qy[2] - m23 * qx[1];
  const T txy = m1 * (qy[1] + qx[2]);
  fv[0] = from_parts<T>(0.0, 0.0);
  fv[1] = -txx;
  fv[2] = -txy;
  fv[3] = -(q[1] * txx + q[2] * txy + kr * qx[3]);
  gv[0] = from_parts<T>(0.0, 0.0);
  gv[1] = -txy;
  gv[2] = -tyy;
  gv[3] = -(q[1] * txy + q[2] * tyy + kr * qy[3]);
}

// ---------------------------------------------------------------- common face flux
// Owned-face common flux scaled by the face metric:  F^num = |S| f_n^com (Eq.
// norm_f_2 with sign(n . grad xi) = +1 on structured meshes), where the normal is
// S/|S| and S = |J| grad(xi) (or grad(eta)) on the '-' element's face.
//   inviscid (Eq. Rosanov): |S| f_n,inv = f . S - (v_g . S) q^c on each side,
//     dissipation 1/2 |lambda|max(S) Gamma~ (q+ - q-), all of eps, U_r, Gamma~ and
//     |lambda| at the averaged primitive state; |lambda| is homogeneous in S.
//   viscous (BR2, Sec. 3.1): q^com = (q+ + q-)/2, grad q^com = (grad q+ + grad q-)/2
//     + eta (r+ + r-)/2 with r-+ = (q^com - q-+) S g'(end) / |J|-+, which sum to
//     (q+ - q-) S g_R'(1) (1/|J|- + 1/|J|+) / 2; the penalty eta (BR2_PENALTY) is folded
//     into lift_end = eta g_R'(1);  |S| f_vis . n = f_vis . S.
// Inviscid part alone: fnum = |S| f_n,inv^com from qm ('-' side) and qp ('+' side); also
// returns dq = qp - qm and the averaged state qa.
template <class T, class G, class GS>
__device__ __forceinline__ void rusanov_common(const T qm[4], const T qp[4], G Sx, G Sy, G ug,
                                               G vg, const GS& gs, T dq[4], T qa[4], T fnum[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) { dq[k] = qp[k] - qm[k]; qa[k] = 0.5 * (qp[k] + qm[k]); }
  // --- normal fluxes of both sides
  T fm[4], fp[4];
  {
    Thermo<T> t;
    thermo(qm, gs, t);
    const G vgS = ug * Sx + vg * Sy;
#pragma unroll
    for (int k = 0; k < 4; ++k) fm[k] = t.f[k] * Sx + t.g[k] * Sy - vgS * t.qc[k];
    thermo(qp, gs, t);
#pragma unroll
    for (int k = 0; k < 4; ++k) fp[k] = t.f[k] * Sx + t.g[k] * Sy - vgS * t.qc[k];
  }
  // --- averaged state: eps, U_r, alpha, c', |lambda|max, Gamma~ (Eqs. theta,
  //     eigenvalues_para, eps_move)
  const T invTa = inv(qa[3]);
  const T rho = qa[0] * invTa * gs.inv_R;
  const T c2 = gs.gamma * gs.R * qa[3];
  const T wx = qa[1] - ug, wy = qa[2] - vg;
  const T w2 = wx * wx + wy * wy;
  // M_mov^2 = |v - v_g|^2 / c^2; eps = min(1, max(kappa M_inf, M_mov)), floored.
  T eps = sqrt_(w2 * inv(c2));
  eps = vmax(as_T<T>(gs.kappa_minf), eps);
  eps = vmin(from_parts<T>(1.0, 0.0), eps);
  eps = vmax(eps, as_T<T>(gs.eps_floor));
  const T ur2 = eps * eps * c2;
  const T beta = (gs.inv_R - gs.inv_cp) * invTa;     // rho_p + rho_T/(rho C_p)
  const T alpha = 0.5 * (1.0 - beta * ur2);
  const G S2 = Sx * Sx + Sy * Sy;
  const T un = wx * Sx + wy * Sy;                     // |S| u_n
  const T unp = un * (1.0 - alpha);
  const T cpr = sqrt_(alpha * alpha * un * un + ur2 * S2);
  T lmax = abs_(un);
  lmax = vmax(lmax, abs_(un));
  lmax = vmax(lmax, abs_(unp + cpr));
  lmax = vmax(lmax, abs_(unp - cpr));
  const T theta = inv(ur2) + invTa * gs.inv_cp;      // 1/U_r^2 - rho_T/(rho C_p)
  const T h = gs.cp * qa[3] + 0.5 * (qa[1] * qa[1] + qa[2] * qa[2]);
  const T rhoT = -rho * invTa;
  // Gamma~ dq with Gamma~ of Eq. preconditioning, rows arranged around d0.
  const T d0 = theta * dq[0] + rhoT * dq[3];
  const T rdu = rho * dq[1], rdv = rho * dq[2];
  T diss[4];
  diss[0] = d0;
  diss[1] = qa[1] * d0 + rdu;
  diss[2] = qa[2] * d0 + rdv;
  diss[3] = h * d0 - dq[0] + qa[1] * rdu + qa[2] * rdv + rho * gs.cp * dq[3];
  const T hl = 0.5 * lmax;
#pragma unroll
  for (int k = 0; k < 4; ++k) fnum[k] = 0.5 * (fm[k] + fp[k]) - hl * diss[k];
}

template <class T, class G, class GS>
__device__ __forceinline__ void face_common(const T qm[4], const T qp[4], const T gm[8],
                                            const T gp[8], G Sx, G Sy, G ug, G vg, G Jm, G Jp,
                                            const GS& gs, double lift_end, T fnum[4], T qcom[4]) {
  T dq[4], qa[4];
  rusanov_common(qm, qp, Sx, Sy, ug, vg, gs, dq, qa, fnum);
#pragma unroll
  for (int k = 0; k < 4; ++k) qcom[k] = qa[k];
  if (gs.viscous) {
    // (r- + r+)/2 = (q+ - q-) S g_R'(1) (1/|J|- + 1/|J|+) / 4
    const G lift = 0.25 * lift_end * (inv(Jm) + inv(Jp));
    T qx[4], qy[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const T jl = dq[k] * lift;
      qx[k] = 0.5 * (gm[k] + gp[k]) + jl * Sx;
      qy[k] = 0.5 * (gm[4 + k] + gp[4 + k]) + jl * Sy;
    }
    T fv[4], gv[4];
    neg_viscous_flux(qa, qx, qy, gs, fv, gv);
#pragma unroll
    for (int k = 0; k < 4; ++k) fnum[k] = fnum[k] + fv[k] * Sx + gv[k] * Sy;
  }
}

// Boundary face (Sec. 3.3): the boundary state qb replaces the missing neighbour, far
// field qb = q_inf, adiabatic no-slip wall qb = (p^-, v_g, T^-).  Inviscid: the
// preconditioned Rusanov flux between the trace qe and qb, the element on the '-' side
// when S points out of the domain (elem_minus), else on the '+' side.  Viscous: q^com =
// qb, grad q^com = grad qe + eta r with the full one-sided lift r = (qb - qe) S g'(end)/|J|
// (dg_end = eta g'(end) of the element's face: +eta g_R'(1) on a T face, eta g_L'(-1) on a
// B face); at a wall the component of grad T^com along S is removed (dT/dn = 0); the flux
// f_vis(qb, grad q^com) . S.  Writes fnum = |S| f_n^com along +S and qb.
// dqinf (nullable): tangent of q_inf carried by dual-number T (parameter sensitivities).
template <class T, class G, class GS>
__device__ __forceinline__ void face_boundary(const T qe[4], const T ge[8], G Sx, G Sy, G ug, G vg,
                                              G Je, const GS& gs, double dg_end, bool elem_minus,
                                              int kind, const double qinf[4], T fnum[4], T qb[4],
                                              const double* dqinf = nullptr) {
  if (kind == BC_WALL) {
    qb[0] = qe[0];
    qb[1] = as_T<T>(ug);
    qb[2] = as_T<T>(vg);
    qb[3] = qe[3];
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) qb[k] = from_parts<T>(qinf[k], dqinf ? dqinf[k] : 0.0);
  }
  T dq[4], qa[4];
  if (elem_minus) rusanov_common(qe, qb, Sx, Sy, ug, vg, gs, dq, qa, fnum);
  else rusanov_common(qb, qe, Sx, Sy, ug, vg, gs, dq, qa, fnum);
  if (gs.viscous) {
    const G lift = dg_end * inv(Je);
    T qx[4], qy[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const T jl = (qb[k] - qe[k]) * lift;
      qx[k] = ge[k] + jl * Sx;
      qy[k] = ge[4 + k] + jl * Sy;
    }
    if (kind == BC_WALL) {
      const T gn = (qx[3] * Sx + qy[3] * Sy) * inv(Sx * Sx + Sy * Sy);
      qx[3] = qx[3] - gn * Sx;
      qy[3] = qy[3] - gn * Sy;
    }
    T fv[4], gv[4];
    neg_viscous_flux(qb, qx, qy, gs, fv, gv);
#pragma unroll
    for (int k = 0; k < 4; ++k) fnum[k] = fnum[k] + fv[k] * Sx + gv[k] * Sy;
  }
}

// Four doubles passed by value to a kernel (the far-field state's tangent).
struct Vec4 {
  double v[4];
};

// ---------------------------------------------------------------- launch geometry
// Elements per block for the point-parallel kernels (one thread per solution point):
// K x floor(128 / n^2) elements, K = 1 or 2 (the tile shape, fixed or chosen per kernel
// by the autotuner; a thread performs the same operations for either K).
template <int N, int K = 1> struct Tile {
  static constexpr int NP = N * N;
  static constexpr int EPB = K * (128 / NP);
  static constexpr int THREADS = EPB * NP;
};

}  // namespace fr
