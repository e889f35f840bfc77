// fr_linear.cu -- the Newton operator A = Gamma/dtau + (a0/dt) M - dR/dq^p (Eq.
// unsteady_pre_discretized_3) as a product of stored local Jacobians, applied forward
// (JVP) or transposed (VJP).
//
// R is a composition of linear maps fixed by the basis and the geometry (local
// gradients, traces, liftings, corrected divergence) and two pointwise nonlinear maps:
//   face map   Phi: (q-, q+, grad q-, grad q+) -> F^num    at each owned flux point,
//   point map  Psi: (q, corrected grad q)      -> (F, G)   at each solution point,
// plus q^c(q) in the GCL term.  fr_linearize evaluates the Jacobians of Phi and Psi at q
// by forward mode (one dual direction per input) and stores them with
// P' = Gamma/dtau + (a0/dt) M - (1/|J|) div(|J| xi_t, |J| eta_t) M at each point.  The
// state q is fixed during a GMRES solve, so the JVP then costs small mat-vecs instead
// of a dual-number residual, and the VJP is the same factors transposed, applied in
// reverse order.
#include <algorithm>
#include <cstdio>
#include "fr_internal.h"
#include "fr_kernels.cuh"

namespace fr {

// ------------------------------------------------------------------ linearisation
// Face map Jacobian at owned flux point o = (e*2 + dir)*N + t:
//   JFQ[r*8 + c][o] = d fnum_r / d (q-_c (c<4) | q+_{c-4}),
//   JFG[r*16 + c][o] = d fnum_r / d (g-_c (c<8) | g+_{c-8}).
template <int N>
__global__ void k_lin_face(Mesh M, Basis B, const double* __restrict__ gf,
                           const double* __restrict__ tq, const double* __restrict__ tg,
                           double* __restrict__ JFQ, double* __restrict__ JFG) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int nf = M.ne * 2 * N;
  if (idx >= nf) return;
  const int e = idx / (2 * N), rem = idx % (2 * N), dir = rem / N, t = rem % N;
  if (!M.on(e)) return;
  const int plus = dir == 0 ? M.right(e) : M.top(e);
  const int fm = dir == 0 ? FACE_R : FACE_T, fp = dir == 0 ? FACE_L : FACE_B;
  const Gas& gas = M.par(e).gas;
  const size_t FNs = (size_t)M.ne * 4 * N;
  if (plus < 0) {   // boundary face above the element: the boundary map's Jacobian in (q-, g-)
    const size_t om = ((size_t)e * 4 + fm) * N + t;
    double qe[4], ge[8];
#pragma unroll
    for (int v = 0; v < 4; ++v) qe[v] = tq[(((size_t)e * 4 + fm) * 4 + v) * N + t];
#pragma unroll
    for (int c = 0; c < 8; ++c) ge[c] = M.viscous ? tg[(((size_t)e * 4 + fm) * 8 + c) * N + t] : 0.0;
    const double Sx = gf[GF_SX * FNs + om], Sy = gf[GF_SY * FNs + om];
    const double ug = gf[GF_UG * FNs + om], vg = gf[GF_VG * FNs + om], Jm = gf[GF_J * FNs + om];
    const int ndir = M.viscous ? 12 : 4;
#pragma unroll 1
    for (int dd = 0; dd < ndir; ++dd) {
      Dual dq[4], dg[8], fnum[4], qb[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) dq[v] = mk(qe[v], dd == v ? 1.0 : 0.0);
#pragma unroll
      for (int c = 0; c < 8; ++c) dg[c] = mk(ge[c], dd == 4 + c ? 1.0 : 0.0);
      face_boundary(dq, dg, Sx, Sy, ug, vg, Jm, gas, B.lift_end, true, -plus, M.par(e).qinf, fnum, qb);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (dd < 4) {
          JFQ[(size_t)(r * 8 + dd) * nf + idx] = fnum[r].d;
          JFQ[(size_t)(r * 8 + 4 + dd) * nf + idx] = 0.0;
        } else {
          JFG[(size_t)(r * 16 + dd - 4) * nf + idx] = fnum[r].d;
          JFG[(size_t)(r * 16 + 8 + dd - 4) * nf + idx] = 0.0;
        }
      }
    }
    return;
  }
  double qm[4], qp[4], gm[8], gp[8];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    qm[v] = tq[(((size_t)e * 4 + fm) * 4 + v) * N + t];
    qp[v] = tq[(((size_t)plus * 4 + fp) * 4 + v) * N + t];
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    gm[c] = M.viscous ? tg[(((size_t)e * 4 + fm) * 8 + c) * N + t] : 0.0;
    gp[c] = M.viscous ? tg[(((size_t)plus * 4 + fp) * 8 + c) * N + t] : 0.0;
  }
  const size_t om = ((size_t)e * 4 + fm) * N + t, op = ((size_t)plus * 4 + fp) * N + t;
  const double Sx = gf[GF_SX * FNs + om], Sy = gf[GF_SY * FNs + om];
  const double ug = gf[GF_UG * FNs + om], vg = gf[GF_VG * FNs + om];
  const double Jm = gf[GF_J * FNs + om], Jp = gf[GF_J * FNs + op];
  const int ndir = M.viscous ? 24 : 8;
#pragma unroll 1
  for (int dd = 0; dd < ndir; ++dd) {
    Dual dqm[4], dqp[4], dgm[8], dgp[8], fnum[4], qcom[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      dqm[v] = mk(qm[v], dd == v ? 1.0 : 0.0);
      dqp[v] = mk(qp[v], dd == 4 + v ? 1.0 : 0.0);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      dgm[c] = mk(gm[c], dd == 8 + c ? 1.0 : 0.0);
      dgp[c] = mk(gp[c], dd == 16 + c ? 1.0 : 0.0);
    }
    face_common(dqm, dqp, dgm, dgp, Sx, Sy, ug, vg, Jm, Jp, gas, B.lift_end, fnum, qcom);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (dd < 8) JFQ[(size_t)(r * 8 + dd) * nf + idx] = fnum[r].d;
      else JFG[(size_t)(r * 16 + dd - 8) * nf + idx] = fnum[r].d;
    }
  }
}

// Boundary faces below row 0 of a bounded mesh (the element on the '+' side), flux point
// b = e*N + t of the first nrow elements:
//   JFQb[r*4 + c][b] = d fnum_r / d qe_c,  JFGb[r*8 + c][b] = d fnum_r / d ge_c.
template <int N>
__global__ void k_lin_face_below(Mesh M, Basis B, const double* __restrict__ gf,
                                 const double* __restrict__ tq, const double* __restrict__ tg,
                                 int nrow, double* __restrict__ JFQb, double* __restrict__ JFGb) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int nb = nrow * N;
  if (idx >= nb) return;
  const int e = idx / N, t = idx % N;
  const int below = M.bottom(e);
  if (below >= 0 || !M.on(e)) return;
  const Gas& gas = M.par(e).gas;
  const size_t FNs = (size_t)M.ne * 4 * N;
  const size_t of = ((size_t)e * 4 + FACE_B) * N + t;
  double qe[4], ge[8];
#pragma unroll
  for (int v = 0; v < 4; ++v) qe[v] = tq[(((size_t)e * 4 + FACE_B) * 4 + v) * N + t];
#pragma unroll
  for (int c = 0; c < 8; ++c) ge[c] = M.viscous ? tg[(((size_t)e * 4 + FACE_B) * 8 + c) * N + t] : 0.0;
  const double Sx = gf[GF_SX * FNs + of], Sy = gf[GF_SY * FNs + of];
  const double ug = gf[GF_UG * FNs + of], vg = gf[GF_VG * FNs + of], Je = gf[GF_J * FNs + of];
  const int ndir = M.viscous ? 12 : 4;
#pragma unroll 1
  for (int dd = 0; dd < ndir; ++dd) {
    Dual dq[4], dg[8], fnum[4], qb[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) dq[v] = mk(qe[v], dd == v ? 1.0 : 0.0);
#pragma unroll
    for (int c = 0; c < 8; ++c) dg[c] = mk(ge[c], dd == 4 + c ? 1.0 : 0.0);
    face_boundary(dq, dg, Sx, Sy, ug, vg, Je, gas, -B.lift_end, false, -below, M.par(e).qinf, fnum, qb);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (dd < 4) JFQb[(size_t)(r * 4 + dd) * nb + idx] = fnum[r].d;
      else JFGb[(size_t)(r * 8 + dd - 4) * nb + idx] = fnum[r].d;
    }
  }
}

// The common solution of a boundary face varies as D_b times the element's trace
// (Sec. 3.3: a far field fixes all of q_b; an adiabatic no-slip wall takes p and T from
// the trace and prescribes the velocity): the diagonal of D_b for variable v.
__device__ __forceinline__ double bc_pass(int kind, int v) {
  return (kind == BC_WALL && (v == 0 || v == 3)) ? 1.0 : 0.0;
}

// Point map Jacobian at solution point o = e*NP + pt:
//   JP[r*4 + c][o] = d (F_r (r<4) | G_{r-4}) / d q_c,
//   JG[r*8 + c][o] = d (F, G)_r / d (corrected grad q)_c (x comps c<4, y comps c>=4),
//   PP[r*4 + c][o] = (Gamma/dtau + a0_dt M - (1/|J|) divst M)_rc.
template <int N>
__global__ void __launch_bounds__(Tile<N>::THREADS)
k_lin_point(const double* __restrict__ q, Mesh M, Basis B, const double* __restrict__ gs,
            const double* __restrict__ gf, const double* __restrict__ gl,
            const double* __restrict__ tq, const double* __restrict__ qcm,
            const double* __restrict__ qcb, double* __restrict__ JP, double* __restrict__ JG,
            double* __restrict__ PP) {
  constexpr int NP = N * N, EPB = Tile<N>::EPB;
  const int le = threadIdx.x / NP, pt = threadIdx.x % NP;
  const int e = blockIdx.x * EPB + le;
  if (le >= EPB || e >= M.ne || !M.on(e)) return;
  const int i = pt % N, j = pt / N;
  const size_t SN = (size_t)M.ne * NP;
  const size_t FNs = (size_t)M.ne * 4 * N;
  const size_t o = (size_t)e * NP + pt;
  const CaseParams& cpar = M.par(e);
  const Gas& gas = cpar.gas;
  const double inv_dtau = cpar.inv_dtau, a0_dt = cpar.a0_dt;
  double qv[4], gc[8];
  const size_t qo = M.qbase(e, NP) + pt, qs = cpar.sn;
#pragma unroll
  for (int v = 0; v < 4; ++v) qv[v] = q[v * qs + qo];
  const double ij = gs[GS_INVJ * SN + o];
  if (M.viscous) {
#pragma unroll
    for (int c = 0; c < 8; ++c) gc[c] = gl[c * SN + o];
    const int qsrc[4] = {M.left(e), e, M.bottom(e), e};
    const int qdir[4] = {0, 0, 1, 1};
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int s = (f < 2) ? j : i;
      const double w = (f == FACE_L) ? B.dgL[i] : (f == FACE_R) ? B.dgR[i]
                     : (f == FACE_B) ? B.dgL[j] : B.dgR[j];
      const size_t of = ((size_t)e * 4 + f) * N + s;
      const double sx = gf[GF_SX * FNs + of] * w * ij, sy = gf[GF_SY * FNs + of] * w * ij;
      // below row 0 of a bounded mesh the common state comes from the boundary buffer
      const bool bface = f == FACE_B && qsrc[f] < 0;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const double qc = bface ? qcb[((size_t)e * 4 + v) * N + s]
                                : qcm[(((size_t)qsrc[f] * 2 + qdir[f]) * 4 + v) * N + s];
        const double jump = qc - tq[(((size_t)e * 4 + f) * 4 + v) * N + s];
        gc[v] += jump * sx;
        gc[4 + v] += jump * sy;
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) gc[c] = 0.0;
  }
  const double sxx = gs[GS_SXX * SN + o], sxy = gs[GS_SXY * SN + o];
  const double sex = gs[GS_SEX * SN + o], sey = gs[GS_SEY * SN + o];
  const double stx = gs[GS_STX * SN + o], ste = gs[GS_STE * SN + o];
  const int ndir = M.viscous ? 12 : 4;
#pragma unroll 1
  for (int dd = 0; dd < ndir; ++dd) {
    Dual dq[4], dx[4], dy[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      dq[v] = mk(qv[v], dd == v ? 1.0 : 0.0);
      dx[v] = mk(gc[v], dd == 4 + v ? 1.0 : 0.0);
      dy[v] = mk(gc[4 + v], dd == 8 + v ? 1.0 : 0.0);
    }
    Thermo<Dual> th;
    thermo(dq, gas, th);
    Dual fx[4], gy[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) { fx[v] = th.f[v]; gy[v] = th.g[v]; }
    if (M.viscous) {
      Dual fv[4], gv[4];
      neg_viscous_flux(dq, dx, dy, gas, fv, gv);
#pragma unroll
      for (int v = 0; v < 4; ++v) { fx[v] = fx[v] + fv[v]; gy[v] = gy[v] + gv[v]; }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const double dF = sxx * fx[v].d + sxy * gy[v].d + stx * th.qc[v].d;
      const double dG = sex * fx[v].d + sey * gy[v].d + ste * th.qc[v].d;
      if (dd < 4) {
        JP[(size_t)(v * 4 + dd) * SN + o] = dF;
        JP[(size_t)((4 + v) * 4 + dd) * SN + o] = dG;
      } else {
        JG[(size_t)(v * 8 + dd - 4) * SN + o] = dF;
        JG[(size_t)((4 + v) * 8 + dd - 4) * SN + o] = dG;
      }
    }
  }
  const double divst = gs[GS_DIVST * SN + o];
  const double ug = gs[GS_UG * SN + o], vg = gs[GS_VG * SN + o];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double w[4] = {0.0, 0.0, 0.0, 0.0}, col[4];
    w[c] = 1.0;
    gamma_m_apply(qv, w, ug, vg, gas, inv_dtau, a0_dt - ij * divst, col);
#pragma unroll
    for (int r = 0; r < 4; ++r) PP[(size_t)(r * 4 + c) * SN + o] = col[r];
  }
}

// ------------------------------------------------------------------ forward (A v)
// Owned flux point: dfnum = JFQ [dq-; dq+] + JFG [dg-; dg+],  dqcom = (dq- + dq+)/2.
template <int N>
__global__ void k_lin_face_apply(Mesh M, const double* __restrict__ tqv,
                                 const double* __restrict__ tgv, const double* __restrict__ JFQ,
                                 const double* __restrict__ JFG, double* __restrict__ fnv,
                                 double* __restrict__ qcv) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int nf = M.ne * 2 * N;
  if (idx >= nf) return;
  const int e = idx / (2 * N), rem = idx % (2 * N), dir = rem / N, t = rem % N;
  if (!M.on(e)) return;
  const int plus = dir == 0 ? M.right(e) : M.top(e);
  const int fm = dir == 0 ? FACE_R : FACE_T, fp = dir == 0 ? FACE_L : FACE_B;
  const bool bnd = plus < 0;   // boundary face above the element: no '+' side
  double x[8];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    x[v] = tqv[(((size_t)e * 4 + fm) * 4 + v) * N + t];
    x[4 + v] = bnd ? 0.0 : tqv[(((size_t)plus * 4 + fp) * 4 + v) * N + t];
  }
  double out[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s = fma(JFQ[(size_t)(r * 8 + c) * nf + idx], x[c], s);
    out[r] = s;
  }
  if (M.viscous) {
    // the viscous flux has no mass component and does not depend on the pressure
    // gradient: row 0 and the columns of p_x, p_y (c % 4 == 0) of JFG are exact zeros
    double g[16];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      g[c] = c % 4 ? tgv[(((size_t)e * 4 + fm) * 8 + c) * N + t] : 0.0;
      g[8 + c] = (c % 4 && !bnd) ? tgv[(((size_t)plus * 4 + fp) * 8 + c) * N + t] : 0.0;
    }
#pragma unroll
    for (int r = 1; r < 4; ++r) {
      double s = out[r];
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c % 4) s = fma(JFG[(size_t)(r * 16 + c) * nf + idx], g[c], s);
      out[r] = s;
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const size_t oo = (((size_t)e * 2 + dir) * 4 + v) * N + t;
    fnv[oo] = out[v];
    qcv[oo] = bnd ? bc_pass(-plus, v) * x[v] : 0.5 * (x[v] + x[4 + v]);
  }
}

// Boundary faces below row 0: dfnum = JFQb dqe + JFGb dge, dqcom = D_b dqe, into
// fbv, qbv [nrow][4][N].
template <int N>
__global__ void k_lin_face_below_apply(Mesh M, const double* __restrict__ tqv,
                                       const double* __restrict__ tgv, const double* __restrict__ JFQb,
                                       const double* __restrict__ JFGb, int nrow,
                                       double* __restrict__ fbv, double* __restrict__ qbv) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int nb = nrow * N;
  if (idx >= nb) return;
  const int e = idx / N, t = idx % N;
  const int below = M.bottom(e);
  if (below >= 0 || !M.on(e)) return;
  double x[4], out[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) x[v] = tqv[(((size_t)e * 4 + FACE_B) * 4 + v) * N + t];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) s = fma(JFQb[(size_t)(r * 4 + c) * nb + idx], x[c], s);
    out[r] = s;
  }
  if (M.viscous) {
    double g[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) g[c] = c % 4 ? tgv[(((size_t)e * 4 + FACE_B) * 8 + c) * N + t] : 0.0;
#pragma unroll
    for (int r = 1; r < 4; ++r) {
      double s = out[r];
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (c % 4) s = fma(JFGb[(size_t)(r * 8 + c) * nb + idx], g[c], s);
      out[r] = s;
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    fbv[((size_t)e * 4 + v) * N + t] = out[v];
    qbv[((size_t)e * 4 + v) * N + t] = bc_pass(-below, v) * x[v];
  }
}

// Solution point: dgc = dg + lifted jumps, d(F,G) = JP dq + JG dgc, then
// A v = P' dq + (1/|J|)(Dc dF + Dc dG + sum_f g_f' dfnum_f).
template <int N, int K = 1>
__global__ void __launch_bounds__(Tile<N, K>::THREADS)
k_lin_elem_apply(const double* __restrict__ v, Mesh M, Basis B,
                 const double* __restrict__ gs, const double* __restrict__ gf,
                 const double* __restrict__ glv, const double* __restrict__ tqv,
                 const double* __restrict__ fnv, const double* __restrict__ qcv,
                 const double* __restrict__ JP, const double* __restrict__ JG,
                 const double* __restrict__ PP, const double* __restrict__ fbv,
                 const double* __restrict__ qbv, double* __restrict__ out) {
  constexpr int NP = N * N, EPB = Tile<N, K>::EPB;
  __shared__ double sF[EPB][4][NP];
  __shared__ double sG[EPB][4][NP];
  const int le = threadIdx.x / NP, pt = threadIdx.x % NP;
  const int e = blockIdx.x * EPB + le;
  const bool live = (le < EPB) && (e < M.ne) && M.on(e);
  const int i = pt % N, j = pt / N;
  const size_t SN = (size_t)M.ne * NP;
  const size_t FNs = (size_t)M.ne * 4 * N;
  const size_t o = (size_t)e * NP + pt;
  double dq[4] = {0, 0, 0, 0}, ij = 0.0;
  const size_t qo = live ? M.qbase(e, NP) + pt : 0, qs = live ? M.qstride(e) : 0;
  if (live) {
#pragma unroll
    for (int c = 0; c < 4; ++c) dq[c] = v[c * qs + qo];
    ij = gs[GS_INVJ * SN + o];
    double fg[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < 4; ++c) s = fma(JP[(size_t)(r * 4 + c) * SN + o], dq[c], s);
      fg[r] = s;
    }
    if (M.viscous) {
      double g[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) g[c] = glv[c * SN + o];
      const int qsrc[4] = {M.left(e), e, M.bottom(e), e};
      const int qdir[4] = {0, 0, 1, 1};
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const int s = (f < 2) ? j : i;
        const double w = (f == FACE_L) ? B.dgL[i] : (f == FACE_R) ? B.dgR[i]
                       : (f == FACE_B) ? B.dgL[j] : B.dgR[j];
        const size_t of = ((size_t)e * 4 + f) * N + s;
        const double sx = gf[GF_SX * FNs + of] * w * ij, sy = gf[GF_SY * FNs + of] * w * ij;
        const bool bface = f == FACE_B && qsrc[f] < 0;   // below row 0 of a bounded mesh
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const double qc = bface ? qbv[((size_t)e * 4 + c) * N + s]
                                  : qcv[(((size_t)qsrc[f] * 2 + qdir[f]) * 4 + c) * N + s];
          const double jump = qc - tqv[(((size_t)e * 4 + f) * 4 + c) * N + s];
          g[c] += jump * sx;
          g[4 + c] += jump * sy;
        }
      }
      // rows of the mass fluxes (r = 0, 4) and columns of p_x, p_y (c = 0, 4) of JG are
      // exact zeros (no viscous mass flux, no pressure-gradient dependence)
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        if (r % 4 == 0) continue;
        double s = fg[r];
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (c % 4) s = fma(JG[(size_t)(r * 8 + c) * SN + o], g[c], s);
        fg[r] = s;
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) { sF[le][r][pt] = fg[r]; sG[le][r][pt] = fg[4 + r]; }
  }
  __syncthreads();
  if (!live) return;
  const int nbL = M.left(e), nbB = M.bottom(e);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    double d = 0.0;
#pragma unroll
    for (int k = 0; k < N; ++k) d = fma(B.Dc[i][k], sF[le][r][j * N + k], d);
#pragma unroll
    for (int k = 0; k < N; ++k) d = fma(B.Dc[j][k], sG[le][r][k * N + i], d);
    d = fma(B.dgL[i], fnv[(((size_t)nbL * 2 + 0) * 4 + r) * N + j], d);
    d = fma(B.dgR[i], fnv[(((size_t)e * 2 + 0) * 4 + r) * N + j], d);
    d = fma(B.dgL[j], nbB < 0 ? fbv[((size_t)e * 4 + r) * N + i]
                              : fnv[(((size_t)nbB * 2 + 1) * 4 + r) * N + i], d);
    d = fma(B.dgR[j], fnv[(((size_t)e * 2 + 1) * 4 + r) * N + i], d);
    double p = 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) p = fma(PP[(size_t)(r * 4 + c) * SN + o], dq[c], p);
    out[r * qs + qo] = fma(ij, d, p);
  }
}

// ------------------------------------------------------------------ transpose (A^T w)
// Element pass: s = w/|J|; adjoints of F, G (Dc^T), of the four faces' fluxes, of the
// corrected gradient, and the point-local part P'^T w + JP^T a(F,G).
//   agl[8][SN]  = JG^T a(F,G) (adjoint of the corrected = local gradient)
//   afn[e][f][4][N], aqc[e][f][4][N]: this element's contributions to the adjoints of
//   the common flux / common solution on its face f (the owning face sums two of them).
template <int N>
__global__ void __launch_bounds__(Tile<N>::THREADS)
k_lin_elem_adjoint(const double* __restrict__ w, Mesh M, Basis B,
                   const double* __restrict__ gs, const double* __restrict__ gf,
                   const double* __restrict__ JP, const double* __restrict__ JG,
                   const double* __restrict__ PP, double* __restrict__ aq,
                   double* __restrict__ agl, double* __restrict__ afn, double* __restrict__ aqc) {
  constexpr int NP = N * N, EPB = Tile<N>::EPB;
  __shared__ double ss[EPB][4][NP];
  __shared__ double sgx[EPB][4][NP];   // adjoint of the corrected gradient, x comps, times S weights later
  __shared__ double sgy[EPB][4][NP];
  const int le = threadIdx.x / NP, pt = threadIdx.x % NP;
  const int e = blockIdx.x * EPB + le;
  const bool live = (le < EPB) && (e < M.ne);
  const int i = pt % N, j = pt / N;
  const size_t SN = (size_t)M.ne * NP;
  const size_t FNs = (size_t)M.ne * 4 * N;
  const size_t o = (size_t)e * NP + pt;
  double wv[4] = {0, 0, 0, 0}, ij = 0.0;
  if (live) {
    ij = gs[GS_INVJ * SN + o];
    const size_t qo = M.qbase(e, NP) + pt, qs = M.qstride(e);
#pragma unroll
    for (int r = 0; r < 4; ++r) { wv[r] = w[r * qs + qo]; ss[le][r][pt] = wv[r] * ij; }
  }
  __syncthreads();
  if (live) {
    // adjoint of (F_r, G_r) at this point
    double aFG[8];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      double aF = 0.0, aG = 0.0;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        aF = fma(B.Dc[k][i], ss[le][r][j * N + k], aF);   // F at (i,j) enters rows (k, j)
        aG = fma(B.Dc[k][j], ss[le][r][k * N + i], aG);   // G at (i,j) enters rows (i, k)
      }
      aFG[r] = aF;
      aFG[4 + r] = aG;
    }
    // point-local part
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
#pragma unroll
      for (int r = 0; r < 4; ++r) s = fma(PP[(size_t)(r * 4 + c) * SN + o], wv[r], s);
#pragma unroll
      for (int r = 0; r < 8; ++r) s = fma(JP[(size_t)(r * 4 + c) * SN + o], aFG[r], s);
      aq[c * SN + o] = s;
    }
    if (M.viscous) {
      // JG's mass rows (r = 0, 4) and pressure-gradient columns (c = 0, 4) are exact zeros
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        double s = 0.0;
#pragma unroll
        for (int r = 0; r < 8; ++r)
          if (r % 4 && c % 4) s = fma(JG[(size_t)(r * 8 + c) * SN + o], aFG[r], s);
        agl[c * SN + o] = s;
        if (c < 4) sgx[le][c][pt] = s * ij; else sgy[le][c - 4][pt] = s * ij;
      }
    }
  }
  __syncthreads();
  if (!live) return;
  // face contributions: thread pt < 4N handles face f = pt / N, line index s = pt % N
  for (int t = pt; t < 4 * N; t += NP) {
    const int f = t / N, s = t % N;
    const bool row = (f == FACE_L || f == FACE_R);
    const double* dg = (f == FACE_L || f == FACE_B) ? B.dgL : B.dgR;
    const size_t of = ((size_t)e * 4 + f) * N + s;
    const double Sx = gf[GF_SX * FNs + of], Sy = gf[GF_SY * FNs + of];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      double a_fn = 0.0, a_qc = 0.0;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const int p2 = row ? s * N + k : k * N + s;   // points on the line of face point s
        a_fn = fma(dg[k], ss[le][r][p2], a_fn);
        if (M.viscous) a_qc = fma(dg[k], Sx * sgx[le][r][p2] + Sy * sgy[le][r][p2], a_qc);
      }
      afn[(((size_t)e * 4 + f) * 4 + r) * N + s] = a_fn;
      aqc[(((size_t)e * 4 + f) * 4 + r) * N + s] = a_qc;
    }
  }
}

// Face pass (owned flux point): sum both sides' contributions, apply the face map's
// transposed Jacobian, write the adjoints of both sides' traces.  The own-trace term of
// the lifted jump (-a_qc) is added here as well.
template <int N>
__global__ void k_lin_face_adjoint(Mesh M, const double* __restrict__ JFQ,
                                   const double* __restrict__ JFG, const double* __restrict__ afn,
                                   const double* __restrict__ aqc, double* __restrict__ atq,
                                   double* __restrict__ atg) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int nf = M.ne * 2 * N;
  if (idx >= nf) return;
  const int e = idx / (2 * N), rem = idx % (2 * N), dir = rem / N, t = rem % N;
  const int plus = dir == 0 ? M.right(e) : M.top(e);
  const int fm = dir == 0 ? FACE_R : FACE_T, fp = dir == 0 ? FACE_L : FACE_B;
  if (plus < 0) {   // boundary face above the element: q^com = D_b q-, no '+' side
    double af[4], aqe[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const size_t im = (((size_t)e * 4 + fm) * 4 + r) * N + t;
      af[r] = afn[im];
      aqe[r] = (bc_pass(-plus, r) - 1.0) * aqc[im];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double sm = aqe[c];
#pragma unroll
      for (int r = 0; r < 4; ++r) sm = fma(JFQ[(size_t)(r * 8 + c) * nf + idx], af[r], sm);
      atq[(((size_t)e * 4 + fm) * 4 + c) * N + t] = sm;
    }
    if (M.viscous) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        double sm = 0.0;
#pragma unroll
        for (int r = 1; r < 4; ++r)
          if (c % 4) sm = fma(JFG[(size_t)(r * 16 + c) * nf + idx], af[r], sm);
        atg[(((size_t)e * 4 + fm) * 8 + c) * N + t] = sm;
      }
    }
    return;
  }
  double afs[4], aqm[4], aqp[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const size_t im = (((size_t)e * 4 + fm) * 4 + r) * N + t;
    const size_t ip = (((size_t)plus * 4 + fp) * 4 + r) * N + t;
    afs[r] = afn[im] + afn[ip];
    const double aqcom = aqc[im] + aqc[ip];
    // q^com = (q- + q+)/2 enters both lifted jumps; each side's own trace enters with -1
    aqm[r] = 0.5 * aqcom - aqc[im];
    aqp[r] = 0.5 * aqcom - aqc[ip];
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double sm = aqm[c], sp = aqp[c];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      sm = fma(JFQ[(size_t)(r * 8 + c) * nf + idx], afs[r], sm);
      sp = fma(JFQ[(size_t)(r * 8 + 4 + c) * nf + idx], afs[r], sp);
    }
    atq[(((size_t)e * 4 + fm) * 4 + c) * N + t] = sm;
    atq[(((size_t)plus * 4 + fp) * 4 + c) * N + t] = sp;
  }
  if (M.viscous) {
    // JFG's mass row and pressure-gradient columns (c % 4 == 0) are exact zeros
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      double sm = 0.0, sp = 0.0;
#pragma unroll
      for (int r = 1; r < 4; ++r) {
        if (c % 4 == 0) continue;
        sm = fma(JFG[(size_t)(r * 16 + c) * nf + idx], afs[r], sm);
        sp = fma(JFG[(size_t)(r * 16 + 8 + c) * nf + idx], afs[r], sp);
      }
      atg[(((size_t)e * 4 + fm) * 8 + c) * N + t] = sm;
      atg[(((size_t)plus * 4 + fp) * 8 + c) * N + t] = sp;
    }
  }
}

// Boundary faces below row 0: the adjoints of the element's B-face trace and gradient
// trace (no other element shares the face).
template <int N>
__global__ void k_lin_face_below_adjoint(Mesh M, const double* __restrict__ JFQb,
                                         const double* __restrict__ JFGb, int nrow,
                                         const double* __restrict__ afn, const double* __restrict__ aqc,
                                         double* __restrict__ atq, double* __restrict__ atg) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int nb = nrow * N;
  if (idx >= nb) return;
  const int e = idx / N, t = idx % N;
  const int below = M.bottom(e);
  if (below >= 0) return;
  double af[4], aqe[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const size_t ib = (((size_t)e * 4 + FACE_B) * 4 + r) * N + t;
    af[r] = afn[ib];
    aqe[r] = (bc_pass(-below, r) - 1.0) * aqc[ib];
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double sm = aqe[c];
#pragma unroll
    for (int r = 0; r < 4; ++r) sm = fma(JFQb[(size_t)(r * 4 + c) * nb + idx], af[r], sm);
    atq[(((size_t)e * 4 + FACE_B) * 4 + c) * N + t] = sm;
  }
  if (M.viscous) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      double sm = 0.0;
#pragma unroll
      for (int r = 1; r < 4; ++r)
        if (c % 4) sm = fma(JFGb[(size_t)(r * 8 + c) * nb + idx], af[r], sm);
      atg[(((size_t)e * 4 + FACE_B) * 8 + c) * N + t] = sm;
    }
  }
}

// Trace pass (solution point): out = aq + l^T atq + (grad^T)(agl + l^T atg).
template <int N>
__global__ void __launch_bounds__(Tile<N>::THREADS)
k_lin_trace_adjoint(Mesh M, Basis B, const double* __restrict__ gs,
                    const double* __restrict__ aq, const double* __restrict__ agl,
                    const double* __restrict__ atq, const double* __restrict__ atg,
                    double* __restrict__ out) {
  constexpr int NP = N * N, EPB = Tile<N>::EPB;
  __shared__ double sbx[EPB][4][NP];
  __shared__ double sby[EPB][4][NP];
  const int le = threadIdx.x / NP, pt = threadIdx.x % NP;
  const int e = blockIdx.x * EPB + le;
  const bool live = (le < EPB) && (e < M.ne);
  const int i = pt % N, j = pt / N;
  const size_t SN = (size_t)M.ne * NP;
  const size_t o = (size_t)e * NP + pt;
  double acc[4] = {0, 0, 0, 0};
  // trace weights of this point on the four faces: L/R lines j (weight l(i)), B/T lines i
  const int lines[4] = {j, j, i, i};
  if (live) {
    const double wts[4] = {B.lL[i], B.lR[i], B.lL[j], B.lR[j]};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double s = aq[c * SN + o];
#pragma unroll
      for (int f = 0; f < 4; ++f) s = fma(wts[f], atq[(((size_t)e * 4 + f) * 4 + c) * N + lines[f]], s);
      acc[c] = s;
    }
    if (M.viscous) {
      const double sxx = gs[GS_SXX * SN + o], sxy = gs[GS_SXY * SN + o];
      const double sex = gs[GS_SEX * SN + o], sey = gs[GS_SEY * SN + o];
      const double ij = gs[GS_INVJ * SN + o];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        double ax = agl[c * SN + o], ay = agl[(4 + c) * SN + o];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          ax = fma(wts[f], atg[(((size_t)e * 4 + f) * 8 + c) * N + lines[f]], ax);
          ay = fma(wts[f], atg[(((size_t)e * 4 + f) * 8 + 4 + c) * N + lines[f]], ay);
        }
        // gx = (sxx dxi + sex deta) ij, gy = (sxy dxi + sey deta) ij
        sbx[le][c][pt] = (sxx * ax + sxy * ay) * ij;   // adjoint of dxi at this point
        sby[le][c][pt] = (sex * ax + sey * ay) * ij;   // adjoint of deta at this point
      }
    }
  }
  __syncthreads();
  if (!live) return;
  if (M.viscous) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double s = acc[c];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        s = fma(B.D[k][i], sbx[le][c][j * N + k], s);   // dxi at (k,j) reads q at (i,j)
        s = fma(B.D[k][j], sby[le][c][k * N + i], s);   // deta at (i,k) reads q at (i,j)
      }
      acc[c] = s;
    }
  }
  const size_t qo = M.qbase(e, NP) + pt, qs = M.qstride(e);
#pragma unroll
  for (int c = 0; c < 4; ++c) out[c * qs + qo] = acc[c];
}

}  // namespace fr

namespace frk {
using namespace fr;

template <int N>
static int linearize_n(fr_ctx* c, const double* q, cudaStream_t s) {
  constexpr int EPB = Tile<N>::EPB, TH = Tile<N>::THREADS;
  const int nblk = (c->ne + EPB - 1) / EPB;
  const bool visc = c->mesh.viscous;
  const int nf = c->ne * 2 * N;
  {
    FR_ACCOUNT(c, KK_TRACE, (double)c->ne * N * N * fr_flops_trace(N, visc), 0.0);
    FR_PROF_BEGIN(c, s);
    k_trace<double, N><<<nblk, TH, 0, s>>>(Buf<double>{const_cast<double*>(q)}, c->mesh, c->basis,
                                           c->gs, Buf<double>{c->gl}, Buf<double>{c->tq},
                                           Buf<double>{c->tg});
    FR_PROF_END(c, s, KK_TRACE);
    FR_LAUNCH_CHECK(c);
  }
  {
    FR_ACCOUNT(c, KK_FACE, (double)nf * fr_flops_face_point(visc), 0.0);
    FR_PROF_BEGIN(c, s);
    k_face<double, N><<<(nf + 127) / 128, 128, 0, s>>>(c->mesh, c->basis, c->gf,
                                                      Buf<double>{c->tq}, Buf<double>{c->tg},
                                                      Buf<double>{c->fn}, Buf<double>{c->qcm});
    FR_PROF_END(c, s, KK_FACE);
    FR_LAUNCH_CHECK(c);
  }
  const int nbf = c->bounded ? c->nx * N : 0;   // flux points of the faces below row 0
  if (nbf > 0) {
    {
      FR_PROF_BEGIN(c, s);
      k_face_below<double, N><<<(nbf + 127) / 128, 128, 0, s>>>(c->mesh, c->basis, c->gf,
                                                                Buf<double>{c->tq}, Buf<double>{c->tg},
                                                                Buf<double>{c->fnb}, Buf<double>{c->qcb},
                                                                c->nx);
      FR_PROF_END(c, s, KK_FACE);
      FR_LAUNCH_CHECK(c);
    }
    {
      FR_ACCOUNT(c, KK_LINEARIZE, (visc ? 12.0 : 4.0) * nbf * FR_JVP_FLOP_FACTOR * fr_flops_face_point(visc), 0.0);
      FR_PROF_BEGIN(c, s);
      k_lin_face_below<N><<<(nbf + 127) / 128, 128, 0, s>>>(c->mesh, c->basis, c->gf, c->tq, c->tg,
                                                            c->nx, c->JFQb, c->JFGb);
      FR_PROF_END(c, s, KK_LINEARIZE);
      FR_LAUNCH_CHECK(c);
    }
  }
  {
    FR_ACCOUNT(c, KK_LINEARIZE, (visc ? 24.0 : 8.0) * nf * FR_JVP_FLOP_FACTOR * fr_flops_face_point(visc), 0.0);
    FR_PROF_BEGIN(c, s);
    k_lin_face<N><<<(nf + 127) / 128, 128, 0, s>>>(c->mesh, c->basis, c->gf, c->tq, c->tg,
                                                   c->JFQ, c->JFG);
    FR_PROF_END(c, s, KK_LINEARIZE);
    FR_LAUNCH_CHECK(c);
  }
  {
    FR_ACCOUNT(c, KK_LINEARIZE, (double)c->ne * N * N * (visc ? 12.0 : 4.0) * FR_JVP_FLOP_FACTOR * 95.0, 0.0);
    FR_PROF_BEGIN(c, s);
    k_lin_point<N><<<nblk, TH, 0, s>>>(q, c->mesh, c->basis, c->gs, c->gf, c->gl, c->tq,
                                       c->qcm, c->qcb, c->JP, c->JG, c->PP);
    FR_PROF_END(c, s, KK_LINEARIZE);
    FR_LAUNCH_CHECK(c);
  }
  c->lin_ready = 1;
  return FR_OK;
}

template <int N>
static int apply_n(fr_ctx* c, const double* v, double* out, bool transpose, cudaStream_t s) {
  constexpr int EPB = Tile<N>::EPB, TH = Tile<N>::THREADS;
  const int nblk = (c->ne + EPB - 1) / EPB;
  const int nf = c->ne * 2 * N;
  const int nbf = c->bounded ? c->nx * N : 0;   // flux points of the faces below row 0
  const bool visc = c->mesh.viscous;
  const double np = (double)c->ne * N * N;
  // algorithmic flops of the linear operator per solution point and per owned flux point
  const double fl_trace = fr_flops_trace(N, visc);
  // (the gradient Jacobians' non-zero part: 3 x 12 at a face point, 6 x 6 at a point)
  const double fl_face = 2.0 * (4 * 8 + (visc ? 3 * 12 : 0)) + 8.0;
  const double fl_elem = 2.0 * (8 * 4 + (visc ? 6 * 6 : 0)) + (visc ? 96.0 : 0.0) +
                         4.0 * (4.0 * N + 8.0 + 8.0 + 2.0);
  if (!transpose) {
    {
      FR_ACCOUNT(c, KK_LIN_APPLY, np * fl_trace, 0.0);
      FR_PROF_BEGIN(c, s);
      if (c->tile.trace == 2)
        k_trace<double, N, double, 2><<<(c->ne + Tile<N, 2>::EPB - 1) / Tile<N, 2>::EPB,
                                        Tile<N, 2>::THREADS, 0, s>>>(
            Buf<double>{const_cast<double*>(v)}, c->mesh, c->basis, c->gs, Buf<double>{c->gl_d},
            Buf<double>{c->tq_d}, Buf<double>{c->tg_d});
      else
        k_trace<double, N><<<nblk, TH, 0, s>>>(Buf<double>{const_cast<double*>(v)}, c->mesh, c->basis,
                                               c->gs, Buf<double>{c->gl_d}, Buf<double>{c->tq_d},
                                               Buf<double>{c->tg_d});
      FR_PROF_END(c, s, KK_LIN_APPLY);
      FR_LAUNCH_CHECK(c);
    }
    {
      FR_ACCOUNT(c, KK_LIN_APPLY, nf * fl_face, 0.0);
      FR_PROF_BEGIN(c, s);
      k_lin_face_apply<N><<<(nf + 127) / 128, 128, 0, s>>>(c->mesh, c->tq_d, c->tg_d, c->JFQ,
                                                           c->JFG, c->fn_d, c->qcm_d);
      FR_PROF_END(c, s, KK_LIN_APPLY);
      FR_LAUNCH_CHECK(c);
    }
    if (nbf > 0) {
      FR_ACCOUNT(c, KK_LIN_APPLY, nbf * fl_face, 0.0);
      FR_PROF_BEGIN(c, s);
      k_lin_face_below_apply<N><<<(nbf + 127) / 128, 128, 0, s>>>(c->mesh, c->tq_d, c->tg_d, c->JFQb,
                                                                  c->JFGb, c->nx, c->fnb_d, c->qcb_d);
      FR_PROF_END(c, s, KK_LIN_APPLY);
      FR_LAUNCH_CHECK(c);
    }
    {
      FR_ACCOUNT(c, KK_LIN_APPLY, np * fl_elem, 0.0);
      FR_PROF_BEGIN(c, s);
      if (c->tile.lin_elem == 2)
        k_lin_elem_apply<N, 2><<<(c->ne + Tile<N, 2>::EPB - 1) / Tile<N, 2>::EPB, Tile<N, 2>::THREADS,
                                 0, s>>>(v, c->mesh, c->basis, c->gs, c->gf, c->gl_d, c->tq_d,
                                         c->fn_d, c->qcm_d, c->JP, c->JG, c->PP, c->fnb_d,
                                         c->qcb_d, out);
      else
        k_lin_elem_apply<N><<<nblk, TH, 0, s>>>(v, c->mesh, c->basis, c->gs, c->gf, c->gl_d,
                                                c->tq_d, c->fn_d, c->qcm_d, c->JP, c->JG, c->PP,
                                                c->fnb_d, c->qcb_d, out);
      FR_PROF_END(c, s, KK_LIN_APPLY);
      FR_LAUNCH_CHECK(c);
    }
  } else {
    {
      FR_ACCOUNT(c, KK_LIN_ADJOINT, np * fl_elem, 0.0);
      FR_PROF_BEGIN(c, s);
      k_lin_elem_adjoint<N><<<nblk, TH, 0, s>>>(v, c->mesh, c->basis, c->gs, c->gf, c->JP,
                                                c->JG, c->PP, c->adj_q, c->gl_d, c->adj_fn, c->adj_qc);
      FR_PROF_END(c, s, KK_LIN_ADJOINT);
      FR_LAUNCH_CHECK(c);
    }
    {
      FR_ACCOUNT(c, KK_LIN_ADJOINT, nf * fl_face, 0.0);
      FR_PROF_BEGIN(c, s);
      k_lin_face_adjoint<N><<<(nf + 127) / 128, 128, 0, s>>>(c->mesh, c->JFQ, c->JFG, c->adj_fn,
                                                             c->adj_qc, c->tq_d, c->tg_d);
      FR_PROF_END(c, s, KK_LIN_ADJOINT);
      FR_LAUNCH_CHECK(c);
    }
    if (nbf > 0) {
      FR_ACCOUNT(c, KK_LIN_ADJOINT, nbf * fl_face, 0.0);
      FR_PROF_BEGIN(c, s);
      k_lin_face_below_adjoint<N><<<(nbf + 127) / 128, 128, 0, s>>>(c->mesh, c->JFQb, c->JFGb, c->nx,
                                                                    c->adj_fn, c->adj_qc, c->tq_d, c->tg_d);
      FR_PROF_END(c, s, KK_LIN_ADJOINT);
      FR_LAUNCH_CHECK(c);
    }
    {
      FR_ACCOUNT(c, KK_LIN_ADJOINT, np * fl_trace, 0.0);
      FR_PROF_BEGIN(c, s);
      k_lin_trace_adjoint<N><<<nblk, TH, 0, s>>>(c->mesh, c->basis, c->gs, c->adj_q, c->gl_d,
                                                 c->tq_d, c->tg_d, out);
      FR_PROF_END(c, s, KK_LIN_ADJOINT);
      FR_LAUNCH_CHECK(c);
    }
  }
  return FR_OK;
}

int linearize(fr_ctx* c, const double* q, double inv_dtau, double a0_dt, cudaStream_t s) {
  // the point-local block P' reads Gamma/dtau and a0/dt from the case parameters
  const int rc = set_operator_terms(c, inv_dtau, a0_dt, s);
  if (rc != FR_OK) return rc;
  switch (c->n) {
    case 2: return linearize_n<2>(c, q, s);
    case 3: return linearize_n<3>(c, q, s);
    case 4: return linearize_n<4>(c, q, s);
    case 5: return linearize_n<5>(c, q, s);
  }
  return FR_ERR_ARG;
}

template <int N>
static int trace_adjoint_n(fr_ctx* c, double* out, cudaStream_t s) {
  constexpr int EPB = Tile<N>::EPB, TH = Tile<N>::THREADS;
  const int nblk = (c->ne + EPB - 1) / EPB;
  FR_ACCOUNT(c, KK_LIN_ADJOINT, (double)c->ne * N * N * fr_flops_trace(N, c->mesh.viscous), 0.0);
  FR_PROF_BEGIN(c, s);
  k_lin_trace_adjoint<N><<<nblk, TH, 0, s>>>(c->mesh, c->basis, c->gs, c->adj_q, c->gl_d, c->tq_d,
                                             c->tg_d, out);
  FR_PROF_END(c, s, KK_LIN_ADJOINT);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

int trace_adjoint(fr_ctx* c, double* out, cudaStream_t s) {
  switch (c->n) {
    case 2: return trace_adjoint_n<2>(c, out, s);
    case 3: return trace_adjoint_n<3>(c, out, s);
    case 4: return trace_adjoint_n<4>(c, out, s);
    case 5: return trace_adjoint_n<5>(c, out, s);
  }
  return FR_ERR_ARG;
}

int apply_linear(fr_ctx* c, const double* v, double* out, bool transpose, cudaStream_t s) {
  if (!c->lin_ready) { snprintf(c->err, sizeof(c->err), "no linearisation stored"); return FR_ERR_ARG; }
  switch (c->n) {
    case 2: return apply_n<2>(c, v, out, transpose, s);
    case 3: return apply_n<3>(c, v, out, transpose, s);
    case 4: return apply_n<4>(c, v, out, transpose, s);
    case 5: return apply_n<5>(c, v, out, transpose, s);
  }
  return FR_ERR_ARG;
}

}  // namespace frk

// ------------------------------------------------------------------ tile-shape autotuner
namespace frk {
using namespace fr;

static __global__ void k_fill(double* __restrict__ p, size_t n, double v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// Median device time of 5 launches of fn after one untimed launch (stream 0, set-up).
template <class F>
static int time_launches(fr_ctx* c, F fn, float* ms) {
  cudaEvent_t ev[6];
  for (auto& e : ev) FR_CUDA_CHECK(c, cudaEventCreate(&e));
  fn();
  FR_CUDA_CHECK(c, cudaGetLastError());
  for (int k = 0; k < 5; ++k) {
    FR_CUDA_CHECK(c, cudaEventRecord(ev[k], 0));
    fn();
  }
  FR_CUDA_CHECK(c, cudaEventRecord(ev[5], 0));
  FR_CUDA_CHECK(c, cudaGetLastError());
  FR_CUDA_CHECK(c, cudaEventSynchronize(ev[5]));
  float t[5];
  for (int k = 0; k < 5; ++k) FR_CUDA_CHECK(c, cudaEventElapsedTime(&t[k], ev[k], ev[k + 1]));
  std::sort(t, t + 5);
  *ms = t[2];
  for (auto& e : ev) cudaEventDestroy(e);
  return FR_OK;
}

// Picks K in {1, 2} for each point-parallel kernel by timing both on this context's own
// sizes and buffers (filled with finite placeholder values; every one of them is
// rewritten before its first real use).  The shapes agree to rounding.
template <int N>
static int autotune_n(fr_ctx* c) {
  const int nb1 = (c->ne + Tile<N, 1>::EPB - 1) / Tile<N, 1>::EPB;
  const int nb2 = (c->ne + Tile<N, 2>::EPB - 1) / Tile<N, 2>::EPB;
  constexpr int T1 = Tile<N, 1>::THREADS, T2 = Tile<N, 2>::THREADS;
  const size_t SN = (size_t)c->ne * c->np2, FNn = (size_t)c->ne * 4 * c->n;
  struct Fill { double* p; size_t n; double v; };
  const Fill fills[] = {{c->gs, GS_COUNT * SN, 1.0}, {c->gf, GF_COUNT * FNn, 1.0}, {c->w_r, c->ndof, 1.0},
                        {c->w_z, c->ndof, 0.5}, {c->JP, 32 * SN, 0.1}, {c->JG, 64 * SN, 0.1},
                        {c->PP, 16 * SN, 0.1}, {c->gl, 8 * SN, 0.1}, {c->gl_d, 8 * SN, 0.1},
                        {c->tq, c->ne * 16 * (size_t)c->n, 1.0}, {c->tq_d, c->ne * 16 * (size_t)c->n, 0.1},
                        {c->fn, c->ne * 8 * (size_t)c->n, 0.1}, {c->fn_d, c->ne * 8 * (size_t)c->n, 0.1},
                        {c->qcm, c->ne * 8 * (size_t)c->n, 1.0}, {c->qcm_d, c->ne * 8 * (size_t)c->n, 0.1}};
  for (const Fill& f : fills) k_fill<<<1024, 256>>>(f.p, f.n, f.v);
  FR_CUDA_CHECK(c, cudaGetLastError());
  const Basis& B = c->basis;
  const Mesh& M = c->mesh;
  const Buf<double> Q{c->w_r}, GL{c->gl}, TQ{c->tq}, TG{c->tg}, FN{c->fn}, QC{c->qcm};
  const Buf<Dual> QD{c->w_r, c->w_z}, GLD{c->gl, c->gl_d}, TQD{c->tq, c->tq_d}, TGD{c->tg, c->tg_d};
  const Buf<Dual> FND{c->fn, c->fn_d}, QCD{c->qcm, c->qcm_d};
  const TimeTerms tt{nullptr, nullptr};
  float a = 0.f, b = 0.f;
  auto pick = [&](int* slot) { *slot = b < a ? 2 : 1; };
  FR_TRY(time_launches(c, [&] { k_trace<double, N><<<nb1, T1>>>(Q, M, B, c->gs, GL, TQ, TG); }, &a));
  FR_TRY(time_launches(c, [&] { k_trace<double, N, double, 2><<<nb2, T2>>>(Q, M, B, c->gs, GL, TQ, TG); }, &b));
  pick(&c->tile.trace);
  FR_TRY(time_launches(c, [&] { k_elem<double, N, MODE_RESID><<<nb1, T1>>>(Q, M, B, c->gs, c->gf, GL, TQ, FN, QC, c->w_t, tt); }, &a));
  FR_TRY(time_launches(c, [&] { k_elem<double, N, MODE_RESID, double, 2><<<nb2, T2>>>(Q, M, B, c->gs, c->gf, GL, TQ, FN, QC, c->w_t, tt); }, &b));
  pick(&c->tile.elem);
  FR_TRY(time_launches(c, [&] { k_trace<Dual, N><<<nb1, T1>>>(QD, M, B, c->gs, GLD, TQD, TGD); }, &a));
  FR_TRY(time_launches(c, [&] { k_trace<Dual, N, double, 2><<<nb2, T2>>>(QD, M, B, c->gs, GLD, TQD, TGD); }, &b));
  pick(&c->tile.trace_d);
  FR_TRY(time_launches(c, [&] { k_elem<Dual, N, MODE_JVP><<<nb1, T1>>>(QD, M, B, c->gs, c->gf, GLD, TQD, FND, QCD, c->w_t, tt); }, &a));
  FR_TRY(time_launches(c, [&] { k_elem<Dual, N, MODE_JVP, double, 2><<<nb2, T2>>>(QD, M, B, c->gs, c->gf, GLD, TQD, FND, QCD, c->w_t, tt); }, &b));
  pick(&c->tile.elem_d);
  FR_TRY(time_launches(c, [&] { k_lin_elem_apply<N><<<nb1, T1>>>(c->w_r, M, B, c->gs, c->gf, c->gl_d, c->tq_d, c->fn_d, c->qcm_d, c->JP, c->JG, c->PP, c->fnb_d, c->qcb_d, c->w_t); }, &a));
  FR_TRY(time_launches(c, [&] { k_lin_elem_apply<N, 2><<<nb2, T2>>>(c->w_r, M, B, c->gs, c->gf, c->gl_d, c->tq_d, c->fn_d, c->qcm_d, c->JP, c->JG, c->PP, c->fnb_d, c->qcb_d, c->w_t); }, &b));
  pick(&c->tile.lin_elem);
  FR_CUDA_CHECK(c, cudaDeviceSynchronize());
  return FR_OK;
}

int autotune_tiles(fr_ctx* c) {
  const int forced = c->cfg.tiles;
  if (forced == 1 || forced == 2) {
    c->tile.trace = c->tile.elem = c->tile.trace_d = c->tile.elem_d = c->tile.lin_elem = forced;
    return FR_OK;
  }
  switch (c->n) {
    case 2: return autotune_n<2>(c);
    case 3: return autotune_n<3>(c);
    case 4: return autotune_n<4>(c);
    case 5: return autotune_n<5>(c);
  }
  return FR_ERR_ARG;
}

}  // namespace frk
