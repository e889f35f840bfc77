// fr_residual.cu -- geometry, residual R(q^p) and its exact forward-mode Jacobian action
// (Wang & Yu, arXiv 1903.06304, Secs. 2.3, 3.1, 3.2) for sm_103a.
//
// One residual evaluation is three launches:
//   trace  (one thread per solution point): local physical gradients by the chain rule
//          and the values of the degree-p interpolants at the 4n flux points;
//   face   (one thread per owned flux point): common flux F^num = |S| f_n^com and q^com,
//          computed once per face and shared by both elements;
//   elem   (one thread per solution point): corrected gradient, viscous flux,
//          computational fluxes F, G, corrected divergence, GCL term, R (optionally the
//          BDF pseudo-step right-hand side, or the Newton operator A v).
// The JVP runs the same kernels with T = Dual (value + tangent).
#include <cstdio>
#include "fr_internal.h"
#include "fr_kernels.cuh"

namespace fr {

// ------------------------------------------------------------------ geometry (Sec. 2.3)
// Bilinear map through the 4 corners: |J|, S_xi = |J| grad(xi) = (y_eta, -x_eta),
// S_eta = |J| grad(eta) = (-y_xi, x_xi), v_g (bilinear in the corner velocities) and
// |J| xi_t = -v_g . S_xi, |J| eta_t = -v_g . S_eta, at solution and flux points; the
// divergence of (|J| xi_t, |J| eta_t) by the interpolant derivative.
struct MapPoint {
  double x_xi, x_eta, y_xi, y_eta, ug, vg;
};

__device__ __forceinline__ MapPoint map_at(const double X[4], const double Y[4],
                                           const double VX[4], const double VY[4], double xi,
                                           double eta) {
  const double N0 = 0.25 * (1 - xi) * (1 - eta), N1 = 0.25 * (1 + xi) * (1 - eta);
  const double N2 = 0.25 * (1 + xi) * (1 + eta), N3 = 0.25 * (1 - xi) * (1 + eta);
  const double a0 = -0.25 * (1 - eta), a1 = 0.25 * (1 - eta), a2 = 0.25 * (1 + eta), a3 = -0.25 * (1 + eta);
  const double b0 = -0.25 * (1 - xi), b1 = -0.25 * (1 + xi), b2 = 0.25 * (1 + xi), b3 = 0.25 * (1 - xi);
  MapPoint m;
  m.x_xi = a0 * X[0] + a1 * X[1] + a2 * X[2] + a3 * X[3];
  m.y_xi = a0 * Y[0] + a1 * Y[1] + a2 * Y[2] + a3 * Y[3];
  m.x_eta = b0 * X[0] + b1 * X[1] + b2 * X[2] + b3 * X[3];
  m.y_eta = b0 * Y[0] + b1 * Y[1] + b2 * Y[2] + b3 * Y[3];
  m.ug = N0 * VX[0] + N1 * VX[1] + N2 * VX[2] + N3 * VX[3];
  m.vg = N0 * VY[0] + N1 * VY[1] + N2 * VY[2] + N3 * VY[3];
  return m;
}

template <int N>
__global__ void k_geometry(const double* __restrict__ corners, const double* __restrict__ vel,
                           int ne, Basis B, double* __restrict__ gs, double* __restrict__ gf) {
  constexpr int NP = N * N;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double X[4], Y[4], VX[4], VY[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    X[a] = corners[e * 8 + 2 * a];
    Y[a] = corners[e * 8 + 2 * a + 1];
    VX[a] = vel[e * 8 + 2 * a];
    VY[a] = vel[e * 8 + 2 * a + 1];
  }
  const size_t SN = (size_t)ne * NP;
  double stx[NP], ste[NP];
#pragma unroll
  for (int j = 0; j < N; ++j) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const MapPoint m = map_at(X, Y, VX, VY, B.xs[i], B.xs[j]);
      const double J = m.x_xi * m.y_eta - m.x_eta * m.y_xi;
      const double sxx = m.y_eta, sxy = -m.x_eta, sex = -m.y_xi, sey = m.x_xi;
      const size_t o = (size_t)e * NP + j * N + i;
      gs[GS_SXX * SN + o] = sxx;
      gs[GS_SXY * SN + o] = sxy;
      gs[GS_SEX * SN + o] = sex;
      gs[GS_SEY * SN + o] = sey;
      stx[j * N + i] = -(m.ug * sxx + m.vg * sxy);
      ste[j * N + i] = -(m.ug * sex + m.vg * sey);
      gs[GS_STX * SN + o] = stx[j * N + i];
      gs[GS_STE * SN + o] = ste[j * N + i];
      gs[GS_INVJ * SN + o] = 1.0 / J;
      gs[GS_J * SN + o] = J;
      gs[GS_UG * SN + o] = m.ug;
      gs[GS_VG * SN + o] = m.vg;
    }
  }
#pragma unroll
  for (int j = 0; j < N; ++j) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double d = 0.0;
#pragma unroll
      for (int k = 0; k < N; ++k) d += B.D[i][k] * stx[j * N + k] + B.D[j][k] * ste[k * N + i];
      gs[GS_DIVST * SN + (size_t)e * NP + j * N + i] = d;
    }
  }
  const size_t FN = (size_t)ne * 4 * N;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
#pragma unroll
    for (int t = 0; t < N; ++t) {
      const double xi = f == FACE_L ? -1.0 : f == FACE_R ? 1.0 : B.xs[t];
      const double eta = f == FACE_B ? -1.0 : f == FACE_T ? 1.0 : B.xs[t];
      const MapPoint m = map_at(X, Y, VX, VY, xi, eta);
      const double J = m.x_xi * m.y_eta - m.x_eta * m.y_xi;
      const bool along_xi = (f == FACE_L || f == FACE_R);
      const size_t o = ((size_t)e * 4 + f) * N + t;
      gf[GF_SX * FN + o] = along_xi ? m.y_eta : -m.y_xi;
      gf[GF_SY * FN + o] = along_xi ? -m.x_eta : m.x_xi;
      gf[GF_J * FN + o] = J;
      gf[GF_UG * FN + o] = m.ug;
      gf[GF_VG * FN + o] = m.vg;
    }
  }
}

__global__ void k_conservative(const double* __restrict__ q, size_t SN, Gas gas,
                               double* __restrict__ qc) {
  const size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (o >= SN) return;
  double qq[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) qq[v] = q[v * SN + o];
  Thermo<double> th;
  thermo(qq, gas, th);
#pragma unroll
  for (int v = 0; v < 4; ++v) qc[v * SN + o] = th.qc[v];
}

// ------------------------------------------------------------------ launchers
template <class T, int N, int MODE>
static int run_pipeline(fr_ctx* c, Buf<T> Q, Buf<T> GL, Buf<T> TQ, Buf<T> TG, Buf<T> FNb,
                        Buf<T> QCb, double* out, TimeTerms tt, JvpTerms jt, cudaStream_t s) {
  constexpr int EPB = Tile<N>::EPB, TH = Tile<N>::THREADS;
  constexpr bool jvp = MODE == MODE_JVP;
  const int nblk = (c->ne + EPB - 1) / EPB;
  const bool visc = c->gas.viscous;
  const double pts = (double)c->ne * N * N, fac = jvp ? FR_JVP_FLOP_FACTOR : 1.0;
  FR_ACCOUNT(c, jvp ? KK_TRACE_JVP : KK_TRACE, fac * pts * fr_flops_trace(N, visc), 0.0);
  FR_ACCOUNT(c, jvp ? KK_FACE_JVP : KK_FACE, fac * 2.0 * c->ne * N * fr_flops_face_point(visc), 0.0);
  FR_ACCOUNT(c, jvp ? KK_ELEM_JVP : KK_ELEM, fac * pts * fr_flops_elem(N, visc), 0.0);
  {
    FR_PROF_BEGIN(c, s);
    k_trace<T, N><<<nblk, TH, 0, s>>>(Q, c->ne, c->basis, c->gas, c->gs, GL, TQ, TG);
    FR_PROF_END(c, s, jvp ? KK_TRACE_JVP : KK_TRACE);
    FR_LAUNCH_CHECK(c);
  }
  {
    const int nf = c->ne * 2 * N;
    FR_PROF_BEGIN(c, s);
    k_face<T, N><<<(nf + 127) / 128, 128, 0, s>>>(c->mesh, c->basis, c->gas, c->gf, TQ, TG, FNb, QCb);
    FR_PROF_END(c, s, jvp ? KK_FACE_JVP : KK_FACE);
    FR_LAUNCH_CHECK(c);
  }
  {
    FR_PROF_BEGIN(c, s);
    k_elem<T, N, MODE><<<nblk, TH, 0, s>>>(Q, c->mesh, c->basis, c->gas, c->gs, c->gf, GL, TQ, FNb,
                                           QCb, out, tt, jt);
    FR_PROF_END(c, s, jvp ? KK_ELEM_JVP : KK_ELEM);
    FR_LAUNCH_CHECK(c);
  }
  return FR_OK;
}

template <int N>
static int residual_n(fr_ctx* c, const double* q, double* out, TimeTerms tt, cudaStream_t s) {
  Buf<double> Q{const_cast<double*>(q)};
  return run_pipeline<double, N, MODE_RESID>(c, Q, Buf<double>{c->gl}, Buf<double>{c->tq},
                                             Buf<double>{c->tg}, Buf<double>{c->fn},
                                             Buf<double>{c->qcm}, out, tt, JvpTerms{0, 0}, s);
}

template <int N>
static int jvp_n(fr_ctx* c, const double* q, const double* v, double* out, JvpTerms jt,
                 cudaStream_t s) {
  Buf<Dual> Q{const_cast<double*>(q), const_cast<double*>(v)};
  TimeTerms tt{nullptr, nullptr, 0, 0, 0};
  return run_pipeline<Dual, N, MODE_JVP>(c, Q, Buf<Dual>{c->gl, c->gl_d}, Buf<Dual>{c->tq, c->tq_d},
                                         Buf<Dual>{c->tg, c->tg_d}, Buf<Dual>{c->fn, c->fn_d},
                                         Buf<Dual>{c->qcm, c->qcm_d}, out, tt, jt, s);
}

}  // namespace fr

// ------------------------------------------------------------------ flop counts
// Itemised in the design notes: thermo 19, viscous flux 18, face common flux 12 (jumps
// and means) + 81 (two normal fluxes) + 80 (preconditioned dissipation) + 75 (BR2 and
// viscous flux), element point 19 + 122 (corrected gradient, viscous flux) + 40 (F, G) +
// 4 (4n + 10) (corrected divergence, GCL term, 1/|J|).
double fr_flops_trace(int n, bool viscous) {
  const double grad = viscous ? 16.0 * n + 24.0 : 0.0;
  return grad + 4.0 * n * (viscous ? 12.0 : 4.0) * (2.0 * n - 1.0) / (n * n);
}
double fr_flops_face_point(bool viscous) { return 12.0 + 81.0 + 80.0 + (viscous ? 75.0 : 0.0); }
double fr_flops_elem(int n, bool viscous) {
  return 19.0 + (viscous ? 122.0 : 0.0) + 40.0 + 4.0 * (4.0 * n + 10.0);
}
// A dual product costs 4 flops (value product, tangent product, fused tangent sum), a
// dual sum 2, a dual by a constant 2: over the kernels' mix of operations the JVP does
// about 3x the flops of the residual.
const double FR_JVP_FLOP_FACTOR = 3.0;

namespace frk {
using namespace fr;

int geometry(fr_ctx* c, const double* corners, const double* vel, cudaStream_t s) {
  const int th = 64, nb = (c->ne + th - 1) / th;
  FR_PROF_BEGIN(c, s);
  switch (c->n) {
    case 2: k_geometry<2><<<nb, th, 0, s>>>(corners, vel, c->ne, c->basis, c->gs, c->gf); break;
    case 3: k_geometry<3><<<nb, th, 0, s>>>(corners, vel, c->ne, c->basis, c->gs, c->gf); break;
    case 4: k_geometry<4><<<nb, th, 0, s>>>(corners, vel, c->ne, c->basis, c->gs, c->gf); break;
    case 5: k_geometry<5><<<nb, th, 0, s>>>(corners, vel, c->ne, c->basis, c->gs, c->gf); break;
    default: return FR_ERR_ARG;
  }
  FR_PROF_END(c, s, KK_GEOM);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

int residual(fr_ctx* c, const double* q, double* out, const double* qcn, const double* qcnm1,
             double a0dt, double a1dt, double a2dt, cudaStream_t s) {
  TimeTerms tt{qcn, qcnm1, a0dt, a1dt, a2dt};
  switch (c->n) {
    case 2: return residual_n<2>(c, q, out, tt, s);
    case 3: return residual_n<3>(c, q, out, tt, s);
    case 4: return residual_n<4>(c, q, out, tt, s);
    case 5: return residual_n<5>(c, q, out, tt, s);
  }
  return FR_ERR_ARG;
}

int jvp(fr_ctx* c, const double* q, const double* v, double inv_dtau, double a0_dt, double* out,
        cudaStream_t s) {
  JvpTerms jt{inv_dtau, a0_dt};
  switch (c->n) {
    case 2: return jvp_n<2>(c, q, v, out, jt, s);
    case 3: return jvp_n<3>(c, q, v, out, jt, s);
    case 4: return jvp_n<4>(c, q, v, out, jt, s);
    case 5: return jvp_n<5>(c, q, v, out, jt, s);
  }
  return FR_ERR_ARG;
}

int conservative(fr_ctx* c, const double* q, double* qc, cudaStream_t s) {
  const size_t SN = (size_t)c->ne * c->np2;
  FR_ACCOUNT(c, KK_CONS, 0.0, 8.0 * 8.0 * SN);
  FR_PROF_BEGIN(c, s);
  k_conservative<<<(unsigned)((SN + 255) / 256), 256, 0, s>>>(q, SN, c->gas, qc);
  FR_PROF_END(c, s, KK_CONS);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

}  // namespace frk
