// fr_kernels.cuh -- the geometry kernel, the three point-parallel kernels of one residual
// / JVP evaluation (trace, face, elem) and the pointwise (Gamma/dtau + a0/dt M) product;
// included by every translation unit that launches them.
#pragma once
#include "fr_device.cuh"

namespace fr {

// ------------------------------------------------------------------ geometry (Sec. 2.3)
// Bilinear map through the 4 corners: |J|, S_xi = |J| grad(xi) = (y_eta, -x_eta),
// S_eta = |J| grad(eta) = (-y_xi, x_xi), v_g (bilinear in the corner velocities) and
// |J| xi_t = -v_g . S_xi, |J| eta_t = -v_g . S_eta, at solution and flux points; the
// divergence of (|J| xi_t, |J| eta_t) by the interpolant derivative.
template <class T>
struct MapPoint {
  T x_xi, x_eta, y_xi, y_eta, ug, vg;
};

template <class T>
__device__ __forceinline__ MapPoint<T> map_at(const T X[4], const T Y[4], const T VX[4],
                                              const T VY[4], double xi, double eta) {
  const double N0 = 0.25 * (1 - xi) * (1 - eta), N1 = 0.25 * (1 + xi) * (1 - eta);
  const double N2 = 0.25 * (1 + xi) * (1 + eta), N3 = 0.25 * (1 - xi) * (1 + eta);
  const double a0 = -0.25 * (1 - eta), a1 = 0.25 * (1 - eta), a2 = 0.25 * (1 + eta), a3 = -0.25 * (1 + eta);
  const double b0 = -0.25 * (1 - xi), b1 = -0.25 * (1 + xi), b2 = 0.25 * (1 + xi), b3 = 0.25 * (1 - xi);
  MapPoint<T> m;
  m.x_xi = a0 * X[0] + a1 * X[1] + a2 * X[2] + a3 * X[3];
  m.y_xi = a0 * Y[0] + a1 * Y[1] + a2 * Y[2] + a3 * Y[3];
  m.x_eta = b0 * X[0] + b1 * X[1] + b2 * X[2] + b3 * X[3];
  m.y_eta = b0 * Y[0] + b1 * Y[1] + b2 * Y[2] + b3 * Y[3];
  m.ug = N0 * VX[0] + N1 * VX[1] + N2 * VX[2] + N3 * VX[3];
  m.vg = N0 * VY[0] + N1 * VY[1] + N2 * VY[2] + N3 * VY[3];
  return m;
}

// T = double: the geometry.  T = Dual: the geometry and its tangent for the corner and
// corner-velocity tangents dcorners, dvel (the parameter-sensitivity path).
template <int N, class T = double>
__global__ void k_geometry(const double* __restrict__ corners, const double* __restrict__ vel,
                           int ne, Basis B, Buf<T> GS, Buf<T> GF,
                           const double* __restrict__ dcorners = nullptr,
                           const double* __restrict__ dvel = nullptr) {
  constexpr int NP = N * N;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  T X[4], Y[4], VX[4], VY[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const size_t i = (size_t)e * 8 + 2 * a;
    X[a] = from_parts<T>(corners[i], dcorners ? dcorners[i] : 0.0);
    Y[a] = from_parts<T>(corners[i + 1], dcorners ? dcorners[i + 1] : 0.0);
    VX[a] = from_parts<T>(vel[i], dvel ? dvel[i] : 0.0);
    VY[a] = from_parts<T>(vel[i + 1], dvel ? dvel[i + 1] : 0.0);
  }
  const size_t SN = (size_t)ne * NP;
  T stx[NP], ste[NP];
#pragma unroll
  for (int j = 0; j < N; ++j) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const MapPoint<T> m = map_at(X, Y, VX, VY, B.xs[i], B.xs[j]);
      const T J = m.x_xi * m.y_eta - m.x_eta * m.y_xi;
      const T sxx = m.y_eta, sxy = -m.x_eta, sex = -m.y_xi, sey = m.x_xi;
      const size_t o = (size_t)e * NP + j * N + i;
      GS.st(GS_SXX * SN + o, sxx);
      GS.st(GS_SXY * SN + o, sxy);
      GS.st(GS_SEX * SN + o, sex);
      GS.st(GS_SEY * SN + o, sey);
      stx[j * N + i] = -(m.ug * sxx + m.vg * sxy);
      ste[j * N + i] = -(m.ug * sex + m.vg * sey);
      GS.st(GS_STX * SN + o, stx[j * N + i]);
      GS.st(GS_STE * SN + o, ste[j * N + i]);
      GS.st(GS_INVJ * SN + o, inv(J));
      GS.st(GS_J * SN + o, J);
      GS.st(GS_UG * SN + o, m.ug);
      GS.st(GS_VG * SN + o, m.vg);
    }
  }
#pragma unroll
  for (int j = 0; j < N; ++j) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T d = from_parts<T>(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < N; ++k) d = d + (B.D[i][k] * stx[j * N + k] + B.D[j][k] * ste[k * N + i]);
      GS.st(GS_DIVST * SN + (size_t)e * NP + j * N + i, d);
    }
  }
  const size_t FN = (size_t)ne * 4 * N;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
#pragma unroll
    for (int t = 0; t < N; ++t) {
      const double xi = f == FACE_L ? -1.0 : f == FACE_R ? 1.0 : B.xs[t];
      const double eta = f == FACE_B ? -1.0 : f == FACE_T ? 1.0 : B.xs[t];
      const MapPoint<T> m = map_at(X, Y, VX, VY, xi, eta);
      const T J = m.x_xi * m.y_eta - m.x_eta * m.y_xi;
      const bool along_xi = (f == FACE_L || f == FACE_R);
      const size_t o = ((size_t)e * 4 + f) * N + t;
      GF.st(GF_SX * FN + o, along_xi ? m.y_eta : -m.y_xi);
      GF.st(GF_SY * FN + o, along_xi ? -m.x_eta : m.x_xi);
      GF.st(GF_J * FN + o, J);
      GF.st(GF_UG * FN + o, m.ug);
      GF.st(GF_VG * FN + o, m.vg);
    }
  }
}


// ------------------------------------------------------------------ topology and parameters
// Periodic structured nx-by-ny block starting at element e0 of a launch, case id cid.
static __global__ void k_fill_topo(int nx, int ny, int e0, int cid, int* __restrict__ nbr,
                            int* __restrict__ ecase) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nx * ny) return;
  const int i = l % nx, j = l / nx;
  const int g = e0 + l;
  nbr[4 * g + FACE_L] = e0 + j * nx + (i == 0 ? nx - 1 : i - 1);
  nbr[4 * g + FACE_R] = e0 + j * nx + (i == nx - 1 ? 0 : i + 1);
  nbr[4 * g + FACE_B] = e0 + (j == 0 ? ny - 1 : j - 1) * nx + i;
  nbr[4 * g + FACE_T] = e0 + (j == ny - 1 ? 0 : j + 1) * nx + i;
  ecase[g] = cid;
}

static __global__ void k_set_case(CaseParams* cp, int cid, CaseParams value) { cp[cid] = value; }

// Bounded in eta (one case from element 0): the faces below row 0 and above row ny-1
// become boundary faces of the given kinds (neighbour -kind).
static __global__ void k_mark_bounds(int nx, int ny, int below, int above, int* __restrict__ nbr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
  nbr[4 * i + FACE_B] = -below;
  nbr[4 * ((ny - 1) * nx + i) + FACE_T] = -above;
}

// ------------------------------------------------------------------ trace kernel
// q^p (and the tangent) of EPB elements staged in shared memory; each thread owns one
// solution point.  Outputs: gl[8][Ne*NP] local gradients (x comps then y comps),
// tq[Ne][4][4][N] state traces, tg[Ne][4][8][N] gradient traces.
template <class T, int N, class G = double, int K = 1>
__global__ void __launch_bounds__(Tile<N, K>::THREADS)
k_trace(Buf<T> Q, Mesh M, Basis B, const double* __restrict__ gs, Buf<T> GL, Buf<T> TQ,
        Buf<T> TG, const double* __restrict__ dgs = nullptr) {
  const int ne = M.ne;
  constexpr int NP = N * N, EPB = Tile<N, K>::EPB;
  __shared__ T sq[EPB][4][NP];
  __shared__ T sg[EPB][8][NP];
  const int le = threadIdx.x / NP, pt = threadIdx.x % NP;
  const int e = blockIdx.x * EPB + le;
  const bool live = (le < EPB) && (e < ne) && M.on(e);
  const int i = pt % N, j = pt / N;
  const size_t SN = (size_t)ne * NP;
  const size_t o = (size_t)e * NP + pt;
  if (live) {
    const size_t qo = M.qbase(e, NP) + pt, qs = M.qstride(e);
#pragma unroll
    for (int v = 0; v < 4; ++v) sq[le][v][pt] = Q.ld(v * qs + qo);
  }
  __syncthreads();
  if (M.viscous) {
    if (live) {
      const G sxx = geo<G>(gs, dgs, GS_SXX * SN + o), sxy = geo<G>(gs, dgs, GS_SXY * SN + o);
      const G sex = geo<G>(gs, dgs, GS_SEX * SN + o), sey = geo<G>(gs, dgs, GS_SEY * SN + o);
      const G ij = geo<G>(gs, dgs, GS_INVJ * SN + o);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        T dxi = B.D[i][0] * sq[le][v][j * N + 0];
        T deta = B.D[j][0] * sq[le][v][0 * N + i];
#pragma unroll
        for (int k = 1; k < N; ++k) {
          dxi = dxi + B.D[i][k] * sq[le][v][j * N + k];
          deta = deta + B.D[j][k] * sq[le][v][k * N + i];
        }
        const T gx = (sxx * dxi + sex * deta) * ij;
        const T gy = (sxy * dxi + sey * deta) * ij;
        sg[le][v][pt] = gx;
        sg[le][4 + v][pt] = gy;
        GL.st(v * SN + o, gx);
        GL.st((4 + v) * SN + o, gy);
      }
    }
    __syncthreads();
  }
  if (!live) return;
  for (int t = pt; t < 4 * N; t += NP) {
    const int f = t / N, s = t % N;
    const double* w = (f == FACE_L || f == FACE_B) ? B.lL : B.lR;
    const bool row = (f == FACE_L || f == FACE_R);  // along xi at fixed eta index s
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      T acc = w[0] * sq[le][c][row ? s * N : s];
#pragma unroll
      for (int k = 1; k < N; ++k) acc = acc + w[k] * sq[le][c][row ? s * N + k : k * N + s];
      TQ.st((((size_t)e * 4 + f) * 4 + c) * N + s, acc);
    }
    if (M.viscous) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        T acc = w[0] * sg[le][c][row ? s * N : s];
#pragma unroll
        for (int k = 1; k < N; ++k) acc = acc + w[k] * sg[le][c][row ? s * N + k : k * N + s];
        TG.st((((size_t)e * 4 + f) * 8 + c) * N + s, acc);
      }
    }
  }
}

// ------------------------------------------------------------------ face kernel
// One thread per owned flux point: xi-faces are owned by their '-' (left) element (its R
// face), eta-faces by their bottom element (its T face).  Outputs fn, qcm [Ne][2][4][N].
template <class T, int N, class G = double>
__global__ void k_face(Mesh M, Basis B, const double* __restrict__ gf, Buf<T> TQ,
                       Buf<T> TG, Buf<T> FN, Buf<T> QC, const double* __restrict__ dgf = nullptr,
                       double dmach = 0.0, Vec4 dqinf = Vec4{}) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M.ne * 2 * N) return;
  const int e = idx / (2 * N), rem = idx % (2 * N), dir = rem / N, t = rem % N;
  if (!M.on(e)) return;
  const int plus = dir == 0 ? M.right(e) : M.top(e);
  const int fm = dir == 0 ? FACE_R : FACE_T, fp = dir == 0 ? FACE_L : FACE_B;
  typename GasOf<G>::type gas = gas_for<G>(M.par(e).gas, dmach);
  const size_t FNs = (size_t)M.ne * 4 * N;
  if (plus < 0) {   // boundary face above the element (Sec. 3.3): the element is on the '-' side
    T qe[4], ge[8];
#pragma unroll
    for (int v = 0; v < 4; ++v) qe[v] = TQ.ld((((size_t)e * 4 + fm) * 4 + v) * N + t);
#pragma unroll
    for (int c = 0; c < 8; ++c)
      ge[c] = M.viscous ? TG.ld((((size_t)e * 4 + fm) * 8 + c) * N + t) : from_parts<T>(0.0, 0.0);
    const size_t om = ((size_t)e * 4 + fm) * N + t;
    T fnum[4], qb[4];
    face_boundary(qe, ge, geo<G>(gf, dgf, GF_SX * FNs + om), geo<G>(gf, dgf, GF_SY * FNs + om),
                  geo<G>(gf, dgf, GF_UG * FNs + om), geo<G>(gf, dgf, GF_VG * FNs + om),
                  geo<G>(gf, dgf, GF_J * FNs + om), gas, B.lift_end, true, -plus, M.par(e).qinf,
                  fnum, qb, dqinf.v);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const size_t oo = (((size_t)e * 2 + dir) * 4 + v) * N + t;
      FN.st(oo, fnum[v]);
      QC.st(oo, qb[v]);
    }
    return;
  }
  T qm[4], qp[4], gm[8], gp[8];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    qm[v] = TQ.ld((((size_t)e * 4 + fm) * 4 + v) * N + t);
    qp[v] = TQ.ld((((size_t)plus * 4 + fp) * 4 + v) * N + t);
  }
  if (M.viscous) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      gm[c] = TG.ld((((size_t)e * 4 + fm) * 8 + c) * N + t);
      gp[c] = TG.ld((((size_t)plus * 4 + fp) * 8 + c) * N + t);
    }
  }
  const size_t om = ((size_t)e * 4 + fm) * N + t, op = ((size_t)plus * 4 + fp) * N + t;
  T fnum[4], qcom[4];
  face_common(qm, qp, gm, gp, geo<G>(gf, dgf, GF_SX * FNs + om), geo<G>(gf, dgf, GF_SY * FNs + om),
              geo<G>(gf, dgf, GF_UG * FNs + om), geo<G>(gf, dgf, GF_VG * FNs + om),
              geo<G>(gf, dgf, GF_J * FNs + om), geo<G>(gf, dgf, GF_J * FNs + op), gas, B.lift_end,
              fnum, qcom);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const size_t oo = (((size_t)e * 2 + dir) * 4 + v) * N + t;
    FN.st(oo, fnum[v]);
    QC.st(oo, qcom[v]);
  }
}

// Boundary faces below row 0 (Sec. 3.3), which no element owns: one thread per flux
// point of the first `nrow` elements, those whose bottom neighbour is a boundary; the
// element is on the '+' side of +eta.  Outputs fb, qb [nrow][4][N].
template <class T, int N, class G = double>
__global__ void k_face_below(Mesh M, Basis B, const double* __restrict__ gf, Buf<T> TQ, Buf<T> TG,
                             Buf<T> FB, Buf<T> QB, int nrow, const double* __restrict__ dgf = nullptr,
                             double dmach = 0.0, Vec4 dqinf = Vec4{}) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nrow * N) return;
  const int e = idx / N, t = idx % N;
  const int below = M.bottom(e);
  if (below >= 0 || !M.on(e)) return;
  typename GasOf<G>::type gas = gas_for<G>(M.par(e).gas, dmach);
  const size_t FNs = (size_t)M.ne * 4 * N;
  T qe[4], ge[8];
#pragma unroll
  for (int v = 0; v < 4; ++v) qe[v] = TQ.ld((((size_t)e * 4 + FACE_B) * 4 + v) * N + t);
#pragma unroll
  for (int c = 0; c < 8; ++c)
    ge[c] = M.viscous ? TG.ld((((size_t)e * 4 + FACE_B) * 8 + c) * N + t) : from_parts<T>(0.0, 0.0);
  const size_t of = ((size_t)e * 4 + FACE_B) * N + t;
  T fnum[4], qb[4];
  face_boundary(qe, ge, geo<G>(gf, dgf, GF_SX * FNs + of), geo<G>(gf, dgf, GF_SY * FNs + of),
                geo<G>(gf, dgf, GF_UG * FNs + of), geo<G>(gf, dgf, GF_VG * FNs + of),
                geo<G>(gf, dgf, GF_J * FNs + of), gas, -B.lift_end, false, -below, M.par(e).qinf,
                fnum, qb, dqinf.v);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    FB.st(((size_t)e * 4 + v) * N + t, fnum[v]);
    QB.st(((size_t)e * 4 + v) * N + t, qb[v]);
  }
}

// ------------------------------------------------------------------ wall traction
// Weighted traction of one wall flux point (the integrand of the force of Sec. 4):
// w (t_x, t_y) with t = -(p - p_inf) n + tau . n, n = sgn S / |S| the unit normal out of
// the body (sgn = +1 below row 0, -1 above the last row), p_inf = R (rho_inf = T_inf = 1),
// tau from grad q^com of the wall (the interior local gradient ge plus the one-sided lift
// of q_b - q^e with q_b = (p^e, v_g, T^e), the component of grad T along S removed), and
// w = wq |S| (wq the Gauss weight).  T is the arithmetic type (dual numbers carry state
// or parameter tangents), G the geometry's type, GS the gas.
template <class T> __device__ __forceinline__ T div_(T a, T b) { return a * inv(b); }
__device__ __forceinline__ double div_(double a, double b) { return a / b; }

template <class T, class G, class GS>
__device__ __forceinline__ void wall_traction(const T qe[4], const T ge[8], G Sx_, G Sy_, G ug, G vg,
                                              G J, const GS& gas, double dg_end, double sgn,
                                              double wq, bool viscous, T& fx, T& fy) {
  const T Sx = as_T<T>(Sx_), Sy = as_T<T>(Sy_);
  const T qb[4] = {qe[0], as_T<T>(ug), as_T<T>(vg), qe[3]};
  const T s2 = Sx * Sx + Sy * Sy;
  const T smag = sqrt_(s2);
  const T nbx = div_(sgn * Sx, smag), nby = div_(sgn * Sy, smag);
  const T dp = qb[0] - as_T<T>(gas.R);
  T tx = -(dp * nbx), ty = -(dp * nby);
  if (viscous) {
    const T lift = div_(as_T<T>(dg_end), as_T<T>(J));
    T gx[4], gy[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const T jl = (qb[k] - qe[k]) * lift;
      gx[k] = ge[k] + jl * Sx;
      gy[k] = ge[4 + k] + jl * Sy;
    }
    const T gn = div_(gx[3] * Sx + gy[3] * Sy, s2);
    gx[3] = gx[3] - gn * Sx;
    gy[3] = gy[3] - gn * Sy;
    T fv[4], gv[4];
    neg_viscous_flux(qb, gx, gy, gas, fv, gv);   // -f_vis, -g_vis
    tx = tx - (fv[1] * nbx + gv[1] * nby);
    ty = ty - (fv[2] * nbx + gv[2] * nby);
  }
  const T w = wq * smag;
  fx = w * tx;
  fy = w * ty;
}

// Force on the wall faces (the numerator of the force coefficients of Sec. 4): the
// weighted tractions of every wall flux point (wall_traction), summed by one block:
// every thread sums a fixed set of flux points and the block sums in a fixed order
// (deterministic).  out[0..1] = (F_x, F_y); with G = Dual (geometry tangents dgf, the
// Mach tangent dmach and the traces' tangents dtq, dtg, e.g. of the local gradients under
// a moving geometry) also out[2..3] = their tangents.
template <int N, class G = double>
__global__ void __launch_bounds__(256) k_wall_force(Mesh M, Basis B, const double* __restrict__ gf,
                                                    const double* __restrict__ tq,
                                                    const double* __restrict__ tg, int nx, int ny,
                                                    int wall_below, int wall_above,
                                                    double* __restrict__ out,
                                                    const double* __restrict__ dgf = nullptr,
                                                    double dmach = 0.0,
                                                    const double* __restrict__ dtq = nullptr,
                                                    const double* __restrict__ dtg = nullptr) {
  __shared__ double red[4][256 / 32];
  typename GasOf<G>::type gas = gas_for<G>(M.par(0).gas, dmach);
  const size_t FNs = (size_t)M.ne * 4 * N;
  G fx = as_T<G>(0.0), fy = as_T<G>(0.0);
  for (int idx = threadIdx.x; idx < 2 * nx * N; idx += blockDim.x) {
    const int side = idx / (nx * N), rem = idx % (nx * N), i = rem / N, t = rem % N;
    if (side == 0 ? !wall_below : !wall_above) continue;
    const int e = side == 0 ? i : (ny - 1) * nx + i;
    const int f = side == 0 ? FACE_B : FACE_T;
    G qe[4], ge[8];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const size_t k = (((size_t)e * 4 + f) * 4 + v) * N + t;
      qe[v] = from_parts<G>(tq[k], dtq ? dtq[k] : 0.0);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const size_t k = (((size_t)e * 4 + f) * 8 + c) * N + t;
      ge[c] = M.viscous ? from_parts<G>(tg[k], dtg ? dtg[k] : 0.0) : as_T<G>(0.0);
    }
    const size_t of = ((size_t)e * 4 + f) * N + t;
    G px, py;
    wall_traction(qe, ge, geo<G>(gf, dgf, GF_SX * FNs + of), geo<G>(gf, dgf, GF_SY * FNs + of),
                  geo<G>(gf, dgf, GF_UG * FNs + of), geo<G>(gf, dgf, GF_VG * FNs + of),
                  geo<G>(gf, dgf, GF_J * FNs + of), gas, side == 0 ? -B.lift_end : B.lift_end,
                  side == 0 ? 1.0 : -1.0, B.ws[t], M.viscous, px, py);
    fx = fx + px;
    fy = fy + py;
  }
  double part[4] = {val(fx), val(fy), tan_(fx), tan_(fy)};
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part[k] += __shfl_down_sync(0xffffffffu, part[k], off);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) red[k][wid] = part[k];
  }
  __syncthreads();
  const int nout = sizeof(G) == sizeof(double) ? 2 : 4;
  if (threadIdx.x < nout) {
    double acc = 0.0;
    for (int w2 = 0; w2 < 256 / 32; ++w2) acc += red[threadIdx.x][w2];
    out[threadIdx.x] = acc;
  }
}

// ------------------------------------------------------------------ element kernel
// MODE_TAN writes only the tangent of R (the parameter-sensitivity path).
enum { MODE_RESID = 0, MODE_JVP = 1, MODE_TAN = 2 };

struct TimeTerms {           // r = R - (a0 q^c + a1 qc_n + a2 qc_nm1)/dt, coefficients per case
  const double* qcn;
  const double* qcnm1;
};

// (inv_dtau Gamma + a0_dt M) w at one point (Eqs. jacobian, preconditioning, theta),
// eps from the point's own v - v_g (Eq. eps_move).
__device__ __forceinline__ void gamma_m_apply(const double q[4], const double w[4], double ug,
                                              double vg, const Gas& gs, double inv_dtau,
                                              double a0_dt, double out[4]) {
  const double invT = 1.0 / q[3];
  const double rho = q[0] * invT * gs.inv_R;
  const double c2 = gs.gamma * gs.R * q[3];
  const double wx = q[1] - ug, wy = q[2] - vg;
  double eps = sqrt((wx * wx + wy * wy) / c2);
  eps = gs.kappa_minf >= eps ? gs.kappa_minf : eps;
  eps = 1.0 <= eps ? 1.0 : eps;
  eps = eps >= gs.eps_floor ? eps : gs.eps_floor;
  const double ur2 = eps * eps * c2;
  const double theta = 1.0 / ur2 + invT * gs.inv_cp;
  const double rho_p = invT * gs.inv_R;
  const double rhoT = -rho * invT;
  const double h = gs.cp * q[3] + 0.5 * (q[1] * q[1] + q[2] * q[2]);
  const double s = inv_dtau + a0_dt;
  const double c0 = inv_dtau * theta + a0_dt * rho_p;
  const double d0 = c0 * w[0] + s * rhoT * w[3];
  const double sr = s * rho;
  out[0] = d0;
  out[1] = q[1] * d0 + sr * w[1];
  out[2] = q[2] * d0 + sr * w[2];
  out[3] = h * d0 - s * w[0] + sr * (q[1] * w[1] + q[2] * w[2]) + sr * gs.cp * w[3];
}

template <class T, int N, int MODE, class G = double, int K = 1>
__global__ void __launch_bounds__(Tile<N, K>::THREADS)
k_elem(Buf<T> Q, Mesh M, Basis B, const double* __restrict__ gs,
       const double* __restrict__ gf, Buf<T> GL, Buf<T> TQ, Buf<T> FN, Buf<T> QC,
       double* __restrict__ out, TimeTerms tt, const double* __restrict__ dgs = nullptr,
       const double* __restrict__ dgf = nullptr, double dmach = 0.0, Buf<T> FB = Buf<T>{},
       Buf<T> QB = Buf<T>{}) {
  constexpr int NP = N * N, EPB = Tile<N, K>::EPB;
  __shared__ T sF[EPB][4][NP];
  __shared__ T sG[EPB][4][NP];
  const int le = threadIdx.x / NP, pt = threadIdx.x % NP;
  const int e = blockIdx.x * EPB + le;
  const bool live = (le < EPB) && (e < M.ne) && M.on(e);
  const int i = pt % N, j = pt / N;
  const size_t SN = (size_t)M.ne * NP;
  const size_t FNs = (size_t)M.ne * 4 * N;
  const size_t o = (size_t)e * NP + pt;
  T q[4];
  Thermo<T> th;
  G ij = from_parts<G>(0.0, 0.0);
  const CaseParams& cpar = M.par(live ? e : 0);
  typename GasOf<G>::type gas = gas_for<G>(cpar.gas, dmach);
  const size_t qo = live ? M.qbase(e, NP) + pt : 0, qs = cpar.sn;
  if (live) {
#pragma unroll
    for (int v = 0; v < 4; ++v) q[v] = Q.ld(v * qs + qo);
    thermo(q, gas, th);
    ij = geo<G>(gs, dgs, GS_INVJ * SN + o);
    T fx[4], gy[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) { fx[v] = th.f[v]; gy[v] = th.g[v]; }
    if (M.viscous) {
      T qx[4], qy[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) { qx[v] = GL.ld(v * SN + o); qy[v] = GL.ld((4 + v) * SN + o); }
      // lifted jumps of the four faces: (q^com_f - q^loc_f) S_f g_f'(.) / |J|
      const int nbL = M.left(e), nbB = M.bottom(e);
      const int qsrc[4] = {nbL, e, nbB, e};
      const int qdir[4] = {0, 0, 1, 1};
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const int s = (f < 2) ? j : i;
        const double w = (f == FACE_L) ? B.dgL[i] : (f == FACE_R) ? B.dgR[i]
                       : (f == FACE_B) ? B.dgL[j] : B.dgR[j];
        const size_t of = ((size_t)e * 4 + f) * N + s;
        const G sx = geo<G>(gf, dgf, GF_SX * FNs + of) * w * ij, sy = geo<G>(gf, dgf, GF_SY * FNs + of) * w * ij;
        // below row 0 of a bounded mesh the common state comes from the boundary buffer
        const bool bface = f == FACE_B && nbB < 0;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const T qcf = bface ? QB.ld(((size_t)e * 4 + v) * N + s)
                              : QC.ld((((size_t)qsrc[f] * 2 + qdir[f]) * 4 + v) * N + s);
          const T jump = qcf - TQ.ld((((size_t)e * 4 + f) * 4 + v) * N + s);
          qx[v] = qx[v] + jump * sx;
          qy[v] = qy[v] + jump * sy;
        }
      }
      T fv[4], gv[4];
      neg_viscous_flux(q, qx, qy, gas, fv, gv);
#pragma unroll
      for (int v = 0; v < 4; ++v) { fx[v] = fx[v] + fv[v]; gy[v] = gy[v] + gv[v]; }
    }
    const G sxx = geo<G>(gs, dgs, GS_SXX * SN + o), sxy = geo<G>(gs, dgs, GS_SXY * SN + o);
    const G sex = geo<G>(gs, dgs, GS_SEX * SN + o), sey = geo<G>(gs, dgs, GS_SEY * SN + o);
    const G stx = geo<G>(gs, dgs, GS_STX * SN + o), ste = geo<G>(gs, dgs, GS_STE * SN + o);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      sF[le][v][pt] = sxx * fx[v] + sxy * gy[v] + stx * th.qc[v];
      sG[le][v][pt] = sex * fx[v] + sey * gy[v] + ste * th.qc[v];
    }
  }
  __syncthreads();
  if (!live) return;
  const int nbL = M.left(e), nbB = M.bottom(e);
  const G divst = geo<G>(gs, dgs, GS_DIVST * SN + o);
  T R[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    T d = B.Dc[i][0] * sF[le][v][j * N + 0];
#pragma unroll
    for (int k = 1; k < N; ++k) d = d + B.Dc[i][k] * sF[le][v][j * N + k];
#pragma unroll
    for (int k = 0; k < N; ++k) d = d + B.Dc[j][k] * sG[le][v][k * N + i];
    d = d + B.dgL[i] * FN.ld((((size_t)nbL * 2 + 0) * 4 + v) * N + j);
    d = d + B.dgR[i] * FN.ld((((size_t)e * 2 + 0) * 4 + v) * N + j);
    d = d + B.dgL[j] * (nbB < 0 ? FB.ld(((size_t)e * 4 + v) * N + i)
                                : FN.ld((((size_t)nbB * 2 + 1) * 4 + v) * N + i));
    d = d + B.dgR[j] * FN.ld((((size_t)e * 2 + 1) * 4 + v) * N + i);
    d = d - th.qc[v] * divst;
    R[v] = -(d * ij);
  }
  if constexpr (MODE == MODE_RESID) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      double r = val(R[v]);
      if (tt.qcn) {
        double acc = cpar.a0dt * val(th.qc[v]) + cpar.a1dt * tt.qcn[v * qs + qo];
        if (tt.qcnm1 && cpar.a2dt != 0.0) acc += cpar.a2dt * tt.qcnm1[v * qs + qo];
        r -= acc;
      }
      out[v * qs + qo] = r;
    }
  } else if constexpr (MODE == MODE_TAN) {
#pragma unroll
    for (int v = 0; v < 4; ++v) out[v * qs + qo] = tan_(R[v]);
  } else {
    double qv[4], wv[4], gm[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) { qv[v] = val(q[v]); wv[v] = tan_(q[v]); }
    gamma_m_apply(qv, wv, gs[GS_UG * SN + o], gs[GS_VG * SN + o], gas, cpar.inv_dtau, cpar.a0_dt, gm);
#pragma unroll
    for (int v = 0; v < 4; ++v) out[v * qs + qo] = gm[v] - tan_(R[v]);
  }
}

}  // namespace fr
