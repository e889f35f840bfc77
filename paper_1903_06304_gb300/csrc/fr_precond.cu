// fr_precond.cu -- element block-Jacobi preconditioner for the Newton operator
//   A = Gamma/dtau + (a0/dt) M - dR/dq^p        (Eq. unsteady_pre_discretized_3)
// Build:  B_e = Gamma_e/dtau + (a0/dt) M_e - dR_e/dq_e  (neighbour states frozen), exact:
//         from the stored local Jacobians (default) or by dual-number forward mode; one
//         CTA per element, 8 columns in flight.
// Factor: power-of-two row/column equilibration, in-place Gauss-Jordan inversion with
//         partial pivoting in FP64 or FP32; stored transposed, scaled, in FP64, FP32 or
//         BF16 (the FP32 inverse rounded).
// Apply:  z_e = Dc (B~_e^-1 (Dr r_e)), FP64 in/out; FP32/BF16 inverses applied with
//         double-float accumulation on the FP32 pipe (default) or in plain FP32.
#include <algorithm>
#include <type_traits>
#include <cstdio>
#include <cuda_bf16.h>
#include "fr_internal.h"
#include "fr_kernels.cuh"
#include "fr_df.cuh"

namespace fr {

constexpr int BG = 8;  // tangent directions processed concurrently per element

// Dynamic shared memory of one direction group (all Dual).
template <int N> struct BlkSmem {
  static constexpr int NP = N * N;
  static constexpr int Q = 0, GLs = Q + 4 * NP, TQs = GLs + 8 * NP, TGs = TQs + 16 * N,
                       FNs = TGs + 32 * N, QCs = FNs + 16 * N, Fs = QCs + 16 * N,
                       Gs = Fs + 4 * NP, SIZE = Gs + 4 * NP;
};

template <int N>
__global__ void __launch_bounds__(BG * N * N)
k_block(const double* __restrict__ q, Mesh M, Basis B, const double* __restrict__ gs,
        const double* __restrict__ gf, const double* __restrict__ tqv,
        const double* __restrict__ tgv, double* __restrict__ Bout) {
  constexpr int NP = N * N, BS = 4 * NP;
  using L = BlkSmem<N>;
  extern __shared__ Dual smem_dual[];
  const int e = blockIdx.x;
  if (!M.on(e)) return;
  const int grp = threadIdx.x / NP, pt = threadIdx.x % NP;
  const int i = pt % N, j = pt / N;
  Dual* S = smem_dual + grp * L::SIZE;
  Dual* sq = S + L::Q;     // [4][NP]
  Dual* sg = S + L::GLs;   // [8][NP]
  Dual* stq = S + L::TQs;  // [4 faces][4][N]
  Dual* stg = S + L::TGs;  // [4 faces][8][N]
  Dual* sfn = S + L::FNs;  // [4 faces][4][N]
  Dual* sqc = S + L::QCs;  // [4 faces][4][N]
  Dual* sF = S + L::Fs;    // [4][NP]
  Dual* sG = S + L::Gs;    // [4][NP]
  const size_t SN = (size_t)M.ne * NP;
  const size_t FNs = (size_t)M.ne * 4 * N;
  const size_t o = (size_t)e * NP + pt;
  const int nbL = M.left(e), nbR = M.right(e), nbB = M.bottom(e), nbT = M.top(e);
  const CaseParams& cpar = M.par(e);
  const Gas& gas = cpar.gas;
  const double inv_dtau = cpar.inv_dtau, a0_dt = cpar.a0_dt;
  double qv[4];
  const size_t qo = M.qbase(e, NP) + pt, qs = cpar.sn;
#pragma unroll
  for (int v = 0; v < 4; ++v) qv[v] = q[v * qs + qo];
  const double sxx = gs[GS_SXX * SN + o], sxy = gs[GS_SXY * SN + o];
  const double sex = gs[GS_SEX * SN + o], sey = gs[GS_SEY * SN + o];
  const double stx = gs[GS_STX * SN + o], ste = gs[GS_STE * SN + o];
  const double ij = gs[GS_INVJ * SN + o], divst = gs[GS_DIVST * SN + o];
  const double ugp = gs[GS_UG * SN + o], vgp = gs[GS_VG * SN + o];

  for (int d0 = 0; d0 < BS; d0 += BG) {
    const int d = d0 + grp;
    const bool act = d < BS;
    // A: seeded state
#pragma unroll
    for (int v = 0; v < 4; ++v) sq[v * NP + pt] = mk(qv[v], (v * NP + pt == d) ? 1.0 : 0.0);
    __syncthreads();
    // B: local gradients
    if (M.viscous) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        Dual dxi = B.D[i][0] * sq[v * NP + j * N];
        Dual deta = B.D[j][0] * sq[v * NP + i];
#pragma unroll
        for (int k = 1; k < N; ++k) {
          dxi = dxi + B.D[i][k] * sq[v * NP + j * N + k];
          deta = deta + B.D[j][k] * sq[v * NP + k * N + i];
        }
        sg[v * NP + pt] = (sxx * dxi + sex * deta) * ij;
        sg[(4 + v) * NP + pt] = (sxy * dxi + sey * deta) * ij;
      }
    }
    __syncthreads();
    // C: own traces
    for (int t = pt; t < 4 * N; t += NP) {
      const int f = t / N, s = t % N;
      const double* w = (f == FACE_L || f == FACE_B) ? B.lL : B.lR;
      const bool row = (f == FACE_L || f == FACE_R);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        Dual acc = w[0] * sq[c * NP + (row ? s * N : s)];
#pragma unroll
        for (int k = 1; k < N; ++k) acc = acc + w[k] * sq[c * NP + (row ? s * N + k : k * N + s)];
        stq[(f * 4 + c) * N + s] = acc;
      }
      if (M.viscous) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          Dual acc = w[0] * sg[c * NP + (row ? s * N : s)];
#pragma unroll
          for (int k = 1; k < N; ++k) acc = acc + w[k] * sg[c * NP + (row ? s * N + k : k * N + s)];
          stg[(f * 8 + c) * N + s] = acc;
        }
      }
    }
    __syncthreads();
    // D: common fluxes on the 4 faces of e, neighbour traces frozen (tangent 0); the
    //    geometry is that of the owning ('-') element, as in the residual.
    for (int t = pt; t < 4 * N; t += NP) {
      const int f = t / N, s = t % N;
      const int nb_f = f == FACE_L ? nbL : f == FACE_R ? nbR : f == FACE_B ? nbB : nbT;
      if (nb_f < 0) {   // boundary face (Sec. 3.3): a function of e's own trace alone
        Dual qe[4], ge[8];
#pragma unroll
        for (int v = 0; v < 4; ++v) qe[v] = stq[(f * 4 + v) * N + s];
#pragma unroll
        for (int c = 0; c < 8; ++c) ge[c] = M.viscous ? stg[(f * 8 + c) * N + s] : mk(0.0, 0.0);
        const size_t of = ((size_t)e * 4 + f) * N + s;
        Dual fnum[4], qb[4];
        face_boundary(qe, ge, gf[GF_SX * FNs + of], gf[GF_SY * FNs + of], gf[GF_UG * FNs + of],
                      gf[GF_VG * FNs + of], gf[GF_J * FNs + of], gas,
                      f == FACE_T ? B.lift_end : -B.lift_end, f == FACE_T, -nb_f, cpar.qinf, fnum, qb);
#pragma unroll
        for (int v = 0; v < 4; ++v) { sfn[(f * 4 + v) * N + s] = fnum[v]; sqc[(f * 4 + v) * N + s] = qb[v]; }
        continue;
      }
      Dual qm[4], qp[4], gm[8], gp[8];
      int own_m;           // element owning the face (its R or T face)
      int fo, fother, other;
      if (f == FACE_R || f == FACE_T) { own_m = e; fo = f; other = (f == FACE_R) ? nbR : nbT; fother = (f == FACE_R) ? FACE_L : FACE_B; }
      else { own_m = (f == FACE_L) ? nbL : nbB; fo = (f == FACE_L) ? FACE_R : FACE_T; other = e; fother = f; }
      const bool e_minus = (own_m == e) && (f == FACE_R || f == FACE_T);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const Dual mine = stq[(f * 4 + v) * N + s];
        const Dual theirs = e_minus ? mk(tqv[(((size_t)other * 4 + fother) * 4 + v) * N + s], 0.0)
                                    : mk(tqv[(((size_t)own_m * 4 + fo) * 4 + v) * N + s], 0.0);
        qm[v] = e_minus ? mine : theirs;
        qp[v] = e_minus ? theirs : mine;
      }
      if (M.viscous) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const Dual mine = stg[(f * 8 + c) * N + s];
          const Dual theirs = e_minus ? mk(tgv[(((size_t)other * 4 + fother) * 8 + c) * N + s], 0.0)
                                      : mk(tgv[(((size_t)own_m * 4 + fo) * 8 + c) * N + s], 0.0);
          gm[c] = e_minus ? mine : theirs;
          gp[c] = e_minus ? theirs : mine;
        }
      }
      const size_t om = ((size_t)own_m * 4 + fo) * N + s;
      const size_t op = ((size_t)other * 4 + fother) * N + s;
      Dual fnum[4], qcom[4];
      face_common(qm, qp, gm, gp, gf[GF_SX * FNs + om], gf[GF_SY * FNs + om], gf[GF_UG * FNs + om],
                  gf[GF_VG * FNs + om], gf[GF_J * FNs + om], gf[GF_J * FNs + op], gas, B.lift_end,
                  fnum, qcom);
#pragma unroll
      for (int v = 0; v < 4; ++v) { sfn[(f * 4 + v) * N + s] = fnum[v]; sqc[(f * 4 + v) * N + s] = qcom[v]; }
    }
    __syncthreads();
    // E: element part at each solution point
    Dual qd[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) qd[v] = sq[v * NP + pt];
    Thermo<Dual> th;
    thermo(qd, gas, th);
    Dual fx[4], gy[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) { fx[v] = th.f[v]; gy[v] = th.g[v]; }
    if (M.viscous) {
      Dual qx[4], qy[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) { qx[v] = sg[v * NP + pt]; qy[v] = sg[(4 + v) * NP + pt]; }
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const int s = (f < 2) ? j : i;
        const double w = (f == FACE_L) ? B.dgL[i] : (f == FACE_R) ? B.dgR[i]
                       : (f == FACE_B) ? B.dgL[j] : B.dgR[j];
        const size_t of = ((size_t)e * 4 + f) * N + s;
        const double sx = gf[GF_SX * FNs + of] * w * ij, sy = gf[GF_SY * FNs + of] * w * ij;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const Dual jump = sqc[(f * 4 + v) * N + s] - stq[(f * 4 + v) * N + s];
          qx[v] = qx[v] + jump * sx;
          qy[v] = qy[v] + jump * sy;
        }
      }
      Dual fv[4], gv[4];
      neg_viscous_flux(qd, qx, qy, gas, fv, gv);
#pragma unroll
      for (int v = 0; v < 4; ++v) { fx[v] = fx[v] + fv[v]; gy[v] = gy[v] + gv[v]; }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      sF[v * NP + pt] = sxx * fx[v] + sxy * gy[v] + stx * th.qc[v];
      sG[v * NP + pt] = sex * fx[v] + sey * gy[v] + ste * th.qc[v];
    }
    __syncthreads();
    if (act) {
      double wt[4], gmv[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) wt[v] = qd[v].d;
      gamma_m_apply(qv, wt, ugp, vgp, gas, inv_dtau, a0_dt, gmv);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        Dual dv = B.Dc[i][0] * sF[v * NP + j * N];
#pragma unroll
        for (int k = 1; k < N; ++k) dv = dv + B.Dc[i][k] * sF[v * NP + j * N + k];
#pragma unroll
        for (int k = 0; k < N; ++k) dv = dv + B.Dc[j][k] * sG[v * NP + k * N + i];
        dv = dv + B.dgL[i] * sfn[(FACE_L * 4 + v) * N + j];
        dv = dv + B.dgR[i] * sfn[(FACE_R * 4 + v) * N + j];
        dv = dv + B.dgL[j] * sfn[(FACE_B * 4 + v) * N + i];
        dv = dv + B.dgR[j] * sfn[(FACE_T * 4 + v) * N + i];
        dv = dv - th.qc[v] * divst;
        const double dR = -(dv.d * ij);
        Bout[((size_t)e * BS + v * NP + pt) * BS + d] = gmv[v] - dR;
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ blocks from the linearisation
// B_e from the stored local Jacobians (fr_linearize): the linearised operator restricted
// to element e with the neighbours' inputs zero, one unit column at a time:
//   traces and local gradient of the unit vector -> face fluxes through e's side of the
//   face Jacobians (columns of q-/g- on e's R, T faces, of q+/g+ on its L, B faces), half
//   of e's trace in the common solution -> corrected gradient -> point Jacobians ->
//   corrected divergence plus the point block P'.
// The element's face and point Jacobians are staged once in shared memory; BG columns
// are in flight, one group of n^2 threads each.
template <int N> struct BlkLinSmem {
  static constexpr int NP = N * N;
  static constexpr int JF = 4 * N * 48;   // [face][s][16 q-entries (r,c) | 32 g-entries (r,c)]
  static constexpr int JPT = 112 * NP;    // [JP 32 | JG 64 | PP 16][point]
  static constexpr int Q = 0, GL = Q + 4 * NP, TQ = GL + 8 * NP, TG = TQ + 16 * N,
                       FN = TG + 32 * N, F = FN + 16 * N, G = F + 4 * NP, SIZE = G + 4 * NP;
  static constexpr size_t BYTES = sizeof(double) * (JF + JPT + (size_t)BG * SIZE);
};

template <int N>
__global__ void __launch_bounds__(BG * N * N)
k_block_lin(Mesh M, Basis B, const double* __restrict__ gs, const double* __restrict__ gf,
            const double* __restrict__ JFQ, const double* __restrict__ JFG,
            const double* __restrict__ JP, const double* __restrict__ JG,
            const double* __restrict__ PP, const double* __restrict__ JFQb,
            const double* __restrict__ JFGb, int nbf, double* __restrict__ Bout) {
  constexpr int NP = N * N, BS = 4 * NP;
  using L = BlkLinSmem<N>;
  extern __shared__ double smd[];
  const int e = blockIdx.x;
  if (!M.on(e)) return;
  const int grp = threadIdx.x / NP, pt = threadIdx.x % NP;
  const int i = pt % N, j = pt / N;
  double* sJF = smd;
  double* sJP = smd + L::JF;
  double* S = smd + L::JF + L::JPT + grp * L::SIZE;
  double* sq = S + L::Q;
  double* sg = S + L::GL;
  double* stq = S + L::TQ;
  double* stg = S + L::TG;
  double* sfn = S + L::FN;
  double* sF = S + L::F;
  double* sG = S + L::G;
  const int nf = M.ne * 2 * N;
  const size_t SN = (size_t)M.ne * NP, FNs = (size_t)M.ne * 4 * N;
  const size_t o = (size_t)e * NP + pt;
  const bool visc = M.viscous;
  // stage this element's side of its four faces' Jacobians and its point Jacobians
  for (int t = threadIdx.x; t < L::JF; t += blockDim.x) {
    const int f = t / (N * 48), rem = t % (N * 48), sp = rem / 48, k = rem % 48;
    const bool minus = (f == FACE_R || f == FACE_T);     // e owns its R and T faces
    const int owner = f == FACE_R || f == FACE_T ? e : f == FACE_L ? M.left(e) : M.bottom(e);
    const int dir = (f == FACE_R || f == FACE_L) ? 0 : 1;
    double val;
    if (owner < 0) {   // boundary face below row 0 of a bounded mesh: e's own trace
      const size_t ib = (size_t)e * N + sp;
      if (k < 16) val = JFQb[(size_t)k * nbf + ib];
      else val = visc ? JFGb[(size_t)(k - 16) * nbf + ib] : 0.0;
      sJF[t] = val;
      continue;
    }
    const size_t idx = ((size_t)owner * 2 + dir) * N + sp;
    if (k < 16) {
      const int r = k / 4, cc = k % 4;
      val = JFQ[(size_t)(r * 8 + (minus ? cc : 4 + cc)) * nf + idx];
    } else {
      const int r = (k - 16) / 8, cc = (k - 16) % 8;
      val = visc ? JFG[(size_t)(r * 16 + (minus ? cc : 8 + cc)) * nf + idx] : 0.0;
    }
    sJF[t] = val;
  }
  for (int t = threadIdx.x; t < L::JPT; t += blockDim.x) {
    const int r = t / NP, pp = t % NP;
    const size_t oo = (size_t)e * NP + pp;
    sJP[t] = r < 32 ? JP[(size_t)r * SN + oo]
           : r < 96 ? (visc ? JG[(size_t)(r - 32) * SN + oo] : 0.0)
                    : PP[(size_t)(r - 96) * SN + oo];
  }
  const double sxx = gs[GS_SXX * SN + o], sxy = gs[GS_SXY * SN + o];
  const double sex = gs[GS_SEX * SN + o], sey = gs[GS_SEY * SN + o];
  const double ij = gs[GS_INVJ * SN + o];
  // lifting weights of the four faces at this point: S_f g_f' / |J|
  double lsx[4], lsy[4];
  // share of e's trace in each face's common solution: 1/2 inside, D_b on a boundary face
  double cs[4][4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int nbf_ = f == FACE_L ? M.left(e) : f == FACE_R ? M.right(e)
                   : f == FACE_B ? M.bottom(e) : M.top(e);
#pragma unroll
    for (int v = 0; v < 4; ++v)
      cs[f][v] = nbf_ >= 0 ? 0.5 : ((-nbf_ == BC_WALL && (v == 0 || v == 3)) ? 1.0 : 0.0);
  }
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int sp = (f < 2) ? j : i;
    const double w = (f == FACE_L) ? B.dgL[i] : (f == FACE_R) ? B.dgR[i]
                   : (f == FACE_B) ? B.dgL[j] : B.dgR[j];
    const size_t of = ((size_t)e * 4 + f) * N + sp;
    lsx[f] = gf[GF_SX * FNs + of] * w * ij;
    lsy[f] = gf[GF_SY * FNs + of] * w * ij;
  }
  __syncthreads();
  for (int d0 = 0; d0 < BS; d0 += BG) {
    const int d = d0 + grp;
    const bool act = d < BS;
    // A: unit column
#pragma unroll
    for (int v = 0; v < 4; ++v) sq[v * NP + pt] = (act && v * NP + pt == d) ? 1.0 : 0.0;
    __syncthreads();
    // B: local gradient
    if (visc) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double dxi = 0.0, deta = 0.0;
#pragma unroll
        for (int k = 0; k < N; ++k) {
          dxi = fma(B.D[i][k], sq[v * NP + j * N + k], dxi);
          deta = fma(B.D[j][k], sq[v * NP + k * N + i], deta);
        }
        sg[v * NP + pt] = (sxx * dxi + sex * deta) * ij;
        sg[(4 + v) * NP + pt] = (sxy * dxi + sey * deta) * ij;
      }
    }
    __syncthreads();
    // C: traces of the column and of its gradient
    for (int t = pt; t < 4 * N; t += NP) {
      const int f = t / N, sp = t % N;
      const double* w = (f == FACE_L || f == FACE_B) ? B.lL : B.lR;
      const bool row = (f == FACE_L || f == FACE_R);
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < N; ++k) acc = fma(w[k], sq[cc * NP + (row ? sp * N + k : k * N + sp)], acc);
        stq[(f * 4 + cc) * N + sp] = acc;
      }
      if (visc) {
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) {
          double acc = 0.0;
#pragma unroll
          for (int k = 0; k < N; ++k) acc = fma(w[k], sg[cc * NP + (row ? sp * N + k : k * N + sp)], acc);
          stg[(f * 8 + cc) * N + sp] = acc;
        }
      }
    }
    __syncthreads();
    // D: face fluxes through e's side of the face Jacobians
    for (int t = pt; t < 4 * N; t += NP) {
      const int f = t / N, sp = t % N;
      const double* jf = sJF + (f * N + sp) * 48;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        double acc = 0.0;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) acc = fma(jf[r * 4 + cc], stq[(f * 4 + cc) * N + sp], acc);
        if (visc && r > 0) {   // exact zeros: mass row, pressure-gradient columns
#pragma unroll
          for (int cc = 0; cc < 8; ++cc)
            if (cc % 4) acc = fma(jf[16 + r * 8 + cc], stg[(f * 8 + cc) * N + sp], acc);
        }
        sfn[(f * 4 + r) * N + sp] = acc;
      }
    }
    __syncthreads();
    // E: corrected gradient (the common solution holds the share cs of e's trace), point
    // fluxes
    double dq[4], g[8];
#pragma unroll
    for (int v = 0; v < 4; ++v) dq[v] = sq[v * NP + pt];
    double fg[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      double acc = 0.0;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) acc = fma(sJP[(r * 4 + cc) * NP + pt], dq[cc], acc);
      fg[r] = acc;
    }
    if (visc) {
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) g[cc] = sg[cc * NP + pt];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const int sp = (f < 2) ? j : i;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const double jump = (cs[f][v] - 1.0) * stq[(f * 4 + v) * N + sp];
          g[v] = fma(jump, lsx[f], g[v]);
          g[4 + v] = fma(jump, lsy[f], g[4 + v]);
        }
      }
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        if (r % 4 == 0) continue;   // exact zeros: mass rows, pressure-gradient columns
        double acc = fg[r];
#pragma unroll
        for (int cc = 0; cc < 8; ++cc)
          if (cc % 4) acc = fma(sJP[(32 + r * 8 + cc) * NP + pt], g[cc], acc);
        fg[r] = acc;
      }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) { sF[v * NP + pt] = fg[v]; sG[v * NP + pt] = fg[4 + v]; }
    __syncthreads();
    // F: corrected divergence, point block, one block entry per row
    if (act) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double dv = 0.0;
#pragma unroll
        for (int k = 0; k < N; ++k) dv = fma(B.Dc[i][k], sF[v * NP + j * N + k], dv);
#pragma unroll
        for (int k = 0; k < N; ++k) dv = fma(B.Dc[j][k], sG[v * NP + k * N + i], dv);
        dv = fma(B.dgL[i], sfn[(FACE_L * 4 + v) * N + j], dv);
        dv = fma(B.dgR[i], sfn[(FACE_R * 4 + v) * N + j], dv);
        dv = fma(B.dgL[j], sfn[(FACE_B * 4 + v) * N + i], dv);
        dv = fma(B.dgR[j], sfn[(FACE_T * 4 + v) * N + i], dv);
        double pv = 0.0;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) pv = fma(sJP[(96 + v * 4 + cc) * NP + pt], dq[cc], pv);
        Bout[((size_t)e * BS + v * NP + pt) * BS + d] = fma(ij, dv, pv);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ factor
template <class W> __device__ __forceinline__ W wabs(W x) { return x < 0 ? -x : x; }

// In-place Gauss-Jordan inversion with partial (row) pivoting of the equilibrated block,
// one CTA per element; writes the transposed scaled inverse and the scales.
template <class W, class S, int N>
__global__ void k_factor(const double* __restrict__ Bin, S* __restrict__ Aout,
                         float* __restrict__ Dr, float* __restrict__ Dc, int* __restrict__ info,
                         Mesh M) {
  constexpr int BS = 4 * N * N, LDA = BS + 1;       // padded rows: conflict-free columns
  extern __shared__ unsigned char smraw[];
  W* A = reinterpret_cast<W*>(smraw);               // [BS][LDA] row-major
  W* col = A + BS * LDA;                            // [BS]
  float* dr = reinterpret_cast<float*>(col + BS);   // [BS]
  float* dc = dr + BS;                              // [BS]
  int* perm = reinterpret_cast<int*>(dc + BS);      // [BS]
  __shared__ int s_piv;
  __shared__ int s_bad;
  const int e = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  if (!M.on(e)) return;
  const double* Be = Bin + (size_t)e * BS * BS;
  if (tid == 0) s_bad = 0;
  // stage the block in the working precision (coalesced); the power-of-two scales below
  // are exact in either precision
  for (int idx = tid; idx < BS * BS; idx += nt) A[(idx / BS) * LDA + idx % BS] = (W)Be[idx];
  __syncthreads();
  // row scales 2^-e with e the exponent of the row's largest |entry|: a warp per row
  for (int r = wid; r < BS; r += nw) {
    W m = 0;
    for (int c2 = lane; c2 < BS; c2 += 32) m = fmax(m, wabs(A[r * LDA + c2]));
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) {
      int ex = 0;
      if (m > (W)0) frexp(m, &ex);
      dr[r] = m > (W)0 ? ldexpf(1.0f, -ex) : 1.0f;
    }
  }
  __syncthreads();
  // column scales of the row-scaled block: a warp per column
  for (int c2 = wid; c2 < BS; c2 += nw) {
    W m = 0;
    for (int r = lane; r < BS; r += 32) m = fmax(m, wabs(A[r * LDA + c2]) * (W)dr[r]);
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) {
      int ex = 0;
      if (m > (W)0) frexp(m, &ex);
      dc[c2] = m > (W)0 ? ldexpf(1.0f, -ex) : 1.0f;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < BS * BS; idx += nt) {
    const int r = idx / BS, c2 = idx % BS;
    A[r * LDA + c2] = A[r * LDA + c2] * (W)dr[r] * (W)dc[c2];
  }
  __syncthreads();
  for (int k = 0; k < BS; ++k) {
    if (tid < 32) {  // pivot search in column k, rows k..BS-1 (first max wins)
      W best = (W)-1;
      int bi = k;
      for (int r = k + tid; r < BS; r += 32) {
        const W a = wabs(A[r * LDA + k]);
        if (a > best) { best = a; bi = r; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const W ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) { s_piv = bi; perm[k] = bi; if (best == (W)0) s_bad = 1; }
    }
    __syncthreads();
    const int pr = s_piv;
    if (pr != k)
      for (int c2 = tid; c2 < BS; c2 += nt) { const W t = A[k * LDA + c2]; A[k * LDA + c2] = A[pr * LDA + c2]; A[pr * LDA + c2] = t; }
    __syncthreads();
    const W piv = A[k * LDA + k];
    const W rp = piv != (W)0 ? (W)1 / piv : (W)0;
    for (int r = tid; r < BS; r += nt) col[r] = A[r * LDA + k];
    __syncthreads();
    for (int c2 = tid; c2 < BS; c2 += nt) A[k * LDA + c2] = (c2 == k ? (W)1 : A[k * LDA + c2]) * rp;
    __syncthreads();
    for (int idx = tid; idx < BS * BS; idx += nt) {
      const int r = idx / BS, c2 = idx % BS;
      if (r == k) continue;
      const W f = col[r];
      const W akc = A[k * LDA + c2];
      A[r * LDA + c2] = (c2 == k ? (W)0 : A[r * LDA + c2]) - f * akc;
    }
    __syncthreads();
  }
  // undo the column interchanges in reverse order
  for (int k = BS - 1; k >= 0; --k) {
    const int pr = perm[k];
    if (pr != k)
      for (int r = tid; r < BS; r += nt) { const W t = A[r * LDA + k]; A[r * LDA + k] = A[r * LDA + pr]; A[r * LDA + pr] = t; }
    __syncthreads();
  }
  // inverse of Dr B Dc is A; store A transposed: Aout[col][row]
  S* Ae = Aout + (size_t)e * BS * BS;
  for (int idx = tid; idx < BS * BS; idx += nt) {
    const int c2 = idx / BS, r = idx % BS;   // coalesced store of the transpose
    Ae[idx] = (S)A[r * LDA + c2];
  }
  for (int r = tid; r < BS; r += nt) { Dr[(size_t)e * BS + r] = dr[r]; Dc[(size_t)e * BS + r] = dc[r]; }
  if (tid == 0) info[e] = s_bad;
}

// ------------------------------------------------------------------ factor on the tensor cores
// Blocked Gauss-Jordan inversion of the equilibrated block on the augmented matrix
// M = [A | I] (FP32 in shared memory, BP = the block size rounded up to 16, the padding an
// identity), panel width 16: the panel's pivots and its elimination run on the FP32 SIMT
// pipe (the panel columns only), then every row of M right of the panel receives the
// rank-16 update M += U M[panel rows] on the tensor cores (mma.sync m16n8k16, BF16
// operands, FP32 accumulation), U the panel's multipliers.  SPLIT = 1 rounds U and the
// panel rows to BF16 once (about 2^-9 relative per update); SPLIT = 3 writes each as a
// sum of two BF16 numbers and accumulates hi*hi + hi*lo + lo*hi (about 2^-16).  The result
// is stored like k_factor's: the transposed inverse of Dr B Dc and the scales.
constexpr int TC_THREADS = 128;
template <int N> struct TcDims {
  static constexpr int BS = 4 * N * N;
  static constexpr int BP = (BS + 15) / 16 * 16;   // padded block size
  static constexpr int LDM = 2 * BP + 4;           // FP32 row stride of M (shifts banks by 4)
  static constexpr int LDW = 33;                   // panel workspace stride (16 + 16 columns)
  static constexpr size_t BYTES = sizeof(float) * ((size_t)BP * LDM + (size_t)BP * LDW + 2 * BP) +
                                  sizeof(int) * BP + 2 * sizeof(__nv_bfloat16) * ((size_t)BP * 16 + 2 * (size_t)BP * 16);
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float& c0, float& c1, float& c2, float& c3, uint32_t a0, uint32_t a1,
                                         uint32_t a2, uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c0), "+f"(c1), "+f"(c2), "+f"(c3)
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <class S, int N, int SPLIT>
__global__ void __launch_bounds__(TC_THREADS) k_factor_tc(const double* __restrict__ Bin, S* __restrict__ Aout,
                                                           float* __restrict__ Dr, float* __restrict__ Dc,
                                                           int* __restrict__ info, Mesh Msh) {
  using D = TcDims<N>;
  constexpr int BS = D::BS, BP = D::BP, LDM = D::LDM, LDW = D::LDW;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* Mx = reinterpret_cast<float*>(smraw);           // [BP][LDM]
  float* Wk = Mx + (size_t)BP * LDM;                      // [BP][LDW]: panel columns | K tracker
  float* dr = Wk + (size_t)BP * LDW;                      // [BP]
  float* dc = dr + BP;                                     // [BP]
  int* piv = reinterpret_cast<int*>(dc + BP);              // [16] (BP reserved)
  __nv_bfloat16* Uh = reinterpret_cast<__nv_bfloat16*>(piv + BP);   // [2][BP][16] (hi, lo)
  __nv_bfloat16* Vt = Uh + 2 * BP * 16;                              // [2][2BP][16] transposed panel rows
  __shared__ int s_piv, s_bad;
  const int e = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  if (!Msh.on(e)) return;
  const double* Be = Bin + (size_t)e * BS * BS;
  if (tid == 0) s_bad = 0;
  for (int idx = tid; idx < BP * 2 * BP; idx += TC_THREADS) {
    const int r = idx / (2 * BP), c2 = idx % (2 * BP);
    float v;
    if (c2 < BP) v = (r < BS && c2 < BS) ? (float)Be[r * BS + c2] : (r == c2 ? 1.f : 0.f);
    else v = (c2 - BP == r) ? 1.f : 0.f;
    Mx[r * LDM + c2] = v;
  }
  __syncthreads();
  // equilibration (powers of two, exact): row scales, then column scales of the row-scaled block
  for (int r = wid; r < BP; r += TC_THREADS / 32) {
    float m = 0.f;
    for (int c2 = lane; c2 < BS; c2 += 32) m = fmaxf(m, fabsf(Mx[r * LDM + c2]));
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) {
      int ex = 0;
      if (m > 0.f && r < BS) frexpf(m, &ex);
      dr[r] = (m > 0.f && r < BS) ? ldexpf(1.0f, -ex) : 1.0f;
    }
  }
  __syncthreads();
  for (int c2 = wid; c2 < BP; c2 += TC_THREADS / 32) {
    float m = 0.f;
    for (int r = lane; r < BS; r += 32) m = fmaxf(m, fabsf(Mx[r * LDM + c2]) * dr[r]);
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) {
      int ex = 0;
      if (m > 0.f && c2 < BS) frexpf(m, &ex);
      dc[c2] = (m > 0.f && c2 < BS) ? ldexpf(1.0f, -ex) : 1.0f;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < BS * BS; idx += TC_THREADS) {
    const int r = idx / BS, c2 = idx % BS;
    Mx[r * LDM + c2] *= dr[r] * dc[c2];
  }
  __syncthreads();
  for (int k0 = 0; k0 < BP; k0 += 16) {
    // (a) pivots of the panel: Gauss-Jordan steps on a copy of its 16 columns
    for (int idx = tid; idx < BP * 16; idx += TC_THREADS) Wk[(idx / 16) * LDW + idx % 16] = Mx[(idx / 16) * LDM + k0 + idx % 16];
    __syncthreads();
    for (int i = 0; i < 16; ++i) {
      const int k = k0 + i;
      if (tid < 32) {
        float best = -1.f;
        int bi = k;
        for (int r = k + tid; r < BP; r += 32) {
          const float a = fabsf(Wk[r * LDW + i]);
          if (a > best) { best = a; bi = r; }
        }
        for (int off = 16; off > 0; off >>= 1) {
          const float ob = __shfl_down_sync(0xffffffffu, best, off);
          const int oi = __shfl_down_sync(0xffffffffu, bi, off);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (tid == 0) { s_piv = bi; piv[i] = bi; if (!(best > 0.f)) s_bad = 1; }
      }
      __syncthreads();
      const int pr = s_piv;
      if (pr != k)
        for (int c2 = tid; c2 < 16; c2 += TC_THREADS) { const float t = Wk[k * LDW + c2]; Wk[k * LDW + c2] = Wk[pr * LDW + c2]; Wk[pr * LDW + c2] = t; }
      __syncthreads();
      const float d = Wk[k * LDW + i];
      const float rp = d != 0.f ? 1.f / d : 0.f;
      __syncthreads();
      for (int c2 = tid; c2 < 16; c2 += TC_THREADS) Wk[k * LDW + c2] *= rp;
      __syncthreads();
      for (int idx = tid; idx < BP * 16; idx += TC_THREADS) {
        const int r = idx / 16, c2 = idx % 16;
        if (r == k || c2 == i) continue;
        Wk[r * LDW + c2] = fmaf(-Wk[r * LDW + i], Wk[k * LDW + c2], Wk[r * LDW + c2]);
      }
      __syncthreads();
      for (int r = tid; r < BP; r += TC_THREADS) if (r != k) Wk[r * LDW + i] = 0.f;
      __syncthreads();
    }
    // (b) the interchanges on the whole rows of M, in order
    for (int i = 0; i < 16; ++i) {
      const int k = k0 + i, pr = piv[i];
      if (pr != k)
        for (int c2 = tid; c2 < 2 * BP; c2 += TC_THREADS) { const float t = Mx[k * LDM + c2]; Mx[k * LDM + c2] = Mx[pr * LDM + c2]; Mx[pr * LDM + c2] = t; }
      __syncthreads();
    }
    // (c) the elimination again without interchanges on [panel | K]: K (the panel's unit
    // columns) becomes T K, and U = T K - K are the multipliers of the rank-16 update
    for (int idx = tid; idx < BP * 32; idx += TC_THREADS) {
      const int r = idx / 32, c2 = idx % 32;
      Wk[r * LDW + c2] = c2 < 16 ? Mx[r * LDM + k0 + c2] : (r == k0 + c2 - 16 ? 1.f : 0.f);
    }
    __syncthreads();
    for (int i = 0; i < 16; ++i) {
      const int k = k0 + i;
      const float d = Wk[k * LDW + i];
      const float rp = d != 0.f ? 1.f / d : 0.f;
      __syncthreads();
      for (int c2 = tid; c2 < 32; c2 += TC_THREADS) Wk[k * LDW + c2] *= rp;
      __syncthreads();
      for (int idx = tid; idx < BP * 32; idx += TC_THREADS) {
        const int r = idx / 32, c2 = idx % 32;
        if (r == k || c2 == i) continue;
        Wk[r * LDW + c2] = fmaf(-Wk[r * LDW + i], Wk[k * LDW + c2], Wk[r * LDW + c2]);
      }
      __syncthreads();
      for (int r = tid; r < BP; r += TC_THREADS) if (r != k) Wk[r * LDW + i] = 0.f;
      __syncthreads();
    }
    // (d) operands in BF16: U (row-major [BP][16]) and the panel rows transposed ([2BP][16])
    const int c0 = k0 + 16, ncols = 2 * BP - c0;
    for (int idx = tid; idx < BP * 16; idx += TC_THREADS) {
      const int r = idx / 16, i = idx % 16;
      const float u = Wk[r * LDW + 16 + i] - (r == k0 + i ? 1.f : 0.f);
      const __nv_bfloat16 hi = __float2bfloat16_rn(u);
      Uh[idx] = hi;
      if (SPLIT == 3) Uh[BP * 16 + idx] = __float2bfloat16_rn(u - __bfloat162float(hi));
    }
    for (int idx = tid; idx < ncols * 16; idx += TC_THREADS) {
      const int n = idx / 16, i = idx % 16;
      const float v = Mx[(k0 + i) * LDM + c0 + n];
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      Vt[idx] = hi;
      if (SPLIT == 3) Vt[2 * BP * 16 + idx] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
    __syncthreads();
    // (e) the panel's columns become unit columns; everything right of it gets M += U V
    for (int idx = tid; idx < BP * 16; idx += TC_THREADS) {
      const int r = idx / 16, i = idx % 16;
      Mx[r * LDM + k0 + i] = (r == k0 + i) ? 1.f : 0.f;
    }
    const int g = lane >> 2, t4 = lane & 3;
    const int ntiles = (BP / 16) * (ncols / 8);
    for (int tile = wid; tile < ntiles; tile += TC_THREADS / 32) {
      const int mt = tile / (ncols / 8), nt8 = tile % (ncols / 8);
      const int r0 = mt * 16, n0 = nt8 * 8;
      float* C0 = Mx + (r0 + g) * LDM + c0 + n0 + 2 * t4;
      float* C1 = Mx + (r0 + g + 8) * LDM + c0 + n0 + 2 * t4;
      float c_0 = C0[0], c_1 = C0[1], c_2 = C1[0], c_3 = C1[1];
#pragma unroll
      for (int ha = 0; ha < (SPLIT == 3 ? 2 : 1); ++ha) {
#pragma unroll
        for (int hb = 0; hb < (SPLIT == 3 ? 2 : 1); ++hb) {
          if (ha == 1 && hb == 1) continue;   // lo x lo is below the split's accuracy
          const __nv_bfloat16* U = Uh + ha * BP * 16;
          const __nv_bfloat16* V = Vt + hb * 2 * BP * 16;
          const uint32_t a0 = *reinterpret_cast<const uint32_t*>(U + (r0 + g) * 16 + 2 * t4);
          const uint32_t a1 = *reinterpret_cast<const uint32_t*>(U + (r0 + g + 8) * 16 + 2 * t4);
          const uint32_t a2 = *reinterpret_cast<const uint32_t*>(U + (r0 + g) * 16 + 2 * t4 + 8);
          const uint32_t a3 = *reinterpret_cast<const uint32_t*>(U + (r0 + g + 8) * 16 + 2 * t4 + 8);
          const uint32_t b0 = *reinterpret_cast<const uint32_t*>(V + (n0 + g) * 16 + 2 * t4);
          const uint32_t b1 = *reinterpret_cast<const uint32_t*>(V + (n0 + g) * 16 + 2 * t4 + 8);
          mma_bf16(c_0, c_1, c_2, c_3, a0, a1, a2, a3, b0, b1);
        }
      }
      C0[0] = c_0; C0[1] = c_1; C1[0] = c_2; C1[1] = c_3;
    }
    __syncthreads();
  }
  // the right half of M is the inverse of the equilibrated (padded) block; store it
  // transposed: Aout[col][row]
  S* Ae = Aout + (size_t)e * BS * BS;
  for (int idx = tid; idx < BS * BS; idx += TC_THREADS) {
    const int c2 = idx / BS, r = idx % BS;
    Ae[idx] = (S)Mx[r * LDM + BP + c2];
  }
  for (int r = tid; r < BS; r += TC_THREADS) { Dr[(size_t)e * BS + r] = dr[r]; Dc[(size_t)e * BS + r] = dc[r]; }
  if (tid == 0) info[e] = s_bad;
}

template <class S> __device__ __forceinline__ float to_f(S x) { return (float)x; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

// z_e = Dc (A^T_stored (Dr r_e)) with four threads per row: thread (part, row) sums the
// columns c = part, part + 4, ... (consecutive rows of one column are adjacent in the
// transposed store: coalesced), two partial sums each; the four parts meet in shared
// memory.  ACC: 0 FP64, 1 FP32, 2 double-float (FP32 pairs with error-free
// transformations, linear to about 2^-44 of the summed magnitudes).
constexpr int APPLY_PARTS = 4;

// With rsub and zadd (both nullable) the same pass forms z_e = zadd_e + B_e^-1 (r - rsub)_e.
// CO = 1 (FP32) or 2 (FP64 coarse arrays): the smoothing step of the two-level
// preconditioner from the coarse solution y0 instead, z_e = (P y0)_e + B_e^-1 (r - A P y0)_e
// with the stored columns A P of the element's stencil members (ci): the four parts of a
// row each sum 15 of its 60 terms (double-float for FP32 arrays, FP64 otherwise).
// One element e by the whole block: A is the element's stored inverse and APe its A P
// columns (CO != 0), in global or shared memory (generic pointers).
template <class S, int ACC, int N, int CO>
__device__ __forceinline__ void apply_elem(int e, const S* __restrict__ A, const void* __restrict__ APe,
                                           const float* __restrict__ Dr, const float* __restrict__ Dc,
                                           const double* __restrict__ r, const Mesh& M,
                                           double* __restrict__ z, const double* __restrict__ rsub,
                                           const double* __restrict__ zadd, bool tr,
                                           const CoarseIn& ci) {
  constexpr int NP = N * N, BS = 4 * NP, BSR = (BS + 31) / 32 * 32;
  constexpr int COLS = (BS + APPLY_PARTS - 1) / APPLY_PARTS;   // columns per thread
  __shared__ double xd[ACC == 0 ? BS : 1];
  __shared__ float xf[ACC == 1 ? BS : 1];
  __shared__ float2 x2[ACC == 2 ? BS : 1];
  __shared__ double pd[ACC == 0 ? APPLY_PARTS : 1][BSR];
  __shared__ float pf[ACC == 1 ? APPLY_PARTS : 1][BSR];
  __shared__ float2 p2[ACC == 2 ? APPLY_PARTS : 1][BSR];
  if (!M.on(e)) return;
  const int part = threadIdx.x / BSR, row = threadIdx.x % BSR;
  // every load of this thread's columns issued before any arithmetic
  S av[COLS];
#pragma unroll
  for (int k = 0; k < COLS; ++k) {
    const int c2 = part + APPLY_PARTS * k;
    av[k] = (row < BS && c2 < BS) ? A[tr ? (size_t)row * BS + c2 : (size_t)c2 * BS + row] : S(0.0f);
  }
  // B^-1 = Dc Ainv Dr from the stored transpose of Ainv; B^-T = Dr Ainv^T Dc
  const float* Din = tr ? Dc : Dr;
  const float* Dout = tr ? Dr : Dc;
  const size_t qo = M.qbase(e, NP), qs = M.qstride(e);
  constexpr int CT = 5 * 12;   // coarse terms of a row: 5 stencil members x 12 P1 coefficients
  constexpr int CPT = (CT + APPLY_PARTS - 1) / APPLY_PARTS;   // coarse terms per thread
  using SC = typename std::conditional<CO == 2, double, float>::type;
  // this thread's A P entries, its input row and scale, loaded with the inverse's columns
  SC apv[CO ? CPT : 1];
  if constexpr (CO != 0) {
    const SC* ap = (const SC*)APe + row;
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
      const int kk = part + APPLY_PARTS * k;
      apv[k] = (row < BS && kk < CT) ? ap[(size_t)kk * BS] : SC(0);
    }
  }
  double rin = 0.0, din = 0.0;
  if (threadIdx.x < BS) {
    const int t = threadIdx.x;
    rin = r[(t / NP) * qs + qo + t % NP];
    din = (double)Din[(size_t)e * BS + t];
  }
  __shared__ double cyd[CO == 2 ? CT : 1];
  __shared__ float cyf[CO == 1 ? CT : 1];
  __shared__ double cpd[CO == 2 ? APPLY_PARTS : 1][CO == 2 ? BSR : 1];
  __shared__ float2 cpf[CO == 1 ? APPLY_PARTS : 1][CO == 1 ? BSR : 1];
  if constexpr (CO != 0) {
    for (int t = threadIdx.x; t < CT; t += blockDim.x) {
      const int cell = ci.nb[(size_t)e * 5 + t / 12];
      if constexpr (CO == 2) cyd[t] = cell >= 0 ? ((const double*)ci.y0)[(size_t)cell * 12 + t % 12] : 0.0;
      else cyf[t] = cell >= 0 ? ((const float*)ci.y0)[(size_t)cell * 12 + t % 12] : 0.0f;
    }
    __syncthreads();
    if (row < BS) {
      if constexpr (CO == 2) {
        double a0 = 0.0;
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
          const int kk = part + APPLY_PARTS * k;
          if (kk < CT) a0 = fma(apv[k], cyd[kk], a0);
        }
        cpd[part][row] = a0;
      } else {
        float h0 = 0.f, l0 = 0.f;
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
          const int kk = part + APPLY_PARTS * k;
          if (kk < CT) df_add(h0, l0, apv[k], make_float2(cyf[kk], 0.f));
        }
        cpf[part][row] = make_float2(h0, l0);
      }
    }
    __syncthreads();
  }
  // the block has at least BS threads: thread t < BS stages input row t
  if (threadIdx.x < BS) {
    const int t = threadIdx.x;
    const int v = t / NP, pt = t % NP;
    const size_t gi = v * qs + qo + pt;
    double rs = rsub ? rsub[gi] : 0.0;
    if constexpr (CO == 2) {
      rs = cpd[0][t];
#pragma unroll
      for (int q = 1; q < APPLY_PARTS; ++q) rs += cpd[q][t];
    } else if constexpr (CO == 1) {
      float sh = cpf[0][t].x, sl = cpf[0][t].y;
#pragma unroll
      for (int q = 1; q < APPLY_PARTS; ++q) df_merge(sh, sl, cpf[q][t].x, cpf[q][t].y);
      rs = (double)sh + (double)sl;
    }
    const double u = (rin - rs) * din;
    if (ACC == 0) xd[t] = u;
    else if (ACC == 1) xf[t] = (float)u;
    else {
      const float hi = __double2float_rn(u);
      x2[t] = make_float2(hi, __double2float_rn(u - (double)hi));
    }
  }
  __syncthreads();
  if (row < BS) {
    if (ACC == 0) {
      double a0 = 0.0, a1 = 0.0;
#pragma unroll
      for (int k = 0; k < COLS; ++k) {
        const int c2 = part + APPLY_PARTS * k;
        if (c2 < BS) {
          if (k & 1) a1 = fma((double)av[k], xd[c2], a1);
          else a0 = fma((double)av[k], xd[c2], a0);
        }
      }
      pd[part][row] = a0 + a1;
    } else if (ACC == 1) {
      float a0 = 0.f, a1 = 0.f;
#pragma unroll
      for (int k = 0; k < COLS; ++k) {
        const int c2 = part + APPLY_PARTS * k;
        if (c2 < BS) {
          if (k & 1) a1 = fmaf(to_f(av[k]), xf[c2], a1);
          else a0 = fmaf(to_f(av[k]), xf[c2], a0);
        }
      }
      pf[part][row] = a0 + a1;
    } else {
      float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
#pragma unroll
      for (int k = 0; k < COLS; ++k) {
        const int c2 = part + APPLY_PARTS * k;
        if (c2 < BS) {
          if (k & 1) df_add(h1, l1, to_f(av[k]), x2[c2]);
          else df_add(h0, l0, to_f(av[k]), x2[c2]);
        }
      }
      // partial sums combined as FP32 pairs: conversions and FP64 additions run on the
      // FP64 pipe, which is slower than all of the two-sum work above
      df_merge(h0, l0, h1, l1);
      p2[part][row] = make_float2(h0, l0);
    }
  }
  __syncthreads();
  if (part != 0 || row >= BS) return;
  double acc;
  if (ACC == 1) {
    float t = pf[0][row];
#pragma unroll
    for (int q = 1; q < APPLY_PARTS; ++q) t += pf[q][row];
    acc = (double)t;
  } else if (ACC == 2) {
    float sh = p2[0][row].x, sl = p2[0][row].y;
#pragma unroll
    for (int q = 1; q < APPLY_PARTS; ++q) df_merge(sh, sl, p2[q][row].x, p2[q][row].y);
    acc = (double)sh + (double)sl;
  } else {
    acc = pd[0][row];
#pragma unroll
    for (int q = 1; q < APPLY_PARTS; ++q) acc += pd[q][row];
  }
  const int v = row / NP, pt = row % NP;
  const size_t gi = v * qs + qo + pt;
  const double zr = acc * (double)Dout[(size_t)e * BS + row];
  if constexpr (CO != 0) {
    // P y0 at this point: c0 + c1 xi + c2 eta of the element's own coefficients (slot 0)
    const int i = pt % N, j = pt / N;
    double c[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) c[m] = CO == 2 ? cyd[3 * v + m] : (double)cyf[3 * v + m];
    z[gi] = fma(c[2], ci.xs[j], fma(c[1], ci.xs[i], c[0])) + zr;
  } else {
    z[gi] = zadd ? zadd[gi] + zr : zr;
  }
}

template <class S, int ACC, int N, int CO = 0>
__global__ void k_apply4(const S* __restrict__ AT, const float* __restrict__ Dr,
                         const float* __restrict__ Dc, const double* __restrict__ r, Mesh M,
                         double* __restrict__ z, const double* __restrict__ rsub,
                         const double* __restrict__ zadd, bool tr, CoarseIn ci = CoarseIn{}) {
  constexpr int BS = 4 * N * N;
  const int e = blockIdx.x;
  apply_elem<S, ACC, N, CO>(e, AT + (size_t)e * BS * BS,
                            CO ? (const char*)ci.AP + (size_t)e * 60 * BS * (CO == 2 ? 8 : 4) : nullptr,
                            Dr, Dc, r, M, z, rsub, zadd, tr, ci);
}

// ------------------------------------------------------------------ bulk-copy pipeline
// mbarrier and bulk-copy (TMA, 1-D cp.async.bulk) primitives in inline PTX.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Waits for phase `parity` of the barrier: spins > 0 potentially blocking tries, spins < 0
// one non-blocking test.  False if the phase has not completed within the budget.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long spins) {
  const unsigned a = smem_u32(bar);
  if (spins < 0) {
    unsigned done;
    asm volatile(
        "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    return done != 0;
  }
  for (long long i = 0; i < spins; ++i) {
    unsigned done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Bytes of one element's slab in the pipeline: the stored inverse, then the A P columns,
// rounded up to 128 bytes.
template <class S, int N, int CO>
struct BulkSlab {
  static constexpr unsigned A = 16u * N * N * N * N * (unsigned)sizeof(S);   // (4 n^2)^2 entries
  static constexpr unsigned P = CO == 0 ? 0u : 60u * 4u * N * N * (CO == 2 ? 8u : 4u);
  static constexpr unsigned SLAB = (A + P + 127u) / 128u * 128u;
};

// The block apply as a persistent kernel fed by bulk copies: each block walks the elements
// e = blockIdx.x, + gridDim.x, ...; one thread keeps the next nst - 1 elements' inverses
// (and A P columns) in flight into an nst-slab shared ring while the block computes the
// current one, so the HBM stream of the stored inverses runs under the arithmetic.  The
// copy sizes and addresses are multiples of 16 bytes for every degree and precision.
// A wait that runs out of its budget sets *err, waits (bounded) for this block's copies
// in flight, and ends the block.
template <class S, int ACC, int N, int CO>
__global__ void k_apply_bulk(const S* __restrict__ AT, const float* __restrict__ Dr,
                             const float* __restrict__ Dc, const double* __restrict__ r, Mesh M,
                             double* __restrict__ z, CoarseIn ci, int nst, long long spins, int* err) {
  using L = BulkSlab<S, N, CO>;
  constexpr int BS = 4 * N * N;
  extern __shared__ __align__(128) unsigned char slab[];
  __shared__ __align__(8) unsigned long long bar[4];
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int i = 0; i < nst; ++i) mbar_init(&bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto elem = [&](int k) { return blockIdx.x + k * (int)gridDim.x; };
  auto issue = [&](int k) {
    const int e = elem(k), st = k % nst;
    unsigned char* dst = slab + (size_t)st * L::SLAB;
    mbar_expect_tx(&bar[st], L::A + L::P);
    bulk_g2s(dst, AT + (size_t)e * BS * BS, L::A, &bar[st]);
    if (CO) bulk_g2s(dst + L::A, (const char*)ci.AP + (size_t)e * L::P, L::P, &bar[st]);
  };
  if (tid == 0)
    for (int k = 0; k < nst - 1 && elem(k) < M.ne; ++k) issue(k);
  int k = 0;
  bool bad = false;
  for (; elem(k) < M.ne; ++k) {
    const int st = k % nst;
    if (tid == 0 && elem(k + nst - 1) < M.ne) issue(k + nst - 1);
    const bool ok = mbar_wait(&bar[st], (unsigned)(k / nst) & 1u, spins);
    if (__syncthreads_or(!ok)) { bad = true; break; }
    const unsigned char* cur = slab + (size_t)st * L::SLAB;
    apply_elem<S, ACC, N, CO>(elem(k), (const S*)cur, cur + L::A, Dr, Dc, r, M, z, nullptr, nullptr,
                              false, ci);
    __syncthreads();   // the slab is refilled nst - 1 elements later
  }
  if (bad && tid == 0) {
    atomicExch(err, 1);
    // copies issued and not consumed: elements k .. k + nst - 1
    for (int j = k; j < k + nst && elem(j) < M.ne; ++j)
      mbar_wait(&bar[j % nst], (unsigned)(j / nst) & 1u, 1LL << 22);
  }
}

}  // namespace fr

namespace frk {
using namespace fr;

template <int N>
static int block_build_n(fr_ctx* c, const double* q, double inv_dtau, double a0_dt, cudaStream_t s) {
  if (c->cfg.block_mode == FR_BLOCK_LINEARIZED) {
    // from the local Jacobians at q (also the operator GMRES applies next)
    FR_TRY(linearize(c, q, inv_dtau, a0_dt, s));
    const bool visc = c->mesh.viscous;
    // per element and unit column: gradient, traces, face products, point products, divergence
    const double per_col = (double)N * N * (16.0 * N + 84.0) + 4.0 * N * (12.0 * N + 34.0);
    FR_ACCOUNT(c, KK_BLOCK, 2.0 * c->ne * c->bsz * (visc ? per_col : 0.5 * per_col), 0.0);
    const size_t smem = BlkLinSmem<N>::BYTES;
    FR_CUDA_CHECK(c, cudaFuncSetAttribute(k_block_lin<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FR_PROF_BEGIN(c, s);
    k_block_lin<N><<<c->ne, BG * N * N, smem, s>>>(c->mesh, c->basis, c->gs, c->gf, c->JFQ, c->JFG,
                                                   c->JP, c->JG, c->PP, c->JFQb, c->JFGb,
                                                   c->bounded ? c->nx * N : 0, c->B64);
    FR_PROF_END(c, s, KK_BLOCK);
    FR_LAUNCH_CHECK(c);
    return FR_OK;
  }
  // dual-number forward mode: value traces of every element (neighbour data of the blocks)
  constexpr int EPB = Tile<N>::EPB, TH = Tile<N>::THREADS;
  const int nblk = (c->ne + EPB - 1) / EPB;
  const bool visc = c->mesh.viscous;
  {
    const int rc = set_operator_terms(c, inv_dtau, a0_dt, s);
    if (rc != FR_OK) return rc;
  }
  FR_ACCOUNT(c, KK_TRACE, (double)c->ne * N * N * fr_flops_trace(N, visc), 0.0);
  // per element and tangent direction: gradients + traces, 4n face points, n^2 element points
  FR_ACCOUNT(c, KK_BLOCK, (double)c->ne * c->bsz * FR_JVP_FLOP_FACTOR *
                              (N * N * (fr_flops_trace(N, visc) + fr_flops_elem(N, visc)) +
                               4.0 * N * fr_flops_face_point(visc)), 0.0);
  {
    FR_PROF_BEGIN(c, s);
    k_trace<double, N><<<nblk, TH, 0, s>>>(Buf<double>{const_cast<double*>(q)}, c->mesh, c->basis,
                                           c->gs, Buf<double>{c->gl}, Buf<double>{c->tq},
                                           Buf<double>{c->tg});
    FR_PROF_END(c, s, KK_TRACE);
    FR_LAUNCH_CHECK(c);
  }
  const size_t smem = (size_t)BG * BlkSmem<N>::SIZE * sizeof(Dual);
  FR_CUDA_CHECK(c, cudaFuncSetAttribute(k_block<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  FR_PROF_BEGIN(c, s);
  k_block<N><<<c->ne, BG * N * N, smem, s>>>(q, c->mesh, c->basis, c->gs, c->gf, c->tq,
                                             c->tg, c->B64);
  FR_PROF_END(c, s, KK_BLOCK);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

// Dynamic shared memory of k_factor<W, S, N> for block size bs = 4 N^2: the padded
// matrix, the pivot column, the two scale vectors and the interchanges.
template <class W>
static size_t factor_smem(int bs) { return (size_t)bs * (bs + 1) * sizeof(W) + bs * sizeof(W) + bs * 4 * 2 + bs * 4; }

template <class W, class S, int N>
static int factor_n(fr_ctx* c, S* out, cudaStream_t s) {
  constexpr int BS = 4 * N * N;
  const size_t smem = factor_smem<W>(BS);
  FR_CUDA_CHECK(c, cudaFuncSetAttribute(k_factor<W, S, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_factor<W, S, N><<<c->ne, 256, smem, s>>>(c->B64, out, c->Dr, c->Dc, c->info, c->mesh);
  return FR_OK;
}

template <class W, class S>
static int factor_t(fr_ctx* c, S* out, cudaStream_t s) {
  switch (c->n) {
    case 2: return factor_n<W, S, 2>(c, out, s);
    case 3: return factor_n<W, S, 3>(c, out, s);
    case 4: return factor_n<W, S, 4>(c, out, s);
    case 5: return factor_n<W, S, 5>(c, out, s);
  }
  return FR_ERR_ARG;
}

template <class S, int N, int SPLIT>
static int factor_tc_n(fr_ctx* c, S* out, cudaStream_t s) {
  const size_t smem = TcDims<N>::BYTES;
  FR_CUDA_CHECK(c, cudaFuncSetAttribute(k_factor_tc<S, N, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_factor_tc<S, N, SPLIT><<<c->ne, TC_THREADS, smem, s>>>(c->B64, out, c->Dr, c->Dc, c->info, c->mesh);
  return FR_OK;
}

template <class S>
static int factor_tc(fr_ctx* c, S* out, cudaStream_t s) {
  const bool split = c->cfg.factor_tc == FR_FACTOR_TC_BF16X3;
  switch (c->n * 2 + (split ? 1 : 0)) {
    case 4: return factor_tc_n<S, 2, 1>(c, out, s);
    case 5: return factor_tc_n<S, 2, 3>(c, out, s);
    case 6: return factor_tc_n<S, 3, 1>(c, out, s);
    case 7: return factor_tc_n<S, 3, 3>(c, out, s);
    case 8: return factor_tc_n<S, 4, 1>(c, out, s);
    case 9: return factor_tc_n<S, 4, 3>(c, out, s);
    case 10: return factor_tc_n<S, 5, 1>(c, out, s);
    case 11: return factor_tc_n<S, 5, 3>(c, out, s);
  }
  return FR_ERR_ARG;
}

static int factor(fr_ctx* c, cudaStream_t s) {
  const int bs = c->bsz;
  if (c->cfg.factor_tc != FR_FACTOR_SIMT) {
    // blocked Gauss-Jordan on [A | I] padded to bp: per panel of 16 the SIMT elimination of
    // its columns twice (2 x 16 rank-1 updates of bp x 16 and bp x 32) and the rank-16
    // update of the columns right of it on the tensor cores (2 bp x 16 x width flops, three
    // products with the split operands)
    const int bp = (bs + 15) / 16 * 16;
    double tc = 0.0, simt = 0.0;
    for (int k0 = 0; k0 < bp; k0 += 16) {
      tc += 2.0 * bp * 16.0 * (2.0 * bp - k0 - 16) * (c->cfg.factor_tc == FR_FACTOR_TC_BF16X3 ? 3.0 : 1.0);
      simt += 2.0 * 16.0 * bp * 48.0;
    }
    FR_ACCOUNT(c, KK_FACTOR, (tc + simt) * c->ne, 0.0);
    FR_PROF_BEGIN(c, s);
    if (c->cfg.prec_dtype == FR_PREC_FP64) FR_TRY(factor_tc<double>(c, (double*)c->Binv, s));
    else if (c->cfg.prec_dtype == FR_PREC_FP32) FR_TRY(factor_tc<float>(c, (float*)c->Binv, s));
    else FR_TRY(factor_tc<__nv_bfloat16>(c, (__nv_bfloat16*)c->Binv, s));
    FR_PROF_END(c, s, KK_FACTOR);
    FR_LAUNCH_CHECK(c);
    return FR_OK;
  }
  // in-place Gauss-Jordan: bs steps of a rank-1 update of bs^2 entries (2 flops each)
  FR_ACCOUNT(c, KK_FACTOR, 2.0 * (double)bs * bs * bs * c->ne, 0.0);
  FR_PROF_BEGIN(c, s);
  // each degree has its own instantiation and attribute value: contexts of several degrees
  // building blocks concurrently from different threads never change one another's
  if (c->cfg.prec_dtype == FR_PREC_FP64)
    FR_TRY(factor_t<double>(c, (double*)c->Binv, s));
  else if (c->cfg.prec_dtype == FR_PREC_FP32)
    FR_TRY(factor_t<float>(c, (float*)c->Binv, s));
  else
    FR_TRY(factor_t<float>(c, (__nv_bfloat16*)c->Binv, s));
  FR_PROF_END(c, s, KK_FACTOR);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

int block_build(fr_ctx* c, const double* q, double inv_dtau, double a0_dt, cudaStream_t s) {
  int rc;
  switch (c->n) {
    case 2: rc = block_build_n<2>(c, q, inv_dtau, a0_dt, s); break;
    case 3: rc = block_build_n<3>(c, q, inv_dtau, a0_dt, s); break;
    case 4: rc = block_build_n<4>(c, q, inv_dtau, a0_dt, s); break;
    case 5: rc = block_build_n<5>(c, q, inv_dtau, a0_dt, s); break;
    default: return FR_ERR_ARG;
  }
  if (rc != FR_OK) return rc;
  return factor(c, s);
}

// The bulk-copy pipeline for one instantiation: its persistent grid (blocks per SM at
// this slab size times the SMs, cached per context) and launch.  False if two slabs do not
// fit in shared memory (the caller falls back to one block per element).
template <class S, int ACC, int N, int CO>
static bool launch_bulk(fr_ctx* c, const double* r, double* z, const CoarseIn& ci, int threads,
                        cudaStream_t s, int* rc) {
  const int nst = c->cfg.apply_bulk;
  const size_t smem = (size_t)nst * BulkSlab<S, N, CO>::SLAB;
  if (smem > 200 * 1024) return false;
  int& grid = c->apply_grid[CO];
  auto kern = k_apply_bulk<S, ACC, N, CO>;
  if (grid == 0) {
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem) != cudaSuccess || per < 1) {
      *rc = FR_ERR_CUDA;
      snprintf(c->err, sizeof(c->err), "bulk apply: launch configuration");
      return true;
    }
    grid = per * nsm;
  }
  const long long spins = c->cfg.wait_spins == 0 ? (1LL << 22) : c->cfg.wait_spins;
  kern<<<std::min(grid, c->ne), threads, smem, s>>>((const S*)c->Binv, c->Dr, c->Dc, r, c->mesh, z,
                                                   ci, nst, spins, c->dev_err);
  *rc = FR_OK;
  return true;
}

template <int CO>
static int apply_impl(fr_ctx* c, const double* r, double* z, const double* rsub,
                      const double* zadd, const CoarseIn& ci, cudaStream_t s) {
  const int bs = c->bsz;
  const double esz = c->cfg.prec_dtype == FR_PREC_FP64 ? 8.0 : c->cfg.prec_dtype == FR_PREC_FP32 ? 4.0 : 2.0;
  // the coarse form also reads the 60 stored columns of A P per row
  const double co_flops = CO ? 2.0 * 60.0 * bs * c->ne : 0.0;
  const double co_bytes = CO ? 60.0 * bs * c->ne * (CO == 1 ? 4.0 : 8.0) : 0.0;
  FR_ACCOUNT(c, KK_APPLY, 2.0 * (double)bs * bs * c->ne + co_flops,
             c->ne * ((double)bs * bs * esz + 2.0 * bs * 4.0) + co_bytes +
                 (2.0 + (rsub ? 1.0 : 0.0) + (zadd ? 1.0 : 0.0)) * 8.0 * c->ndof);
  FR_PROF_BEGIN(c, s);
  // Double-float accumulation keeps the preconditioner linear to near FP64 round-off (the
  // stored inverse rounded once); plain FP32 accumulation also rounds the input and every
  // partial sum, a state-dependent perturbation that left-preconditioned GMRES cannot get
  // below on stiff cases
  const bool df = c->cfg.apply_accum == FR_ACCUM_DF64;
  const bool tr = c->transposed != 0;   // B^-T in the adjoint solve
  const int nt4 = APPLY_PARTS * ((bs + 31) / 32 * 32);
  const int acc = c->cfg.prec_dtype == FR_PREC_FP64 ? 0 : df ? 2 : 1;
  if (c->cfg.apply_bulk && !tr && !rsub && !zadd) {
    int rc = FR_OK;
    bool done = false;
    const bool f32 = c->cfg.prec_dtype == FR_PREC_FP32;
    switch (c->n * 10 + acc) {
#define FR_BULK_CASE(NN)                                                                            \
      case NN * 10 + 0: done = launch_bulk<double, 0, NN, CO>(c, r, z, ci, nt4, s, &rc); break;      \
      case NN * 10 + 1: done = f32 ? launch_bulk<float, 1, NN, CO>(c, r, z, ci, nt4, s, &rc)         \
                                   : launch_bulk<__nv_bfloat16, 1, NN, CO>(c, r, z, ci, nt4, s, &rc); break; \
      case NN * 10 + 2: done = f32 ? launch_bulk<float, 2, NN, CO>(c, r, z, ci, nt4, s, &rc)         \
                                   : launch_bulk<__nv_bfloat16, 2, NN, CO>(c, r, z, ci, nt4, s, &rc); break;
      FR_BULK_CASE(2) FR_BULK_CASE(3) FR_BULK_CASE(4) FR_BULK_CASE(5)
#undef FR_BULK_CASE
      default: return FR_ERR_ARG;
    }
    if (done) {
      if (rc != FR_OK) return rc;
      FR_PROF_END(c, s, KK_APPLY);
      FR_LAUNCH_CHECK(c);
      return FR_OK;
    }
  }
  switch (c->n * 10 + acc) {
#define FR_APPLY_CASE(NN)                                                                      \
    case NN * 10 + 0: k_apply4<double, 0, NN, CO><<<c->ne, nt4, 0, s>>>((const double*)c->Binv, c->Dr, c->Dc, r, c->mesh, z, rsub, zadd, tr, ci); break; \
    case NN * 10 + 1: if (c->cfg.prec_dtype == FR_PREC_FP32)                                  \
        k_apply4<float, 1, NN, CO><<<c->ne, nt4, 0, s>>>((const float*)c->Binv, c->Dr, c->Dc, r, c->mesh, z, rsub, zadd, tr, ci); \
      else k_apply4<__nv_bfloat16, 1, NN, CO><<<c->ne, nt4, 0, s>>>((const __nv_bfloat16*)c->Binv, c->Dr, c->Dc, r, c->mesh, z, rsub, zadd, tr, ci); \
      break;                                                                                   \
    case NN * 10 + 2: if (c->cfg.prec_dtype == FR_PREC_FP32)                                  \
        k_apply4<float, 2, NN, CO><<<c->ne, nt4, 0, s>>>((const float*)c->Binv, c->Dr, c->Dc, r, c->mesh, z, rsub, zadd, tr, ci); \
      else k_apply4<__nv_bfloat16, 2, NN, CO><<<c->ne, nt4, 0, s>>>((const __nv_bfloat16*)c->Binv, c->Dr, c->Dc, r, c->mesh, z, rsub, zadd, tr, ci); \
      break;
    FR_APPLY_CASE(2) FR_APPLY_CASE(3) FR_APPLY_CASE(4) FR_APPLY_CASE(5)
#undef FR_APPLY_CASE
    default: return FR_ERR_ARG;
  }
  FR_PROF_END(c, s, KK_APPLY);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

int block_apply(fr_ctx* c, const double* r, double* z, cudaStream_t s) {
  return apply_impl<0>(c, r, z, nullptr, nullptr, CoarseIn{}, s);
}

int block_apply_fused(fr_ctx* c, const double* r, const double* t, const double* z0, double* z,
                      cudaStream_t s) {
  return apply_impl<0>(c, r, z, t, z0, CoarseIn{}, s);
}

int block_apply_coarse(fr_ctx* c, const double* r, double* z, const CoarseIn& ci, int co,
                       cudaStream_t s) {
  if (co == 1) return apply_impl<1>(c, r, z, nullptr, nullptr, ci, s);
  return apply_impl<2>(c, r, z, nullptr, nullptr, ci, s);
}

}  // namespace frk
