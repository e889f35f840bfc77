// fr_mg.cu -- two-level preconditioner for the Newton operator of Sec. 3.2: a coarse
// correction on the discontinuous linear (P1) space, solved by an agglomeration multigrid
// V-cycle, followed by the element block-Jacobi step.
//
// The paper preconditions restarted GMRES with per-process ILU(0) (Sec. 4, parallel
// setting); element blocks alone stall on low-Mach BDF2 steps once the preconditioned
// dissipation's pressure coupling (growing as p^2/h) dominates the time term
// gamma M^2 a0/dt, because element-local solves do not reach the smooth, domain-wide
// pressure modes.  This adds them back:
//
//   M^-1 r = z0 + B^-1 (r - A z0),   z0 = P V(P^T r)
//
// P maps per element and variable the coefficients (c0, c1, c2) of c0 + c1 xi + c2 eta to
// the solution points; V is one V-cycle on the Galerkin operators: A_0 = P^T A P (from the
// stored local Jacobians: each element's response to a neighbour's P1 function through
// their shared face, and its diagonal block times its own; or, with the dual-number
// operator, from coloured products of A with the elements' P1 functions), A_{l+1} = Q^T A_l Q with
// Q the exact map of a 2 x 2 agglomerate's P1 function to its children; damped 12 x 12
// block-Jacobi sweeps on every level but a case's last, which (<= 4 cells) is solved by
// its dense inverse.  A in the smoothing step is the operator of the build: the columns
// A P of every element's stencil members on its own rows, which form A_0, are stored, so
// A z0 = (A P) y0 costs no operator product.  Fixed
// summation orders, no atomics on data: the preconditioner is a fixed linear map between
// builds (up to the rounding of the coarse arithmetic).
//
// Layout for GB300: the coarse levels are stored and swept in the configured coarse
// precision (FP32 by default: a coarse sweep is 72 multiply-adds per coefficient, which
// the FP64 pipe -- 2 FMA per clock per SM -- would make the largest cost of an iteration;
// the build arithmetic stays FP64).  Levels with more than TAIL cells of a case run in
// tiles over all SMs, two launches per level and cycle (sweeps, residual and restriction
// on the way down; prolongation and sweeps on the way up), each block recomputing the
// halo its sweeps need; the remaining small levels of each case, with the dense solve, run
// in one block per case, the phases separated by block barriers; the restriction from the
// solution points is one launch, and the prolongation back, A z0 and the block-Jacobi
// step are the block apply's single pass.  An application thus costs 2 L + 3 launches for
// L tiled levels, whatever the number of sweeps.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>
#include "fr_internal.h"

namespace {

constexpr int NB = 12;          // P1 coefficients per cell (4 variables x 3)
constexpr int SL = 5;           // stencil slots per cell (self + 4 neighbours)
constexpr int BLK = NB * NB;    // entries of one 12 x 12 block
constexpr int MAXFIN = 4;       // cells of a case solved exactly
constexpr int DN = MAXFIN * NB; // leading dimension of the dense inverses
constexpr int TAIL = 16;        // levels of a case with at most this many cells: one block
constexpr int TAIL_THREADS = 256;

// Reference-coordinate basis value of mode m (1, xi, eta) at point (i, j).
__device__ __forceinline__ double phi(const fr::Basis& B, int m, int i, int j) {
  return m == 0 ? 1.0 : (m == 1 ? B.xs[i] : B.xs[j]);
}

// Q_m,a: coefficient of fine mode a in the child for coarse mode m (qo = s_a f_x, s_b f_y,
// f_x, f_y): c0 + c1 X + c2 Y = (c0 + c1 s_a f_x + c2 s_b f_y) + c1 f_x xi + c2 f_y eta.
__device__ __forceinline__ double qmap(const double* qo, int a, int m) {
  if (a == 0) return m == 0 ? 1.0 : (m == 1 ? qo[0] : qo[1]);
  if (a == 1) return m == 1 ? qo[2] : 0.0;
  return m == 2 ? qo[3] : 0.0;
}

// Device view of one level; the coefficient arrays hold S (float or double).
template <class S>
struct Lv {
  int nc;
  const int* nb;        // [nc][5]
  const int* mode;      // [nc]: 1 = swept by the multi-block kernels of this level
  const int* parent;    // [nc]
  const int* children;  // [nc of the next level][4]
  const double* qo;     // [nc][4]
  const S* A;           // [nc][5][12][12]
  const S* Dinv;        // [nc][12][12]
  S *x, *y, *b;         // [nc][12]
  const S* Ainv;        // [nfin][48][48]
};



// ---------------------------------------------------------------- fine <-> level 0
// Seeds of the level-0 Galerkin products: P1 function k of every element of colour col.
template <int N>
__global__ void k_p1_seed(fr::Mesh mesh, fr::Basis B, const int* __restrict__ colour, int col,
                          int k, double* __restrict__ x) {
  constexpr int NP = N * N;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)mesh.ne * NP) return;
  const int e = (int)(t / NP), pt = (int)(t % NP);
  const size_t base = mesh.qbase(e, NP), qs = mesh.qstride(e);
  const double val = colour[e] == col ? phi(B, k % 3, pt % N, pt / N) : 0.0;
#pragma unroll
  for (int v = 0; v < 4; ++v) x[v * qs + base + pt] = v == k / 3 ? val : 0.0;
}

// Column k of the level-0 blocks: P^T y on every element whose stencil holds a member of
// colour col (the seed's response on e comes from that member alone), and the response
// itself, the column (A P)_{e,s} e_k of the smoothing step, into AP [Ne][5][12][4 n^2].
// One thread per element row; the first 12 of an element also form the block column.
template <int N, class S>
__global__ void k_p1_gather(fr::Mesh mesh, fr::Basis B, const int* __restrict__ colslot, int ncol,
                            int col, int k, const double* __restrict__ y, S* __restrict__ A,
                            S* __restrict__ AP) {
  constexpr int NP = N * N, BS = 4 * NP;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)mesh.ne * BS) return;
  const int e = (int)(t / BS), r = (int)(t % BS);
  const int s = colslot[(size_t)e * ncol + col];
  if (s < 0) return;
  const size_t base = mesh.qbase(e, NP), qs = mesh.qstride(e);
  AP[(((size_t)e * SL + s) * NB + k) * BS + r] = (S)y[(r / NP) * qs + base + r % NP];
  if (r >= NB) return;
  const int v = r / 3, m = r % 3;
  double acc = 0.0;
  for (int pt = 0; pt < NP; ++pt) acc = fma(phi(B, m, pt % N, pt / N), y[v * qs + base + pt], acc);
  A[(((size_t)e * SL + s) * NB + r) * NB + k] = (S)acc;
}

// Level-0 operators and A P columns from the stored local Jacobians (the build without
// operator products).  Element e's rows respond to the P1 function (mode k) of a stencil
// member f != e only through their shared face: f's trace and local-gradient trace on it
// (by the basis' derivative and interpolation weights and f's metrics), the face Jacobian
// of f's side gives the change of the common flux, the common solution moves by half of
// f's trace and lifts into e's corrected gradient, and e's point Jacobians and corrected
// divergence give the rows.  A member reached through two faces (a 2-wide periodic
// direction) sums both.  The self columns are e's diagonal block times its own P1
// functions.  Each column is projected in FP64 onto e's P1 functions for the block of A_0
// and stored rounded to S for the smoothing step.  One block per element, G groups of n^2
// threads, one (member, mode) column per group and round.
template <int N> struct GalSmem {
  static constexpr int NP = N * N, BS = 4 * NP;
  static constexpr int G = 128 / NP > 0 ? 128 / NP : 1;
  static constexpr int JF = 4 * N * 48;            // neighbour side of e's four faces
  static constexpr int JGE = 64 * NP;              // e's point Jacobians in the corrected gradient
  static constexpr int SELF = 12 * BS;             // self columns
  // per group: f's gradient (x, y) at its points, traces (value, gx, gy), flux change,
  // F, G and the column
  static constexpr int GX = 0, GY = GX + NP, TQ = GY + NP, TGX = TQ + N, TGY = TGX + N,
                       DF = TGY + N, F = DF + 4 * N, GG = F + 4 * NP, COL = GG + 4 * NP,
                       PER = COL + 4 * NP;
  static constexpr size_t BYTES = sizeof(double) * (JF + JGE + SELF + (size_t)G * PER);
};

template <int N, class S>
__global__ void __launch_bounds__(GalSmem<N>::G * N * N)
k_mg_galerkin_lin(fr::Mesh M, fr::Basis B, const double* __restrict__ gs, const double* __restrict__ gf,
                  const double* __restrict__ JFQ, const double* __restrict__ JFG,
                  const double* __restrict__ JG, const double* __restrict__ B64,
                  const int* __restrict__ nb0, S* __restrict__ A0, S* __restrict__ AP) {
  using namespace fr;
  using L = GalSmem<N>;
  constexpr int NP = L::NP, BS = L::BS, G = L::G;
  extern __shared__ double smg[];
  double* sJF = smg;
  double* sJG = sJF + L::JF;
  double* sSelf = sJG + L::JGE;
  const int e = blockIdx.x;
  if (!M.on(e)) return;
  const int grp = threadIdx.x / NP, pt = threadIdx.x % NP;
  const int i = pt % N, j = pt / N;
  double* W = sSelf + L::SELF + (size_t)grp * L::PER;
  const bool visc = M.viscous;
  const int nf = M.ne * 2 * N;
  const size_t SN = (size_t)M.ne * NP, FNs = (size_t)M.ne * 4 * N;
  const int nbf[4] = {M.left(e), M.right(e), M.bottom(e), M.top(e)};   // FACE_L, R, B, T
  // neighbour side of each face's Jacobian: q entries (r, c) then g entries (r, c)
  for (int t = threadIdx.x; t < L::JF; t += blockDim.x) {
    const int f = t / (N * 48), rem = t % (N * 48), sp = rem / 48, k = rem % 48;
    double val = 0.0;
    if (nbf[f] >= 0) {
      const bool own = (f == FACE_R || f == FACE_T);   // e owns it: the neighbour is '+'
      const int owner = own ? e : nbf[f];
      const int dir = (f == FACE_R || f == FACE_L) ? 0 : 1;
      const size_t idx = ((size_t)owner * 2 + dir) * N + sp;
      if (k < 16) {
        const int r = k / 4, cc = k % 4;
        val = JFQ[(size_t)(r * 8 + (own ? 4 + cc : cc)) * nf + idx];
      } else if (visc) {
        const int r = (k - 16) / 8, cc = (k - 16) % 8;
        val = JFG[(size_t)(r * 16 + (own ? 8 + cc : cc)) * nf + idx];
      }
    }
    sJF[t] = val;
  }
  for (int t = threadIdx.x; t < L::JGE; t += blockDim.x)
    sJG[t] = visc ? JG[(size_t)(t / NP) * SN + (size_t)e * NP + t % NP] : 0.0;
  // self columns: B_e P_e (FP64)
  for (int t = threadIdx.x; t < L::SELF; t += blockDim.x) {
    const int k = t / BS, row = t % BS, v = k / 3, m = k % 3;
    const double* brow = B64 + ((size_t)e * BS + row) * BS + (size_t)v * NP;
    double acc = 0.0;
    for (int q = 0; q < NP; ++q) acc = fma(brow[q], phi(B, m, q % N, q / N), acc);
    sSelf[t] = acc;
  }
  // e's lifting weights at this point
  const size_t o = (size_t)e * NP + pt;
  const double ij = gs[GS_INVJ * SN + o];
  double lsx[4], lsy[4];
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
  // the self slot: A_0 block and stored columns
  for (int t = threadIdx.x; t < NB * BS; t += blockDim.x) {
    const int k = t / BS, row = t % BS;
    AP[(((size_t)e * SL + 0) * NB + k) * BS + row] = (S)sSelf[t];
  }
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    const int r = t / NB, k = t % NB, v = r / 3, m = r % 3;
    double acc = 0.0;
    for (int q = 0; q < NP; ++q) acc = fma(phi(B, m, q % N, q / N), sSelf[k * BS + v * NP + q], acc);
    A0[(((size_t)e * SL + 0) * NB + r) * NB + k] = (S)acc;
  }
  // neighbour slots: tasks (slot 1..4, mode) in rounds of G
  for (int t0 = 0; t0 < 4 * NB; t0 += G) {
    const int task = t0 + grp;
    const int slot = 1 + task / NB, k = task % NB, v = k / 3, m = k % 3;
    const int cell = task < 4 * NB ? nb0[(size_t)e * SL + slot] : -1;
    double col[4] = {0.0, 0.0, 0.0, 0.0};   // this point's rows (variables 0..3)
    for (int fe = 0; fe < 4; ++fe) {
      const bool act = cell >= 0 && nbf[fe] == cell;
      const int f = act ? cell : e;
      // f's face opposite fe, and the line of f's points ending at each face point
      const int fp = fe == FACE_L ? FACE_R : fe == FACE_R ? FACE_L : fe == FACE_B ? FACE_T : FACE_B;
      // 1: local gradient of the P1 function on f (variable v only)
      if (act && visc) {
        const size_t of = (size_t)f * NP + pt;
        double dxi = 0.0, deta = 0.0;
#pragma unroll
        for (int q = 0; q < N; ++q) {
          dxi = fma(B.D[i][q], phi(B, m, q, j), dxi);
          deta = fma(B.D[j][q], phi(B, m, i, q), deta);
        }
        const double fij = gs[GS_INVJ * SN + of];
        W[L::GX + pt] = (gs[GS_SXX * SN + of] * dxi + gs[GS_SEX * SN + of] * deta) * fij;
        W[L::GY + pt] = (gs[GS_SXY * SN + of] * dxi + gs[GS_SEY * SN + of] * deta) * fij;
      }
      __syncthreads();
      // 2: traces on f's face fp
      if (act && pt < N) {
        const int sp = pt;
        const double* w = (fp == FACE_L || fp == FACE_B) ? B.lL : B.lR;
        const bool row = (fp == FACE_L || fp == FACE_R);
        double tq = 0.0, tx = 0.0, ty = 0.0;
#pragma unroll
        for (int q = 0; q < N; ++q) {
          const int ii = row ? q : sp, jj = row ? sp : q;
          tq = fma(w[q], phi(B, m, ii, jj), tq);
          if (visc) {
            tx = fma(w[q], W[L::GX + jj * N + ii], tx);
            ty = fma(w[q], W[L::GY + jj * N + ii], ty);
          }
        }
        W[L::TQ + sp] = tq;
        W[L::TGX + sp] = tx;
        W[L::TGY + sp] = ty;
      }
      __syncthreads();
      // 3: change of the common flux on the shared face (only variable v's columns)
      for (int t = pt; act && t < 4 * N; t += NP) {
        const int r = t / N, sp = t % N;
        const double* jf = sJF + (fe * N + sp) * 48;
        double acc = jf[r * 4 + v] * W[L::TQ + sp];
        if (visc && r > 0) {
          acc = fma(jf[16 + r * 8 + v], W[L::TGX + sp], acc);
          acc = fma(jf[16 + r * 8 + 4 + v], W[L::TGY + sp], acc);
        }
        W[L::DF + r * N + sp] = acc;
      }
      // 4: e's fluxes from its corrected gradient (half of f's trace lifted through fe)
      if (act && visc) {
        const int sp = (fe < 2) ? j : i;
        const double half = 0.5 * W[L::TQ + sp];
        const double gx = half * lsx[fe], gy = half * lsy[fe];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const double val = (r % 4 == 0) ? 0.0
                           : fma(sJG[(r * 8 + v) * NP + pt], gx, sJG[(r * 8 + 4 + v) * NP + pt] * gy);
          if (r < 4) W[L::F + r * NP + pt] = val;
          else W[L::GG + (r - 4) * NP + pt] = val;
        }
      }
      __syncthreads();
      // 5: e's rows: corrected divergence of the fluxes and the face term of fe
      if (act) {
        const double dgw = (fe == FACE_L) ? B.dgL[i] : (fe == FACE_R) ? B.dgR[i]
                         : (fe == FACE_B) ? B.dgL[j] : B.dgR[j];
        const int sp = (fe < 2) ? j : i;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          double d = 0.0;
          if (visc) {
#pragma unroll
            for (int q = 0; q < N; ++q) d = fma(B.Dc[i][q], W[L::F + r * NP + j * N + q], d);
#pragma unroll
            for (int q = 0; q < N; ++q) d = fma(B.Dc[j][q], W[L::GG + r * NP + q * N + i], d);
          }
          d = fma(dgw, W[L::DF + r * N + sp], d);
          col[r] = fma(ij, d, col[r]);
        }
      }
      __syncthreads();
    }
    // the column to shared memory, stored and projected
    if (cell >= 0) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        W[L::COL + r * NP + pt] = col[r];
        AP[(((size_t)e * SL + slot) * NB + k) * BS + r * NP + pt] = (S)col[r];
      }
    }
    __syncthreads();
    for (int t = pt; cell >= 0 && t < NB; t += NP) {
      const int rv = t / 3, rm = t % 3;
      double acc = 0.0;
      for (int q = 0; q < NP; ++q) acc = fma(phi(B, rm, q % N, q / N), W[L::COL + rv * NP + q], acc);
      A0[(((size_t)e * SL + slot) * NB + t) * NB + k] = (S)acc;
    }
    __syncthreads();
  }
}

// b0 = P^T r (per element: 12 sums over its points, FP64, stored in S)
template <int N, class S>
__global__ void k_p1_restrict(fr::Mesh mesh, fr::Basis B, const double* __restrict__ r,
                              S* __restrict__ b0) {
  constexpr int NP = N * N;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)mesh.ne * NB) return;
  const int e = (int)(t / NB), row = (int)(t % NB);
  const size_t base = mesh.qbase(e, NP), qs = mesh.qstride(e);
  const int v = row / 3, m = row % 3;
  double acc = 0.0;
  for (int pt = 0; pt < NP; ++pt) acc = fma(phi(B, m, pt % N, pt / N), r[v * qs + base + pt], acc);
  b0[t] = (S)acc;
}

// ---------------------------------------------------------------- transposed preconditioner
// M^-1 = B^-1 + (I - B^-1 A) P V P^T with V the V-cycle on A's Galerkin operators, so
//   M^-T r = u + P V' (P^T r - (A P)^T u),   u = B^-T r,
// where V' = V^T is the same V-cycle on the transposed operators (the Galerkin operators of
// A^T are the transposes of A's, and a cycle with equal pre- and post-smoothing by damped
// block Jacobi transposes into the cycle on the transposed blocks).

// A^T's stencil blocks: block s of cell c is the transpose of block s' of member f = nb(c, s)
// (s' = the slot of c in f's stencil); diagonal inverses transposed for the smoothed cells.
template <class S>
__global__ void k_mg_transpose(Lv<S> L, const int* __restrict__ rslot, S* __restrict__ AT,
                               S* __restrict__ DinvT) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)L.nc * SL * BLK) return;
  const int c = (int)(t / (SL * BLK)), s = (int)(t / BLK % SL), ij = (int)(t % BLK);
  const int i = ij / NB, j = ij % NB;
  const int f = L.nb[c * SL + s];
  AT[t] = f >= 0 ? L.A[(((size_t)f * SL + rslot[c * SL + s]) * NB + j) * NB + i] : S(0);
  if (s == 0 && L.parent[c] >= 0) DinvT[((size_t)c * NB + i) * NB + j] = L.Dinv[((size_t)c * NB + j) * NB + i];
}

// Dense inverses of the finishing cases, transposed in their (12 m)^2 corner.
template <class S>
__global__ void k_mg_transpose_dense(const S* __restrict__ Ainv, const int* __restrict__ fin, int nfin,
                                     S* __restrict__ AinvT) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nfin * DN * DN) return;
  const int f = (int)(t / (DN * DN)), ij = (int)(t % (DN * DN)), i = ij / DN, j = ij % DN;
  const int m = fin[2 * f + 1] * NB;
  AinvT[t] = (i < m && j < m) ? Ainv[(size_t)f * DN * DN + (size_t)j * DN + i] : S(0);
}

// b0 = P^T r - (A P)^T u: row (e, k) sums the P1 projection of r and, over the stencil
// members g of e, the stored column of e's mode k on g's rows against u on g (FP64 sums).
template <int N, class S>
__global__ void k_p1_restrict_t(fr::Mesh mesh, fr::Basis B, const double* __restrict__ r,
                                const double* __restrict__ u, const S* __restrict__ AP,
                                const int* __restrict__ nb0, const int* __restrict__ rslot0,
                                S* __restrict__ b0) {
  constexpr int NP = N * N, BS = 4 * NP;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)mesh.ne * NB) return;
  const int e = (int)(t / NB), k = (int)(t % NB), v = k / 3, m = k % 3;
  const size_t base = mesh.qbase(e, NP), qs = mesh.qstride(e);
  double acc = 0.0;
  for (int pt = 0; pt < NP; ++pt) acc = fma(phi(B, m, pt % N, pt / N), r[v * qs + base + pt], acc);
  for (int jj = 0; jj < SL; ++jj) {
    const int g = nb0[(size_t)e * SL + jj];
    if (g < 0) continue;
    const S* ap = AP + (((size_t)g * SL + rslot0[(size_t)e * SL + jj]) * NB + k) * BS;
    const size_t gb = mesh.qbase(g, NP), gs = mesh.qstride(g);
    for (int row = 0; row < BS; ++row) acc = fma(-(double)ap[row], u[(row / NP) * gs + gb + row % NP], acc);
  }
  b0[t] = (S)acc;
}

// z = u + P y0 (FP64 out)
template <int N, class S>
__global__ void k_p1_prolong_add(fr::Mesh mesh, fr::Basis B, const S* __restrict__ y0,
                                 const double* __restrict__ u, double* __restrict__ z) {
  constexpr int NP = N * N;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)mesh.ne * NP) return;
  const int e = (int)(t / NP), pt = (int)(t % NP);
  const size_t base = mesh.qbase(e, NP), qs = mesh.qstride(e);
  const double xi = B.xs[pt % N], eta = B.xs[pt / N];
  const S* c = y0 + (size_t)e * NB;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const size_t gi = v * qs + base + pt;
    z[gi] = u[gi] + fma((double)c[3 * v + 2], eta, fma((double)c[3 * v + 1], xi, (double)c[3 * v]));
  }
}

// ---------------------------------------------------------------- multi-block levels
// A level of a case with more than TAIL cells (and at least 3 in each direction, so that a
// cell's four neighbours are distinct) runs in tiles of TX x TX cells, one block per tile
// with one thread per row of every cell of the tile and its halo, two launches per V-cycle:
//   down: the NU smoothing sweeps, the residual and the restriction to the parents;
//   up:   the prolongation of the parents' correction and the NU smoothing sweeps.
// A Jacobi sweep reads the neighbours' previous values, so each block recomputes a halo of
// NU cells around its tile (each sweep one cell less), in shared memory, instead of
// waiting for the other blocks: identical arithmetic on every copy, one launch per phase
// group instead of one per sweep.  The down pass writes the smoothed values to x and the
// parents' right-hand sides; the up pass reads x and the parents' results and writes the
// level's result to y (a block never reads what another block of the same launch writes).
constexpr int TX = 4;   // tile side: (TX + 2 NU)^2 x 12 threads, one per region row

struct CaseLevel {
  int nx, ny, off, bounded;
};

// Global cell at tile position (a, b) of a region with halo h: -1 outside a bounded mesh.
__device__ __forceinline__ int region_cell(const CaseLevel& g, int i0, int j0, int h, int a, int b) {
  int i = i0 - h + a, j = j0 - h + b;
  i = ((i % g.nx) + g.nx) % g.nx;
  if (g.bounded) {
    if (j < 0 || j >= g.ny) return -1;
  } else {
    j = ((j % g.ny) + g.ny) % g.ny;
  }
  return g.off + j * g.nx + i;
}

// Stencil slot of direction d (0 self, 1 left, 2 right, 3 below, 4 above) of a cell in row
// j: the slots list the distinct members in this order with absent ones left out.
__device__ __forceinline__ int dir_slot(const CaseLevel& g, int j, int d) {
  if (d < 3) return d;
  const bool below = !g.bounded || j > 0;
  const bool above = !g.bounded || j < g.ny - 1;
  if (d == 3) return below ? 3 : -1;
  return above ? (below ? 4 : 3) : -1;
}

// Row r of the operator block in stencil slot s of cell c (12 contiguous entries at a
// 48- or 96-byte multiple: 16-byte aligned), zeros for an absent slot (s < 0).
__device__ __forceinline__ void load_row12(const float* A, int c, int s, int r, float out[NB]) {
  if (s < 0) {
#pragma unroll
    for (int k = 0; k < NB; ++k) out[k] = 0.f;
    return;
  }
  const float4* p = reinterpret_cast<const float4*>(A + (((size_t)c * SL + s) * NB + r) * NB);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float4 v = p[q];
    out[4 * q] = v.x; out[4 * q + 1] = v.y; out[4 * q + 2] = v.z; out[4 * q + 3] = v.w;
  }
}
__device__ __forceinline__ void load_row12(const double* A, int c, int s, int r, double out[NB]) {
  if (s < 0) {
#pragma unroll
    for (int k = 0; k < NB; ++k) out[k] = 0.0;
    return;
  }
  const double2* p = reinterpret_cast<const double2*>(A + (((size_t)c * SL + s) * NB + r) * NB);
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const double2 v = p[q];
    out[2 * q] = v.x; out[2 * q + 1] = v.y;
  }
}

// Row r of (A x)_c: the five operator rows loaded first (vector loads), then the products.
template <class S>
__device__ __forceinline__ S row_product(const Lv<S>& L, int c, int r, const S* x) {
  S av[SL][NB];
  int nb[SL];
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    nb[s] = L.nb[c * SL + s];
    load_row12(L.A, c, nb[s] >= 0 ? s : -1, r, av[s]);
  }
  S acc = S(0);
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    if (nb[s] < 0) continue;
    const S* xf = x + (size_t)nb[s] * NB;
#pragma unroll
    for (int k = 0; k < NB; ++k) acc = fma(av[s][k], xf[k], acc);
  }
  return acc;
}

// r-th row of b - A x at region position (a, b) (cell c, row j of its case) with the
// neighbours' values in the region array xs (stride RX).
template <class S, int RX>
__device__ __forceinline__ S region_residual(const Lv<S>& L, const CaseLevel& g, int c, int j, int a, int bb,
                                             int r, const S* bs, const S (*xs)[NB]) {
  const int da[5] = {0, -1, 1, 0, 0}, db[5] = {0, 0, 0, -1, 1};
  // the five operator rows first (16-byte vector loads, absent members as zeros), then the
  // products: one round trip to memory instead of five
  S av[5][NB];
#pragma unroll
  for (int d = 0; d < 5; ++d) load_row12(L.A, c, dir_slot(g, j, d), r, av[d]);
  S acc = bs[r];
#pragma unroll
  for (int d = 0; d < 5; ++d) {
    const S* xn = xs[(bb + db[d]) * RX + a + da[d]];
#pragma unroll
    for (int k = 0; k < NB; ++k) acc = fma(-av[d][k], xn[k], acc);
  }
  return acc;
}

struct Tile {
  int k, i0, j0, pad;
};

// Dynamic shared memory of the tiled kernels: four region arrays of 12 coefficients and
// the region's cell indices.
template <class S, int NU>
constexpr size_t tile_smem() {
  return (size_t)4 * (TX + 2 * NU) * (TX + 2 * NU) * NB * sizeof(S) + (size_t)(TX + 2 * NU) * (TX + 2 * NU) * sizeof(int);
}

template <class S, int NU>
__global__ void __launch_bounds__((TX + 2 * NU) * (TX + 2 * NU) * NB, 2) k_mg_down(Lv<S> L, const CaseLevel* __restrict__ cl, const Tile* __restrict__ tiles,
                                                 S omega, S* __restrict__ bn) {
  constexpr int RX = TX + 2 * NU, RN = RX * RX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S (*sb)[NB] = reinterpret_cast<S (*)[NB]>(smem_raw);
  S (*x0)[NB] = sb + RN;
  S (*x1)[NB] = x0 + RN;
  S (*res)[NB] = x1 + RN;
  int* cell = reinterpret_cast<int*>(res + RN);
  const Tile T = tiles[blockIdx.x];
  const CaseLevel g = cl[T.k];
  // one thread per region row (RN * NB == blockDim): its row of D^-1 and of b, loaded first
  const int tp = threadIdx.x / NB, tr = threadIdx.x % NB;
  const int tc = region_cell(g, T.i0, T.j0, NU, tp % RX, tp / RX);
  S drow[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) drow[k] = tc >= 0 ? L.Dinv[((size_t)tc * NB + tr) * NB + k] : S(0);
  sb[tp][tr] = tc >= 0 ? L.b[(size_t)tc * NB + tr] : S(0);
  if (tr == 0) cell[tp] = tc;
  __syncthreads();
  // sweep 1 from zero: x = omega D^-1 b on the whole region
  {
    S acc = S(0);
#pragma unroll
    for (int k = 0; k < NB; ++k) acc = fma(drow[k], sb[tp][k], acc);
    x0[tp][tr] = omega * acc;
  }
  __syncthreads();
  S (*cur)[NB] = x0;
  S (*nxt)[NB] = x1;
  for (int sw = 1; sw < NU; ++sw) {
    // residual on the positions at least sw cells inside the region, then the update
    for (int t = threadIdx.x; t < RN * NB; t += blockDim.x) {
      const int p = t / NB, r = t % NB, a = p % RX, b = p / RX, c = cell[p];
      if (a < sw || a >= RX - sw || b < sw || b >= RX - sw || c < 0) continue;
      const int j = (c - g.off) / g.nx;
      res[p][r] = region_residual<S, RX>(L, g, c, j, a, b, r, sb[p], cur);
    }
    __syncthreads();
    {
      const int a = tp % RX, b = tp / RX;
      if (!(a < sw || a >= RX - sw || b < sw || b >= RX - sw || tc < 0)) {
        S acc = S(0);
#pragma unroll
        for (int k = 0; k < NB; ++k) acc = fma(drow[k], res[tp][k], acc);
        nxt[tp][tr] = cur[tp][tr] + omega * acc;
      }
    }
    __syncthreads();
    S (*tmp)[NB] = cur; cur = nxt; nxt = tmp;
  }
  // residual and smoothed values on the tile's own cells
  for (int t = threadIdx.x; t < TX * TX * NB; t += blockDim.x) {
    const int q = t / NB, r = t % NB, a = NU + q % TX, b = NU + q / TX, p = b * RX + a;
    const int i = T.i0 + q % TX, jj = T.j0 + q / TX, c = cell[p];
    if (i >= g.nx || jj >= g.ny || c < 0) continue;
    res[p][r] = region_residual<S, RX>(L, g, c, jj, a, b, r, sb[p], cur);
    L.x[(size_t)c * NB + r] = cur[p][r];
  }
  __syncthreads();
  // restriction to the parents of the tile (tiles start at even cells and have an even
  // side: a parent's children are all in its tile)
  constexpr int PX = TX / 2;
  for (int t = threadIdx.x; t < PX * PX * NB; t += blockDim.x) {
    const int q = t / NB, r = t % NB;
    const int i = T.i0 + 2 * (q % PX), jj = T.j0 + 2 * (q / PX);
    if (i >= g.nx || jj >= g.ny) continue;
    const int c00 = g.off + jj * g.nx + i;
    const int P = L.parent[c00];
    const int v = r / 3, m = r % 3;
    double acc = 0.0;
    for (int qq = 0; qq < 4; ++qq) {
      const int ch = L.children[P * 4 + qq];
      if (ch < 0) continue;
      const int ci = (ch - g.off) % g.nx, cj = (ch - g.off) / g.nx;
      const int p = (cj - T.j0 + NU) * RX + (ci - T.i0 + NU);
      const double* o = L.qo + (size_t)ch * 4;
      for (int a = 0; a < 3; ++a) acc = fma(qmap(o, a, m), (double)res[p][3 * v + a], acc);
    }
    bn[(size_t)P * NB + r] = (S)acc;
  }
}

template <class S, int NU>
__global__ void __launch_bounds__((TX + 2 * NU) * (TX + 2 * NU) * NB, 2) k_mg_up(Lv<S> L, const CaseLevel* __restrict__ cl, const Tile* __restrict__ tiles,
                                               S omega, const S* __restrict__ xp) {
  constexpr int RX = TX + 2 * NU, RN = RX * RX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S (*sb)[NB] = reinterpret_cast<S (*)[NB]>(smem_raw);
  S (*x0)[NB] = sb + RN;
  S (*x1)[NB] = x0 + RN;
  S (*res)[NB] = x1 + RN;
  int* cell = reinterpret_cast<int*>(res + RN);
  const Tile T = tiles[blockIdx.x];
  const CaseLevel g = cl[T.k];
  // one thread per region row (RN * NB == blockDim): its row of D^-1, loaded first
  const int tp = threadIdx.x / NB, tr = threadIdx.x % NB;
  const int tc = region_cell(g, T.i0, T.j0, NU, tp % RX, tp / RX);
  S drow[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) drow[k] = tc >= 0 ? L.Dinv[((size_t)tc * NB + tr) * NB + k] : S(0);
  if (tr == 0) cell[tp] = tc;
  __syncthreads();
  // the smoothed values plus the parents' correction, on the whole region
  for (int t = threadIdx.x; t < RN * NB; t += blockDim.x) {
    const int p = t / NB, r = t % NB, c = cell[p];
    S val = S(0), bv = S(0);
    if (c >= 0) {
      const int v = r / 3, a = r % 3;
      const double* o = L.qo + (size_t)c * 4;
      const S* X = xp + (size_t)L.parent[c] * NB + 3 * v;
      double acc = 0.0;
      for (int m = 0; m < 3; ++m) acc = fma(qmap(o, a, m), (double)X[m], acc);
      val = L.x[(size_t)c * NB + r] + (S)acc;
      bv = L.b[(size_t)c * NB + r];
    }
    x0[p][r] = val;
    sb[p][r] = bv;
  }
  __syncthreads();
  S (*cur)[NB] = x0;
  S (*nxt)[NB] = x1;
  for (int sw = 1; sw <= NU; ++sw) {
    for (int t = threadIdx.x; t < RN * NB; t += blockDim.x) {
      const int p = t / NB, r = t % NB, a = p % RX, b = p / RX, c = cell[p];
      if (a < sw || a >= RX - sw || b < sw || b >= RX - sw || c < 0) continue;
      const int j = (c - g.off) / g.nx;
      res[p][r] = region_residual<S, RX>(L, g, c, j, a, b, r, sb[p], cur);
    }
    __syncthreads();
    {
      const int a = tp % RX, b = tp / RX;
      if (!(a < sw || a >= RX - sw || b < sw || b >= RX - sw || tc < 0)) {
        S acc = S(0);
#pragma unroll
        for (int k = 0; k < NB; ++k) acc = fma(drow[k], res[tp][k], acc);
        nxt[tp][tr] = cur[tp][tr] + omega * acc;
      }
    }
    __syncthreads();
    S (*tmp)[NB] = cur; cur = nxt; nxt = tmp;
  }
  for (int t = threadIdx.x; t < TX * TX * NB; t += blockDim.x) {
    const int q = t / NB, r = t % NB, a = NU + q % TX, b = NU + q / TX, p = b * RX + a;
    const int i = T.i0 + q % TX, jj = T.j0 + q / TX, c = cell[p];
    if (i >= g.nx || jj >= g.ny || c < 0) continue;
    L.y[(size_t)c * NB + r] = cur[p][r];
  }
}

// ---------------------------------------------------------------- single-block tail
// The levels of one case from `lev0` on (each at most TAIL cells) and its exact solve, in
// one block: down (pre-smoothing, residual, restriction), the dense solve on the case's
// last level, up (prolongation, post-smoothing).  A sweep is two phases: y = b - A x for
// every cell, then x += omega D^-1 y in place (a phase reads only what the previous one
// wrote).
struct TailCase {
  int lev0, nlev;             // first level of the tail, levels of the case in total
  int off[16], cnt[16];       // the case's cells on each level
  int fin;                    // index of the case's dense inverse on its last level
};

template <class S>
__device__ void tail_sweep(const Lv<S>& L, int off, int cnt, S omega, bool first) {
  for (int t = threadIdx.x; t < cnt * NB; t += blockDim.x) {
    const int c = off + t / NB, r = t % NB;
    L.y[(size_t)c * NB + r] = L.b[(size_t)c * NB + r] - (first ? S(0) : row_product(L, c, r, L.x));
  }
  __syncthreads();
  for (int t = threadIdx.x; t < cnt * NB; t += blockDim.x) {
    const int c = off + t / NB, r = t % NB;
    const S* d = L.Dinv + ((size_t)c * NB + r) * NB;
    const S* yc = L.y + (size_t)c * NB;
    S acc = S(0);
#pragma unroll
    for (int k = 0; k < NB; ++k) acc = fma(d[k], yc[k], acc);
    L.x[(size_t)c * NB + r] = (first ? S(0) : L.x[(size_t)c * NB + r]) + omega * acc;
  }
  __syncthreads();
}

template <class S>
__global__ void __launch_bounds__(TAIL_THREADS) k_mg_tail(const Lv<S>* __restrict__ lev,
                                                         const TailCase* __restrict__ tc,
                                                         const int* __restrict__ cases, int nu,
                                                         S omega) {
  const TailCase T = tc[cases[blockIdx.x]];
  const int last = T.nlev - 1;
  for (int l = T.lev0; l < last; ++l) {
    const Lv<S> L = lev[l];
    const int off = T.off[l], cnt = T.cnt[l];
    for (int it = 0; it < nu; ++it) tail_sweep(L, off, cnt, omega, it == 0);
    for (int t = threadIdx.x; t < cnt * NB; t += blockDim.x) {
      const int c = off + t / NB, r = t % NB;
      L.y[(size_t)c * NB + r] = L.b[(size_t)c * NB + r] - row_product(L, c, r, L.x);
    }
    __syncthreads();
    const Lv<S> Nn = lev[l + 1];
    for (int t = threadIdx.x; t < T.cnt[l + 1] * NB; t += blockDim.x) {
      const int I = T.off[l + 1] + t / NB, r = t % NB, v = r / 3, m = r % 3;
      double acc = 0.0;
      for (int q = 0; q < 4; ++q) {
        const int c = L.children[I * 4 + q];
        if (c < 0) continue;
        const double* o = L.qo + (size_t)c * 4;
        for (int a = 0; a < 3; ++a) acc = fma(qmap(o, a, m), (double)L.y[(size_t)c * NB + 3 * v + a], acc);
      }
      Nn.b[(size_t)I * NB + r] = (S)acc;
    }
    __syncthreads();
  }
  {
    const Lv<S> L = lev[last];
    const int off = T.off[last], m = T.cnt[last] * NB;
    const S* Ai = L.Ainv + (size_t)T.fin * DN * DN;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
      S acc = S(0);
      for (int k = 0; k < m; ++k) acc = fma(Ai[r * DN + k], L.b[(size_t)off * NB + k], acc);
      L.x[(size_t)off * NB + r] = acc;
    }
    __syncthreads();
  }
  for (int l = last - 1; l >= T.lev0; --l) {
    const Lv<S> L = lev[l];
    const Lv<S> Nn = lev[l + 1];
    const int off = T.off[l], cnt = T.cnt[l];
    for (int t = threadIdx.x; t < cnt * NB; t += blockDim.x) {
      const int c = off + t / NB, r = t % NB, v = r / 3, a = r % 3;
      const double* o = L.qo + (size_t)c * 4;
      const S* X = Nn.x + (size_t)L.parent[c] * NB + 3 * v;
      double acc = 0.0;
      for (int m = 0; m < 3; ++m) acc = fma(qmap(o, a, m), (double)X[m], acc);
      L.x[(size_t)c * NB + r] += (S)acc;
    }
    __syncthreads();
    for (int it = 0; it < nu; ++it) tail_sweep(L, off, cnt, omega, false);
  }
  // the result of the first level of the tail goes to y, where the tiled levels and the
  // prolongation to the solution points read each level's result
  {
    const Lv<S> L = lev[T.lev0];
    for (int t = threadIdx.x; t < T.cnt[T.lev0] * NB; t += blockDim.x)
      L.y[(size_t)T.off[T.lev0] * NB + t] = L.x[(size_t)T.off[T.lev0] * NB + t];
  }
}

// ---------------------------------------------------------------- build kernels
// Dinv = inverse of the diagonal (slot 0) block of every cell that is smoothed (parent
// >= 0); *bad counts singular blocks.  One warp per cell: Gauss-Jordan with partial
// pivoting on [A | I] in FP64, lane c < 24 holding column c of the 12 x 24 array in
// registers (the pivot search by the pivot column's lane, the row operations by every
// lane on its own column with the multipliers broadcast from that lane).
template <class S>
__global__ void k_mg_invert_diag(Lv<S> L, S* __restrict__ Dinv, int* __restrict__ bad) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= L.nc || L.parent[c] < 0) return;
  const S* src = L.A + (size_t)c * SL * BLK;   // slot 0: the diagonal block
  double col[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i)
    col[i] = lane < NB ? (double)src[i * NB + lane] : (lane < 2 * NB && i == lane - NB ? 1.0 : 0.0);
  bool singular = false;
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    // pivot row: the largest |a[i][k]|, i >= k (lane k searches its column)
    int p = k;
    double best = 0.0;
#pragma unroll
    for (int i = 0; i < NB; ++i)
      if (i >= k && fabs(col[i]) > best) { best = fabs(col[i]); p = i; }
    p = __shfl_sync(0xffffffffu, p, k);
    best = __shfl_sync(0xffffffffu, best, k);
    if (!(best > 0.0)) { singular = true; break; }
    // swap rows k and p in every column
    double rk = 0.0, rp = 0.0;
#pragma unroll
    for (int i = 0; i < NB; ++i) { if (i == k) rk = col[i]; if (i == p) rp = col[i]; }
#pragma unroll
    for (int i = 0; i < NB; ++i) { if (i == k) col[i] = rp; else if (i == p) col[i] = rk; }
    // scale row k by the pivot, then eliminate column k from every other row
    const double piv = __shfl_sync(0xffffffffu, rp, k);
    const double inv = 1.0 / piv;
    double rowk = 0.0;
#pragma unroll
    for (int i = 0; i < NB; ++i) if (i == k) { col[i] *= inv; rowk = col[i]; }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const double f = __shfl_sync(0xffffffffu, col[i], k);   // a[i][k] after the swap
      if (i != k) col[i] = fma(-f, rowk, col[i]);
    }
  }
  if (singular) {
    if (lane == 0) atomicAdd(bad, 1);
    return;
  }
  S* dst = Dinv + (size_t)c * BLK;
  if (lane >= NB && lane < 2 * NB) {
#pragma unroll
    for (int i = 0; i < NB; ++i) dst[i * NB + (lane - NB)] = (S)col[i];
  }
}

// Dense inverse of each finishing case: its cells' blocks assembled into one (12 m)^2
// matrix in shared memory (m <= 4) and inverted by Gauss-Jordan with partial pivoting in
// FP64, the block's threads sharing each elimination step.
template <class S>
__global__ void k_mg_coarsest(Lv<S> L, const int* __restrict__ fin, S* __restrict__ Ainv,
                              int* __restrict__ bad) {
  __shared__ double a[DN * DN];
  __shared__ double inv[DN * DN];
  __shared__ double col[DN];
  __shared__ int piv;
  const int f = blockIdx.x, c0 = fin[2 * f], cnt = fin[2 * f + 1], m = cnt * NB;
  for (int t = threadIdx.x; t < DN * DN; t += blockDim.x) {
    a[t] = 0.0;
    inv[t] = (t / DN == t % DN) ? 1.0 : 0.0;
  }
  __syncthreads();
  // rows of cell c0 + i; one column block per distinct stencil member of the case
  for (int t = threadIdx.x; t < cnt * SL * BLK; t += blockDim.x) {
    const int i = t / (SL * BLK), s = (t / BLK) % SL, rk = t % BLK;
    const int ci = c0 + i, fj = L.nb[ci * SL + s];
    if (fj < 0) continue;
    const int j = fj - c0, r = rk / NB, k = rk % NB;
    a[(i * NB + r) * DN + j * NB + k] = (double)L.A[((size_t)ci * SL + s) * BLK + rk];
  }
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      double best = fabs(a[k * DN + k]);
      for (int i = k + 1; i < m; ++i)
        if (fabs(a[i * DN + k]) > best) { best = fabs(a[i * DN + k]); p = i; }
      if (!(best > 0.0)) { atomicAdd(bad, 1); p = -1; }
      piv = p;
    }
    __syncthreads();
    const int p = piv;
    if (p < 0) break;
    if (p != k) {
      for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double t = a[k * DN + j]; a[k * DN + j] = a[p * DN + j]; a[p * DN + j] = t;
        t = inv[k * DN + j]; inv[k * DN + j] = inv[p * DN + j]; inv[p * DN + j] = t;
      }
    }
    __syncthreads();
    const double d = 1.0 / a[k * DN + k];
    __syncthreads();   // every thread has read the pivot before row k is scaled
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      a[k * DN + j] *= d;
      inv[k * DN + j] *= d;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) col[i] = a[i * DN + k];
    __syncthreads();
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int i = t / m, j = t % m;
      if (i == k) continue;
      a[i * DN + j] = fma(-col[i], a[k * DN + j], a[i * DN + j]);
      inv[i * DN + j] = fma(-col[i], inv[k * DN + j], inv[i * DN + j]);
    }
    __syncthreads();
  }
  S* dst = Ainv + (size_t)f * DN * DN;
  for (int t = threadIdx.x; t < DN * DN; t += blockDim.x) dst[t] = (S)inv[t];
}

// A_{l+1} = Q^T A_l Q: entry (r, k) of coarse block (I, S) sums, over the children c of I
// and their slots s whose member's parent is slot S of I, Q_c^T A_l[c][s] Q_f (FP64).
template <class S>
__global__ void k_mg_galerkin(Lv<S> L, const int* __restrict__ gslot, int nc_next,
                              const int* __restrict__ nb_next, S* __restrict__ An) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nc_next * SL * BLK) return;
  const int I = (int)(t / (SL * BLK)), Sl = (int)((t / BLK) % SL), rk = (int)(t % BLK);
  if (nb_next[I * SL + Sl] < 0) { An[t] = S(0); return; }
  const int r = rk / NB, k = rk % NB;
  const int v = r / 3, m = r % 3, w = k / 3, mk = k % 3;
  double acc = 0.0;
  for (int q = 0; q < 4; ++q) {
    const int c = L.children[I * 4 + q];
    if (c < 0) continue;
    const double* oc = L.qo + (size_t)c * 4;
    for (int s = 0; s < SL; ++s) {
      if (gslot[c * SL + s] != Sl) continue;
      const int f = L.nb[c * SL + s];
      const double* of = L.qo + (size_t)f * 4;
      const S* a = L.A + ((size_t)c * SL + s) * BLK;
      for (int ap = 0; ap < 3; ++ap) {
        const double qa = qmap(oc, ap, m);
        if (qa == 0.0) continue;
        double inner = 0.0;
        for (int bp = 0; bp < 3; ++bp)
          inner = fma((double)a[(3 * v + ap) * NB + 3 * w + bp], qmap(of, bp, mk), inner);
        acc = fma(qa, inner, acc);
      }
    }
  }
  An[t] = (S)acc;
}

unsigned blocks_for(long long n, int th) { return (unsigned)((n + th - 1) / th); }

template <class T> int dalloc(fr_ctx* c, T** p, size_t count) {
  if (*p) { cudaFree(*p); *p = nullptr; }
  if (count == 0) return FR_OK;
  FR_CUDA_CHECK(c, cudaMalloc((void**)p, count * sizeof(T)));
  return FR_OK;
}

template <class T> int upload(fr_ctx* c, T** p, const std::vector<T>& h) {
  FR_TRY(dalloc(c, p, h.size()));
  if (!h.empty()) FR_CUDA_CHECK(c, cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return FR_OK;
}

int op_apply(fr_ctx* c, const double* q, const double* x, double inv_dtau, double a0_dt, double* out,
             cudaStream_t s) {
  if (c->cfg.jvp_mode == FR_JVP_LINEARIZED) return frk::apply_linear(c, x, out, false, s);
  return frk::jvp(c, q, x, inv_dtau, a0_dt, out, s);
}

// The level as the kernels see it: A's operators, or with tr the transposed hierarchy's.
template <class S>
Lv<S> view(const MgLevel& l, bool tr = false) {
  Lv<S> v;
  v.nc = l.nc;
  v.nb = l.nb;
  v.mode = l.mode;
  v.parent = l.parent;
  v.children = l.children;
  v.qo = l.qo;
  v.A = (const S*)(tr ? l.AT : l.A);
  v.Dinv = (const S*)(tr ? l.DinvT : l.Dinv);
  v.x = (S*)l.x;
  v.y = (S*)l.y;
  v.b = (S*)l.b;
  v.Ainv = (const S*)(tr ? l.AinvT : l.Ainv);
  return v;
}

// Cells of one level of one case: an nx x ny grid (periodic in xi, in eta unless bounded).
struct CaseGrid {
  int nx, ny, off;
};

void stencil_of(const CaseGrid& g, bool bounded, int i, int j, int* out) {
  int cand[5] = {g.off + j * g.nx + i, g.off + j * g.nx + (i + g.nx - 1) % g.nx,
                 g.off + j * g.nx + (i + 1) % g.nx, -1, -1};
  if (!bounded || j > 0) cand[3] = g.off + ((j + g.ny - 1) % g.ny) * g.nx + i;
  if (!bounded || j < g.ny - 1) cand[4] = g.off + ((j + 1) % g.ny) * g.nx + i;
  int n = 0;
  for (int k = 0; k < 5; ++k) {
    if (cand[k] < 0) continue;
    bool dup = false;
    for (int q = 0; q < n; ++q) dup = dup || out[q] == cand[k];
    if (!dup) out[n++] = cand[k];
  }
  for (int k = n; k < SL; ++k) out[k] = -1;
}

template <int N, class S>
int build_level0(fr_ctx* c, const double* q, double inv_dtau, double a0_dt, cudaStream_t s) {
  constexpr int NP = N * N;
  MgLevel& L0 = c->mg[0];
  if (c->cfg.jvp_mode == FR_JVP_LINEARIZED) {
    // from the local Jacobians stored at q (the operator GMRES applies) and the element
    // blocks of the same build
    using GL = GalSmem<N>;
    FR_CUDA_CHECK(c, cudaFuncSetAttribute(k_mg_galerkin_lin<N, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)GL::BYTES));
    FR_PROF_BEGIN(c, s);
    k_mg_galerkin_lin<N, S><<<c->ne, GL::G * NP, GL::BYTES, s>>>(c->mesh, c->basis, c->gs, c->gf, c->JFQ,
                                                                c->JFG, c->JG, c->B64, L0.nb, (S*)L0.A,
                                                                (S*)c->mg_ap);
    FR_PROF_END(c, s, KK_COARSE);
    FR_LAUNCH_CHECK(c);
    // per element: 48 neighbour columns (traces, face products, lifted fluxes, divergence)
    // and 12 self columns, each projected on 12 P1 functions
    FR_ACCOUNT(c, KK_COARSE, 2.0 * c->ne * (48.0 * NP * (4.0 * N + 24.0 + 2.0 * NB) + 12.0 * 4 * NP * NP + 60.0 * NB * NP), 0.0);
    return FR_OK;
  }
  const long long npts = (long long)c->ne * NP;
  // one operator product per colour and P1 function
  for (int col = 0; col < c->mg_ncol; ++col) {
    for (int k = 0; k < NB; ++k) {
      {
        FR_PROF_BEGIN(c, s);
        k_p1_seed<N><<<blocks_for(npts, 256), 256, 0, s>>>(c->mesh, c->basis, c->mg_colslot, col, k, c->mg_x);
        FR_PROF_END(c, s, KK_COARSE);
        FR_LAUNCH_CHECK(c);
      }
      FR_TRY(op_apply(c, q, c->mg_x, inv_dtau, a0_dt, c->mg_y, s));
      {
        FR_PROF_BEGIN(c, s);
        k_p1_gather<N, S><<<blocks_for((long long)c->ne * 4 * NP, 256), 256, 0, s>>>(
            c->mesh, c->basis, c->mg_colslot + (size_t)c->ne, c->mg_ncol, col, k, c->mg_y, (S*)L0.A,
            (S*)c->mg_ap);
        FR_PROF_END(c, s, KK_COARSE);
        FR_LAUNCH_CHECK(c);
      }
    }
  }
  FR_ACCOUNT(c, KK_COARSE, (double)c->mg_ncol * NB * c->ne * NB * 2.0 * NP, 0.0);
  return FR_OK;
}

template <class S>
int build_levels(fr_ctx* c, cudaStream_t s) {
  for (size_t l = 0; l < c->mg.size(); ++l) {
    MgLevel& L = c->mg[l];
    const Lv<S> V = view<S>(L);
    FR_PROF_BEGIN(c, s);
    k_mg_invert_diag<S><<<blocks_for((long long)L.nc * 32, 128), 128, 0, s>>>(V, (S*)L.Dinv, c->mg_bad);
    if (L.nfin > 0) k_mg_coarsest<S><<<L.nfin, 128, 0, s>>>(V, L.fin, (S*)L.Ainv, c->mg_bad);
    if (l + 1 < c->mg.size()) {
      const MgLevel& Nx = c->mg[l + 1];
      k_mg_galerkin<S><<<blocks_for((long long)Nx.nc * SL * BLK, 256), 256, 0, s>>>(
          V, L.gslot, Nx.nc, Nx.nb, (S*)Nx.A);
    }
    FR_PROF_END(c, s, KK_COARSE);
    FR_LAUNCH_CHECK(c);
    FR_ACCOUNT(c, KK_COARSE, 2.0 * NB * NB * NB * L.nc, 0.0);
  }
  return FR_OK;
}

// b0 = P^T r (the prolongation back is fused into the block apply)
template <int N, class S>
int fine_restrict(fr_ctx* c, const double* r, cudaStream_t s) {
  constexpr int NP = N * N;
  FR_PROF_BEGIN(c, s);
  k_p1_restrict<N, S><<<blocks_for((long long)c->ne * NB, 256), 256, 0, s>>>(c->mesh, c->basis, r, (S*)c->mg[0].b);
  FR_PROF_END(c, s, KK_COARSE);
  FR_LAUNCH_CHECK(c);
  FR_ACCOUNT(c, KK_COARSE, 2.0 * NB * c->ne * NP, 8.0 * 4.0 * c->ne * NP + (double)sizeof(S) * NB * c->ne);
  return FR_OK;
}

template <class S>
int launch_tail(fr_ctx* c, const MgLevel& L, cudaStream_t s, bool tr) {
  FR_PROF_BEGIN(c, s);
  k_mg_tail<S><<<L.ntail, TAIL_THREADS, 0, s>>>((const Lv<S>*)(tr ? c->mg_views_t : c->mg_views), (const TailCase*)c->mg_tc,
                                                 L.tail, c->cfg.mg_sweeps, (S)c->cfg.mg_omega);
  FR_PROF_END(c, s, KK_COARSE);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

// One V-cycle: the tails of the cases that are small from level 0 on, then per tiled level
// the down pass (and the tails of the cases whose single-block part starts below it), then
// the up passes in reverse order; every level's result ends in y.
template <class S, int NU>
int vcycle_n(fr_ctx* c, cudaStream_t s, bool tr) {
  const S om = (S)c->cfg.mg_omega;
  if (tile_smem<S, NU>() > 48 * 1024) {
    FR_CUDA_CHECK(c, cudaFuncSetAttribute(k_mg_down<S, NU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem<S, NU>()));
    FR_CUDA_CHECK(c, cudaFuncSetAttribute(k_mg_up<S, NU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem<S, NU>()));
  }
  if (c->mg[0].ntail > 0) FR_TRY(launch_tail<S>(c, c->mg[0], s, tr));
  size_t ltop = 0;
  while (ltop < c->mg.size() && c->mg[ltop].ntiles > 0) ++ltop;
  for (size_t l = 0; l < ltop; ++l) {
    MgLevel& L = c->mg[l];
    MgLevel& Nx = c->mg[l + 1];
    {
      FR_PROF_BEGIN(c, s);
      k_mg_down<S, NU><<<L.ntiles, (TX + 2 * NU) * (TX + 2 * NU) * NB, tile_smem<S, NU>(), s>>>(view<S>(L, tr), (const CaseLevel*)L.cl, (const Tile*)L.tiles, om, (S*)Nx.b);
      FR_PROF_END(c, s, KK_COARSE);
      FR_LAUNCH_CHECK(c);
    }
    if (Nx.ntail > 0) FR_TRY(launch_tail<S>(c, Nx, s, tr));
  }
  for (size_t l = ltop; l-- > 0;) {
    MgLevel& L = c->mg[l];
    MgLevel& Nx = c->mg[l + 1];
    FR_PROF_BEGIN(c, s);
    k_mg_up<S, NU><<<L.ntiles, (TX + 2 * NU) * (TX + 2 * NU) * NB, tile_smem<S, NU>(), s>>>(view<S>(L, tr), (const CaseLevel*)L.cl, (const Tile*)L.tiles, om, (const S*)Nx.y);
    FR_PROF_END(c, s, KK_COARSE);
    FR_LAUNCH_CHECK(c);
  }
  for (size_t l = 0; l < ltop; ++l) {
    const MgLevel& L = c->mg[l];
    const double cells = (double)L.nsweep;
    // per cycle and cell: (2 NU + 1) residual rows of 5 blocks and 2 NU inverse rows of 12
    FR_ACCOUNT(c, KK_COARSE, cells * NB * 2.0 * ((2.0 * NU + 1.0) * SL * NB + 2.0 * NU * NB),
               (double)sizeof(S) * cells * ((2.0 * NU + 1.0) * SL * BLK + 2.0 * NU * BLK));
  }
  return FR_OK;
}

template <class S>
int vcycle(fr_ctx* c, cudaStream_t s, bool tr = false) {
  return c->cfg.mg_sweeps == 1 ? vcycle_n<S, 1>(c, s, tr) : vcycle_n<S, 2>(c, s, tr);
}

template <class S>
int apply_t(fr_ctx* c, const double* q, const double* r, double* z, double inv_dtau, double a0_dt,
            cudaStream_t s) {
  int rc;
  switch (c->n) {
    case 2: rc = fine_restrict<2, S>(c, r, s); break;
    case 3: rc = fine_restrict<3, S>(c, r, s); break;
    case 4: rc = fine_restrict<4, S>(c, r, s); break;
    case 5: rc = fine_restrict<5, S>(c, r, s); break;
    default: return FR_ERR_ARG;
  }
  if (rc != FR_OK) return rc;
  FR_TRY(vcycle<S>(c, s));
  // z = z0 + B^-1 (r - A z0) with z0 = P y0: the block apply prolongs y0 and forms A z0 from
  // the build's stored columns A P, in one pass
  CoarseIn ci;
  ci.AP = c->mg_ap;
  ci.y0 = c->mg[0].y;
  ci.nb = c->mg[0].nb;
  for (int i = 0; i < c->n; ++i) ci.xs[i] = c->basis.xs[i];
  return frk::block_apply_coarse(c, r, z, ci, sizeof(S) == sizeof(float) ? 1 : 2, s);
}

// z = M^-T r: u = B^-T r, b0 = P^T r - (A P)^T u, the cycle on the transposed hierarchy,
// z = u + P y0 (the transposed hierarchy built by mg_transpose for this build)
template <int N, class S>
int apply_tr_n(fr_ctx* c, const double* r, double* z, cudaStream_t s) {
  constexpr int NP = N * N;
  double* u = c->mg_x;
  FR_TRY(frk::block_apply(c, r, u, s));   // c->transposed: B^-T
  MgLevel& L0 = c->mg[0];
  {
    FR_PROF_BEGIN(c, s);
    k_p1_restrict_t<N, S><<<blocks_for((long long)c->ne * NB, 256), 256, 0, s>>>(
        c->mesh, c->basis, r, u, (const S*)c->mg_ap, L0.nb, L0.rslot, (S*)L0.b);
    FR_PROF_END(c, s, KK_COARSE);
    FR_LAUNCH_CHECK(c);
  }
  FR_TRY(vcycle<S>(c, s, true));
  {
    FR_PROF_BEGIN(c, s);
    k_p1_prolong_add<N, S><<<blocks_for((long long)c->ne * NP, 256), 256, 0, s>>>(c->mesh, c->basis,
                                                                                (const S*)L0.y, u, z);
    FR_PROF_END(c, s, KK_COARSE);
    FR_LAUNCH_CHECK(c);
  }
  return FR_OK;
}

template <class S>
int apply_tr(fr_ctx* c, const double* r, double* z, cudaStream_t s) {
  switch (c->n) {
    case 2: return apply_tr_n<2, S>(c, r, z, s);
    case 3: return apply_tr_n<3, S>(c, r, z, s);
    case 4: return apply_tr_n<4, S>(c, r, z, s);
    case 5: return apply_tr_n<5, S>(c, r, z, s);
  }
  return FR_ERR_ARG;
}

template <class S>
int transpose_levels(fr_ctx* c, cudaStream_t s) {
  std::vector<Lv<S>> views;
  for (MgLevel& L : c->mg) {
    const size_t esz = sizeof(S), n12 = (size_t)L.nc * NB;
    if (!L.AT) FR_CUDA_CHECK(c, cudaMalloc(&L.AT, n12 * SL * NB * esz));
    if (!L.DinvT) {
      FR_CUDA_CHECK(c, cudaMalloc(&L.DinvT, n12 * NB * esz));
      FR_CUDA_CHECK(c, cudaMemset(L.DinvT, 0, n12 * NB * esz));
    }
    if (L.nfin > 0 && !L.AinvT) FR_CUDA_CHECK(c, cudaMalloc(&L.AinvT, (size_t)L.nfin * DN * DN * esz));
    FR_PROF_BEGIN(c, s);
    k_mg_transpose<S><<<blocks_for((long long)L.nc * SL * BLK, 256), 256, 0, s>>>(view<S>(L), L.rslot,
                                                                                 (S*)L.AT, (S*)L.DinvT);
    if (L.nfin > 0)
      k_mg_transpose_dense<S><<<blocks_for((long long)L.nfin * DN * DN, 256), 256, 0, s>>>(
          (const S*)L.Ainv, L.fin, L.nfin, (S*)L.AinvT);
    FR_PROF_END(c, s, KK_COARSE);
    FR_LAUNCH_CHECK(c);
    views.push_back(view<S>(L, true));
  }
  FR_CUDA_CHECK(c, cudaMemcpyAsync(c->mg_views_t, views.data(), views.size() * sizeof(Lv<S>),
                                   cudaMemcpyHostToDevice, s));
  FR_CUDA_CHECK(c, cudaStreamSynchronize(s));   // views is a host temporary
  c->mg_t_ready = 1;
  return FR_OK;
}

template <class S>
int upload_views(fr_ctx* c) {
  std::vector<Lv<S>> views;
  for (const MgLevel& L : c->mg) views.push_back(view<S>(L));
  FR_CUDA_CHECK(c, cudaMemcpy(c->mg_views, views.data(), views.size() * sizeof(Lv<S>), cudaMemcpyHostToDevice));
  return FR_OK;
}

}  // namespace

namespace frk {

void mg_free(fr_ctx* c) {
  for (MgLevel& l : c->mg) {
    int* is[] = {l.nb, l.cell_case, l.parent, l.children, l.gslot, l.fin, l.mode, l.tail, l.rslot};
    for (int* p : is) if (p) cudaFree(p);
    void* vs[] = {l.A, l.Dinv, l.x, l.y, l.b, l.Ainv, l.tiles, l.cl, l.AT, l.DinvT, l.AinvT};
    for (void* p : vs) if (p) cudaFree(p);
    if (l.qo) cudaFree(l.qo);
  }
  c->mg.clear();
  if (c->mg_colslot) { cudaFree(c->mg_colslot); c->mg_colslot = nullptr; }
  double** fs[] = {&c->mg_x, &c->mg_y};
  for (double** p : fs) if (*p) { cudaFree(*p); *p = nullptr; }
  if (c->mg_ap) { cudaFree(c->mg_ap); c->mg_ap = nullptr; }
  if (c->mg_bad) { cudaFree(c->mg_bad); c->mg_bad = nullptr; }
  if (c->mg_views) { cudaFree(c->mg_views); c->mg_views = nullptr; }
  if (c->mg_views_t) { cudaFree(c->mg_views_t); c->mg_views_t = nullptr; }
  c->mg_t_ready = 0;
  if (c->mg_tc) { cudaFree(c->mg_tc); c->mg_tc = nullptr; }
  c->mg_ncol = 0;
  c->mg_q = nullptr;
}

int mg_setup(fr_ctx* c) {
  mg_free(c);
  if (c->cfg.precond != FR_PRECOND_TWO_LEVEL) return FR_OK;
  const bool bounded = c->bounded != 0;
  const bool f64 = c->cfg.mg_prec == FR_PREC_FP64;
  const size_t esz = f64 ? sizeof(double) : sizeof(float);
  // level grids of every case, cells numbered case after case
  std::vector<CaseGrid> grids(c->ncases);
  int off = 0;
  for (int k = 0; k < c->ncases; ++k) {
    grids[k] = CaseGrid{c->cps[k].nx, c->cps[k].ny, off};
    off += c->cps[k].nx * c->cps[k].ny;
  }
  std::vector<char> done(c->ncases, 0);
  std::vector<TailCase> tcs(c->ncases);
  for (int k = 0; k < c->ncases; ++k) {
    std::memset(&tcs[k], 0, sizeof(TailCase));
    tcs[k].lev0 = -1;
    tcs[k].fin = -1;
  }
  std::vector<std::vector<int>> h_nb, h_case, h_parent, h_children, h_gslot, h_fin, h_mode, h_tail;
  std::vector<std::vector<double>> h_qo;
  std::vector<int> h_nsweep;
  std::vector<std::vector<Tile>> h_tiles;
  std::vector<std::vector<CaseLevel>> h_cls;
  while (true) {
    const int lev = (int)h_nb.size();
    int nc = 0;
    for (int k = 0; k < c->ncases; ++k) if (!done[k]) nc += grids[k].nx * grids[k].ny;
    if (nc == 0) break;
    if (lev >= 16) { snprintf(c->err, sizeof(c->err), "two-level set-up: too many levels"); return FR_ERR_ARG; }
    std::vector<int> nb((size_t)nc * SL), cs(nc), parent(nc, -1), gsl((size_t)nc * SL, -1), fin;
    std::vector<int> mode(nc, 0), tail;
    std::vector<Tile> tiles;
    std::vector<CaseLevel> cls(c->ncases, CaseLevel{0, 0, 0, 0});
    std::vector<double> qo((size_t)nc * 4, 0.0);
    std::vector<CaseGrid> next(c->ncases);
    int noff = 0, nsweep = 0;
    for (int k = 0; k < c->ncases; ++k) {
      if (done[k]) continue;
      const CaseGrid& g = grids[k];
      const int cnt = g.nx * g.ny;
      TailCase& T = tcs[k];
      T.off[lev] = g.off;
      T.cnt[lev] = cnt;
      T.nlev = lev + 1;
      if ((cnt <= TAIL || g.nx < 3 || g.ny < 3) && T.lev0 < 0) { T.lev0 = lev; tail.push_back(k); }
      if (cnt <= MAXFIN) {
        T.fin = (int)fin.size() / 2;
        fin.push_back(g.off);
        fin.push_back(cnt);
      } else {
        next[k] = CaseGrid{(g.nx + 1) / 2, (g.ny + 1) / 2, noff};
        noff += next[k].nx * next[k].ny;
      }
    }
    for (int k = 0; k < c->ncases; ++k) {
      if (done[k]) continue;
      const CaseGrid& g = grids[k];
      const bool cont = g.nx * g.ny > MAXFIN;
      const bool swept = tcs[k].lev0 < 0;   // not yet in the case's single-block kernel
      cls[k] = CaseLevel{g.nx, g.ny, g.off, bounded ? 1 : 0};
      if (swept)
        for (int j0 = 0; j0 < g.ny; j0 += TX)
          for (int i0 = 0; i0 < g.nx; i0 += TX) tiles.push_back(Tile{k, i0, j0, 0});
      for (int j = 0; j < g.ny; ++j) {
        for (int i = 0; i < g.nx; ++i) {
          const int cell = g.off + j * g.nx + i;
          stencil_of(g, bounded, i, j, &nb[(size_t)cell * SL]);
          cs[cell] = k;
          mode[cell] = swept ? 1 : 0;
          nsweep += swept ? 1 : 0;
          if (!cont) continue;
          const CaseGrid& G = next[k];
          const int I = i / 2, J = j / 2;
          parent[cell] = G.off + J * G.nx + I;
          const bool sx = 2 * I + 1 < g.nx, sy = 2 * J + 1 < g.ny;
          const double fx = sx ? 0.5 : 1.0, fy = sy ? 0.5 : 1.0;
          const double sa = sx ? (double)(2 * (i - 2 * I) - 1) : 0.0;
          const double sb = sy ? (double)(2 * (j - 2 * J) - 1) : 0.0;
          qo[(size_t)cell * 4 + 0] = sa * fx;
          qo[(size_t)cell * 4 + 1] = sb * fy;
          qo[(size_t)cell * 4 + 2] = fx;
          qo[(size_t)cell * 4 + 3] = fy;
        }
      }
    }
    h_nb.push_back(nb);
    h_case.push_back(cs);
    h_parent.push_back(parent);
    h_gslot.push_back(gsl);
    h_qo.push_back(qo);
    h_fin.push_back(fin);
    h_mode.push_back(mode);
    h_tail.push_back(tail);
    h_nsweep.push_back(nsweep);
    h_tiles.push_back(tiles);
    h_cls.push_back(cls);
    for (int k = 0; k < c->ncases; ++k) {
      if (done[k]) continue;
      if (grids[k].nx * grids[k].ny <= MAXFIN) done[k] = 1;
      else grids[k] = next[k];
    }
  }
  const size_t nlev = h_nb.size();
  // children and parent slots from the next level's stencils
  for (size_t l = 0; l + 1 < nlev; ++l) {
    const int ncn = (int)h_case[l + 1].size();
    std::vector<int> ch((size_t)ncn * 4, -1);
    const int nc = (int)h_case[l].size();
    for (int cell = 0; cell < nc; ++cell) {
      const int P = h_parent[l][cell];
      if (P < 0) continue;
      int q = 0;
      while (q < 4 && ch[(size_t)P * 4 + q] >= 0) ++q;
      if (q == 4) { snprintf(c->err, sizeof(c->err), "two-level set-up: more than 4 children"); return FR_ERR_ARG; }
      ch[(size_t)P * 4 + q] = cell;
      for (int s = 0; s < SL; ++s) {
        const int f = h_nb[l][(size_t)cell * SL + s];
        if (f < 0) continue;
        const int F = h_parent[l][f];
        int Sl = -1;
        for (int t = 0; t < SL; ++t) if (h_nb[l + 1][(size_t)P * SL + t] == F) Sl = t;
        if (Sl < 0) { snprintf(c->err, sizeof(c->err), "two-level set-up: parent stencil mismatch"); return FR_ERR_ARG; }
        h_gslot[l][(size_t)cell * SL + s] = Sl;
      }
    }
    h_children.push_back(ch);
  }
  h_children.push_back({});
  c->mg.resize(nlev);
  for (size_t l = 0; l < nlev; ++l) {
    MgLevel& L = c->mg[l];
    L.nc = (int)h_case[l].size();
    L.nfin = (int)h_fin[l].size() / 2;
    L.ntail = (int)h_tail[l].size();
    L.nsweep = h_nsweep[l];
    FR_TRY(upload(c, &L.nb, h_nb[l]));
    {
      // the slot of each cell in the stencil of each of its members
      std::vector<int> rs(h_nb[l].size(), -1);
      for (int cell = 0; cell < (int)h_case[l].size(); ++cell)
        for (int s2 = 0; s2 < SL; ++s2) {
          const int f = h_nb[l][(size_t)cell * SL + s2];
          if (f < 0) continue;
          for (int t = 0; t < SL; ++t)
            if (h_nb[l][(size_t)f * SL + t] == cell) rs[(size_t)cell * SL + s2] = t;
          if (rs[(size_t)cell * SL + s2] < 0) {
            snprintf(c->err, sizeof(c->err), "two-level set-up: stencils not symmetric");
            return FR_ERR_ARG;
          }
        }
      FR_TRY(upload(c, &L.rslot, rs));
    }
    FR_TRY(upload(c, &L.cell_case, h_case[l]));
    FR_TRY(upload(c, &L.parent, h_parent[l]));
    FR_TRY(upload(c, &L.gslot, h_gslot[l]));
    FR_TRY(upload(c, &L.qo, h_qo[l]));
    FR_TRY(upload(c, &L.children, h_children[l]));
    FR_TRY(upload(c, &L.fin, h_fin[l]));
    FR_TRY(upload(c, &L.mode, h_mode[l]));
    FR_TRY(upload(c, &L.tail, h_tail[l]));
    L.ntiles = (int)h_tiles[l].size();
    if (L.ntiles > 0) {
      FR_CUDA_CHECK(c, cudaMalloc(&L.tiles, h_tiles[l].size() * sizeof(Tile)));
      FR_CUDA_CHECK(c, cudaMemcpy(L.tiles, h_tiles[l].data(), h_tiles[l].size() * sizeof(Tile), cudaMemcpyHostToDevice));
    }
    FR_CUDA_CHECK(c, cudaMalloc(&L.cl, h_cls[l].size() * sizeof(CaseLevel)));
    FR_CUDA_CHECK(c, cudaMemcpy(L.cl, h_cls[l].data(), h_cls[l].size() * sizeof(CaseLevel), cudaMemcpyHostToDevice));
    const size_t n12 = (size_t)L.nc * NB;
    void** bufs[] = {&L.A, &L.Dinv, &L.x, &L.y, &L.b, &L.Ainv};
    const size_t counts[] = {n12 * SL * NB, n12 * NB, n12, n12, n12, (size_t)L.nfin * DN * DN};
    for (int i = 0; i < 6; ++i) {
      if (counts[i] == 0) continue;
      FR_CUDA_CHECK(c, cudaMalloc(bufs[i], counts[i] * esz));
      FR_CUDA_CHECK(c, cudaMemset(*bufs[i], 0, counts[i] * esz));
    }
  }
  FR_CUDA_CHECK(c, cudaMalloc(&c->mg_tc, tcs.size() * sizeof(TailCase)));
  FR_CUDA_CHECK(c, cudaMemcpy(c->mg_tc, tcs.data(), tcs.size() * sizeof(TailCase), cudaMemcpyHostToDevice));
  FR_CUDA_CHECK(c, cudaMalloc(&c->mg_views, nlev * std::max(sizeof(Lv<double>), sizeof(Lv<float>))));
  FR_CUDA_CHECK(c, cudaMalloc(&c->mg_views_t, nlev * std::max(sizeof(Lv<double>), sizeof(Lv<float>))));
  FR_TRY(f64 ? upload_views<double>(c) : upload_views<float>(c));
  // level 0: greedy colouring in which no stencil holds two members of one colour
  const int ne = c->ne;
  const std::vector<int>& nb0 = h_nb[0];
  std::vector<std::vector<int>> members_of(ne);
  for (int e = 0; e < ne; ++e)
    for (int s = 0; s < SL; ++s)
      if (nb0[(size_t)e * SL + s] >= 0) members_of[nb0[(size_t)e * SL + s]].push_back(e);
  std::vector<int> colour(ne, -1);
  int ncol = 0;
  for (int f = 0; f < ne; ++f) {
    std::vector<char> used(64, 0);
    for (int e : members_of[f])
      for (int s = 0; s < SL; ++s) {
        const int g = nb0[(size_t)e * SL + s];
        if (g >= 0 && colour[g] >= 0 && colour[g] < 64) used[colour[g]] = 1;
      }
    int col = 0;
    while (col < 64 && used[col]) ++col;
    if (col == 64) { snprintf(c->err, sizeof(c->err), "two-level set-up: colouring failed"); return FR_ERR_ARG; }
    colour[f] = col;
    ncol = std::max(ncol, col + 1);
  }
  // colslot layout on the device: [Ne] colours, then [Ne][ncol] slots
  std::vector<int> cslot((size_t)ne + (size_t)ne * ncol, -1);
  for (int e = 0; e < ne; ++e) cslot[e] = colour[e];
  for (int e = 0; e < ne; ++e)
    for (int s = 0; s < SL; ++s) {
      const int f = nb0[(size_t)e * SL + s];
      if (f >= 0) cslot[(size_t)ne + (size_t)e * ncol + colour[f]] = s;
    }
  c->mg_ncol = ncol;
  FR_TRY(upload(c, &c->mg_colslot, cslot));
  FR_TRY(dalloc(c, &c->mg_x, c->ndof));
  FR_TRY(dalloc(c, &c->mg_y, c->ndof));
  // the build's A P columns, zero where a stencil slot is unused
  const size_t nap = (size_t)ne * SL * NB * c->bsz;
  FR_CUDA_CHECK(c, cudaMalloc(&c->mg_ap, nap * esz));
  FR_CUDA_CHECK(c, cudaMemset(c->mg_ap, 0, nap * esz));
  FR_TRY(dalloc(c, &c->mg_bad, 1));
  FR_CUDA_CHECK(c, cudaMemset(c->mg_bad, 0, sizeof(int)));
  return FR_OK;
}

int mg_build(fr_ctx* c, const double* q, double inv_dtau, double a0_dt, cudaStream_t s) {
  if (c->cfg.precond != FR_PRECOND_TWO_LEVEL) return FR_OK;
  c->mg_t_ready = 0;
  if (c->mg.empty()) { snprintf(c->err, sizeof(c->err), "two-level preconditioner not set up"); return FR_ERR_ARG; }
  c->mg_q = q;
  c->mg_inv_dtau = inv_dtau;
  c->mg_a0_dt = a0_dt;
  const bool f64 = c->cfg.mg_prec == FR_PREC_FP64;
  int rc;
  switch (c->n * 2 + (f64 ? 1 : 0)) {
    case 4: rc = build_level0<2, float>(c, q, inv_dtau, a0_dt, s); break;
    case 5: rc = build_level0<2, double>(c, q, inv_dtau, a0_dt, s); break;
    case 6: rc = build_level0<3, float>(c, q, inv_dtau, a0_dt, s); break;
    case 7: rc = build_level0<3, double>(c, q, inv_dtau, a0_dt, s); break;
    case 8: rc = build_level0<4, float>(c, q, inv_dtau, a0_dt, s); break;
    case 9: rc = build_level0<4, double>(c, q, inv_dtau, a0_dt, s); break;
    case 10: rc = build_level0<5, float>(c, q, inv_dtau, a0_dt, s); break;
    case 11: rc = build_level0<5, double>(c, q, inv_dtau, a0_dt, s); break;
    default: return FR_ERR_ARG;
  }
  if (rc != FR_OK) return rc;
  return f64 ? build_levels<double>(c, s) : build_levels<float>(c, s);
}

int mg_transpose(fr_ctx* c, cudaStream_t s) {
  if (c->cfg.precond != FR_PRECOND_TWO_LEVEL || c->mg.empty()) return FR_OK;
  return c->cfg.mg_prec == FR_PREC_FP64 ? transpose_levels<double>(c, s) : transpose_levels<float>(c, s);
}

int precond_apply(fr_ctx* c, const double* q, const double* r, double* z, double inv_dtau,
                  double a0_dt, cudaStream_t s) {
  if (c->cfg.precond != FR_PRECOND_TWO_LEVEL) return block_apply(c, r, z, s);
  if (c->transposed) {
    // M^-T with the transposed hierarchy of the last build, else the transposed blocks alone
    if (!c->mg_t_ready) return block_apply(c, r, z, s);
    if (c->cfg.mg_prec == FR_PREC_FP64) return apply_tr<double>(c, r, z, s);
    return apply_tr<float>(c, r, z, s);
  }
  if (c->cfg.mg_prec == FR_PREC_FP64) return apply_t<double>(c, q, r, z, inv_dtau, a0_dt, s);
  return apply_t<float>(c, q, r, z, inv_dtau, a0_dt, s);
}

}  // namespace frk
