// fr_adjoint.cu -- building blocks of the discrete adjoint of the BDF2 march (Sec. 3.2)
// for force objectives (Sec. 4): the gradient of a weighted wall force with respect to the
// state, the transposed pointwise Jacobian of the conservative variables and their Mach
// derivative.  The paper differentiates nothing; these are the exact derivatives of its
// discrete quantities, formed by forward mode over the same device functions the residual
// and the force use (no separate derivative formulas to keep in step).
#include <cstdio>
#include <vector>
#include "fr_internal.h"
#include "fr_kernels.cuh"

namespace fr {

// Adjoints of the wall faces' traces: for every wall flux point, the derivatives of
// wx F_x + wy F_y (its weighted traction, wall_traction) with respect to the interior
// trace q^e (4) and the trace of the local gradient (8), by one dual direction each,
// written to atq [Ne][4 faces][4][N] and atg [Ne][4][8][N] at the wall faces (the caller
// zeroes the rest).
template <int N>
__global__ void k_wall_force_adjoint(Mesh M, Basis B, const double* __restrict__ gf,
                                     const double* __restrict__ tq, const double* __restrict__ tg,
                                     int nx, int ny, int wall_below, int wall_above, double wx,
                                     double wy, double* __restrict__ atq, double* __restrict__ atg) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2 * nx * N) return;
  const int side = idx / (nx * N), rem = idx % (nx * N), i = rem / N, t = rem % N;
  if (side == 0 ? !wall_below : !wall_above) return;
  const int e = side == 0 ? i : (ny - 1) * nx + i;
  const int f = side == 0 ? FACE_B : FACE_T;
  const Gas& gas = M.par(0).gas;
  const size_t FNs = (size_t)M.ne * 4 * N;
  const size_t of = ((size_t)e * 4 + f) * N + t;
  double qv[4], gv[8];
#pragma unroll
  for (int v = 0; v < 4; ++v) qv[v] = tq[(((size_t)e * 4 + f) * 4 + v) * N + t];
#pragma unroll
  for (int c = 0; c < 8; ++c) gv[c] = M.viscous ? tg[(((size_t)e * 4 + f) * 8 + c) * N + t] : 0.0;
  const double Sx = gf[GF_SX * FNs + of], Sy = gf[GF_SY * FNs + of];
  const double ug = gf[GF_UG * FNs + of], vg = gf[GF_VG * FNs + of], J = gf[GF_J * FNs + of];
  const int ndir = M.viscous ? 12 : 4;
#pragma unroll 1
  for (int dd = 0; dd < ndir; ++dd) {
    Dual qe[4], ge[8], px, py;
#pragma unroll
    for (int v = 0; v < 4; ++v) qe[v] = mk(qv[v], dd == v ? 1.0 : 0.0);
#pragma unroll
    for (int c = 0; c < 8; ++c) ge[c] = mk(gv[c], dd == 4 + c ? 1.0 : 0.0);
    wall_traction(qe, ge, Sx, Sy, ug, vg, J, gas, side == 0 ? -B.lift_end : B.lift_end,
                  side == 0 ? 1.0 : -1.0, B.ws[t], M.viscous, px, py);
    const double d = wx * px.d + wy * py.d;
    if (dd < 4) atq[(((size_t)e * 4 + f) * 4 + dd) * N + t] = d;
    else atg[(((size_t)e * 4 + f) * 8 + dd - 4) * N + t] = d;
  }
}

// out = beta out + alpha (dq^c/dq^p)^T w at every solution point (thermo's conservative
// variables differentiated in each primitive direction).  beta = 0 does not read out.
__global__ void k_conservative_adjoint(const double* __restrict__ q, const double* __restrict__ w,
                                       size_t SN, int np2, Mesh M, double alpha, double beta,
                                       double* __restrict__ out) {
  const size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (o >= SN) return;
  const int e = (int)(o / np2);
  const size_t qo = M.qbase(e, np2) + o % np2, qs = M.qstride(e);
  double qq[4], ww[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) { qq[v] = q[v * qs + qo]; ww[v] = w[v * qs + qo]; }
  const Gas& gas = M.par(e).gas;
#pragma unroll 1
  for (int c = 0; c < 4; ++c) {
    Dual qd[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) qd[v] = mk(qq[v], v == c ? 1.0 : 0.0);
    Thermo<Dual> th;
    thermo(qd, gas, th);
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < 4; ++r) s = fma(ww[r], th.qc[r].d, s);
    const size_t gi = c * qs + qo;
    out[gi] = beta == 0.0 ? alpha * s : fma(alpha, s, beta * out[gi]);
  }
}

// edot[e] = sum over element e's points of w . dq^c/dM_inf at fixed q^p (the gas constants'
// Mach tangent), one warp per element.
__global__ void k_conservative_dmach(const double* __restrict__ q, const double* __restrict__ w,
                                     int np2, Mesh M, double* __restrict__ edot) {
  const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (e >= M.ne) return;
  const size_t qo = M.qbase(e, np2), qs = M.qstride(e);
  const GasD gas = gas_tangent(M.par(e).gas, 1.0);
  double s = 0.0;
  for (int pt = lane; pt < np2; pt += 32) {
    Dual qd[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) qd[v] = mk(q[v * qs + qo + pt], 0.0);
    Thermo<Dual> th;
    thermo(qd, gas, th);
#pragma unroll
    for (int v = 0; v < 4; ++v) s = fma(w[v * qs + qo + pt], th.qc[v].d, s);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) edot[e] = s;
}

}  // namespace fr

namespace frk {
using namespace fr;

template <int N>
static int wall_force_vjp_n(fr_ctx* c, const double* q, double wx, double wy, double* out,
                            cudaStream_t s) {
  constexpr int EPB = Tile<N>::EPB, TH = Tile<N>::THREADS;
  const int nblk = (c->ne + EPB - 1) / EPB;
  const size_t ne = c->ne, SN = ne * N * N;
  // traces of q (values), then the trace adjoints: zero except at the wall faces
  k_trace<double, N><<<nblk, TH, 0, s>>>(Buf<double>{const_cast<double*>(q)}, c->mesh, c->basis,
                                         c->gs, Buf<double>{c->gl}, Buf<double>{c->tq}, Buf<double>{c->tg});
  FR_LAUNCH_CHECK(c);
  FR_CUDA_CHECK(c, cudaMemsetAsync(c->tq_d, 0, ne * 16 * N * sizeof(double), s));
  FR_CUDA_CHECK(c, cudaMemsetAsync(c->tg_d, 0, ne * 32 * N * sizeof(double), s));
  FR_CUDA_CHECK(c, cudaMemsetAsync(c->adj_q, 0, 4 * SN * sizeof(double), s));
  FR_CUDA_CHECK(c, cudaMemsetAsync(c->gl_d, 0, 8 * SN * sizeof(double), s));
  const int nw = 2 * c->nx * N;
  k_wall_force_adjoint<N><<<(nw + 127) / 128, 128, 0, s>>>(c->mesh, c->basis, c->gf, c->tq, c->tg,
                                                           c->nx, c->ny, c->bc_below == FR_BC_WALL,
                                                           c->bc_above == FR_BC_WALL, wx, wy,
                                                           c->tq_d, c->tg_d);
  FR_LAUNCH_CHECK(c);
  // transposed traces and local gradients back to the solution points
  return trace_adjoint(c, out, s);
}

int wall_force_vjp(fr_ctx* c, const double* q, double wx, double wy, double alpha, double beta,
                   double* out, cudaStream_t s) {
  int rc = FR_ERR_ARG;
  double* tmp = c->w_t;
  switch (c->n) {
    case 2: rc = wall_force_vjp_n<2>(c, q, wx, wy, tmp, s); break;
    case 3: rc = wall_force_vjp_n<3>(c, q, wx, wy, tmp, s); break;
    case 4: rc = wall_force_vjp_n<4>(c, q, wx, wy, tmp, s); break;
    case 5: rc = wall_force_vjp_n<5>(c, q, wx, wy, tmp, s); break;
  }
  if (rc != FR_OK) return rc;
  if (beta == 0.0) return scale(c, tmp, alpha, out, s);
  return axpby(c, alpha, tmp, beta, out, s);
}

int conservative_vjp(fr_ctx* c, const double* q, const double* w, double alpha, double beta,
                     double* out, cudaStream_t s) {
  const size_t SN = (size_t)c->ne * c->np2;
  FR_ACCOUNT(c, KK_CONS, 4.0 * 60.0 * SN, 8.0 * SN * (beta == 0.0 ? 12.0 : 16.0));
  FR_PROF_BEGIN(c, s);
  k_conservative_adjoint<<<(unsigned)((SN + 255) / 256), 256, 0, s>>>(q, w, SN, c->np2, c->mesh,
                                                                      alpha, beta, out);
  FR_PROF_END(c, s, KK_CONS);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

int conservative_dmach(fr_ctx* c, const double* q, const double* w, double* out_h, cudaStream_t s) {
  if (!c->edot) FR_CUDA_CHECK(c, cudaMalloc((void**)&c->edot, (size_t)c->ne * sizeof(double)));
  const int wb = (int)(((size_t)c->ne * 32 + 255) / 256);
  k_conservative_dmach<<<wb, 256, 0, s>>>(q, w, c->np2, c->mesh, c->edot);
  FR_LAUNCH_CHECK(c);
  // the elements' sums added on the host in element order (deterministic)
  std::vector<double> h(c->ne);
  FR_CUDA_CHECK(c, cudaMemcpyAsync(h.data(), c->edot, (size_t)c->ne * sizeof(double),
                                   cudaMemcpyDeviceToHost, s));
  FR_CUDA_CHECK(c, cudaStreamSynchronize(s));
  double acc = 0.0;
  for (double x : h) acc += x;
  *out_h = acc;
  return FR_OK;
}

}  // namespace frk
