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
#include <cstring>
#include "fr_internal.h"
#include "fr_kernels.cuh"

namespace fr {

__global__ void k_conservative(const double* __restrict__ q, size_t SN, int np2, Mesh M,
                               double* __restrict__ qc) {
  const size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (o >= SN) return;
  const int e = (int)(o / np2);
  const size_t qo = M.qbase(e, np2) + o % np2, qs = M.qstride(e);
  double qq[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) qq[v] = q[v * qs + qo];
  Thermo<double> th;
  thermo(qq, M.par(e).gas, th);
#pragma unroll
  for (int v = 0; v < 4; ++v) qc[v * qs + qo] = th.qc[v];
}

// ------------------------------------------------------------------ launchers
template <class T, int N, int MODE>
static int run_pipeline(fr_ctx* c, Buf<T> Q, Buf<T> GL, Buf<T> TQ, Buf<T> TG, Buf<T> FNb,
                        Buf<T> QCb, Buf<T> FBb, Buf<T> QBb, double* out, TimeTerms tt,
                        cudaStream_t s) {
  constexpr bool jvp = MODE == MODE_JVP;
  const int kt = jvp ? c->tile.trace_d : c->tile.trace, ke = jvp ? c->tile.elem_d : c->tile.elem;
  const int nb1 = (c->ne + Tile<N, 1>::EPB - 1) / Tile<N, 1>::EPB;
  const int nb2 = (c->ne + Tile<N, 2>::EPB - 1) / Tile<N, 2>::EPB;
  const bool visc = c->mesh.viscous;
  const double pts = (double)c->ne * N * N, fac = jvp ? FR_JVP_FLOP_FACTOR : 1.0;
  FR_ACCOUNT(c, jvp ? KK_TRACE_JVP : KK_TRACE, fac * pts * fr_flops_trace(N, visc), 0.0);
  FR_ACCOUNT(c, jvp ? KK_FACE_JVP : KK_FACE, fac * 2.0 * c->ne * N * fr_flops_face_point(visc), 0.0);
  FR_ACCOUNT(c, jvp ? KK_ELEM_JVP : KK_ELEM, fac * pts * fr_flops_elem(N, visc), 0.0);
  {
    FR_PROF_BEGIN(c, s);
    if (kt == 2)
      k_trace<T, N, double, 2><<<nb2, Tile<N, 2>::THREADS, 0, s>>>(Q, c->mesh, c->basis, c->gs, GL, TQ, TG);
    else
      k_trace<T, N><<<nb1, Tile<N, 1>::THREADS, 0, s>>>(Q, c->mesh, c->basis, c->gs, GL, TQ, TG);
    FR_PROF_END(c, s, jvp ? KK_TRACE_JVP : KK_TRACE);
    FR_LAUNCH_CHECK(c);
  }
  {
    const int nf = c->ne * 2 * N;
    FR_PROF_BEGIN(c, s);
    k_face<T, N><<<(nf + 127) / 128, 128, 0, s>>>(c->mesh, c->basis, c->gf, TQ, TG, FNb, QCb);
    FR_PROF_END(c, s, jvp ? KK_FACE_JVP : KK_FACE);
    FR_LAUNCH_CHECK(c);
  }
  if (c->bounded) {   // the faces below row 0 (the faces above the last row are in k_face)
    const int nbf = c->nx * N;
    FR_PROF_BEGIN(c, s);
    k_face_below<T, N><<<(nbf + 127) / 128, 128, 0, s>>>(c->mesh, c->basis, c->gf, TQ, TG, FBb, QBb,
                                                         c->nx);
    FR_PROF_END(c, s, jvp ? KK_FACE_JVP : KK_FACE);
    FR_LAUNCH_CHECK(c);
  }
  {
    FR_PROF_BEGIN(c, s);
    if (ke == 2)
      k_elem<T, N, MODE, double, 2><<<nb2, Tile<N, 2>::THREADS, 0, s>>>(
          Q, c->mesh, c->basis, c->gs, c->gf, GL, TQ, FNb, QCb, out, tt, nullptr, nullptr, 0.0,
          FBb, QBb);
    else
      k_elem<T, N, MODE><<<nb1, Tile<N, 1>::THREADS, 0, s>>>(Q, c->mesh, c->basis, c->gs, c->gf,
                                                            GL, TQ, FNb, QCb, out, tt, nullptr,
                                                            nullptr, 0.0, FBb, QBb);
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
                                             Buf<double>{c->qcm}, Buf<double>{c->fnb},
                                             Buf<double>{c->qcb}, out, tt, s);
}

template <int N>
static int jvp_n(fr_ctx* c, const double* q, const double* v, double* out, cudaStream_t s) {
  Buf<Dual> Q{const_cast<double*>(q), const_cast<double*>(v)};
  TimeTerms tt{nullptr, nullptr};
  return run_pipeline<Dual, N, MODE_JVP>(c, Q, Buf<Dual>{c->gl, c->gl_d}, Buf<Dual>{c->tq, c->tq_d},
                                         Buf<Dual>{c->tg, c->tg_d}, Buf<Dual>{c->fn, c->fn_d},
                                         Buf<Dual>{c->qcm, c->qcm_d}, Buf<Dual>{c->fnb, c->fnb_d},
                                         Buf<Dual>{c->qcb, c->qcb_d}, out, tt, s);
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

int set_case_params(fr_ctx* c, int cid, const CaseParams& p, cudaStream_t s) {
  k_set_case<<<1, 1, 0, s>>>(c->cp, cid, p);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

// The single-case context keeps a host copy of case 0's parameters and rewrites the
// device copy only when a call changes them (stream-ordered, by a one-thread kernel).
int set_time_terms(fr_ctx* c, double a0dt, double a1dt, double a2dt, cudaStream_t s) {
  if (c->external_terms) return FR_OK;
  CaseParams& h = c->cp_h;
  if (h.a0dt == a0dt && h.a1dt == a1dt && h.a2dt == a2dt) return FR_OK;
  h.a0dt = a0dt; h.a1dt = a1dt; h.a2dt = a2dt;
  return set_case_params(c, 0, h, s);
}

int set_operator_terms(fr_ctx* c, double inv_dtau, double a0_dt, cudaStream_t s) {
  if (c->external_terms) return FR_OK;
  CaseParams& h = c->cp_h;
  if (h.inv_dtau == inv_dtau && h.a0_dt == a0_dt) return FR_OK;
  h.inv_dtau = inv_dtau; h.a0_dt = a0_dt;
  return set_case_params(c, 0, h, s);
}

// The whole case table from the host copies c->cps, staged through pinned memory.  The
// host waits for the previous staged upload to complete before it rewrites the staging
// area, so a caller may change c->cps again right after this returns.
int upload_cases(fr_ctx* c, cudaStream_t s) {
  BatchWork& b = c->bw;
  if (!b.cp_stage || !b.staged) { snprintf(c->err, sizeof(c->err), "no batch workspace"); return FR_ERR_ARG; }
  FR_CUDA_CHECK(c, cudaEventSynchronize(b.staged));
  std::memcpy(b.cp_stage, c->cps.data(), c->ncases * sizeof(CaseParams));
  FR_CUDA_CHECK(c, cudaMemcpyAsync(c->cp, b.cp_stage, c->ncases * sizeof(CaseParams),
                                   cudaMemcpyHostToDevice, s));
  FR_CUDA_CHECK(c, cudaEventRecord(b.staged, s));
  return FR_OK;
}

int fill_topology(fr_ctx* c, int nx, int ny, int e0, int cid, cudaStream_t s) {
  k_fill_topo<<<(nx * ny + 127) / 128, 128, 0, s>>>(nx, ny, e0, cid, c->nbr, c->ecase);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

int mark_bounds(fr_ctx* c, int nx, int ny, int below, int above, cudaStream_t s) {
  k_mark_bounds<<<(nx + 127) / 128, 128, 0, s>>>(nx, ny, below, above, c->nbr);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

template <int N>
static int wall_force_n(fr_ctx* c, const double* q, double* force_h, cudaStream_t s) {
  constexpr int EPB = Tile<N>::EPB, TH = Tile<N>::THREADS;
  k_trace<double, N><<<(c->ne + EPB - 1) / EPB, TH, 0, s>>>(Buf<double>{const_cast<double*>(q)}, c->mesh,
                                                           c->basis, c->gs, Buf<double>{c->gl},
                                                           Buf<double>{c->tq}, Buf<double>{c->tg});
  FR_LAUNCH_CHECK(c);
  k_wall_force<N><<<1, 256, 0, s>>>(c->mesh, c->basis, c->gf, c->tq, c->tg, c->nx, c->ny,
                                    c->bc_below == FR_BC_WALL, c->bc_above == FR_BC_WALL, c->red);
  FR_LAUNCH_CHECK(c);
  FR_CUDA_CHECK(c, cudaMemcpyAsync(force_h, c->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  FR_CUDA_CHECK(c, cudaStreamSynchronize(s));
  return FR_OK;
}

int wall_force(fr_ctx* c, const double* q, double* force_h, cudaStream_t s) {
  switch (c->n) {
    case 2: return wall_force_n<2>(c, q, force_h, s);
    case 3: return wall_force_n<3>(c, q, force_h, s);
    case 4: return wall_force_n<4>(c, q, force_h, s);
    case 5: return wall_force_n<5>(c, q, force_h, s);
  }
  return FR_ERR_ARG;
}

int geometry(fr_ctx* c, const double* corners, const double* vel, cudaStream_t s) {
  const int th = 64, nb = (c->ne + th - 1) / th;
  FR_PROF_BEGIN(c, s);
  switch (c->n) {
    case 2: k_geometry<2><<<nb, th, 0, s>>>(corners, vel, c->ne, c->basis, Buf<double>{c->gs}, Buf<double>{c->gf}); break;
    case 3: k_geometry<3><<<nb, th, 0, s>>>(corners, vel, c->ne, c->basis, Buf<double>{c->gs}, Buf<double>{c->gf}); break;
    case 4: k_geometry<4><<<nb, th, 0, s>>>(corners, vel, c->ne, c->basis, Buf<double>{c->gs}, Buf<double>{c->gf}); break;
    case 5: k_geometry<5><<<nb, th, 0, s>>>(corners, vel, c->ne, c->basis, Buf<double>{c->gs}, Buf<double>{c->gf}); break;
    default: return FR_ERR_ARG;
  }
  FR_PROF_END(c, s, KK_GEOM);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

int residual(fr_ctx* c, const double* q, double* out, const double* qcn, const double* qcnm1,
             double a0dt, double a1dt, double a2dt, cudaStream_t s) {
  if (qcn) {
    const int rc = set_time_terms(c, a0dt, a1dt, a2dt, s);
    if (rc != FR_OK) return rc;
  }
  TimeTerms tt{qcn, qcnm1};
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
  const int rc = set_operator_terms(c, inv_dtau, a0_dt, s);
  if (rc != FR_OK) return rc;
  switch (c->n) {
    case 2: return jvp_n<2>(c, q, v, out, s);
    case 3: return jvp_n<3>(c, q, v, out, s);
    case 4: return jvp_n<4>(c, q, v, out, s);
    case 5: return jvp_n<5>(c, q, v, out, s);
  }
  return FR_ERR_ARG;
}

int conservative(fr_ctx* c, const double* q, double* qc, cudaStream_t s) {
  const size_t SN = (size_t)c->ne * c->np2;
  FR_ACCOUNT(c, KK_CONS, 0.0, 8.0 * 8.0 * SN);
  FR_PROF_BEGIN(c, s);
  k_conservative<<<(unsigned)((SN + 255) / 256), 256, 0, s>>>(q, SN, c->np2, c->mesh, qc);
  FR_PROF_END(c, s, KK_CONS);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

}  // namespace frk
