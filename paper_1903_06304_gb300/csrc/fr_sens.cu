// fr_sens.cu -- sensitivities of the residual R(q^p; M_inf, corners, corner velocities) to
// its parameters, contracted with a weight vector w (the parameter part of a discrete
// adjoint): w . dR/dM_inf, w . dR/d(corner coordinates) and w . dR/d(corner velocities).
//
// Forward mode: the residual kernels run over dual numbers with the geometry (and the
// Mach-dependent gas constants) carrying the tangent of one parameter direction.  A
// corner of element e moves only e's geometry, which enters R on e and on its four face
// neighbours; elements whose closed neighbourhoods are disjoint are perturbed together
// (a distance-2 colouring of the periodic element grid), and each one's sensitivity is
// the sum of w . dR over its neighbourhood.  Exact to rounding, no step size.
#include <cstdio>
#include <cstring>
#include "fr_internal.h"
#include "fr_kernels.cuh"

namespace fr {

// 1-D colour of column i of n: i mod 3 on the first 3 floor(n/3) columns, then one colour
// per remaining column, so that equal colours are at cyclic distance >= 3.
__host__ __device__ __forceinline__ int colour1d(int i, int n) {
  const int full = 3 * (n / 3);
  return i < full ? i % 3 : 3 + (i - full);
}
__host__ __device__ __forceinline__ int ncolour1d(int n) { return n % 3 == 0 ? 3 : 3 + n % 3; }

__device__ __forceinline__ int elem_colour(const Mesh& M, int e) {
  const CaseParams& c = M.par(e);
  const int l = e - c.e0, i = l % c.nx, j = l / c.nx;
  return colour1d(i, c.nx) * 5 + colour1d(j, c.ny);
}

// seed[e][a][xy] = 1 for the chosen corner a and coordinate xy of colour-k elements.
__global__ void k_sens_seed(Mesh M, int k, int a, int xy, double* __restrict__ seed) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M.ne) return;
  const bool on = elem_colour(M, e) == k;
#pragma unroll
  for (int t = 0; t < 8; ++t) seed[(size_t)e * 8 + t] = (on && t == 2 * a + xy) ? 1.0 : 0.0;
}

// edot[e] = sum over element e's entries of w . r (one warp per element).
__global__ void k_sens_edot(Mesh M, int np2, const double* __restrict__ w,
                            const double* __restrict__ r, double* __restrict__ edot) {
  const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (e >= M.ne) return;
  const size_t qo = M.qbase(e, np2), qs = M.qstride(e);
  double s = 0.0;
  for (int t = lane; t < 4 * np2; t += 32) {
    const size_t i = (size_t)(t / np2) * qs + qo + t % np2;
    s = fma(w[i], r[i], s);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) edot[e] = s;
}

// out[e][a][xy] = edot over e's closed neighbourhood (each distinct element once), for
// the colour-k elements.
__global__ void k_sens_gather(Mesh M, int k, int a, int xy, const double* __restrict__ edot,
                              double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M.ne || elem_colour(M, e) != k) return;
  const int nb[4] = {M.left(e), M.right(e), M.bottom(e), M.top(e)};
  double s = edot[e];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    bool dup = nb[f] == e || nb[f] < 0;   // a boundary face has no neighbour
    for (int g = 0; g < f; ++g) dup = dup || nb[g] == nb[f];
    if (!dup) s += edot[nb[f]];
  }
  out[(size_t)e * 8 + 2 * a + xy] = s;
}

}  // namespace fr

namespace frk {
using namespace fr;

// R' = tangent of R for the corner / velocity tangents (dcorn, dvel, either may be null),
// the Mach tangent dmach and the far-field state's tangent dqinf, into c->rtan.
template <int N>
static int tangent_pass(fr_ctx* c, const double* q, const double* corners, const double* vel,
                        const double* dcorn, const double* dvel, double dmach, Vec4 dqinf,
                        cudaStream_t s) {
  constexpr int EPB = Tile<N>::EPB, TH = Tile<N>::THREADS;
  const int ne = c->ne, nblk = (ne + EPB - 1) / EPB, nf = ne * 2 * N;
  k_geometry<N, Dual><<<(ne + 63) / 64, 64, 0, s>>>(corners, vel, ne, c->basis, Buf<Dual>{c->sgs, c->sdgs},
                                                    Buf<Dual>{c->sgf, c->sdgf}, dcorn, dvel);
  FR_LAUNCH_CHECK(c);
  const Buf<Dual> Q{const_cast<double*>(q), c->zero};
  const Buf<Dual> GL{c->gl, c->gl_d}, TQ{c->tq, c->tq_d}, TG{c->tg, c->tg_d};
  const Buf<Dual> FN{c->fn, c->fn_d}, QC{c->qcm, c->qcm_d};
  k_trace<Dual, N, Dual><<<nblk, TH, 0, s>>>(Q, c->mesh, c->basis, c->sgs, GL, TQ, TG, c->sdgs);
  FR_LAUNCH_CHECK(c);
  k_face<Dual, N, Dual><<<(nf + 127) / 128, 128, 0, s>>>(c->mesh, c->basis, c->sgf, TQ, TG, FN, QC,
                                                         c->sdgf, dmach, dqinf);
  FR_LAUNCH_CHECK(c);
  const Buf<Dual> FB{c->fnb, c->fnb_d}, QB{c->qcb, c->qcb_d};
  if (c->bounded) {   // the faces below row 0
    const int nbf = c->nx * N;
    k_face_below<Dual, N, Dual><<<(nbf + 127) / 128, 128, 0, s>>>(c->mesh, c->basis, c->sgf, TQ, TG, FB,
                                                                  QB, c->nx, c->sdgf, dmach, dqinf);
    FR_LAUNCH_CHECK(c);
  }
  k_elem<Dual, N, MODE_TAN, Dual><<<nblk, TH, 0, s>>>(Q, c->mesh, c->basis, c->sgs, c->sgf, GL, TQ, FN,
                                                      QC, c->rtan, TimeTerms{nullptr, nullptr},
                                                      c->sdgs, c->sdgf, dmach, FB, QB);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

static int tangent(fr_ctx* c, const double* q, const double* corners, const double* vel,
                   const double* dcorn, const double* dvel, double dmach, cudaStream_t s,
                   Vec4 dqinf = Vec4{}) {
  switch (c->n) {
    case 2: return tangent_pass<2>(c, q, corners, vel, dcorn, dvel, dmach, dqinf, s);
    case 3: return tangent_pass<3>(c, q, corners, vel, dcorn, dvel, dmach, dqinf, s);
    case 4: return tangent_pass<4>(c, q, corners, vel, dcorn, dvel, dmach, dqinf, s);
    case 5: return tangent_pass<5>(c, q, corners, vel, dcorn, dvel, dmach, dqinf, s);
  }
  return FR_ERR_ARG;
}

// Tangents (F_x', F_y') of the wall force at fixed q along the direction of the last
// tangent pass: its geometry (sgf, sdgf) and dual traces (tq, tg with their tangents, the
// local gradients moving with the geometry), and the Mach tangent dmach; into out[0..3]
// (values, tangents).
template <int N>
static int wall_force_tangent_n(fr_ctx* c, double dmach, double* out, cudaStream_t s) {
  k_wall_force<N, Dual><<<1, 256, 0, s>>>(c->mesh, c->basis, c->sgf, c->tq, c->tg, c->nx, c->ny,
                                          c->bc_below == FR_BC_WALL, c->bc_above == FR_BC_WALL, out,
                                          c->sdgf, dmach, c->tq_d, c->tg_d);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

static int wall_force_tangent(fr_ctx* c, double dmach, double* out, cudaStream_t s) {
  switch (c->n) {
    case 2: return wall_force_tangent_n<2>(c, dmach, out, s);
    case 3: return wall_force_tangent_n<3>(c, dmach, out, s);
    case 4: return wall_force_tangent_n<4>(c, dmach, out, s);
    case 5: return wall_force_tangent_n<5>(c, dmach, out, s);
  }
  return FR_ERR_ARG;
}

template <class T> static int lazy_alloc(fr_ctx* c, T** p, size_t n) {
  if (*p) return FR_OK;
  FR_CUDA_CHECK(c, cudaMalloc((void**)p, n * sizeof(T)));
  return FR_OK;
}

// workspace of the tangent passes (allocated once per mesh), zero state tangent
static int sens_alloc(fr_ctx* c, cudaStream_t s) {
  const size_t ne = c->ne, SN = ne * c->np2, FN = ne * 4 * c->n;
  FR_TRY(lazy_alloc(c, &c->sgs, GS_COUNT * SN));
  FR_TRY(lazy_alloc(c, &c->sdgs, GS_COUNT * SN));
  FR_TRY(lazy_alloc(c, &c->sgf, GF_COUNT * FN));
  FR_TRY(lazy_alloc(c, &c->sdgf, GF_COUNT * FN));
  FR_TRY(lazy_alloc(c, &c->seed, 8 * ne));
  FR_TRY(lazy_alloc(c, &c->edot, ne));
  FR_TRY(lazy_alloc(c, &c->zero, c->ndof));
  FR_TRY(lazy_alloc(c, &c->rtan, c->ndof));
  FR_CUDA_CHECK(c, cudaMemsetAsync(c->zero, 0, c->ndof * sizeof(double), s));
  return FR_OK;
}

// sum of w . r over the elements, added on the host in element order (deterministic)
static int wdot(fr_ctx* c, const double* w, const double* r, double* out_h, cudaStream_t s) {
  const int wb = (int)(((size_t)c->ne * 32 + 255) / 256);
  k_sens_edot<<<wb, 256, 0, s>>>(c->mesh, c->np2, w, r, c->edot);
  FR_LAUNCH_CHECK(c);
  std::vector<double> h(c->ne);
  FR_CUDA_CHECK(c, cudaMemcpyAsync(h.data(), c->edot, (size_t)c->ne * sizeof(double), cudaMemcpyDeviceToHost, s));
  FR_CUDA_CHECK(c, cudaStreamSynchronize(s));
  double acc = 0.0;
  for (double x : h) acc += x;
  *out_h = acc;
  return FR_OK;
}

}  // namespace frk

extern "C" int fr_param_vjp(fr_ctx* c, const double* q, const double* w, const double* corners,
                            const double* vel, double* dmach, double* dcorners, double* dvel,
                            void* stream) {
  using namespace fr;
  if (!c) return FR_ERR_ARG;
  if (c->ne <= 0) { snprintf(c->err, sizeof(c->err), "fr_set_mesh has not been called"); return FR_ERR_ARG; }
  if (!q || !w || !corners || !vel) return FR_ERR_ARG;
  if (c->ncases != 1) { snprintf(c->err, sizeof(c->err), "fr_param_vjp: single-case contexts only"); return FR_ERR_ARG; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  FR_TRY(frk::sens_alloc(c, s));
  const size_t ne = c->ne;
  const int eb = (int)((ne + 127) / 128), wb = (int)((ne * 32 + 255) / 256);
  if (dmach) {
    FR_TRY(frk::tangent(c, q, corners, vel, nullptr, nullptr, 1.0, s));
    FR_TRY(frk::wdot(c, w, c->rtan, dmach, s));
  }
  const int ncol = ncolour1d(c->cps[0].nx) * 5;   // colour ids i * 5 + j, j < ncolour1d(ny)
  const int ncj = ncolour1d(c->cps[0].ny);
  for (int kind = 0; kind < 2; ++kind) {
    double* out = kind == 0 ? dcorners : dvel;
    if (!out) continue;
    for (int k = 0; k < ncol; ++k) {
      if (k % 5 >= ncj) continue;
      for (int a = 0; a < 4; ++a) {
        for (int xy = 0; xy < 2; ++xy) {
          k_sens_seed<<<eb, 128, 0, s>>>(c->mesh, k, a, xy, c->seed);
          FR_LAUNCH_CHECK(c);
          FR_TRY(frk::tangent(c, q, corners, vel, kind == 0 ? c->seed : nullptr,
                              kind == 1 ? c->seed : nullptr, 0.0, s));
          k_sens_edot<<<wb, 256, 0, s>>>(c->mesh, c->np2, w, c->rtan, c->edot);
          FR_LAUNCH_CHECK(c);
          k_sens_gather<<<eb, 128, 0, s>>>(c->mesh, k, a, xy, c->edot, out);
          FR_LAUNCH_CHECK(c);
        }
      }
    }
  }
  return FR_OK;
}

extern "C" int fr_param_jvp(fr_ctx* c, const double* q, const double* w, const double* corners,
                            const double* vel, const double* dcorners, const double* dvel,
                            double dmach, const double* dqinf_h, double* wdR_h, double* dforce_h,
                            void* stream) {
  using namespace fr;
  if (!c) return FR_ERR_ARG;
  if (c->ne <= 0) { snprintf(c->err, sizeof(c->err), "fr_set_mesh has not been called"); return FR_ERR_ARG; }
  if (!q || !corners || !vel || (wdR_h && !w)) return FR_ERR_ARG;
  if (c->ncases != 1) { snprintf(c->err, sizeof(c->err), "fr_param_jvp: single-case contexts only"); return FR_ERR_ARG; }
  if (dforce_h && (!c->bounded || (c->bc_below != FR_BC_WALL && c->bc_above != FR_BC_WALL))) {
    snprintf(c->err, sizeof(c->err), "fr_param_jvp: the mesh has no wall faces");
    return FR_ERR_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  FR_TRY(frk::sens_alloc(c, s));
  Vec4 dq{};
  if (dqinf_h) for (int k = 0; k < 4; ++k) dq.v[k] = dqinf_h[k];
  FR_TRY(frk::tangent(c, q, corners, vel, dcorners, dvel, dmach, s, dq));
  if (wdR_h) FR_TRY(frk::wdot(c, w, c->rtan, wdR_h, s));
  if (dforce_h) {
    FR_TRY(frk::wall_force_tangent(c, dmach, c->red, s));
    double h4[4];
    FR_CUDA_CHECK(c, cudaMemcpyAsync(h4, c->red, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    FR_CUDA_CHECK(c, cudaStreamSynchronize(s));
    dforce_h[0] = h4[2];
    dforce_h[1] = h4[3];
  }
  return FR_OK;
}
