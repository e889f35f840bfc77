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
    bool dup = nb[f] == e;
    for (int g = 0; g < f; ++g) dup = dup || nb[g] == nb[f];
    if (!dup) s += edot[nb[f]];
  }
  out[(size_t)e * 8 + 2 * a + xy] = s;
}

}  // namespace fr

namespace frk {
using namespace fr;

// R' = tangent of R for the corner / velocity tangents (dcorn, dvel, either may be null)
// and the Mach tangent dmach, into c->rtan.
template <int N>
static int tangent_pass(fr_ctx* c, const double* q, const double* corners, const double* vel,
                        const double* dcorn, const double* dvel, double dmach, cudaStream_t s) {
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
                                                         c->sdgf, dmach);
  FR_LAUNCH_CHECK(c);
  k_elem<Dual, N, MODE_TAN, Dual><<<nblk, TH, 0, s>>>(Q, c->mesh, c->basis, c->sgs, c->sgf, GL, TQ, FN,
                                                      QC, c->rtan, TimeTerms{nullptr, nullptr},
                                                      c->sdgs, c->sdgf, dmach);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

static int tangent(fr_ctx* c, const double* q, const double* corners, const double* vel,
                   const double* dcorn, const double* dvel, double dmach, cudaStream_t s) {
  switch (c->n) {
    case 2: return tangent_pass<2>(c, q, corners, vel, dcorn, dvel, dmach, s);
    case 3: return tangent_pass<3>(c, q, corners, vel, dcorn, dvel, dmach, s);
    case 4: return tangent_pass<4>(c, q, corners, vel, dcorn, dvel, dmach, s);
    case 5: return tangent_pass<5>(c, q, corners, vel, dcorn, dvel, dmach, s);
  }
  return FR_ERR_ARG;
}

template <class T> static int lazy_alloc(fr_ctx* c, T** p, size_t n) {
  if (*p) return FR_OK;
  FR_CUDA_CHECK(c, cudaMalloc((void**)p, n * sizeof(T)));
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
  if (c->bounded) { snprintf(c->err, sizeof(c->err), "fr_param_vjp: not available on bounded meshes"); return FR_ERR_ARG; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t ne = c->ne, SN = ne * c->np2, FN = ne * 4 * c->n;
  FR_TRY(frk::lazy_alloc(c, &c->sgs, GS_COUNT * SN));
  FR_TRY(frk::lazy_alloc(c, &c->sdgs, GS_COUNT * SN));
  FR_TRY(frk::lazy_alloc(c, &c->sgf, GF_COUNT * FN));
  FR_TRY(frk::lazy_alloc(c, &c->sdgf, GF_COUNT * FN));
  FR_TRY(frk::lazy_alloc(c, &c->seed, 8 * ne));
  FR_TRY(frk::lazy_alloc(c, &c->edot, ne));
  FR_TRY(frk::lazy_alloc(c, &c->zero, c->ndof));
  FR_TRY(frk::lazy_alloc(c, &c->rtan, c->ndof));
  FR_CUDA_CHECK(c, cudaMemsetAsync(c->zero, 0, c->ndof * sizeof(double), s));
  const int eb = (int)((ne + 127) / 128), wb = (int)((ne * 32 + 255) / 256);
  if (dmach) {
    FR_TRY(frk::tangent(c, q, corners, vel, nullptr, nullptr, 1.0, s));
    k_sens_edot<<<wb, 256, 0, s>>>(c->mesh, c->np2, w, c->rtan, c->edot);
    FR_LAUNCH_CHECK(c);
    // the elements' dot products summed on the host in element order (deterministic)
    std::vector<double> h(ne);
    FR_CUDA_CHECK(c, cudaMemcpyAsync(h.data(), c->edot, ne * sizeof(double), cudaMemcpyDeviceToHost, s));
    FR_CUDA_CHECK(c, cudaStreamSynchronize(s));
    double acc = 0.0;
    for (size_t e = 0; e < ne; ++e) acc += h[e];
    *dmach = acc;
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
