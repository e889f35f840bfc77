// fr_krylov.cu -- FP64 vector kernels of restarted GMRES with CGS2 (Sec. 3.2) and the
// pseudo-step residual norms.  Reductions are deterministic: a fixed grid writes one
// partial per block and the last block to finish sums the partials in a fixed order.
#include <cstdio>
#include "fr_internal.h"

namespace fr {

constexpr int RT = 256;    // threads per reduction block
constexpr int MAXV = 32;   // Krylov vectors handled per launch

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  return x;
}

// Block sums of nv per-thread values: partial[k * gridDim.x + blockIdx.x].  The last
// block to finish (atomic ticket, no waiting) then sums the partials of every k in a
// fixed order and writes out[k]: one launch per reduction, deterministic result.
// Warp sums of NA values per lane by recursive halving: at each of the 5 steps a lane
// keeps the half of its values selected by one bit of its lane index and adds the
// partner's copy of that half, so lane l ends with the warp sum of value l (values
// padded to 32).  31 additions per lane instead of 5 NA.
template <int NA>
__device__ __forceinline__ double warp_transpose_sum(double (&acc)[NA]) {
  double a[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) a[k] = k < NA ? acc[k] : 0.0;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int half = 16; half >= 1; half >>= 1) {
    const bool up = (lane & half) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const double send = up ? a[k] : a[k + half];
      const double keep = up ? a[k + half] : a[k];
      a[k] = keep + __shfl_xor_sync(0xffffffffu, send, half);
    }
  }
  return a[0];
}

// Block sums of nv per-thread values: partial[k * gridDim.x + blockIdx.x].  The last
// block to finish (atomic ticket, no waiting) then sums the partials of every k in a
// fixed order and writes out[k]: one launch per reduction, deterministic result.
// Returns true in the last block (after out[] is written and visible to the block).
template <int NA>
__device__ __forceinline__ bool block_reduce_store(double (&acc)[NA], int nv, double* partial,
                                                   double* out, unsigned int* ticket) {
  __shared__ double sm[NA][RT / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (NA >= 8) {
    const double s = warp_transpose_sum(acc);
    if (lane < nv && lane < NA) sm[lane][wid] = s;
  } else {
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      if (k < nv) {
        const double s = warp_sum(acc[k]);
        if (lane == 0) sm[k][wid] = s;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < RT / 32; ++w) s += sm[threadIdx.x][w];
    partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // final pass: warp w sums the partials of k = w, w + 8, ... in a fixed order
  const int nb = gridDim.x;
  for (int k = wid; k < nv; k += RT / 32) {
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += ((volatile double*)partial)[(size_t)k * nb + b];
    s = warp_sum(s);
    if (lane == 0) out[k] = s;
  }
  if (threadIdx.x == 0) *ticket = 0u;
  __threadfence_block();
  __syncthreads();
  return true;
}

__device__ void gm_givens(GmresState* st, const double* h1, const double* h2, const double* nrm2);

// MODE 0: dots  out_k = <V_k, w>
// MODE 1: w -= sum_k h_k V_k, then out_k = <V_k, w>       (CGS2 second pass)
// MODE 2: w -= sum_k h_k V_k, then out_0 = <w, w>
// NV (a multiple of 4, >= nv) sizes the unrolled loops, so that a launch issues FP64
// work for at most 3 vectors beyond the nv it is given.
template <int MODE, int NV>
__global__ void __launch_bounds__(RT) k_krylov(const double* __restrict__ V, size_t ld, int nv,
                                               const double* __restrict__ h, double* w, size_t n,
                                               double* __restrict__ partial, double* out,
                                               unsigned int* ticket, GmresState* gst) {
  if (gst) nv = gst->j + 1;   // device-resident Arnoldi: nv = newest basis index + 1
  if (nv > NV) nv = NV;
  constexpr int NA = MODE == 2 ? 1 : NV;
  double acc[NA];
#pragma unroll
  for (int k = 0; k < NA; ++k) acc[k] = 0.0;
  double hk[NV];
  if (MODE != 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) hk[k] = k < nv ? h[k] : 0.0;
  }
  // pairs of entries through 16-byte loads, two pairs in flight per thread (n and ld
  // are even: 4 variables per point)
  const size_t n2 = n / 2, ld2 = ld / 2;
  const double2* V2 = reinterpret_cast<const double2*>(V);
  double2* w2 = reinterpret_cast<double2*>(w);
  const size_t stride = (size_t)gridDim.x * RT;
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n2; i += 2 * stride) {
    const bool two = i + stride < n2;
    double2 xa = w2[i], xb = two ? w2[i + stride] : make_double2(0.0, 0.0);
    if (MODE != 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        if (k < nv) {
          const double2 va = V2[k * ld2 + i];
          const double2 vb = two ? V2[k * ld2 + i + stride] : make_double2(0.0, 0.0);
          xa.x = fma(-hk[k], va.x, xa.x);
          xa.y = fma(-hk[k], va.y, xa.y);
          xb.x = fma(-hk[k], vb.x, xb.x);
          xb.y = fma(-hk[k], vb.y, xb.y);
        }
      }
      w2[i] = xa;
      if (two) w2[i + stride] = xb;
    }
    if (MODE == 2) {
      acc[0] = fma(xa.x, xa.x, acc[0]);
      acc[0] = fma(xa.y, xa.y, acc[0]);
      acc[0] = fma(xb.x, xb.x, acc[0]);
      acc[0] = fma(xb.y, xb.y, acc[0]);
    } else {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        if (k < nv) {
          const double2 va = V2[k * ld2 + i];
          const double2 vb = two ? V2[k * ld2 + i + stride] : make_double2(0.0, 0.0);
          acc[k] = fma(va.x, xa.x, acc[k]);
          acc[k] = fma(va.y, xa.y, acc[k]);
          acc[k] = fma(vb.x, xb.x, acc[k]);
          acc[k] = fma(vb.y, xb.y, acc[k]);
        }
      }
    }
  }
  const bool last = block_reduce_store(acc, MODE == 2 ? 1 : nv, partial, out, ticket);
  // the norm pass of a device-resident Arnoldi step closes it with the Givens update
  if (MODE == 2 && gst && last && threadIdx.x == 0) gm_givens(gst, h - FR_MAX_RESTART, h, out);
}

// out_0 = ||r[continuity row]||^2, out_1 = ||r||^2
__global__ void __launch_bounds__(RT) k_norms(const double* __restrict__ r, size_t sn, size_t n,
                                              double* __restrict__ partial, double* out,
                                              unsigned int* ticket) {
  double acc[2];
  acc[0] = 0.0;
  acc[1] = 0.0;
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
    const double x = r[i];
    if (i < sn) acc[0] = fma(x, x, acc[0]);
    acc[1] = fma(x, x, acc[1]);
  }
  block_reduce_store(acc, 2, partial, out, ticket);
}

__global__ void k_scale(const double* __restrict__ x, double a, double* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], b * y[i]);
}

__global__ void k_axpy_multi(const double* __restrict__ V, size_t ld, int nv,
                             const double* __restrict__ h, double* __restrict__ w, size_t n) {
  double hk[MAXV];
#pragma unroll
  for (int k = 0; k < MAXV; ++k) hk[k] = k < nv ? h[k] : 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double x = w[i];
#pragma unroll
    for (int k = 0; k < MAXV; ++k)
      if (k < nv) x = fma(-hk[k], V[k * ld + i], x);
    w[i] = x;
  }
}

__global__ void k_lincomb(const double* __restrict__ V, size_t ld, int nv, const double* __restrict__ y,
                          double* __restrict__ u, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < nv; ++k) s = fma(y[k], V[k * ld + i], s);
    u[i] = s;
  }
}

// ------------------------------------------------------------------ device-resident Arnoldi
// One restart cycle's Hessenberg matrix, Givens rotations and residual estimates live on
// the device so that iterations are queued without a host round trip.
__global__ void k_gm_copy_in(const double* __restrict__ V, size_t ld, const GmresState* st,
                             double* __restrict__ dst, size_t n) {
  const size_t base = (size_t)st->j * ld;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = V[base + i];
}

// Column j of H from the CGS2 projections h1 + h2 and ||w||, the previous rotations, a
// new rotation, the residual estimate |g_{j+1}| and the stopping test (one thread).
__device__ void gm_givens(GmresState* st, const double* h1, const double* h2, const double* nrm2) {
  if (st->done) return;
  const int j = st->j;
  constexpr int L = GmresState::LD;
  const double hn = sqrt(nrm2[0]);
  if (!isfinite(hn)) { st->nonfinite = 1; st->done = 1; return; }
  for (int i = 0; i <= j; ++i) st->H[i * L + j] = h1[i] + h2[i];
  st->H[(j + 1) * L + j] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = st->H[i * L + j], b = st->H[(i + 1) * L + j];
    st->H[i * L + j] = st->cs[i] * a + st->sn[i] * b;
    st->H[(i + 1) * L + j] = -st->sn[i] * a + st->cs[i] * b;
  }
  const double den = hypot(st->H[j * L + j], st->H[(j + 1) * L + j]);
  st->cs[j] = st->H[j * L + j] / den;
  st->sn[j] = st->H[(j + 1) * L + j] / den;
  st->H[j * L + j] = den;
  st->H[(j + 1) * L + j] = 0.0;
  st->g[j + 1] = -st->sn[j] * st->g[j];
  st->g[j] = st->cs[j] * st->g[j];
  st->j = j + 1;
  st->inv_hn = hn > 0.0 ? 1.0 / hn : 0.0;
  if (fabs(st->g[j + 1]) <= st->tol || hn == 0.0 || j + 1 >= st->jmax) st->done = 1;
}

// V[j] = w / ||w|| with j the index the Givens update wrote; the same values go to next,
// the input of the following iteration's operator.
__global__ void k_gm_store(const double* __restrict__ w, const GmresState* st,
                           double* __restrict__ V, size_t ld, double* __restrict__ next, size_t n) {
  const size_t base = (size_t)st->j * ld;
  const double s = st->inv_hn;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double x = w[i] * s;
    V[base + i] = x;
    next[i] = x;
  }
}

// Back substitution H[0:k,0:k] y = g[0:k], k = j (one thread).
__global__ void k_gm_trisolve(GmresState* st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  constexpr int L = GmresState::LD;
  const int k = st->j;
  for (int i = k - 1; i >= 0; --i) {
    double acc = st->g[i];
    for (int l = i + 1; l < k; ++l) acc -= st->H[i * L + l] * st->y[l];
    st->y[i] = acc / st->H[i * L + i];
  }
}

}  // namespace fr

namespace frk {
using namespace fr;

static int grid_for(const fr_ctx* c) { return c->red_blocks; }

// Launch k_krylov<MODE, NV> with NV = nv_bound rounded up to a multiple of 4.
template <int MODE>
static void launch_krylov(int nv_bound, int g, cudaStream_t s, const double* V, size_t ld, int nv,
                          const double* h, double* w, size_t n, double* partial, double* out,
                          unsigned int* ticket, GmresState* jdev) {
  switch ((nv_bound + 3) / 4) {
#define FR_KRYLOV_CASE(q) \
    case q: k_krylov<MODE, 4 * q><<<g, RT, 0, s>>>(V, ld, nv, h, w, n, partial, out, ticket, jdev); break;
    FR_KRYLOV_CASE(1) FR_KRYLOV_CASE(2) FR_KRYLOV_CASE(3) FR_KRYLOV_CASE(4)
    FR_KRYLOV_CASE(5) FR_KRYLOV_CASE(6) FR_KRYLOV_CASE(7)
    default: k_krylov<MODE, 32><<<g, RT, 0, s>>>(V, ld, nv, h, w, n, partial, out, ticket, jdev); break;
#undef FR_KRYLOV_CASE
  }
}

template <int MODE>
static int krylov(fr_ctx* c, const double* V, int nv, const double* h, double* w, double* out,
                  cudaStream_t s) {
  if (nv < 1 || nv > MAXV) { snprintf(c->err, sizeof(c->err), "krylov: nv=%d", nv); return FR_ERR_ARG; }
  const int g = grid_for(c);
  FR_ACCOUNT(c, KK_KRYLOV, (MODE == 0 ? 2.0 : 4.0) * nv * c->ndof,
             8.0 * c->ndof * (nv + 1 + (MODE != 0 ? 1 : 0)));
  FR_PROF_BEGIN(c, s);
  launch_krylov<MODE>(nv, g, s, V, c->ndof, nv, h, w, c->ndof, c->red, out, c->ticket, nullptr);
  FR_PROF_END(c, s, KK_KRYLOV);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

int dots(fr_ctx* c, const double* V, int nv, const double* w, double* out, cudaStream_t s) {
  return krylov<0>(c, V, nv, nullptr, const_cast<double*>(w), out, s);
}
int axpy_dots(fr_ctx* c, const double* V, int nv, const double* h, double* w, double* out, cudaStream_t s) {
  return krylov<1>(c, V, nv, h, w, out, s);
}
int axpy_norm(fr_ctx* c, const double* V, int nv, const double* h, double* w, double* out, cudaStream_t s) {
  return krylov<2>(c, V, nv, h, w, out, s);
}
int norms(fr_ctx* c, const double* r, double* out, cudaStream_t s) {
  const int g = grid_for(c);
  FR_ACCOUNT(c, KK_KRYLOV, 2.0 * c->ndof, 8.0 * c->ndof);
  FR_PROF_BEGIN(c, s);
  k_norms<<<g, RT, 0, s>>>(r, (size_t)c->ne * c->np2, c->ndof, c->red, out, c->ticket);
  FR_PROF_END(c, s, KK_KRYLOV);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}
int scale(fr_ctx* c, const double* x, double a, double* y, cudaStream_t s) {
  FR_ACCOUNT(c, KK_VECTOR, 1.0 * c->ndof, 16.0 * c->ndof);
{ FR_PROF_BEGIN(c, s); k_scale<<<grid_for(c), RT, 0, s>>>(x, a, y, c->ndof); FR_PROF_END(c, s, KK_VECTOR); }
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}
int axpby(fr_ctx* c, double a, const double* x, double b, double* y, cudaStream_t s) {
  FR_ACCOUNT(c, KK_VECTOR, 3.0 * c->ndof, 24.0 * c->ndof);
{ FR_PROF_BEGIN(c, s); k_axpby<<<grid_for(c), RT, 0, s>>>(a, x, b, y, c->ndof); FR_PROF_END(c, s, KK_VECTOR); }
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}
// w -= sum_k h_k V_k (nv <= 32), no reduction
int axpy(fr_ctx* c, const double* V, int nv, const double* h, double* w, cudaStream_t s) {
  FR_ACCOUNT(c, KK_VECTOR, 2.0 * nv * c->ndof, 8.0 * c->ndof * (nv + 2));
{ FR_PROF_BEGIN(c, s); k_axpy_multi<<<grid_for(c), RT, 0, s>>>(V, c->ndof, nv, h, w, c->ndof); FR_PROF_END(c, s, KK_VECTOR); }
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}
// One Arnoldi iteration's reductions and Givens update with the basis index on the device.
int gm_copy_in(fr_ctx* c, double* dst, cudaStream_t s) {
  FR_ACCOUNT(c, KK_VECTOR, 0.0, 16.0 * c->ndof);
  FR_PROF_BEGIN(c, s);
  k_gm_copy_in<<<grid_for(c), RT, 0, s>>>(c->V, c->ndof, c->gst, dst, c->ndof);
  FR_PROF_END(c, s, KK_VECTOR);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}
int gm_orthogonalize(fr_ctx* c, double* w, double* next, int nv_bound, cudaStream_t s) {
  const int g = grid_for(c);
  GmresState* jd = c->gst;
  constexpr int M = FR_MAX_RESTART;
  FR_ACCOUNT(c, KK_KRYLOV, 8.0 * nv_bound * c->ndof + 2.0 * c->ndof, 8.0 * c->ndof * (3.0 * nv_bound + 5.0));
  {
    FR_PROF_BEGIN(c, s);
    launch_krylov<0>(nv_bound, g, s, c->V, c->ndof, 0, nullptr, w, c->ndof, c->red, c->dsc, c->ticket, jd);
    FR_PROF_END(c, s, KK_KRYLOV);
    FR_LAUNCH_CHECK(c);
  }
  {
    FR_PROF_BEGIN(c, s);
    launch_krylov<1>(nv_bound, g, s, c->V, c->ndof, 0, c->dsc, w, c->ndof, c->red, c->dsc + M, c->ticket, jd);
    FR_PROF_END(c, s, KK_KRYLOV);
    FR_LAUNCH_CHECK(c);
  }
  {
    FR_PROF_BEGIN(c, s);
    launch_krylov<2>(nv_bound, g, s, c->V, c->ndof, 0, c->dsc + M, w, c->ndof, c->red, c->dsc + 2 * M, c->ticket, jd);
    FR_PROF_END(c, s, KK_KRYLOV);
    FR_LAUNCH_CHECK(c);
  }
  {
    FR_ACCOUNT(c, KK_VECTOR, 1.0 * c->ndof, 24.0 * c->ndof);
    FR_PROF_BEGIN(c, s);
    k_gm_store<<<grid_for(c), RT, 0, s>>>(w, c->gst, c->V, c->ndof, next, c->ndof);
    FR_PROF_END(c, s, KK_VECTOR);
    FR_LAUNCH_CHECK(c);
  }
  return FR_OK;
}
int gm_trisolve(fr_ctx* c, cudaStream_t s) {
  FR_PROF_BEGIN(c, s);
  k_gm_trisolve<<<1, 32, 0, s>>>(c->gst);
  FR_PROF_END(c, s, KK_KRYLOV);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}
int lincomb(fr_ctx* c, const double* V, int nv, const double* y, double* u, cudaStream_t s) {
  FR_ACCOUNT(c, KK_VECTOR, 2.0 * nv * c->ndof, 8.0 * c->ndof * (nv + 1));
{ FR_PROF_BEGIN(c, s); k_lincomb<<<grid_for(c), RT, 0, s>>>(V, c->ndof, nv, y, u, c->ndof); FR_PROF_END(c, s, KK_VECTOR); }
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

}  // namespace frk
