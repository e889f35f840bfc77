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
__device__ __forceinline__ void block_reduce_store(double (&acc)[MAXV], int nv, double* partial,
                                                   double* out, unsigned int* ticket) {
  __shared__ double sm[MAXV][RT / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < MAXV; ++k) {
    if (k < nv) {
      const double s = warp_sum(acc[k]);
      if (lane == 0) sm[k][wid] = s;
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
  if (!last) return;
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
}

// MODE 0: dots  out_k = <V_k, w>
// MODE 1: w -= sum_k h_k V_k, then out_k = <V_k, w>       (CGS2 second pass)
// MODE 2: w -= sum_k h_k V_k, then out_0 = <w, w>
template <int MODE>
__global__ void __launch_bounds__(RT) k_krylov(const double* __restrict__ V, size_t ld, int nv,
                                               const double* __restrict__ h, double* w, size_t n,
                                               double* __restrict__ partial, double* out,
                                               unsigned int* ticket) {
  double acc[MAXV];
#pragma unroll
  for (int k = 0; k < MAXV; ++k) acc[k] = 0.0;
  double hk[MAXV];
  if (MODE != 0) {
#pragma unroll
    for (int k = 0; k < MAXV; ++k) hk[k] = k < nv ? h[k] : 0.0;
  }
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
    double x = w[i];
    if (MODE != 0) {
#pragma unroll
      for (int k = 0; k < MAXV; ++k)
        if (k < nv) x = fma(-hk[k], V[k * ld + i], x);
      w[i] = x;
    }
    if (MODE == 2) {
      acc[0] = fma(x, x, acc[0]);
    } else {
#pragma unroll
      for (int k = 0; k < MAXV; ++k)
        if (k < nv) acc[k] = fma(V[k * ld + i], x, acc[k]);
    }
  }
  block_reduce_store(acc, MODE == 2 ? 1 : nv, partial, out, ticket);
}

// out_0 = ||r[continuity row]||^2, out_1 = ||r||^2
__global__ void __launch_bounds__(RT) k_norms(const double* __restrict__ r, size_t sn, size_t n,
                                              double* __restrict__ partial, double* out,
                                              unsigned int* ticket) {
  double acc[MAXV];
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

}  // namespace fr

namespace frk {
using namespace fr;

static int grid_for(const fr_ctx* c) { return c->red_blocks; }

template <int MODE>
static int krylov(fr_ctx* c, const double* V, int nv, const double* h, double* w, double* out,
                  cudaStream_t s) {
  if (nv < 1 || nv > MAXV) { snprintf(c->err, sizeof(c->err), "krylov: nv=%d", nv); return FR_ERR_ARG; }
  const int g = grid_for(c);
  FR_ACCOUNT(c, KK_KRYLOV, (MODE == 0 ? 2.0 : 4.0) * nv * c->ndof,
             8.0 * c->ndof * (nv + 1 + (MODE != 0 ? 1 : 0)));
  FR_PROF_BEGIN(c, s);
  k_krylov<MODE><<<g, RT, 0, s>>>(V, c->ndof, nv, h, w, c->ndof, c->red, out, c->ticket);
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
int lincomb(fr_ctx* c, const double* V, int nv, const double* y, double* u, cudaStream_t s) {
  FR_ACCOUNT(c, KK_VECTOR, 2.0 * nv * c->ndof, 8.0 * c->ndof * (nv + 1));
{ FR_PROF_BEGIN(c, s); k_lincomb<<<grid_for(c), RT, 0, s>>>(V, c->ndof, nv, y, u, c->ndof); FR_PROF_END(c, s, KK_VECTOR); }
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

}  // namespace frk
