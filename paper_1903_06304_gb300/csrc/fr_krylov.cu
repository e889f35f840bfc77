// fr_krylov.cu -- FP64 vector kernels of restarted GMRES with CGS2 (Sec. 3.2) and the
// pseudo-step residual norms.  Reductions are deterministic: a fixed grid writes one
// partial per block and a second launch sums the partials in a fixed order.
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

// Sum nv per-thread values over the block; thread 0 writes partial[k * nblk + blockIdx.x].
__device__ __forceinline__ void block_store(double (&acc)[MAXV], int nv, double* partial) {
  __shared__ double sm[MAXV][RT / 32];
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
}

// MODE 0: dots  partial_k = <V_k, w>
// MODE 1: w -= sum_k h_k V_k, then partial_k = <V_k, w>       (CGS2 second pass)
// MODE 2: w -= sum_k h_k V_k, then partial_0 = <w, w>
template <int MODE>
__global__ void __launch_bounds__(RT) k_krylov(const double* __restrict__ V, size_t ld, int nv,
                                               const double* __restrict__ h, double* w, size_t n,
                                               double* __restrict__ partial) {
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
  block_store(acc, MODE == 2 ? 1 : nv, partial);
}

// out[k] = sum over blocks of partial[k][*] (one thread per k, fixed order)
__global__ void k_finish(const double* __restrict__ partial, int nblk, int nv, double* out) {
  const int k = threadIdx.x;
  if (k >= nv) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(size_t)k * nblk + b];
  out[k] = s;
}

// partial_0 = ||r[continuity row]||^2, partial_1 = ||r||^2
__global__ void __launch_bounds__(RT) k_norms(const double* __restrict__ r, size_t sn, size_t n,
                                              double* __restrict__ partial) {
  double acc[MAXV];
  acc[0] = 0.0;
  acc[1] = 0.0;
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
    const double x = r[i];
    if (i < sn) acc[0] = fma(x, x, acc[0]);
    acc[1] = fma(x, x, acc[1]);
  }
  block_store(acc, 2, partial);
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
  k_krylov<MODE><<<g, RT, 0, s>>>(V, c->ndof, nv, h, w, c->ndof, c->red);
  FR_LAUNCH_CHECK(c);
  const int nk = MODE == 2 ? 1 : nv;
  k_finish<<<1, 32, 0, s>>>(c->red, g, nk, out);
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
  k_norms<<<g, RT, 0, s>>>(r, (size_t)c->ne * c->np2, c->ndof, c->red);
  FR_LAUNCH_CHECK(c);
  k_finish<<<1, 32, 0, s>>>(c->red, g, 2, out);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}
int scale(fr_ctx* c, const double* x, double a, double* y, cudaStream_t s) {
  k_scale<<<grid_for(c), RT, 0, s>>>(x, a, y, c->ndof);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}
int axpby(fr_ctx* c, double a, const double* x, double b, double* y, cudaStream_t s) {
  k_axpby<<<grid_for(c), RT, 0, s>>>(a, x, b, y, c->ndof);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}
// w -= sum_k h_k V_k (nv <= 32), no reduction
int axpy(fr_ctx* c, const double* V, int nv, const double* h, double* w, cudaStream_t s) {
  k_axpy_multi<<<grid_for(c), RT, 0, s>>>(V, c->ndof, nv, h, w, c->ndof);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}
int lincomb(fr_ctx* c, const double* V, int nv, const double* y, double* u, cudaStream_t s) {
  k_lincomb<<<grid_for(c), RT, 0, s>>>(V, c->ndof, nv, y, u, c->ndof);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

}  // namespace frk
