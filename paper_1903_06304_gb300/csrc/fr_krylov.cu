// fr_krylov.cu -- FP64 vector kernels of restarted GMRES with CGS2 (Sec. 3.2) and the
// pseudo-step residual norms.  Reductions are deterministic: a fixed grid writes one
// partial per block and the last block to finish sums the partials in a fixed order.
#include <algorithm>
#include <cstdio>
#include "fr_internal.h"
#include "fr_df.cuh"

namespace fr {

constexpr int RT = 256;    // threads per reduction block
constexpr int MAXV = 32;   // Krylov vectors handled per launch

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  return x;
}

// Sum of pp[0 .. count) by one warp in a fixed order: lane l adds pp[l + 32 i], four
// independent loads in flight (L2 reads: the partials come from other blocks after a
// fence), then a warp sum.
__device__ __forceinline__ double warp_sum_partials(const double* pp, int count) {
  const int lane = threadIdx.x & 31;
  double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
  int p = lane;
  for (; p + 96 < count; p += 128) {
    t0 += __ldcg(pp + p);
    t1 += __ldcg(pp + p + 32);
    t2 += __ldcg(pp + p + 64);
    t3 += __ldcg(pp + p + 96);
  }
  for (; p < count; p += 32) t0 += __ldcg(pp + p);
  return warp_sum((t0 + t1) + (t2 + t3));
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
// of the nb blocks b0 .. b0 + nb - 1 that share the ticket to finish (atomic ticket, no
// waiting) then sums their partials of every k in a fixed order and writes out[k]: one
// launch per reduction, deterministic result.  A whole-grid reduction passes b0 = 0,
// nb = gridDim.x; a batched one passes the block range of one case.  Returns true in the
// last block (after out[] is written and visible to the block).
template <int NA>
__device__ __forceinline__ bool block_reduce_store(double (&acc)[NA], int nv, double* partial,
                                                   double* out, unsigned int* ticket, int b0,
                                                   int nb) {
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
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == (unsigned)nb - 1;
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // final pass: warp w sums the partials of k = w, w + 8, ... in a fixed order
  const size_t ld = gridDim.x;
  for (int k = wid; k < nv; k += RT / 32) {
    const double s = warp_sum_partials(partial + (size_t)k * ld + b0, nb);
    if (lane == 0) out[k] = s;
  }
  if (threadIdx.x == 0) *ticket = 0u;
  __threadfence_block();
  __syncthreads();
  return true;
}

__device__ void gm_givens(GmresState* st, const double* h1, const double* h2, const double* nrm2);

// The streaming part of one reduction pass over pairs i = start, start + stride, ...
// below end, two pairs in flight per thread (16-byte loads; vector lengths and offsets
// are even: 4 variables per point).
// MODE 0: acc_k += <V_k, w>
// MODE 1: w -= sum_k h_k V_k, then acc_k += <V_k, w>       (CGS2 second pass)
// MODE 2: w -= sum_k h_k V_k, then acc_0 += <w, w>
template <int MODE, int NV, int NA>
__device__ __forceinline__ void krylov_pairs(const double2* __restrict__ V2, size_t ld2, double2* w2,
                                             int nv, const double (&hk)[NV], double (&acc)[NA],
                                             size_t start, size_t end, size_t stride) {
  for (size_t i = start; i < end; i += 2 * stride) {
    const bool two = i + stride < end;
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
}

// One reduction pass over the whole vector (modes as above; out_k the reduced sums).
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
#pragma unroll
  for (int k = 0; k < NV; ++k) hk[k] = (MODE != 0 && k < nv) ? h[k] : 0.0;
  const size_t stride = (size_t)gridDim.x * RT;
  krylov_pairs<MODE, NV>(reinterpret_cast<const double2*>(V), ld / 2, reinterpret_cast<double2*>(w),
                         nv, hk, acc, blockIdx.x * (size_t)RT + threadIdx.x, n / 2, stride);
  const bool last = block_reduce_store(acc, MODE == 2 ? 1 : nv, partial, out, ticket, 0, gridDim.x);
  // the norm pass of a device-resident Arnoldi step closes it with the Givens update
  if (MODE == 2 && gst && last && threadIdx.x < 32) gm_givens(gst, h - FR_MAX_RESTART, h, out);
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
  block_reduce_store(acc, 2, partial, out, ticket, 0, gridDim.x);
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
// the device (one GmresState per case) so that iterations are queued without a host
// round trip.

// Column j of H from the CGS2 projections h1 + h2 and ||w||, the previous rotations, a
// new rotation, the residual estimate |g_{j+1}| and the stopping test.  Called by the 32
// lanes of one warp: the column, cosines and sines are staged in shared memory in
// parallel, lane 0 applies the rotations (the running entry in a register, no global
// round trip per rotation), and the rotated column is written back in parallel.
__device__ void gm_givens(GmresState* st, const double* h1, const double* h2, const double* nrm2) {
  constexpr int L = GmresState::LD;
  __shared__ double col[L + 1], rc[L], rs[L];
  const int lane = threadIdx.x & 31;
  if (st->done) return;
  const int j = st->j;
  const double hn = sqrt(nrm2[0]);
  if (!isfinite(hn)) {
    __syncwarp();
    if (lane == 0) { st->nonfinite = 1; st->done = 1; }
    return;
  }
  for (int i = lane; i <= j; i += 32) col[i] = h2 ? h1[i] + h2[i] : h1[i];
  for (int i = lane; i < j; i += 32) { rc[i] = st->cs[i]; rs[i] = st->sn[i]; }
  __syncwarp();
  if (lane == 0) {
    double a = col[0];   // entry i of the column after rotations 0 .. i-1
    for (int i = 0; i < j; ++i) {
      const double b = col[i + 1];
      col[i] = rc[i] * a + rs[i] * b;
      a = -rs[i] * a + rc[i] * b;
    }
    const double den = hypot(a, hn);
    const double cj = a / den, sj = hn / den;
    col[j] = den;
    col[j + 1] = 0.0;
    st->cs[j] = cj;
    st->sn[j] = sj;
    const double gj = st->g[j];
    st->g[j + 1] = -sj * gj;
    st->g[j] = cj * gj;
    st->j = j + 1;
    st->inv_hn = hn > 0.0 ? 1.0 / hn : 0.0;
    if (fabs(st->g[j + 1]) <= st->tol || hn == 0.0 || j + 1 >= st->jmax) st->done = 1;
  }
  __syncwarp();
  for (int i = lane; i <= j + 1; i += 32) st->H[i * L + j] = col[i];
}

// Back substitution H[0:k,0:k] y = g[0:k], k = j (one thread).
__device__ void gm_trisolve(GmresState* st) {
  constexpr int L = GmresState::LD;
  const int k = st->j;
  for (int i = k - 1; i >= 0; --i) {
    double acc = st->g[i];
    for (int l = i + 1; l < k; ++l) acc -= st->H[i * L + l] * st->y[l];
    st->y[i] = acc / st->H[i * L + i];
  }
}

// ------------------------------------------------------------------ batched (per-case) forms
// The vectors of a batch hold its cases one after another.  Block b of a launch works on
// the pair range [blo[b], bhi[b]) of case bcase[b]; case k owns blocks cb0[k] ..
// cb0[k] + cnb[k] - 1.  Reductions are per case: the last of a case's blocks to finish
// sums that case's partials.  Each case has its own GMRES state; the Arnoldi passes skip
// a case whose cycle has stopped.  Per-case scalars: dsc[k * BDS + ...] with the first
// projections at [0, BM), the second at [BM, 2BM), ||w||^2 at 2BM, norms at 3BM.
constexpr int BM = GmresState::LD;
constexpr int BDS = 4 * BM;

// Per case: ||r[continuity row]||^2 and ||r||^2 at dsc[k * BDS + 3BM + 0..1]; the
// continuity row of case k ends at entry mend[k].
__global__ void __launch_bounds__(RT) k_bnorms(const double* __restrict__ r, BatchSegs sg,
                                               const long long* __restrict__ mend,
                                               double* __restrict__ partial, double* dsc,
                                               unsigned int* tickets) {
  const int k = sg.bcase[blockIdx.x];
  const size_t me = (size_t)mend[k];
  double acc[2] = {0.0, 0.0};
  const double2* r2 = reinterpret_cast<const double2*>(r);
  for (size_t i = (size_t)sg.blo[blockIdx.x] + threadIdx.x; i < (size_t)sg.bhi[blockIdx.x]; i += RT) {
    const double2 x = r2[i];
    const double xx = x.x * x.x, yy = x.y * x.y;
    if (2 * i < me) acc[0] += xx;
    if (2 * i + 1 < me) acc[0] += yy;
    acc[1] += xx + yy;
  }
  block_reduce_store(acc, 2, partial, dsc + (size_t)k * BDS + 3 * BM, tickets + k, sg.cb0[k], sg.cnb[k]);
}

// ---- Arnoldi passes of high occupancy.  The reductions above hold one accumulator per
// basis vector in every thread, which limits them to one 256-thread block per SM and
// leaves them waiting on loads.  Here the dot products run on a 2-D grid (pair range x
// group of KG vectors, a few accumulators per thread) and the updates w -= V h on a grid
// of SPLIT blocks per pair range (one accumulator per thread, coefficients in shared
// memory): the same FP64 operations with four to eight times the warps in flight.
constexpr int KG = 4;       // vectors per block of the dot-product pass
constexpr int SPLIT = 4;    // blocks per pair range of the update passes

// This block's nw sums acc[0..nw) go to partial[(k0 + q) * ld + pidx]; the last of the
// `target` blocks sharing the ticket writes out[q] = sum of partial[q * ld + p] over p in
// [first, first + count), q < nout, in a fixed order.  True in the last block.
template <int NA>
__device__ __forceinline__ bool seg_reduce(double (&acc)[NA], int nw, int k0, double* partial,
                                           size_t ld, size_t pidx, double* out, int nout,
                                           unsigned int* ticket, unsigned int target,
                                           size_t first, int count) {
  __shared__ double sm[NA][RT / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if constexpr (NA == 4) {
    // four values: the xor-16 and xor-8 exchanges each halve the set a lane carries, the
    // last three sum over the remaining lane bits; lane 8 q ends with the warp sum of
    // value q (6 additions per lane instead of 20)
    const bool u16 = (lane & 16) != 0, u8 = (lane & 8) != 0;
    double a0 = u16 ? acc[2] : acc[0], a1 = u16 ? acc[3] : acc[1];
    const double s0 = u16 ? acc[0] : acc[2], s1 = u16 ? acc[1] : acc[3];
    a0 += __shfl_xor_sync(0xffffffffu, s0, 16);
    a1 += __shfl_xor_sync(0xffffffffu, s1, 16);
    double v = u8 ? a1 : a0;
    const double sv = u8 ? a0 : a1;
    v += __shfl_xor_sync(0xffffffffu, sv, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    if ((lane & 7) == 0) sm[lane >> 3][wid] = v;
  } else {
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const double t = warp_sum(acc[q]);
      if (lane == 0) sm[q][wid] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x < nw) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < RT / 32; ++w) t += sm[threadIdx.x][w];
    partial[(size_t)(k0 + threadIdx.x) * ld + pidx] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == target - 1;
  __syncthreads();
  if (!last) return false;
  __threadfence();
  for (int q = wid; q < nout; q += RT / 32) {
    const double t = warp_sum_partials(partial + (size_t)q * ld + first, count);
    if (lane == 0) out[q] = t;
  }
  if (threadIdx.x == 0) *ticket = 0u;
  __threadfence_block();
  __syncthreads();
  return true;
}

// ds[out_off + k] = <V_k, w>, k < nv, per case (block (b, g): range b, vectors g KG ..).
__global__ void __launch_bounds__(RT) k_vdots(const double* __restrict__ V, size_t ld,
                                              const double* __restrict__ w, BatchSegs sg,
                                              double* __restrict__ partial, double* dsc,
                                              int out_off, unsigned int* tickets,
                                              const GmresState* gst) {
  const int b = blockIdx.x, g = blockIdx.y;
  const int k = sg.bcase[b];
  const GmresState* st = gst + k;
  if (st->done) return;
  const int nv = st->j + 1;
  const int ng = (nv + KG - 1) / KG;
  if (g >= ng) return;
  const int k0 = g * KG, nw = min(KG, nv - k0);
  double acc[KG] = {0.0, 0.0, 0.0, 0.0};
  const double2* V2 = reinterpret_cast<const double2*>(V);
  const double2* w2 = reinterpret_cast<const double2*>(w);
  const size_t ld2 = ld / 2;
  const size_t lo = (size_t)sg.blo[b], hi = (size_t)sg.bhi[b];
  for (size_t i = lo + threadIdx.x; i < hi; i += 2 * RT) {
    const bool two = i + RT < hi;
    const double2 xa = w2[i], xb = two ? w2[i + RT] : make_double2(0.0, 0.0);
#pragma unroll
    for (int q = 0; q < KG; ++q) {
      if (q < nw) {
        const double2 va = V2[(k0 + q) * ld2 + i];
        const double2 vb = two ? V2[(k0 + q) * ld2 + i + RT] : make_double2(0.0, 0.0);
        acc[q] = fma(va.x, xa.x, acc[q]);
        acc[q] = fma(va.y, xa.y, acc[q]);
        acc[q] = fma(vb.x, xb.x, acc[q]);
        acc[q] = fma(vb.y, xb.y, acc[q]);
      }
    }
  }
  seg_reduce(acc, nw, k0, partial, gridDim.x, b, dsc + (size_t)k * BDS + out_off, nv,
             tickets + k, (unsigned)(sg.cnb[k] * ng), (size_t)sg.cb0[k], sg.cnb[k]);
}

// w -= sum_{k < nv} h_k V_k with h = ds[h_off ..], per case; with NORM also ||w||^2 per
// case into ds[2BM] and, in the case's last block, the Givens update of the cycle.
template <bool NORM>
__global__ void __launch_bounds__(RT) k_vaxpy(const double* __restrict__ V, size_t ld, double* w,
                                              BatchSegs sg, double* __restrict__ partial,
                                              double* dsc, int h_off, unsigned int* tickets,
                                              GmresState* gst, int two_pass) {
  __shared__ double hs[GmresState::LD + 1];
  const int b = blockIdx.x, part = blockIdx.y;
  const int k = sg.bcase[b];
  GmresState* st = gst + k;
  if (st->done) return;
  const int nv = st->j + 1;
  double* ds = dsc + (size_t)k * BDS;
  for (int q = threadIdx.x; q < nv; q += RT) hs[q] = ds[h_off + q];
  __syncthreads();
  const size_t lo0 = (size_t)sg.blo[b], hi0 = (size_t)sg.bhi[b], len = hi0 - lo0;
  const size_t lo = lo0 + len * part / SPLIT, hi = lo0 + len * (part + 1) / SPLIT;
  const double2* V2 = reinterpret_cast<const double2*>(V);
  double2* w2 = reinterpret_cast<double2*>(w);
  const size_t ld2 = ld / 2;
  double acc[1] = {0.0};
  for (size_t i = lo + threadIdx.x; i < hi; i += RT) {
    double2 x = w2[i];
    int q = 0;
    for (; q + 8 <= nv; q += 8) {   // eight independent loads in flight, the sums in order
      double2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = V2[(q + u) * ld2 + i];
#pragma unroll
      for (int u = 0; u < 8; ++u) { x.x = fma(-hs[q + u], v[u].x, x.x); x.y = fma(-hs[q + u], v[u].y, x.y); }
    }
    for (; q + 4 <= nv; q += 4) {   // four independent loads in flight
      const double2 v0 = V2[(q + 0) * ld2 + i], v1 = V2[(q + 1) * ld2 + i];
      const double2 v2 = V2[(q + 2) * ld2 + i], v3 = V2[(q + 3) * ld2 + i];
      x.x = fma(-hs[q], v0.x, x.x); x.y = fma(-hs[q], v0.y, x.y);
      x.x = fma(-hs[q + 1], v1.x, x.x); x.y = fma(-hs[q + 1], v1.y, x.y);
      x.x = fma(-hs[q + 2], v2.x, x.x); x.y = fma(-hs[q + 2], v2.y, x.y);
      x.x = fma(-hs[q + 3], v3.x, x.x); x.y = fma(-hs[q + 3], v3.y, x.y);
    }
    for (; q < nv; ++q) {
      const double2 v = V2[q * ld2 + i];
      x.x = fma(-hs[q], v.x, x.x);
      x.y = fma(-hs[q], v.y, x.y);
    }
    w2[i] = x;
    if (NORM) {
      acc[0] = fma(x.x, x.x, acc[0]);
      acc[0] = fma(x.y, x.y, acc[0]);
    }
  }
  if (!NORM) return;
  const size_t pb = (size_t)b * SPLIT + part;
  const bool last = seg_reduce(acc, 1, 0, partial, (size_t)gridDim.x * SPLIT, pb, ds + 2 * BM, 1,
                               tickets + k, (unsigned)(sg.cnb[k] * SPLIT),
                               (size_t)sg.cb0[k] * SPLIT, sg.cnb[k] * SPLIT);
  if (last && threadIdx.x < 32) gm_givens(st, ds, two_pass ? ds + BM : nullptr, ds + 2 * BM);
}

// CGS2 middle step in one pass: w -= sum_k h1_k V_k over this block's part of a range
// (one pair per thread, kept in shared memory), then <V_k, w> of the updated part for
// every k < nv (warp q takes k = q, q + 8, ...), reduced per case into ds[BM ..].
__global__ void __launch_bounds__(RT) k_vaxdots(const double* __restrict__ V, size_t ld, double* w,
                                                BatchSegs sg, double* __restrict__ partial,
                                                double* dsc, unsigned int* tickets,
                                                GmresState* gst) {
  __shared__ double hs[GmresState::LD + 1];
  __shared__ double2 ws[RT];
  __shared__ double sums[GmresState::LD + 1];
  __shared__ bool last;
  const int b = blockIdx.x, part = blockIdx.y;
  const int k = sg.bcase[b];
  GmresState* st = gst + k;
  if (st->done) return;
  const int nv = st->j + 1;
  double* ds = dsc + (size_t)k * BDS;
  for (int q = threadIdx.x; q < nv; q += RT) hs[q] = ds[q];
  __syncthreads();
  const size_t lo0 = (size_t)sg.blo[b], hi0 = (size_t)sg.bhi[b], len0 = hi0 - lo0;
  const size_t lo = lo0 + len0 * part / SPLIT, hi = lo0 + len0 * (part + 1) / SPLIT;
  const int len = (int)(hi - lo);   // <= RT: a range holds at most 4 RT pairs
  const double2* V2 = reinterpret_cast<const double2*>(V);
  double2* w2 = reinterpret_cast<double2*>(w);
  const size_t ld2 = ld / 2;
  if (threadIdx.x < len) {
    const size_t i = lo + threadIdx.x;
    double2 x = w2[i];
    int q = 0;
    for (; q + 8 <= nv; q += 8) {   // eight independent loads in flight, the sums in order
      double2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = V2[(q + u) * ld2 + i];
#pragma unroll
      for (int u = 0; u < 8; ++u) { x.x = fma(-hs[q + u], v[u].x, x.x); x.y = fma(-hs[q + u], v[u].y, x.y); }
    }
    for (; q + 4 <= nv; q += 4) {
      const double2 v0 = V2[(q + 0) * ld2 + i], v1 = V2[(q + 1) * ld2 + i];
      const double2 v2 = V2[(q + 2) * ld2 + i], v3 = V2[(q + 3) * ld2 + i];
      x.x = fma(-hs[q], v0.x, x.x); x.y = fma(-hs[q], v0.y, x.y);
      x.x = fma(-hs[q + 1], v1.x, x.x); x.y = fma(-hs[q + 1], v1.y, x.y);
      x.x = fma(-hs[q + 2], v2.x, x.x); x.y = fma(-hs[q + 2], v2.y, x.y);
      x.x = fma(-hs[q + 3], v3.x, x.x); x.y = fma(-hs[q + 3], v3.y, x.y);
    }
    for (; q < nv; ++q) {
      const double2 v = V2[q * ld2 + i];
      x.x = fma(-hs[q], v.x, x.x);
      x.y = fma(-hs[q], v.y, x.y);
    }
    w2[i] = x;
    ws[threadIdx.x] = x;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // warp wid takes vectors q = wid + 16 i and q2 = q + 8 together (each w pair loaded once
  // for both); past nv the second stream repeats the first and is not stored
  for (int q = wid; q < nv; q += 2 * (RT / 32)) {
    const int q2 = q + RT / 32;
    const bool has2 = q2 < nv;
    const double2* vq = V2 + q * ld2 + lo;
    const double2* vr = V2 + (has2 ? q2 : q) * ld2 + lo;
    double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
    int t = lane;
    for (; t + 32 < len; t += 64) {
      const double2 xa = ws[t], xb = ws[t + 32];
      const double2 va = vq[t], vb = vq[t + 32], ra = vr[t], rb = vr[t + 32];
      a0 = fma(va.x, xa.x, a0); a0 = fma(va.y, xa.y, a0);
      a1 = fma(vb.x, xb.x, a1); a1 = fma(vb.y, xb.y, a1);
      b0 = fma(ra.x, xa.x, b0); b0 = fma(ra.y, xa.y, b0);
      b1 = fma(rb.x, xb.x, b1); b1 = fma(rb.y, xb.y, b1);
    }
    if (t < len) {
      const double2 xa = ws[t], va = vq[t], ra = vr[t];
      a0 = fma(va.x, xa.x, a0); a0 = fma(va.y, xa.y, a0);
      b0 = fma(ra.x, xa.x, b0); b0 = fma(ra.y, xa.y, b0);
    }
    // two values: the xor-16 exchange leaves lanes 0-15 the first, 16-31 the second
    const bool up = (lane & 16) != 0;
    double v = up ? b0 + b1 : a0 + a1;
    const double sv = up ? a0 + a1 : b0 + b1;
    v += __shfl_xor_sync(0xffffffffu, sv, 16);
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) sums[q] = v;
    if (lane == 16 && has2) sums[q2] = v;
  }
  __syncthreads();
  const size_t ldp = (size_t)gridDim.x * SPLIT, pb = (size_t)b * SPLIT + part;
  if (threadIdx.x < nv) partial[(size_t)threadIdx.x * ldp + pb] = sums[threadIdx.x];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(tickets + k, 1u) == (unsigned)(sg.cnb[k] * SPLIT) - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const size_t first = (size_t)sg.cb0[k] * SPLIT;
  const int count = sg.cnb[k] * SPLIT;
  for (int q = wid; q < nv; q += RT / 32) {
    const double t = warp_sum_partials(partial + (size_t)q * ldp + first, count);
    if (lane == 0) ds[BM + q] = t;
  }
  if (threadIdx.x == 0) tickets[k] = 0u;
}

// V[j] = next = w * inv_hn per case, j the case's newest basis index.  With init set the
// cycle's first vector is written for every case (inv_hn = 0 gives zeros for a case that
// does not iterate); otherwise stopped cases are skipped.
__global__ void k_bgm_store(const double* __restrict__ w, const GmresState* gst, double* __restrict__ V,
                            size_t ld, double* __restrict__ next, BatchSegs sg, int init) {
  const GmresState* st = gst + sg.bcase[blockIdx.x];
  if (!init && st->done) return;
  const double s = st->inv_hn;
  const size_t base = (size_t)st->j * (ld / 2);
  const double2* w2 = reinterpret_cast<const double2*>(w);
  double2* V2 = reinterpret_cast<double2*>(V);
  double2* n2 = reinterpret_cast<double2*>(next);
  for (size_t i = (size_t)sg.blo[blockIdx.x] + threadIdx.x; i < (size_t)sg.bhi[blockIdx.x]; i += RT) {
    const double2 x = w2[i];
    const double2 y = make_double2(x.x * s, x.y * s);
    V2[base + i] = y;
    n2[i] = y;
  }
}

// u = sum_{i < j} y_i V_i per case (zero for a case with no iteration in the cycle).
__global__ void k_blincomb(const double* __restrict__ V, size_t ld, const GmresState* gst,
                           double* __restrict__ u, BatchSegs sg) {
  const GmresState* st = gst + sg.bcase[blockIdx.x];
  const int nk = st->j;
  const double2* V2 = reinterpret_cast<const double2*>(V);
  double2* u2 = reinterpret_cast<double2*>(u);
  const size_t ld2 = ld / 2;
  for (size_t i = (size_t)sg.blo[blockIdx.x] + threadIdx.x; i < (size_t)sg.bhi[blockIdx.x]; i += RT) {
    double2 acc = make_double2(0.0, 0.0);
    for (int q = 0; q < nk; ++q) {
      const double2 v = V2[q * ld2 + i];
      acc.x = fma(st->y[q], v.x, acc.x);
      acc.y = fma(st->y[q], v.y, acc.y);
    }
    u2[i] = acc;
  }
}

// y += coef[k] x over case k's entries.
__global__ void k_baxpy_case(const double* __restrict__ coef, const double* __restrict__ x,
                             double* __restrict__ y, BatchSegs sg) {
  const double a = coef[sg.bcase[blockIdx.x]];
  if (a == 0.0) return;
  const double2* x2 = reinterpret_cast<const double2*>(x);
  double2* y2 = reinterpret_cast<double2*>(y);
  for (size_t i = (size_t)sg.blo[blockIdx.x] + threadIdx.x; i < (size_t)sg.bhi[blockIdx.x]; i += RT) {
    const double2 a2 = x2[i];
    double2 b2 = y2[i];
    b2.x = fma(a, a2.x, b2.x);
    b2.y = fma(a, a2.y, b2.y);
    y2[i] = b2;
  }
}

// Block k: back substitution of case k; thread k of block 0 gathers the stop state.
__global__ void k_bgm_trisolve(GmresState* gst) {
  if (threadIdx.x == 0) gm_trisolve(gst + blockIdx.x);
}
// out[k] = (j, jmax, done, nonfinite) of case k; out[ncases].x = the context's error flag
// (a bounded device wait that ran out).
__global__ void k_bgm_status(const GmresState* gst, int ncases, int4* out, const int* err) {
  for (int k = threadIdx.x; k < ncases; k += blockDim.x) {
    const GmresState* st = gst + k;
    out[k] = make_int4(st->j, st->jmax, st->done, st->nonfinite);
  }
  if (threadIdx.x == 0) out[ncases] = make_int4(*err, 0, 0, 0);
}

// ---- Fused Arnoldi step (arnoldi_fused): the whole CGS2 (or CGS) step of every case in
// one launch.  Block g owns a contiguous part [flo[g], fhi[g]) of one case's pairs, thread
// t the pairs t + FT i (i < PT), held in registers for the whole step: w is read once and
// V[j+1] and next are written once.  The step's reductions (V^T w once or twice, ||w||^2)
// meet at barriers of the case's blocks: each block writes its sums, arrives with one
// atomic add on the case's counter and waits until the case's nb blocks have arrived;
// then every block adds the nb blocks' sums itself, in a fixed order, so no block has to
// release the others and all of them hold identical bits.  The Givens update of the
// column is computed by every block in the same arithmetic; the case's first block writes
// it to the GMRES state.  Blocks of FT threads, at most as many as the GPU holds at once
// (occupancy x SMs), so a case's blocks are all resident while they wait on one another;
// every wait is bounded (wait_spins), and a wait that runs out sets the context's error
// flag and ends its block.
constexpr int FT = 512;    // threads per block of the fused step (two blocks per SM)
constexpr int FW = FT / 32;

struct FusedSegs {
  const int* fcase;              // [G] case of block g
  const long long* flo;          // [G] first pair of block g
  const long long* fhi;          // [G] one past its last pair
  const int* fb0;                // [ncases] first block of case k
  const int* fnb;                // [ncases] its block count
  double* part;                  // [3][BM][G] block sums of the step's three barriers
  unsigned long long* arrive;    // [ncases] arrivals at the case's barriers (a multiple of
                                 // the case's block count between launches)
  int G;
};

// Barrier `phase` (0, 1, 2 of a step) of the blocks of case k carrying the sums vals[q]
// (shared, q < nv): on a true return out[q] (shared) holds the sum over the case's blocks,
// added in block order.  Barrier b of a case ends when the counter reaches (b + 1) nb; each
// phase has its own buffer of sums, written once per launch.  False: this block's wait ran
// out (error flag set) and the block must leave.
__device__ bool fused_barrier_sum(const double* vals, int nv, int k, int phase, const FusedSegs& F,
                                  double* out, long long spins, int* err) {
  __shared__ int s_ok;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int gb0 = F.fb0[k], nb = F.fnb[k];
  const size_t G = (size_t)F.G;
  double* P = F.part + (size_t)phase * BM * G;
  if (tid < nv) P[(size_t)tid * G + blockIdx.x] = vals[tid];
  __syncthreads();
  if (tid == 0) {
    // the block's sums are ordered before its arrival by the block barrier and this fence
    __threadfence();
    const unsigned long long old = atomicAdd(F.arrive + k, 1ull);
    const unsigned long long target = old - old % (unsigned long long)nb + (unsigned long long)nb;
    int ok = 1;
    if (old + 1 != target) {
      ok = 0;
      const long long n = spins < 0 ? 1 : spins;
      for (long long i = 0; i < n; ++i) {
        if (*(volatile unsigned long long*)(F.arrive + k) >= target) { ok = 1; break; }
        if (spins >= 0) __nanosleep(20);
      }
      if (!ok) atomicExch(err, 1);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  if (!s_ok) return false;
  for (int q = wid; q < nv; q += FW) {
    const double v = warp_sum_partials(P + (size_t)q * G + gb0, nb);
    if (lane == 0) out[q] = v;
  }
  __syncthreads();
  return true;
}

// Warp sums of eight values per lane by recursive halving (bits 16, 8, 4 of the lane
// index pick the half a lane keeps), then the last two lane bits: lane l with l % 4 == 0
// ends with the sum of value 4 b16 + 2 b8 + b4 (9 additions per lane instead of 40).
__device__ __forceinline__ double warp_sum8(double (&a)[8]) {
  const int lane = threadIdx.x & 31;
  const bool u16 = (lane & 16) != 0, u8 = (lane & 8) != 0, u4 = (lane & 4) != 0;
  double b[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const double keep = u16 ? a[m + 4] : a[m], send = u16 ? a[m] : a[m + 4];
    b[m] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  double c[2];
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const double keep = u8 ? b[m + 2] : b[m], send = u8 ? b[m] : b[m + 2];
    c[m] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const double keep = u4 ? c[1] : c[0], send = u4 ? c[0] : c[1];
  double v = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

// This block's sums of <V_q, x> over its pairs (thread t: pairs t + FT i, i < PT) for
// q < nv into sums[q]: eight vectors at a time per thread, warp sums by warp_sum8, the
// FW warp sums of each vector added in warp order.
template <int PT>
__device__ __forceinline__ void fused_dots(const double2* V2, size_t ld2, size_t lo, int len,
                                           const double2 (&x)[PT], int nv,
                                           double (*wsum)[FW], double* sums) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int q0 = 0; q0 < nv; q0 += 8) {
    double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < PT; ++i) {
      const int t = tid + FT * i;
      if (t < len) {
        double2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          v[u] = q0 + u < nv ? V2[(size_t)(q0 + u) * ld2 + lo + t] : make_double2(0.0, 0.0);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          acc[u] = fma(v[u].x, x[i].x, acc[u]);
          acc[u] = fma(v[u].y, x[i].y, acc[u]);
        }
      }
    }
    const double s = warp_sum8(acc);
    const int u = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    if ((lane & 3) == 0 && q0 + u < nv) wsum[q0 + u][wid] = s;
  }
  __syncthreads();
  for (int q = wid; q < nv; q += FW) {
    const double t = warp_sum(lane < FW ? wsum[q][lane] : 0.0);
    if (lane == 0) sums[q] = t;
  }
  __syncthreads();
}

// x -= sum_{q < nv} h[q] V_q over this thread's pairs (eight loads in flight, the sums in
// order of q).
template <int PT>
__device__ __forceinline__ void fused_axpy(const double2* V2, size_t ld2, size_t lo, int len,
                                           double2 (&x)[PT], int nv, const double* h) {
#pragma unroll
  for (int i = 0; i < PT; ++i) {
    const int t = threadIdx.x + FT * i;
    if (t >= len) continue;
    const size_t p = lo + t;
    double2 y = x[i];
    int q = 0;
    for (; q + 8 <= nv; q += 8) {
      double2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = V2[(size_t)(q + u) * ld2 + p];
#pragma unroll
      for (int u = 0; u < 8; ++u) { y.x = fma(-h[q + u], v[u].x, y.x); y.y = fma(-h[q + u], v[u].y, y.y); }
    }
    for (; q < nv; ++q) {
      const double2 v = V2[(size_t)q * ld2 + p];
      y.x = fma(-h[q], v.x, y.x);
      y.y = fma(-h[q], v.y, y.y);
    }
    x[i] = y;
  }
}

// One Arnoldi step of every case whose cycle runs: h1 = V^T w; (CGS2) w -= V h1, h2 = V^T w;
// w -= V h2 (h1 for CGS); ||w||^2; the Givens update of column j (the arithmetic of
// gm_givens, in every block; the case's first block writes the state); V[j+1] = next =
// w / ||w|| unless the cycle stopped.
template <int PT>
__global__ void __launch_bounds__(FT, 2) k_arnoldi_fused(double* V, size_t ld, const double* __restrict__ w,
                                                         double* __restrict__ next, FusedSegs F,
                                                         GmresState* gst, int two_pass, long long spins,
                                                         int* err) {
  constexpr int L = GmresState::LD;
  __shared__ double wsum[BM][FW];
  __shared__ double h1[BM], h2[BM], sums[BM], col[L + 1], rc[L], rs[L];
  __shared__ double s_g, s_tol, s_inv_hn;
  __shared__ int s_jmax, s_done, s_nonfinite;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int k = F.fcase[blockIdx.x];
  GmresState* st = gst + k;
  if (st->done) return;
  const int j = st->j, nv = j + 1;
  const size_t lo = (size_t)F.flo[blockIdx.x];
  const int len = (int)((size_t)F.fhi[blockIdx.x] - lo);
  const double2* V2 = reinterpret_cast<const double2*>(V);
  const size_t ld2 = ld / 2;
  const double2* w2 = reinterpret_cast<const double2*>(w);
  double2 x[PT];
#pragma unroll
  for (int i = 0; i < PT; ++i) {
    const int t = tid + FT * i;
    x[i] = t < len ? w2[lo + t] : make_double2(0.0, 0.0);
  }
  // the rotation inputs, read before this block's first arrival: the case's first block
  // rewrites them only after every block has passed the last barrier
  for (int i = tid; i < j; i += FT) { rc[i] = st->cs[i]; rs[i] = st->sn[i]; }
  if (tid == 0) { s_g = st->g[j]; s_tol = st->tol; s_jmax = st->jmax; }
  // h1 = V^T w
  fused_dots<PT>(V2, ld2, lo, len, x, nv, wsum, sums);
  if (!fused_barrier_sum(sums, nv, k, 0, F, h1, spins, err)) return;
  const double* h = h1;
  int phase = 1;
  if (two_pass) {
    // w -= V h1; h2 = V^T w
    fused_axpy<PT>(V2, ld2, lo, len, x, nv, h1);
    fused_dots<PT>(V2, ld2, lo, len, x, nv, wsum, sums);
    if (!fused_barrier_sum(sums, nv, k, 1, F, h2, spins, err)) return;
    h = h2;
    phase = 2;
  }
  // w -= V h; ||w||^2
  fused_axpy<PT>(V2, ld2, lo, len, x, nv, h);
  double a = 0.0;
#pragma unroll
  for (int i = 0; i < PT; ++i) {
    a = fma(x[i].x, x[i].x, a);   // pairs past len hold zeros
    a = fma(x[i].y, x[i].y, a);
  }
  a = warp_sum(a);
  if (lane == 0) wsum[0][wid] = a;
  __syncthreads();
  if (wid == 0) {
    const double t = warp_sum(lane < FW ? wsum[0][lane] : 0.0);
    if (lane == 0) sums[0] = t;
  }
  __syncthreads();
  double* nrm = sums + 1;
  if (!fused_barrier_sum(sums, 1, k, phase, F, nrm, spins, err)) return;
  // Givens update of column j
  for (int i = tid; i <= j; i += FT) col[i] = two_pass ? h1[i] + h2[i] : h1[i];
  __syncthreads();
  if (tid == 0) {
    const double hn = sqrt(nrm[0]);
    s_nonfinite = !isfinite(hn);
    if (s_nonfinite) {
      s_done = 1;
    } else {
      double aa = col[0];
      for (int i = 0; i < j; ++i) {
        const double bb = col[i + 1];
        col[i] = rc[i] * aa + rs[i] * bb;
        aa = -rs[i] * aa + rc[i] * bb;
      }
      const double den = hypot(aa, hn);
      const double cj = aa / den, sj = hn / den;
      col[j] = den;
      col[j + 1] = 0.0;
      rc[j] = cj;
      rs[j] = sj;
      const double g1 = -sj * s_g;
      s_g = cj * s_g;
      sums[0] = g1;
      s_inv_hn = hn > 0.0 ? 1.0 / hn : 0.0;
      s_done = (fabs(g1) <= s_tol || hn == 0.0 || j + 1 >= s_jmax) ? 1 : 0;
    }
  }
  __syncthreads();
  if (blockIdx.x == F.fb0[k]) {
    if (s_nonfinite) {
      if (tid == 0) { st->nonfinite = 1; st->done = 1; }
    } else {
      if (tid == 0) {
        st->cs[j] = rc[j];
        st->sn[j] = rs[j];
        st->g[j + 1] = sums[0];
        st->g[j] = s_g;
        st->j = j + 1;
        st->inv_hn = s_inv_hn;
        st->done = s_done;
      }
      for (int i = tid; i <= j + 1; i += FT) st->H[i * L + j] = col[i];
    }
  }
  if (s_done) return;
  // V[j+1] = next = w / ||w||
  const double s = s_inv_hn;
  double2* Vw = reinterpret_cast<double2*>(V) + (size_t)(j + 1) * ld2;
  double2* n2 = reinterpret_cast<double2*>(next);
#pragma unroll
  for (int i = 0; i < PT; ++i) {
    const int t = tid + FT * i;
    if (t < len) {
      const double2 y = make_double2(x[i].x * s, x[i].y * s);
      Vw[lo + t] = y;
      n2[lo + t] = y;
    }
  }
}

// ---- Double-float Arnoldi (krylov_arith = FR_KRYLOV_DF64).  The basis is stored as FP32
// pairs: entry i of vector q is the float2 (hi, lo) in the 8 bytes an FP64 entry would
// take, so a pair of entries is one 16-byte float4 (h0, l0, h1, l1).  The products, sums
// and updates of the Gram-Schmidt passes run on the FP32 pipe with error-free
// transformations (about 2^-48 relative); the FP64 pipe only converts w on entry and
// exit of a pass and sums the per-block partials.  w, next and the Hessenberg data stay
// FP64.

// One double-float per thread for each of NA values: warp sums, then the warps of the
// block merged by thread q < nw into one FP64 partial[(k0 + q) * ld + pidx]; the last of
// the `target` blocks sharing the ticket sums the partials as seg_reduce does.
template <int NA>
__device__ __forceinline__ bool seg_reduce_df(float (&ah)[NA], float (&al)[NA], int nw, int k0,
                                              double* partial, size_t ld, size_t pidx, double* out,
                                              int nout, unsigned int* ticket, unsigned int target,
                                              size_t first, int count) {
  __shared__ float2 sm[NA][RT / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    float h = ah[q], l = al[q];
    df_warp_sum(h, l);
    if (lane == 0) sm[q][wid] = make_float2(h, l);
  }
  __syncthreads();
  if (threadIdx.x < nw) {
    float h = 0.0f, l = 0.0f;
#pragma unroll
    for (int w = 0; w < RT / 32; ++w) df_merge(h, l, sm[threadIdx.x][w].x, sm[threadIdx.x][w].y);
    partial[(size_t)(k0 + threadIdx.x) * ld + pidx] = df_value(h, l);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == target - 1;
  __syncthreads();
  if (!last) return false;
  __threadfence();
  for (int q = wid; q < nout; q += RT / 32) {
    const double t = warp_sum_partials(partial + (size_t)q * ld + first, count);
    if (lane == 0) out[q] = t;
  }
  if (threadIdx.x == 0) *ticket = 0u;
  __threadfence_block();
  __syncthreads();
  return true;
}

__device__ __forceinline__ float4 df_split2(double2 x) {
  const float2 a = df_split(x.x), b = df_split(x.y);
  return make_float4(a.x, a.y, b.x, b.y);
}

// k_vdots with a double-float basis.
__global__ void __launch_bounds__(RT) k_vdots_df(const float4* __restrict__ V4, size_t ld,
                                                 const double* __restrict__ w, BatchSegs sg,
                                                 double* __restrict__ partial, double* dsc,
                                                 int out_off, unsigned int* tickets,
                                                 const GmresState* gst) {
  const int b = blockIdx.x, g = blockIdx.y;
  const int k = sg.bcase[b];
  const GmresState* st = gst + k;
  if (st->done) return;
  const int nv = st->j + 1;
  const int ng = (nv + KG - 1) / KG;
  if (g >= ng) return;
  const int k0 = g * KG, nw = min(KG, nv - k0);
  float ah[KG] = {0.0f, 0.0f, 0.0f, 0.0f}, al[KG] = {0.0f, 0.0f, 0.0f, 0.0f};
  const double2* w2 = reinterpret_cast<const double2*>(w);
  const size_t ld2 = ld / 2;
  const size_t lo = (size_t)sg.blo[b], hi = (size_t)sg.bhi[b];
  for (size_t i = lo + threadIdx.x; i < hi; i += 2 * RT) {
    const bool two = i + RT < hi;
    const float4 xa = df_split2(w2[i]);
    const float4 xb = two ? df_split2(w2[i + RT]) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
    for (int q = 0; q < KG; ++q) {
      if (q < nw) {
        const float4 va = V4[(k0 + q) * ld2 + i];
        const float4 vb = two ? V4[(k0 + q) * ld2 + i + RT] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        df_fma(ah[q], al[q], va.x, va.y, xa.x, xa.y);
        df_fma(ah[q], al[q], va.z, va.w, xa.z, xa.w);
        df_fma(ah[q], al[q], vb.x, vb.y, xb.x, xb.y);
        df_fma(ah[q], al[q], vb.z, vb.w, xb.z, xb.w);
      }
    }
  }
  seg_reduce_df(ah, al, nw, k0, partial, gridDim.x, b, dsc + (size_t)k * BDS + out_off, nv,
                tickets + k, (unsigned)(sg.cnb[k] * ng), (size_t)sg.cb0[k], sg.cnb[k]);
}

// x -= sum_{q < nv} h_q V_q for one pair of entries (x as two double-floats).
__device__ __forceinline__ void df_pair_update(float4& x, const float2* hs, const float4* V4,
                                               size_t ld2, size_t i, int nv) {
  int q = 0;
  for (; q + 2 <= nv; q += 2) {   // two independent loads in flight
    const float4 v0 = V4[(q + 0) * ld2 + i], v1 = V4[(q + 1) * ld2 + i];
    const float2 h0 = hs[q], h1 = hs[q + 1];
    df_fms(x.x, x.y, h0.x, h0.y, v0.x, v0.y);
    df_fms(x.z, x.w, h0.x, h0.y, v0.z, v0.w);
    df_fms(x.x, x.y, h1.x, h1.y, v1.x, v1.y);
    df_fms(x.z, x.w, h1.x, h1.y, v1.z, v1.w);
  }
  if (q < nv) {
    const float4 v = V4[q * ld2 + i];
    const float2 h = hs[q];
    df_fms(x.x, x.y, h.x, h.y, v.x, v.y);
    df_fms(x.z, x.w, h.x, h.y, v.z, v.w);
  }
}

// k_vaxpy with a double-float basis.
template <bool NORM>
__global__ void __launch_bounds__(RT) k_vaxpy_df(const float4* __restrict__ V4, size_t ld, double* w,
                                                 BatchSegs sg, double* __restrict__ partial,
                                                 double* dsc, int h_off, unsigned int* tickets,
                                                 GmresState* gst, int two_pass) {
  __shared__ float2 hs[GmresState::LD + 1];
  const int b = blockIdx.x, part = blockIdx.y;
  const int k = sg.bcase[b];
  GmresState* st = gst + k;
  if (st->done) return;
  const int nv = st->j + 1;
  double* ds = dsc + (size_t)k * BDS;
  for (int q = threadIdx.x; q < nv; q += RT) hs[q] = df_split(ds[h_off + q]);
  __syncthreads();
  const size_t lo0 = (size_t)sg.blo[b], hi0 = (size_t)sg.bhi[b], len = hi0 - lo0;
  const size_t lo = lo0 + len * part / SPLIT, hi = lo0 + len * (part + 1) / SPLIT;
  double2* w2 = reinterpret_cast<double2*>(w);
  const size_t ld2 = ld / 2;
  float nh[1] = {0.0f}, nl[1] = {0.0f};
  for (size_t i = lo + threadIdx.x; i < hi; i += RT) {
    float4 x = df_split2(w2[i]);
    df_pair_update(x, hs, V4, ld2, i, nv);
    w2[i] = make_double2(df_value(x.x, x.y), df_value(x.z, x.w));
    if (NORM) {
      df_fma(nh[0], nl[0], x.x, x.y, x.x, x.y);
      df_fma(nh[0], nl[0], x.z, x.w, x.z, x.w);
    }
  }
  if (!NORM) return;
  const size_t pb = (size_t)b * SPLIT + part;
  const bool last = seg_reduce_df(nh, nl, 1, 0, partial, (size_t)gridDim.x * SPLIT, pb, ds + 2 * BM, 1,
                                  tickets + k, (unsigned)(sg.cnb[k] * SPLIT),
                                  (size_t)sg.cb0[k] * SPLIT, sg.cnb[k] * SPLIT);
  if (last && threadIdx.x < 32) gm_givens(st, ds, two_pass ? ds + BM : nullptr, ds + 2 * BM);
}

// k_vaxdots with a double-float basis: the updated part of w is kept in shared memory as
// double-floats for the second projections.
__global__ void __launch_bounds__(RT) k_vaxdots_df(const float4* __restrict__ V4, size_t ld, double* w,
                                                   BatchSegs sg, double* __restrict__ partial,
                                                   double* dsc, unsigned int* tickets,
                                                   GmresState* gst) {
  __shared__ float2 hs[GmresState::LD + 1];
  __shared__ float4 ws[RT];
  __shared__ double sums[GmresState::LD + 1];
  __shared__ bool last;
  const int b = blockIdx.x, part = blockIdx.y;
  const int k = sg.bcase[b];
  GmresState* st = gst + k;
  if (st->done) return;
  const int nv = st->j + 1;
  double* ds = dsc + (size_t)k * BDS;
  for (int q = threadIdx.x; q < nv; q += RT) hs[q] = df_split(ds[q]);
  __syncthreads();
  const size_t lo0 = (size_t)sg.blo[b], hi0 = (size_t)sg.bhi[b], len0 = hi0 - lo0;
  const size_t lo = lo0 + len0 * part / SPLIT, hi = lo0 + len0 * (part + 1) / SPLIT;
  const int len = (int)(hi - lo);   // <= RT: a range holds at most 4 RT pairs
  double2* w2 = reinterpret_cast<double2*>(w);
  const size_t ld2 = ld / 2;
  if (threadIdx.x < len) {
    const size_t i = lo + threadIdx.x;
    float4 x = df_split2(w2[i]);
    df_pair_update(x, hs, V4, ld2, i, nv);
    w2[i] = make_double2(df_value(x.x, x.y), df_value(x.z, x.w));
    ws[threadIdx.x] = x;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = wid; q < nv; q += RT / 32) {
    const float4* vq = V4 + q * ld2 + lo;
    float h0 = 0.0f, l0 = 0.0f, h1 = 0.0f, l1 = 0.0f;
    int t = lane;
    for (; t + 32 < len; t += 64) {
      const float4 va = vq[t], vb = vq[t + 32];
      const float4 xa = ws[t], xb = ws[t + 32];
      df_fma(h0, l0, va.x, va.y, xa.x, xa.y);
      df_fma(h0, l0, va.z, va.w, xa.z, xa.w);
      df_fma(h1, l1, vb.x, vb.y, xb.x, xb.y);
      df_fma(h1, l1, vb.z, vb.w, xb.z, xb.w);
    }
    if (t < len) {
      const float4 va = vq[t], xa = ws[t];
      df_fma(h0, l0, va.x, va.y, xa.x, xa.y);
      df_fma(h0, l0, va.z, va.w, xa.z, xa.w);
    }
    df_merge(h0, l0, h1, l1);
    df_warp_sum(h0, l0);
    if (lane == 0) sums[q] = df_value(h0, l0);
  }
  __syncthreads();
  const size_t ldp = (size_t)gridDim.x * SPLIT, pb = (size_t)b * SPLIT + part;
  if (threadIdx.x < nv) partial[(size_t)threadIdx.x * ldp + pb] = sums[threadIdx.x];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(tickets + k, 1u) == (unsigned)(sg.cnb[k] * SPLIT) - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const size_t first = (size_t)sg.cb0[k] * SPLIT;
  const int count = sg.cnb[k] * SPLIT;
  for (int q = wid; q < nv; q += RT / 32) {
    const double t = warp_sum_partials(partial + (size_t)q * ldp + first, count);
    if (lane == 0) ds[BM + q] = t;
  }
  if (threadIdx.x == 0) tickets[k] = 0u;
}

// k_bgm_store with a double-float basis: next = w inv_hn in FP64, V[j] = its split.
__global__ void k_bgm_store_df(const double* __restrict__ w, const GmresState* gst, float4* __restrict__ V4,
                               size_t ld, double* __restrict__ next, BatchSegs sg, int init) {
  const GmresState* st = gst + sg.bcase[blockIdx.x];
  if (!init && st->done) return;
  const double s = st->inv_hn;
  const size_t base = (size_t)st->j * (ld / 2);
  const double2* w2 = reinterpret_cast<const double2*>(w);
  double2* n2 = reinterpret_cast<double2*>(next);
  for (size_t i = (size_t)sg.blo[blockIdx.x] + threadIdx.x; i < (size_t)sg.bhi[blockIdx.x]; i += RT) {
    const double2 x = w2[i];
    const double2 y = make_double2(__dmul_rn(x.x, s), __dmul_rn(x.y, s));
    V4[base + i] = df_split2(y);
    n2[i] = y;
  }
}

// k_blincomb with a double-float basis.
__global__ void k_blincomb_df(const float4* __restrict__ V4, size_t ld, const GmresState* gst,
                              double* __restrict__ u, BatchSegs sg) {
  __shared__ float2 ys[GmresState::LD];
  const GmresState* st = gst + sg.bcase[blockIdx.x];
  const int nk = st->j;
  for (int q = threadIdx.x; q < nk; q += blockDim.x) ys[q] = df_split(st->y[q]);
  __syncthreads();
  double2* u2 = reinterpret_cast<double2*>(u);
  const size_t ld2 = ld / 2;
  for (size_t i = (size_t)sg.blo[blockIdx.x] + threadIdx.x; i < (size_t)sg.bhi[blockIdx.x]; i += RT) {
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int q = 0; q < nk; ++q) {
      const float4 v = V4[q * ld2 + i];
      df_fma(acc.x, acc.y, ys[q].x, ys[q].y, v.x, v.y);
      df_fma(acc.z, acc.w, ys[q].x, ys[q].y, v.z, v.w);
    }
    u2[i] = make_double2(df_value(acc.x, acc.y), df_value(acc.z, acc.w));
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
int check_device_waits(fr_ctx* c, cudaStream_t s) {
  int h = 0;
  FR_CUDA_CHECK(c, cudaMemcpyAsync(&h, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  FR_CUDA_CHECK(c, cudaStreamSynchronize(s));
  if (h == 0) return FR_OK;
  FR_CUDA_CHECK(c, cudaMemsetAsync(c->dev_err, 0, sizeof(int), s));
  FR_TRY(fused_reset(c, s));
  snprintf(c->err, sizeof(c->err), "a bounded device wait ran out of its budget (wait_spins)");
  return FR_ERR_TIMEOUT;
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

// ------------------------------------------------------------------ batched launchers
namespace frk {
using namespace fr;

template <class T> static int bw_alloc(fr_ctx* c, T** p, size_t n) {
  FR_CUDA_CHECK(c, cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T)));
  return FR_OK;
}
template <class T> static int bw_alloc_host(fr_ctx* c, T** p, size_t n) {
  FR_CUDA_CHECK(c, cudaMallocHost((void**)p, std::max<size_t>(n, 1) * sizeof(T)));
  return FR_OK;
}

void batch_free(fr_ctx* c) {
  BatchWork& b = c->bw;
  void* dev[] = {b.bcase, b.cb0, b.cnb, b.blo, b.bhi, b.mend, b.partial, b.tickets, b.dsc, b.gst,
                 b.status, b.coef, b.fz_case, b.fz_b0, b.fz_nb, b.fz_lo, b.fz_hi, b.fz_part,
                 b.fz_arrive};
  for (void* p : dev) if (p) cudaFree(p);
  void* host[] = {b.hsc, b.gst_h, b.status_h, b.coef_h, b.cp_stage};
  for (void* p : host) if (p) cudaFreeHost(p);
  if (b.staged) cudaEventDestroy(b.staged);
  b = BatchWork();
}

// Block table of the fused Arnoldi step: the smallest PT (pairs per thread, or the one
// arnoldi_fused names) whose blocks (each case's pairs split evenly, at most PT FT pairs
// a block) the GPU holds at once; fz_pt = 0 when none does.
// (the largest shared-memory carveout is requested first, so that the launch has the
// shared memory the occupancy figure assumes)
template <int PT> static cudaError_t fused_occupancy(int* out) {
  const cudaError_t e = cudaFuncSetAttribute(k_arnoldi_fused<PT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                             (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_arnoldi_fused<PT>, FT, 0);
}
static int fused_blocks_per_sm(int pt, int* out) {
  cudaError_t e = cudaErrorInvalidValue;
  switch (pt) {
    case 1: e = fused_occupancy<1>(out); break;
    case 2: e = fused_occupancy<2>(out); break;
    case 4: e = fused_occupancy<4>(out); break;
  }
  return e == cudaSuccess ? 0 : 1;
}

static int fused_setup(fr_ctx* c) {
  BatchWork& b = c->bw;
  b.fz_pt = b.fz_G = 0;
  if (c->cfg.arnoldi_fused == 0) return FR_OK;
  const int nc = c->ncases;
  int dev = 0, nsm = 0;
  FR_CUDA_CHECK(c, cudaGetDevice(&dev));
  FR_CUDA_CHECK(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int want = c->cfg.arnoldi_fused;
  int pt = 0, G = 0;
  // first the smallest part size with at most one block per SM (fewer blocks per barrier,
  // two pairs per thread in flight: measured the faster shape), else the smallest that
  // the GPU holds at once
  for (int pass = 0; pass < 2 && pt == 0; ++pass) {
    for (int cand : {1, 2, 4}) {
      if (want > 1 && cand != want) continue;
      int per_sm = 0;
      if (fused_blocks_per_sm(cand, &per_sm)) {
        snprintf(c->err, sizeof(c->err), "fused Arnoldi: occupancy query failed");
        return FR_ERR_CUDA;
      }
      long long g = 0;
      for (int k = 0; k < nc; ++k) {
        const long long np = 2LL * c->cps[k].sn;
        g += std::max<long long>(1, (np + (long long)cand * FT - 1) / ((long long)cand * FT));
      }
      const long long cap = pass == 0 ? std::min<long long>(nsm, (long long)per_sm * nsm) : (long long)per_sm * nsm;
      if (g <= cap) { pt = cand; G = (int)g; break; }
    }
  }
  if (pt == 0) return FR_OK;
  std::vector<int> fcase, fb0(nc), fnb(nc);
  std::vector<long long> flo, fhi;
  for (int k = 0; k < nc; ++k) {
    const long long p0 = c->cps[k].off / 2, np = 2LL * c->cps[k].sn;
    const int nb = (int)std::max<long long>(1, (np + (long long)pt * FT - 1) / ((long long)pt * FT));
    fb0[k] = (int)fcase.size();
    fnb[k] = nb;
    for (int q = 0; q < nb; ++q) {
      fcase.push_back(k);
      flo.push_back(p0 + np * q / nb);
      fhi.push_back(p0 + np * (q + 1) / nb);
    }
  }
  if (bw_alloc(c, &b.fz_case, G) || bw_alloc(c, &b.fz_lo, G) || bw_alloc(c, &b.fz_hi, G) ||
      bw_alloc(c, &b.fz_b0, nc) || bw_alloc(c, &b.fz_nb, nc) ||
      bw_alloc(c, &b.fz_part, (size_t)3 * BM * G) || bw_alloc(c, &b.fz_arrive, nc))
    return FR_ERR_CUDA;
  FR_CUDA_CHECK(c, cudaMemcpy(b.fz_case, fcase.data(), G * sizeof(int), cudaMemcpyHostToDevice));
  FR_CUDA_CHECK(c, cudaMemcpy(b.fz_lo, flo.data(), G * sizeof(long long), cudaMemcpyHostToDevice));
  FR_CUDA_CHECK(c, cudaMemcpy(b.fz_hi, fhi.data(), G * sizeof(long long), cudaMemcpyHostToDevice));
  FR_CUDA_CHECK(c, cudaMemcpy(b.fz_b0, fb0.data(), nc * sizeof(int), cudaMemcpyHostToDevice));
  FR_CUDA_CHECK(c, cudaMemcpy(b.fz_nb, fnb.data(), nc * sizeof(int), cudaMemcpyHostToDevice));
  FR_CUDA_CHECK(c, cudaMemset(b.fz_arrive, 0, nc * sizeof(unsigned long long)));
  b.fz_pt = pt;
  b.fz_G = G;
  return FR_OK;
}

// The barrier counters of the fused step back to their resting value after a wait ran out
// and left a barrier half passed.
int fused_reset(fr_ctx* c, cudaStream_t s) {
  BatchWork& b = c->bw;
  if (!b.fz_arrive) return FR_OK;
  FR_CUDA_CHECK(c, cudaMemsetAsync(b.fz_arrive, 0, c->ncases * sizeof(unsigned long long), s));
  return FR_OK;
}

// Blocks of each case in proportion to its length: at most 4 pairs per thread (a range
// holds at most 4 RT pairs, one pair per thread of each of the SPLIT parts).
int batch_setup(fr_ctx* c) {
  batch_free(c);
  BatchWork& b = c->bw;
  const int nc = c->ncases;
  std::vector<int> bcase, cb0(nc), cnb(nc);
  std::vector<long long> blo, bhi, mend(nc);
  for (int k = 0; k < nc; ++k) {
    const long long p0 = c->cps[k].off / 2, np = 2LL * c->cps[k].sn;
    const int nb = (int)std::max<long long>(1, (np + 4 * RT - 1) / (4 * RT));
    cb0[k] = (int)bcase.size();
    cnb[k] = nb;
    mend[k] = c->cps[k].off + c->cps[k].sn;
    for (int q = 0; q < nb; ++q) {
      bcase.push_back(k);
      blo.push_back(p0 + np * q / nb);
      bhi.push_back(p0 + np * (q + 1) / nb);
    }
  }
  b.nblk = (int)bcase.size();
  if (bw_alloc(c, &b.bcase, b.nblk) || bw_alloc(c, &b.blo, b.nblk) || bw_alloc(c, &b.bhi, b.nblk) ||
      bw_alloc(c, &b.cb0, nc) || bw_alloc(c, &b.cnb, nc) || bw_alloc(c, &b.mend, nc) ||
      bw_alloc(c, &b.partial, (size_t)GmresState::LD * SPLIT * b.nblk) || bw_alloc(c, &b.tickets, nc) ||
      bw_alloc(c, &b.dsc, (size_t)BDS * nc) || bw_alloc(c, &b.gst, nc) ||
      bw_alloc(c, &b.status, nc + 1) || bw_alloc(c, &b.coef, nc) ||
      bw_alloc_host(c, &b.hsc, (size_t)BDS * nc) || bw_alloc_host(c, &b.gst_h, nc) ||
      bw_alloc_host(c, &b.status_h, nc + 1) || bw_alloc_host(c, &b.coef_h, nc) ||
      bw_alloc_host(c, &b.cp_stage, nc))
    return FR_ERR_CUDA;
  FR_CUDA_CHECK(c, cudaEventCreateWithFlags(&b.staged, cudaEventDisableTiming));
  FR_CUDA_CHECK(c, cudaMemcpy(b.bcase, bcase.data(), b.nblk * sizeof(int), cudaMemcpyHostToDevice));
  FR_CUDA_CHECK(c, cudaMemcpy(b.blo, blo.data(), b.nblk * sizeof(long long), cudaMemcpyHostToDevice));
  FR_CUDA_CHECK(c, cudaMemcpy(b.bhi, bhi.data(), b.nblk * sizeof(long long), cudaMemcpyHostToDevice));
  FR_CUDA_CHECK(c, cudaMemcpy(b.cb0, cb0.data(), nc * sizeof(int), cudaMemcpyHostToDevice));
  FR_CUDA_CHECK(c, cudaMemcpy(b.cnb, cnb.data(), nc * sizeof(int), cudaMemcpyHostToDevice));
  FR_CUDA_CHECK(c, cudaMemcpy(b.mend, mend.data(), nc * sizeof(long long), cudaMemcpyHostToDevice));
  FR_CUDA_CHECK(c, cudaMemset(b.tickets, 0, nc * sizeof(unsigned int)));
  FR_CUDA_CHECK(c, cudaMemset(b.gst, 0, nc * sizeof(GmresState)));
  b.sg = BatchSegs{b.bcase, b.blo, b.bhi, b.cb0, b.cnb};
  return fused_setup(c);
}

// The device-resident cycle stores its basis as double-floats when krylov_arith asks.
static bool df_basis(const fr_ctx* c) { return c->cfg.krylov_arith == FR_KRYLOV_DF64; }

int bk_norms(fr_ctx* c, const double* r, cudaStream_t s) {
  FR_ACCOUNT(c, KK_KRYLOV, 2.0 * c->ndof, 8.0 * c->ndof);
  FR_PROF_BEGIN(c, s);
  k_bnorms<<<c->bw.nblk, RT, 0, s>>>(r, c->bw.sg, c->bw.mend, c->bw.partial, c->bw.dsc, c->bw.tickets);
  FR_PROF_END(c, s, KK_KRYLOV);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

int bk_init(fr_ctx* c, const double* r, double* next, cudaStream_t s) {
  FR_ACCOUNT(c, KK_VECTOR, 1.0 * c->ndof, 24.0 * c->ndof);
  FR_PROF_BEGIN(c, s);
  if (df_basis(c))
    k_bgm_store_df<<<c->bw.nblk, RT, 0, s>>>(r, c->bw.gst, reinterpret_cast<float4*>(c->V), c->ndof, next,
                                             c->bw.sg, 1);
  else
    k_bgm_store<<<c->bw.nblk, RT, 0, s>>>(r, c->bw.gst, c->V, c->ndof, next, c->bw.sg, 1);
  FR_PROF_END(c, s, KK_VECTOR);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

int bk_orthogonalize(fr_ctx* c, double* w, double* next, int nv_bound, cudaStream_t s) {
  BatchWork& b = c->bw;
  const dim3 gdots(b.nblk, (nv_bound + KG - 1) / KG), gaxpy(b.nblk, SPLIT);
  const bool two = c->cfg.orthog == FR_ORTHO_CGS2;
  // CGS2: h1 = V^T w; (w -= V h1, h2 = V^T w); (w -= V h2, ||w||, Givens); V[j+1] = w/||w||
  // CGS:  h1 = V^T w; (w -= V h1, ||w||, Givens); V[j+1] = w/||w||
  FR_ACCOUNT(c, KK_KRYLOV, (two ? 8.0 : 4.0) * nv_bound * c->ndof + 2.0 * c->ndof,
             8.0 * c->ndof * ((two ? 4.0 : 2.0) * nv_bound + 6.0));
  const bool df = df_basis(c);
  if (!df && b.fz_pt > 0) {
    // the whole step in one launch: V read once per pass, w once, V[j+1] and next written once
    FR_ACCOUNT(c, KK_KRYLOV, (two ? 8.0 : 4.0) * nv_bound * c->ndof + 3.0 * c->ndof,
               8.0 * c->ndof * ((two ? 4.0 : 2.0) * nv_bound + 3.0));
    const FusedSegs F{b.fz_case, b.fz_lo, b.fz_hi, b.fz_b0, b.fz_nb, b.fz_part, b.fz_arrive, b.fz_G};
    const long long spins = c->cfg.wait_spins == 0 ? (1LL << 22) : c->cfg.wait_spins;
    FR_PROF_BEGIN(c, s);
    switch (b.fz_pt) {
#define FR_FUSED_CASE(P)                                                                          \
  case P:                                                                                         \
    k_arnoldi_fused<P><<<b.fz_G, FT, 0, s>>>(c->V, c->ndof, w, next, F, b.gst, two ? 1 : 0,       \
                                             spins, c->dev_err);                                  \
    break;
      FR_FUSED_CASE(1)
      FR_FUSED_CASE(2)
      FR_FUSED_CASE(4)
#undef FR_FUSED_CASE
    }
    FR_PROF_END(c, s, KK_KRYLOV);
    FR_LAUNCH_CHECK(c);
    return FR_OK;
  }
  const float4* V4 = reinterpret_cast<const float4*>(c->V);
  {
    FR_PROF_BEGIN(c, s);
    if (df) k_vdots_df<<<gdots, RT, 0, s>>>(V4, c->ndof, w, b.sg, b.partial, b.dsc, 0, b.tickets, b.gst);
    else k_vdots<<<gdots, RT, 0, s>>>(c->V, c->ndof, w, b.sg, b.partial, b.dsc, 0, b.tickets, b.gst);
    FR_PROF_END(c, s, KK_KRYLOV);
    FR_LAUNCH_CHECK(c);
  }
  if (two) {
    FR_PROF_BEGIN(c, s);
    if (df) k_vaxdots_df<<<gaxpy, RT, 0, s>>>(V4, c->ndof, w, b.sg, b.partial, b.dsc, b.tickets, b.gst);
    else k_vaxdots<<<gaxpy, RT, 0, s>>>(c->V, c->ndof, w, b.sg, b.partial, b.dsc, b.tickets, b.gst);
    FR_PROF_END(c, s, KK_KRYLOV);
    FR_LAUNCH_CHECK(c);
  }
  {
    FR_PROF_BEGIN(c, s);
    if (df)
      k_vaxpy_df<true><<<gaxpy, RT, 0, s>>>(V4, c->ndof, w, b.sg, b.partial, b.dsc, two ? BM : 0,
                                            b.tickets, b.gst, two ? 1 : 0);
    else
      k_vaxpy<true><<<gaxpy, RT, 0, s>>>(c->V, c->ndof, w, b.sg, b.partial, b.dsc, two ? BM : 0,
                                         b.tickets, b.gst, two ? 1 : 0);
    FR_PROF_END(c, s, KK_KRYLOV);
    FR_LAUNCH_CHECK(c);
  }
  {
    FR_ACCOUNT(c, KK_VECTOR, 1.0 * c->ndof, 24.0 * c->ndof);
    FR_PROF_BEGIN(c, s);
    if (df)
      k_bgm_store_df<<<b.nblk, RT, 0, s>>>(w, b.gst, reinterpret_cast<float4*>(c->V), c->ndof, next, b.sg, 0);
    else
      k_bgm_store<<<b.nblk, RT, 0, s>>>(w, b.gst, c->V, c->ndof, next, b.sg, 0);
    FR_PROF_END(c, s, KK_VECTOR);
    FR_LAUNCH_CHECK(c);
  }
  return FR_OK;
}

int bk_finish(fr_ctx* c, double* u, cudaStream_t s) {
  {
    FR_PROF_BEGIN(c, s);
    k_bgm_trisolve<<<c->ncases, 32, 0, s>>>(c->bw.gst);
    FR_PROF_END(c, s, KK_KRYLOV);
    FR_LAUNCH_CHECK(c);
  }
  {
    FR_ACCOUNT(c, KK_VECTOR, 2.0 * GmresState::LD * c->ndof, 8.0 * c->ndof * (GmresState::LD + 1));
    FR_PROF_BEGIN(c, s);
    if (df_basis(c))
      k_blincomb_df<<<c->bw.nblk, RT, 0, s>>>(reinterpret_cast<const float4*>(c->V), c->ndof, c->bw.gst, u,
                                              c->bw.sg);
    else
      k_blincomb<<<c->bw.nblk, RT, 0, s>>>(c->V, c->ndof, c->bw.gst, u, c->bw.sg);
    FR_PROF_END(c, s, KK_VECTOR);
    FR_LAUNCH_CHECK(c);
  }
  return FR_OK;
}

int bk_status(fr_ctx* c, cudaStream_t s) {
  {
    FR_PROF_BEGIN(c, s);
    k_bgm_status<<<1, 256, 0, s>>>(c->bw.gst, c->ncases, c->bw.status, c->dev_err);
    FR_PROF_END(c, s, KK_KRYLOV);
    FR_LAUNCH_CHECK(c);
  }
  FR_CUDA_CHECK(c, cudaMemcpyAsync(c->bw.status_h, c->bw.status, (c->ncases + 1) * sizeof(int4),
                                   cudaMemcpyDeviceToHost, s));
  return FR_OK;
}

int bk_axpy_case(fr_ctx* c, const double* coef, const double* x, double* y, cudaStream_t s) {
  FR_ACCOUNT(c, KK_VECTOR, 2.0 * c->ndof, 24.0 * c->ndof);
  FR_PROF_BEGIN(c, s);
  k_baxpy_case<<<c->bw.nblk, RT, 0, s>>>(coef, x, y, c->bw.sg);
  FR_PROF_END(c, s, KK_VECTOR);
  FR_LAUNCH_CHECK(c);
  return FR_OK;
}

}  // namespace frk
