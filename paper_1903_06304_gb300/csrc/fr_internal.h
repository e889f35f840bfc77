// fr_internal.h -- context layout and kernel launchers shared by the library's
// translation units (not part of the public C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "fr_device.cuh"
#include "../../include/fr.h"

struct fr_ctx {
  fr_config cfg;
  int p, n, np2, bsz;
  int nx, ny, ne;
  size_t ndof;
  fr::Basis basis;
  fr::Gas gas;
  fr::Mesh mesh;
  // geometry (Sec. 2.3)
  double* gs = nullptr;   // [GS_COUNT][Ne*np2]
  double* gf = nullptr;   // [GF_COUNT][Ne*4*n]
  // residual intermediates: value and tangent copies
  double *tq = nullptr, *tg = nullptr, *gl = nullptr, *fn = nullptr, *qcm = nullptr;
  double *tq_d = nullptr, *tg_d = nullptr, *gl_d = nullptr, *fn_d = nullptr, *qcm_d = nullptr;
  // element blocks
  double* B64 = nullptr;     // [Ne][b][b] unfactored
  void* Binv = nullptr;      // scaled inverse, transposed, in the configured precision
  float* Dr = nullptr;       // [Ne][b] row scales
  float* Dc = nullptr;       // [Ne][b] column scales
  int* info = nullptr;       // [Ne] singular flags
  int blocks_ready = 0;
  // Krylov workspace
  double* V = nullptr;       // [(m+1)][ndof]
  double *w_r = nullptr, *w_z = nullptr, *w_x = nullptr, *w_t = nullptr, *w_u = nullptr;
  double* red = nullptr;     // reduction partials
  double* dsc = nullptr;     // small device scalars
  double* hsc = nullptr;     // pinned host mirror of dsc
  int red_blocks = 0;
  long long launches = 0;
  char err[512];
};

namespace frk {
int geometry(fr_ctx* c, const double* corners, const double* vel, cudaStream_t s);
int residual(fr_ctx* c, const double* q, double* out, const double* qcn, const double* qcnm1,
             double a0dt, double a1dt, double a2dt, cudaStream_t s);
int jvp(fr_ctx* c, const double* q, const double* v, double inv_dtau, double a0_dt, double* out,
        cudaStream_t s);
int conservative(fr_ctx* c, const double* q, double* qc, cudaStream_t s);
int block_build(fr_ctx* c, const double* q, double inv_dtau, double a0_dt, cudaStream_t s);
int block_apply(fr_ctx* c, const double* r, double* z, cudaStream_t s);
// Krylov primitives (deterministic reductions over a fixed grid)
int dots(fr_ctx* c, const double* V, int nv, const double* w, double* out_dev, cudaStream_t s);
int axpy_dots(fr_ctx* c, const double* V, int nv, const double* h_dev, double* w, double* out_dev,
              cudaStream_t s);
int axpy_norm(fr_ctx* c, const double* V, int nv, const double* h_dev, double* w, double* out_dev,
              cudaStream_t s);
int norms(fr_ctx* c, const double* r, double* out_dev, cudaStream_t s);
int scale(fr_ctx* c, const double* x, double a, double* y, cudaStream_t s);
int lincomb(fr_ctx* c, const double* V, int nv, const double* y_dev, double* u, cudaStream_t s);
int axpy(fr_ctx* c, const double* V, int nv, const double* h_dev, double* w, cudaStream_t s);
int axpby(fr_ctx* c, double a, const double* x, double b, double* y, cudaStream_t s);
}  // namespace frk

#define FR_CUDA_CHECK(c, expr)                                                       \
  do {                                                                               \
    cudaError_t e_ = (expr);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      snprintf((c)->err, sizeof((c)->err), "%s: %s (%s:%d)", #expr,                  \
               cudaGetErrorString(e_), __FILE__, __LINE__);                          \
      return FR_ERR_CUDA;                                                            \
    }                                                                                \
  } while (0)

#define FR_LAUNCH_CHECK(c)                                                           \
  do {                                                                               \
    (c)->launches++;                                                                 \
    cudaError_t e_ = cudaGetLastError();                                             \
    if (e_ != cudaSuccess) {                                                         \
      snprintf((c)->err, sizeof((c)->err), "launch: %s (%s:%d)",                     \
               cudaGetErrorString(e_), __FILE__, __LINE__);                          \
      return FR_ERR_CUDA;                                                            \
    }                                                                                \
  } while (0)
