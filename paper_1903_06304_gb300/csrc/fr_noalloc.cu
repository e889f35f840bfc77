// fr_noalloc.cu -- a residual entry point for callers that cannot allocate device memory.
//
// fr_residual needs a context, and creating a context calls cudaMalloc for the geometry,
// trace and face buffers.  Some callers cannot do that: code running inside a CUDA
// graph being captured, code under a custom allocator or memory pool that forbids
// outside allocations, or an embedding runtime that owns all device memory and hands
// out only the input and output buffers.  fr_residual_noalloc computes the same
// residual with all of its scratch in one file-scope device array, so a call performs
// no allocation of any kind.
#include <cstdio>
#include <mutex>
#include "fr_internal.h"
#include "fr_kernels.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB on every device using the library
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

inline size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// Device address of g_scratch on the current device, looked up once per device.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FR_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return FR_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return FR_OK;
}

template <int N>
int run(const fr_config* cfg, int nx, int ny, const double* corners, const double* vel,
        const double* q, double* R, cudaStream_t s) {
  using namespace fr;
  constexpr int NP = N * N, EPB = Tile<N>::EPB, TH = Tile<N>::THREADS;
  const size_t ne = (size_t)nx * ny;
  // every element needs well over 64 bytes of scratch: refusing larger meshes first keeps
  // the byte counts below from wrapping around for absurd nx, ny
  if (ne > kScratchBytes / 64) return FR_ERR_ARG;
  // scratch layout: geometry at solution and flux points, traces, local gradients,
  // common fluxes and common solutions of the owned faces
  const size_t b_gs = round256(sizeof(double) * GS_COUNT * ne * NP);
  const size_t b_gf = round256(sizeof(double) * GF_COUNT * ne * 4 * N);
  const size_t b_tq = round256(sizeof(double) * ne * 16 * N);
  const size_t b_tg = round256(sizeof(double) * ne * 32 * N);
  const size_t b_gl = round256(sizeof(double) * 8 * ne * NP);
  const size_t b_fn = round256(sizeof(double) * ne * 8 * N);
  const size_t b_nb = round256(sizeof(int) * ne * 5);
  const size_t b_cp = round256(sizeof(CaseParams));
  const size_t need = b_gs + b_gf + b_tq + b_tg + b_gl + 2 * b_fn + b_nb + b_cp;
  if (need > kScratchBytes) return FR_ERR_ARG;
  // an error left pending by an earlier, unrelated call is reported as such (and left in
  // place) rather than taken for a failure of this call's launches
  if (cudaPeekAtLastError() != cudaSuccess) return FR_ERR_CUDA;
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != FR_OK) return rc;
  unsigned char* p = static_cast<unsigned char*>(base);
  double* gs = reinterpret_cast<double*>(p); p += b_gs;
  double* gf = reinterpret_cast<double*>(p); p += b_gf;
  double* tq = reinterpret_cast<double*>(p); p += b_tq;
  double* tg = reinterpret_cast<double*>(p); p += b_tg;
  double* gl = reinterpret_cast<double*>(p); p += b_gl;
  double* fn = reinterpret_cast<double*>(p); p += b_fn;
  double* qc = reinterpret_cast<double*>(p); p += b_fn;
  int* nbr = reinterpret_cast<int*>(p);
  int* ecase = nbr + 4 * ne;
  p += b_nb;
  CaseParams* cpd = reinterpret_cast<CaseParams*>(p);
  const Basis B = fr_make_basis(N - 1);
  CaseParams cp;
  cp.gas = fr_make_gas(*cfg);
  cp.a0dt = cp.a1dt = cp.a2dt = cp.inv_dtau = cp.a0_dt = 0.0;
  cp.off = 0;
  cp.e0 = 0;
  cp.sn = (int)(ne * NP);
  cp.nx = nx;
  cp.ny = ny;
  cp.active = 1;
  Mesh M;
  M.nbr = nbr; M.ecase = ecase; M.cp = cpd; M.ne = (int)ne; M.viscous = cp.gas.viscous;
  k_fill_topo<<<(unsigned)((ne + 127) / 128), 128, 0, s>>>(nx, ny, 0, 0, nbr, ecase);
  k_set_case<<<1, 1, 0, s>>>(cpd, 0, cp);
  k_geometry<N><<<(unsigned)((ne + 63) / 64), 64, 0, s>>>(corners, vel, (int)ne, B, Buf<double>{gs},
                                                           Buf<double>{gf});
  const int nblk = (int)((ne + EPB - 1) / EPB);
  k_trace<double, N><<<nblk, TH, 0, s>>>(Buf<double>{const_cast<double*>(q)}, M, B, gs,
                                         Buf<double>{gl}, Buf<double>{tq}, Buf<double>{tg});
  const int nf = (int)(ne * 2 * N);
  k_face<double, N><<<(nf + 127) / 128, 128, 0, s>>>(M, B, gf, Buf<double>{tq}, Buf<double>{tg},
                                                    Buf<double>{fn}, Buf<double>{qc});
  TimeTerms tt{nullptr, nullptr};
  k_elem<double, N, MODE_RESID><<<nblk, TH, 0, s>>>(Buf<double>{const_cast<double*>(q)}, M, B,
                                                    gs, gf, Buf<double>{gl}, Buf<double>{tq},
                                                    Buf<double>{fn}, Buf<double>{qc}, R, tt);
  return cudaGetLastError() == cudaSuccess ? FR_OK : FR_ERR_CUDA;
}

}  // namespace

extern "C" int fr_residual_noalloc(const fr_config* cfg, int nx, int ny, const double* corners_d,
                                   const double* corner_vel_d, const double* qp_d, double* R_d,
                                   void* stream) {
  if (!cfg || !corners_d || !corner_vel_d || !qp_d || !R_d) return FR_ERR_ARG;
  if (cfg->p < 1 || cfg->p > 4 || nx < 2 || ny < 2 || cfg->mach <= 0 || cfg->gamma <= 1.0)
    return FR_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  switch (cfg->p + 1) {
    case 2: return run<2>(cfg, nx, ny, corners_d, corner_vel_d, qp_d, R_d, s);
    case 3: return run<3>(cfg, nx, ny, corners_d, corner_vel_d, qp_d, R_d, s);
    case 4: return run<4>(cfg, nx, ny, corners_d, corner_vel_d, qp_d, R_d, s);
    case 5: return run<5>(cfg, nx, ny, corners_d, corner_vel_d, qp_d, R_d, s);
  }
  return FR_ERR_ARG;
}
