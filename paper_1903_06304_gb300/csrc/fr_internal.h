// fr_internal.h -- context layout and kernel launchers shared by the library's
// translation units (not part of the public C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <functional>
#include <vector>
#include "fr_device.cuh"
#include "../../include/fr.h"

// Device-resident state of one GMRES restart cycle (restart <= 128).
struct GmresState {
  static constexpr int LD = 128;   // longest restart cycle kept on the device
  // header: set by the host at the start of a cycle (everything before H)
  double tol;      // absolute tolerance tol_res * ||b||
  double inv_hn;   // 1/||w|| of the newest vector
  int j;           // newest basis index = iterations done in this cycle
  int jmax;        // iteration limit of this cycle
  int done;
  int nonfinite;
  double g[LD + 1], cs[LD], sn[LD], y[LD];
  // Hessenberg matrix: column j is written by the Givens update of iteration j
  double H[(LD + 1) * LD];
};

// Per-case partition of a batch's vectors for the batched vector kernels: block b works
// on the pair range [blo[b], bhi[b]) of case bcase[b]; case k owns blocks cb0[k] ..
// cb0[k] + cnb[k] - 1 (device arrays).
struct BatchSegs {
  const int* bcase;
  const long long* blo;
  const long long* bhi;
  const int* cb0;
  const int* cnb;
};

// Workspace of the batched Krylov and Newton loops (allocated by frk::batch_setup).
struct BatchWork {
  int nblk = 0;                    // blocks of one batched vector launch
  BatchSegs sg{};
  int *bcase = nullptr, *cb0 = nullptr, *cnb = nullptr;
  long long *blo = nullptr, *bhi = nullptr, *mend = nullptr;
  double* partial = nullptr;       // [32][nblk x 4]: up to 32 sums per block of a split pass
  unsigned int* tickets = nullptr; // [ncases], kept at 0
  double* dsc = nullptr;           // [ncases][128] per-case scalars
  double* hsc = nullptr;           // pinned mirror
  GmresState* gst = nullptr;       // [ncases]
  GmresState* gst_h = nullptr;     // pinned mirror
  int4* status = nullptr;          // [ncases] (j, jmax, done, nonfinite), [ncases].x = error flag
  int4* status_h = nullptr;
  // fused Arnoldi step (arnoldi_fused, fr_krylov.cu): pairs per thread (0: the step does
  // not fit the resident blocks and runs as split passes), block table, sums, barrier state
  int fz_pt = 0, fz_G = 0;
  int *fz_case = nullptr, *fz_b0 = nullptr, *fz_nb = nullptr;
  long long *fz_lo = nullptr, *fz_hi = nullptr;
  double* fz_part = nullptr;               // [3][BM][G] block sums of the three barriers
  unsigned long long* fz_arrive = nullptr;  // [ncases] barrier arrivals
  double* coef = nullptr;          // [ncases] per-case coefficients
  double* coef_h = nullptr;        // pinned staging
  fr::CaseParams* cp_stage = nullptr;   // pinned staging of the case table
  cudaEvent_t staged = nullptr;    // the last upload from pinned staging has completed
};

// One level of the two-level preconditioner's coarse hierarchy (fr_mg.cu): cells carry
// 12 P1 coefficients (4 variables x mean, xi slope, eta slope).  Level 0 has one cell per
// element; level l+1 agglomerates 2 x 2 cells of level l within each case.  A case whose
// level has at most 4 cells is solved there exactly (dense inverse); its cells have
// parent -1.  The coefficient arrays hold the coarse precision (cfg.mg_prec: float or
// double); mode[c] = 1 marks the cells that this level's multi-block kernels sweep (the
// rest belong to a case whose remaining levels run in its single-block kernel).
struct MgLevel {
  int nc = 0;                 // cells (all cases)
  int nsweep = 0;             // cells with mode 1
  int *nb = nullptr;          // [nc][5] distinct stencil members, slot 0 = self, -1 unused
  int *cell_case = nullptr;   // [nc]
  int *mode = nullptr;        // [nc]
  void *A = nullptr;          // [nc][5][12][12] operator blocks by stencil slot
  void *Dinv = nullptr;       // [nc][12][12] inverse diagonal blocks (cells with a parent)
  void *x = nullptr, *y = nullptr, *b = nullptr;   // [nc][12] cycle vectors
  int *parent = nullptr;      // [nc] cell of level l+1, -1 for a case finishing here
  double *qo = nullptr;       // [nc][4]: s_a f_x, s_b f_y, f_x, f_y of the cell in its parent
  int *children = nullptr;    // [nc of level l+1][4], -1 unused
  int *gslot = nullptr;       // [nc][5]: slot of parent(nb[c][s]) in parent(c)'s stencil
  int nfin = 0;               // cases finishing at this level
  int *fin = nullptr;         // [nfin][2]: first cell, cell count
  void *Ainv = nullptr;       // [nfin][48][48] dense inverses (row-major, count*12 used)
  int ntail = 0;              // cases whose single-block kernel starts at this level
  int *tail = nullptr;        // [ntail] their case indices
  int ntiles = 0;             // tiles of the tiled kernels on this level
  void *tiles = nullptr;      // [ntiles] (case, first column, first row)
  void *cl = nullptr;         // [ncases] each case's grid on this level
  // the transposed hierarchy (A^T's Galerkin operators are the transposes of A's): the
  // slot of c in the stencil of each member, and A^T's blocks, diagonal inverses and dense
  // inverses, built on demand for the adjoint solve
  int *rslot = nullptr;       // [nc][5]
  void *AT = nullptr, *DinvT = nullptr, *AinvT = nullptr;
};

// Input of the block apply fused with the coarse correction (level-0 cells are the
// elements): z = P y0 + B^-1 (r - (A P) y0), with AP [Ne][5][12][b] and y0 [Ne][12] in
// the coarse precision, the level-0 stencils nb [Ne][5] and the solution points xs.
struct CoarseIn {
  const void* AP = nullptr;
  const void* y0 = nullptr;
  const int* nb = nullptr;
  double xs[5] = {0, 0, 0, 0, 0};
};

// Kernel classes for the optional per-kernel timing (fr_profile) and launch counts.
enum FrKernel {
  KK_GEOM, KK_TRACE, KK_FACE, KK_ELEM, KK_TRACE_JVP, KK_FACE_JVP, KK_ELEM_JVP, KK_BLOCK,
  KK_FACTOR, KK_APPLY, KK_KRYLOV, KK_VECTOR, KK_CONS, KK_LINEARIZE, KK_LIN_APPLY,
  KK_LIN_ADJOINT, KK_COARSE, KK_COUNT
};

struct FrProfPair {
  cudaEvent_t a, b;
  int kind;
};
struct FrProf {
  bool on = false;
  std::vector<cudaEvent_t> pool;   // reusable events
  size_t used = 0;                 // events handed out since the last read
  std::vector<FrProfPair> pairs;   // recorded launches since the last read
  double ms[KK_COUNT] = {};
  long long n[KK_COUNT] = {};
};

// Tile shapes (K of Tile<N, K>) of the point-parallel kernels: residual and dual JVP
// trace / element passes and the element pass of the linearised operator.
struct TileChoice {
  int trace = 1, elem = 1, trace_d = 1, elem_d = 1, lin_elem = 1;
};

// A captured chunk of GMRES iterations (CUDA graph) and the launch / algorithmic counts
// one replay adds.
struct GraphEntry {
  int start, count, tag;
  const void* q;
  cudaGraphExec_t exec;
  long long launches;
  long long by_kind[KK_COUNT];
  double flops[KK_COUNT], bytes[KK_COUNT];
};

struct fr_ctx {
  fr_config cfg;
  int p, n, np2, bsz;
  int nx, ny, ne;
  size_t ndof;
  fr::Basis basis;
  fr::Gas gas;                 // host copy of case 0's gas
  fr::Mesh mesh;               // device topology and case table of the launches
  int* nbr = nullptr;          // [Ne][4] face neighbours
  int* ecase = nullptr;        // [Ne] case of each element
  fr::CaseParams* cp = nullptr;  // [ncases] device
  fr::CaseParams cp_h;         // host copy of case 0's parameters
  std::vector<fr::CaseParams> cps;   // host copies of every case's parameters
  int ncases = 1;
  bool external_terms = false;  // time and operator terms are set per case by the caller
  BatchWork bw;                 // batched loops (cases of one degree and viscous switch)
  std::vector<GraphEntry> graphs;   // captured GMRES chunks (fr_api.cu)
  TileChoice tile;                  // tile shapes (fr_linear.cu autotune_tiles)
  // parameter sensitivities (fr_sens.cu): geometry values and tangents, seeds, per-element
  // dot products, a zero state tangent and the residual tangent
  double *sgs = nullptr, *sdgs = nullptr, *sgf = nullptr, *sdgf = nullptr;
  double *seed = nullptr, *edot = nullptr, *zero = nullptr, *rtan = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream used only for capturing
  // geometry (Sec. 2.3)
  double* gs = nullptr;   // [GS_COUNT][Ne*np2]
  double* gf = nullptr;   // [GF_COUNT][Ne*4*n]
  // residual intermediates: value and tangent copies
  double *tq = nullptr, *tg = nullptr, *gl = nullptr, *fn = nullptr, *qcm = nullptr;
  double *tq_d = nullptr, *tg_d = nullptr, *gl_d = nullptr, *fn_d = nullptr, *qcm_d = nullptr;
  // bounded meshes (fr_set_mesh_bounded): boundary kinds below row 0 / above row ny-1 and
  // the common flux and state of the faces below row 0, [nx][4][n] (value and tangent)
  int bounded = 0, bc_below = 0, bc_above = 0;
  double *fnb = nullptr, *fnb_d = nullptr, *qcb = nullptr, *qcb_d = nullptr;
  // element blocks
  double* B64 = nullptr;     // [Ne][b][b] unfactored
  void* Binv = nullptr;      // scaled inverse, transposed, in the configured precision
  float* Dr = nullptr;       // [Ne][b] row scales
  float* Dc = nullptr;       // [Ne][b] column scales
  int* info = nullptr;       // [Ne] singular flags
  int blocks_ready = 0;
  // stored local Jacobians of the Newton operator (fr_linear.cu)
  double *JFQ = nullptr, *JFG = nullptr;           // face map: [32|64][Ne*2n]
  double *JP = nullptr, *JG = nullptr, *PP = nullptr;  // point map: [32|64|16][Ne*n^2]
  double *JFQb = nullptr, *JFGb = nullptr;         // faces below row 0: [16|32][nx*n]
  double *adj_q = nullptr, *adj_fn = nullptr, *adj_qc = nullptr;  // transpose work
  int lin_ready = 0;
  int transposed = 0;   // set during fr_adjoint_solve: GMRES applies A^T and B^-T
  int* dev_err = nullptr;   // set by a device wait that ran out of its budget (read by
                            // check_device_waits, which clears it)
  int apply_grid[3] = {0, 0, 0};   // persistent grid of the bulk-copy apply, per coarse form
  // two-level preconditioner (cfg.precond == FR_PRECOND_TWO_LEVEL, fr_mg.cu)
  std::vector<MgLevel> mg;
  int mg_ncol = 0;                 // colours of the level-0 Galerkin products
  int *mg_colslot = nullptr;       // [Ne][ncol]: stencil slot of colour k's member, -1
  double *mg_x = nullptr, *mg_y = nullptr;   // fine seeds and products of the build
  // the build's Newton operator applied to the P1 functions of each stencil member,
  // restricted to the element's rows, [Ne][5][12][b] in the coarse precision (the
  // smoothing step's A z0 = (A P) y0 without an operator product)
  void *mg_ap = nullptr;
  int *mg_bad = nullptr;           // singular coarse blocks met by the builds (device)
  void *mg_views = nullptr;        // device copies of the level views (single-block kernels)
  void *mg_views_t = nullptr;      // the same for the transposed hierarchy
  int mg_t_ready = 0;              // the transposed hierarchy matches the last build
  void *mg_tc = nullptr;           // [ncases] per-case level ranges of the single-block kernels
  const double* mg_q = nullptr;    // state of the last build (dual-number operator)
  double mg_inv_dtau = 0.0, mg_a0_dt = 0.0;
  // Krylov workspace
  double* V = nullptr;       // [(m+1)][ndof]
  double *w_r = nullptr, *w_z = nullptr, *w_x = nullptr, *w_t = nullptr, *w_u = nullptr;
  double* red = nullptr;     // reduction partials
  unsigned int* ticket = nullptr;  // last-block counter of the reductions (kept at 0)
  double* dsc = nullptr;     // small device scalars
  double* hsc = nullptr;     // pinned host mirror of dsc
  int red_blocks = 0;
  long long launches = 0;
  long long launches_by_kind[KK_COUNT] = {};
  double alg_flops[KK_COUNT] = {};   // algorithmic FP64/FP32 flops issued per class
  double alg_bytes[KK_COUNT] = {};   // algorithmic DRAM bytes (streaming kernels)
  FrProf prof;
  char err[512];
};

// Algorithmic FP flops per solution point of the point-parallel kernels (see the design
// notes for the itemised count; +,-,*,/,sqrt = 1 flop, FMA = 2).
double fr_flops_trace(int n, bool viscous);
double fr_flops_face_point(bool viscous);   // per owned flux point
double fr_flops_elem(int n, bool viscous);
extern const double FR_JVP_FLOP_FACTOR;     // dual-number cost over the value cost

#define FR_ACCOUNT(c, k, flops, bytes) \
  do {                                 \
    (c)->alg_flops[(k)] += (flops);    \
    (c)->alg_bytes[(k)] += (bytes);    \
  } while (0)

// Timing of one launch when profiling is on: a pair of events around it on its stream.
cudaEvent_t fr_prof_begin(fr_ctx* c, cudaStream_t s);
void fr_prof_end(fr_ctx* c, cudaStream_t s, cudaEvent_t begin, int kind);

#define FR_PROF_BEGIN(c, s) cudaEvent_t fr_ev_ = (c)->prof.on ? fr_prof_begin((c), (s)) : nullptr
#define FR_PROF_END(c, s, k)                                           \
  do {                                                                  \
    (c)->launches_by_kind[(k)]++;                                       \
    if (fr_ev_) fr_prof_end((c), (s), fr_ev_, (k));                     \
  } while (0)

// 1-D FR basis (Sec. 3.1) and nondimensional gas (Sec. 2.1) of a configuration; host
// only, no allocation.
fr::Basis fr_make_basis(int p);
fr::Gas fr_make_gas(const fr_config& c);

// Issue `count` GMRES iterations starting at basis index `start` through issue(stream):
// directly while profiling or with cfg.graphs off, otherwise by replaying a CUDA graph
// captured on first use (keyed by start, count, tag and q).  Every launch inside a chunk
// must take fixed arguments for a given key.
int gm_chunk(fr_ctx* c, int start, int count, int tag, const void* q,
             const std::function<int(cudaStream_t)>& issue, cudaStream_t s);
void graphs_free(fr_ctx* c);

// Topology, case table and workspace of ncases doubly periodic boxes of nxs[k] x nys[k]
// elements, numbered case after case; params supplies each case's gas and terms (its
// layout fields are filled here).  Synchronous.
int fr_setup_cases(fr_ctx* c, int ncases, const int* nxs, const int* nys,
                   const fr::CaseParams* params);

namespace frk {
int set_case_params(fr_ctx* c, int cid, const fr::CaseParams& p, cudaStream_t s);
int set_time_terms(fr_ctx* c, double a0dt, double a1dt, double a2dt, cudaStream_t s);
int set_operator_terms(fr_ctx* c, double inv_dtau, double a0_dt, cudaStream_t s);
int fill_topology(fr_ctx* c, int nx, int ny, int e0, int cid, cudaStream_t s);
// boundary faces below row 0 and above row ny-1 of the single case (neighbour -kind)
int mark_bounds(fr_ctx* c, int nx, int ny, int below, int above, cudaStream_t s);
// force on the wall faces of a bounded mesh into force_h[2] (host; synchronises s)
int wall_force(fr_ctx* c, const double* q, double* force_h, cudaStream_t s);
int geometry(fr_ctx* c, const double* corners, const double* vel, cudaStream_t s);
int residual(fr_ctx* c, const double* q, double* out, const double* qcn, const double* qcnm1,
             double a0dt, double a1dt, double a2dt, cudaStream_t s);
int jvp(fr_ctx* c, const double* q, const double* v, double inv_dtau, double a0_dt, double* out,
        cudaStream_t s);
int conservative(fr_ctx* c, const double* q, double* qc, cudaStream_t s);
int block_build(fr_ctx* c, const double* q, double inv_dtau, double a0_dt, cudaStream_t s);
int block_apply(fr_ctx* c, const double* r, double* z, cudaStream_t s);
// z = z0 + B^-1 (r - t) in one pass (the smoothing step of the two-level preconditioner)
int block_apply_fused(fr_ctx* c, const double* r, const double* t, const double* z0, double* z,
                      cudaStream_t s);
// z = P y0 + B^-1 (r - (A P) y0) in one pass (co = 1: FP32 coarse arrays, 2: FP64)
int block_apply_coarse(fr_ctx* c, const double* r, double* z, const CoarseIn& ci, int co,
                       cudaStream_t s);
// Two-level preconditioner (fr_mg.cu): topology and workspace of the coarse hierarchy
// (host-built, synchronous; nothing unless cfg.precond asks for it), its build at q after
// the element blocks, and the configured preconditioner z = M^-1 r (block Jacobi, or the
// coarse correction followed by block-Jacobi smoothing with the current operator at q).
int mg_setup(fr_ctx* c);
void mg_free(fr_ctx* c);
int mg_build(fr_ctx* c, const double* q, double inv_dtau, double a0_dt, cudaStream_t s);
// the transposed hierarchy of the last build (for M^-T in the adjoint solve)
int mg_transpose(fr_ctx* c, cudaStream_t s);
int precond_apply(fr_ctx* c, const double* q, const double* r, double* z, double inv_dtau,
                  double a0_dt, cudaStream_t s);
int linearize(fr_ctx* c, const double* q, double inv_dtau, double a0_dt, cudaStream_t s);
int apply_linear(fr_ctx* c, const double* v, double* out, bool transpose, cudaStream_t s);
// out = transposed traces and local gradients of the trace adjoints in tq_d / tg_d plus
// the point adjoints adj_q and gradient adjoints gl_d (the last pass of the VJP)
int trace_adjoint(fr_ctx* c, double* out, cudaStream_t s);
// Adjoint building blocks (fr_adjoint.cu): out = beta out + alpha d(wx F_x + wy F_y)/dq
// (uses w_t), out = beta out + alpha (dq^c/dq)^T w, and sum of w . dq^c/dM at fixed q.
int wall_force_vjp(fr_ctx* c, const double* q, double wx, double wy, double alpha, double beta,
                   double* out, cudaStream_t s);
int conservative_vjp(fr_ctx* c, const double* q, const double* w, double alpha, double beta,
                     double* out, cudaStream_t s);
int conservative_dmach(fr_ctx* c, const double* q, const double* w, double* out_h, cudaStream_t s);
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
// Batched (per-case) forms; scalars of case k at bw.dsc + k * 128.
int batch_setup(fr_ctx* c);
int fused_reset(fr_ctx* c, cudaStream_t s);   // fused Arnoldi barriers back to rest
void batch_free(fr_ctx* c);
int bk_norms(fr_ctx* c, const double* r, cudaStream_t s);         // -> [k][96..97]
int bk_init(fr_ctx* c, const double* r, double* next, cudaStream_t s);
int bk_orthogonalize(fr_ctx* c, double* w, double* next, int nv_bound, cudaStream_t s);
int bk_finish(fr_ctx* c, double* u, cudaStream_t s);              // trisolve + combination
int bk_status(fr_ctx* c, cudaStream_t s);                         // -> bw.status_h (async)
int bk_axpy_case(fr_ctx* c, const double* coef_dev, const double* x, double* y, cudaStream_t s);
int upload_cases(fr_ctx* c, cudaStream_t s);                      // c->cps -> device
// FR_ERR_TIMEOUT (and the flag cleared) if a device wait ran out of its budget since the
// last check (synchronises s).
int check_device_waits(fr_ctx* c, cudaStream_t s);
// Tile shapes: forced by cfg.tiles (1 or 2) or timed on the context's own buffers
// (cfg.tiles = 0).  Synchronous; called once at mesh set-up.
int autotune_tiles(fr_ctx* c);
// Per-case continuity-row and full norms of r (synchronises; bad[k] set for non-finite).
int case_norms(fr_ctx* c, const double* r, std::vector<double>& mass, std::vector<double>& all,
               std::vector<char>& bad, cudaStream_t s);
// Restarted GMRES(m <= 128) of every active case with device-resident Arnoldi (fr_batch.cu);
// inv_dtau, a0_dt feed the dual-number operator of a single-case context (a batch reads
// its terms from the case table).
int gmres_cases(fr_ctx* c, const double* q, const double* b, double* x, double inv_dtau,
                double a0_dt, const std::vector<char>& active, std::vector<int>& iters,
                std::vector<char>& failed, cudaStream_t s);
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

#define FR_TRY(expr)                 \
  do {                               \
    int rc_ = (expr);                \
    if (rc_ != FR_OK) return rc_;    \
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
