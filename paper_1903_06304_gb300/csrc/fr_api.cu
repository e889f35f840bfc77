// fr_api.cu -- C ABI of the GB300 preconditioned FR/CPR implicit hot path: context and
// workspace, the 1-D FR basis (Sec. 3.1), restarted right-preconditioned GMRES with CGS2
// and the pseudo-time Newton loops of Sec. 3.2 (BDF2 dual time, steady PTC with SER).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include "fr_internal.h"

namespace {

// ------------------------------------------------------------------ 1-D basis (Sec. 3.1)
// Legendre P_k(x) and P_k'(x) by the three-term recurrence.
void legendre(int k, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (k == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int m = 1; m < k; ++m) {
    const double p2 = ((2 * m + 1) * x * p1 - m * p0) / (m + 1);
    const double d2 = d0 + (2 * m + 1) * p1;  // P'_{m+1} = P'_{m-1} + (2m+1) P_m
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *P = p1;
  *dP = d1;
}

// Gauss-Legendre points: roots of P_n by Newton iteration from Chebyshev-like guesses.
void gauss_points(int n, double* xs) {
  for (int k = 0; k < n; ++k) {
    double x = -std::cos(M_PI * (k + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(n, x, &P, &dP);
      const double dx = P / dP;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    xs[k] = x;
  }
}

}  // namespace

fr::Basis fr_make_basis(int p) {
  fr::Basis B;
  std::memset(&B, 0, sizeof(B));
  const int n = p + 1;
  double xs[fr::MAXN];
  gauss_points(n, xs);
  for (int i = 0; i < n; ++i) B.xs[i] = xs[i];
  // Gauss weights w_i = 2 / ((1 - x_i^2) P_n'(x_i)^2)
  for (int i = 0; i < n; ++i) {
    double P, dP;
    legendre(n, xs[i], &P, &dP);
    B.ws[i] = 2.0 / ((1.0 - xs[i] * xs[i]) * dP * dP);
  }
  // barycentric weights
  double bw[fr::MAXN];
  for (int k = 0; k < n; ++k) {
    double prod = 1.0;
    for (int m = 0; m < n; ++m) if (m != k) prod *= (xs[k] - xs[m]);
    bw[k] = 1.0 / prod;
  }
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int k = 0; k < n; ++k) {
      if (k == i) continue;
      B.D[i][k] = (bw[k] / bw[i]) / (xs[i] - xs[k]);
      diag -= B.D[i][k];
    }
    B.D[i][i] = diag;
  }
  for (int k = 0; k < n; ++k) {
    double a = 1.0, b = 1.0;
    for (int m = 0; m < n; ++m) {
      if (m == k) continue;
      a *= (-1.0 - xs[m]) / (xs[k] - xs[m]);
      b *= (1.0 - xs[m]) / (xs[k] - xs[m]);
    }
    B.lL[k] = a;
    B.lR[k] = b;
  }
  // g_R = (P_{p+1} + P_p)/2, g_L(x) = g_R(-x):  g_R'(x) = (P'_{p+1} + P'_p)/2,
  // g_L'(x) = -g_R'(-x).
  auto dgr = [p](double x) {
    double P1, dP1, P0, dP0;
    legendre(p + 1, x, &P1, &dP1);
    legendre(p, x, &P0, &dP0);
    return 0.5 * (dP1 + dP0);
  };
  for (int i = 0; i < n; ++i) {
    B.dgR[i] = dgr(xs[i]);
    B.dgL[i] = -dgr(-xs[i]);
  }
  // BR2 face lifting: eta g_R'(1) with the penalty eta = BR2_PENALTY
  B.lift_end = fr::BR2_PENALTY * 0.5 * (p + 1) * (p + 1);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) B.Dc[i][k] = B.D[i][k] - B.dgL[i] * B.lL[k] - B.dgR[i] * B.lR[k];
  return B;
}

fr::Gas fr_make_gas(const fr_config& c) {
  fr::Gas g;
  const double M2 = c.mach * c.mach;
  g.gamma = c.gamma;
  g.R = 1.0 / (c.gamma * M2);
  g.inv_R = c.gamma * M2;
  g.cp = 1.0 / ((c.gamma - 1.0) * M2);
  g.inv_cp = (c.gamma - 1.0) * M2;
  g.inv_gm1 = 1.0 / (c.gamma - 1.0);
  g.mu = 1.0;
  g.viscous = c.re > 0.0;
  g.inv_re = g.viscous ? 1.0 / c.re : 0.0;
  g.k_cond = g.mu * g.cp / c.prandtl;
  g.kappa_minf = c.kappa * c.mach;
  g.eps_floor = c.eps_floor;
  return g;
}

void graphs_free(fr_ctx* c) {
  for (GraphEntry& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

int gm_chunk(fr_ctx* c, int start, int count, int tag, const void* q,
             const std::function<int(cudaStream_t)>& issue, cudaStream_t s) {
  if (!c->cfg.graphs || c->prof.on) return issue(s);
  for (GraphEntry& g : c->graphs) {
    if (g.start == start && g.count == count && g.tag == tag && g.q == q) {
      FR_CUDA_CHECK(c, cudaGraphLaunch(g.exec, s));
      c->launches += g.launches;
      for (int k = 0; k < KK_COUNT; ++k) {
        c->launches_by_kind[k] += g.by_kind[k];
        c->alg_flops[k] += g.flops[k];
        c->alg_bytes[k] += g.bytes[k];
      }
      return FR_OK;
    }
  }
  // capture on a private stream (capture executes nothing), replay on s; the counters
  // advanced during capture stand for this first replay
  if (!c->cap_stream) FR_CUDA_CHECK(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  GraphEntry e;
  std::memset(&e, 0, sizeof(e));
  e.start = start; e.count = count; e.tag = tag; e.q = q;
  const long long l0 = c->launches;
  long long k0[KK_COUNT];
  double f0[KK_COUNT], b0[KK_COUNT];
  for (int k = 0; k < KK_COUNT; ++k) { k0[k] = c->launches_by_kind[k]; f0[k] = c->alg_flops[k]; b0[k] = c->alg_bytes[k]; }
  FR_CUDA_CHECK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  const int rc = issue(c->cap_stream);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &graph);
  if (rc != FR_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
  if (ce != cudaSuccess || !graph) {
    snprintf(c->err, sizeof(c->err), "graph capture: %s", cudaGetErrorString(ce));
    return FR_ERR_CUDA;
  }
  const cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    snprintf(c->err, sizeof(c->err), "graph instantiate: %s", cudaGetErrorString(ie));
    return FR_ERR_CUDA;
  }
  e.launches = c->launches - l0;
  for (int k = 0; k < KK_COUNT; ++k) {
    e.by_kind[k] = c->launches_by_kind[k] - k0[k];
    e.flops[k] = c->alg_flops[k] - f0[k];
    e.bytes[k] = c->alg_bytes[k] - b0[k];
  }
  c->graphs.push_back(e);
  FR_CUDA_CHECK(c, cudaGraphLaunch(e.exec, s));
  return FR_OK;
}

namespace {

template <class T> int dev_alloc(fr_ctx* c, T** p, size_t count) {
  if (*p) { cudaFree(*p); *p = nullptr; }
  if (count == 0) return FR_OK;
  FR_CUDA_CHECK(c, cudaMalloc((void**)p, count * sizeof(T)));
  return FR_OK;
}

void free_mesh(fr_ctx* c) {
  double** ds[] = {&c->gs, &c->gf, &c->tq, &c->tg, &c->gl, &c->fn, &c->qcm, &c->tq_d, &c->tg_d,
                   &c->gl_d, &c->fn_d, &c->qcm_d, &c->B64, &c->V, &c->w_r, &c->w_z, &c->w_x,
                   &c->w_t, &c->w_u, &c->red, &c->JFQ, &c->JFG, &c->JP, &c->JG, &c->PP,
                   &c->adj_q, &c->adj_fn, &c->adj_qc, &c->sgs, &c->sdgs, &c->sgf, &c->sdgf,
                   &c->seed, &c->edot, &c->zero, &c->rtan, &c->fnb, &c->fnb_d, &c->qcb,
                   &c->qcb_d, &c->JFQb, &c->JFGb};
  for (double** p : ds) if (*p) { cudaFree(*p); *p = nullptr; }
  if (c->Binv) { cudaFree(c->Binv); c->Binv = nullptr; }
  if (c->Dr) { cudaFree(c->Dr); c->Dr = nullptr; }
  if (c->Dc) { cudaFree(c->Dc); c->Dc = nullptr; }
  if (c->info) { cudaFree(c->info); c->info = nullptr; }
  if (c->ticket) { cudaFree(c->ticket); c->ticket = nullptr; }
  if (c->dev_err) { cudaFree(c->dev_err); c->dev_err = nullptr; }
  if (c->nbr) { cudaFree(c->nbr); c->nbr = nullptr; }
  if (c->ecase) { cudaFree(c->ecase); c->ecase = nullptr; }
  c->blocks_ready = 0;
  c->lin_ready = 0;
  c->bounded = c->bc_below = c->bc_above = 0;
  frk::batch_free(c);
  frk::mg_free(c);
  graphs_free(c);
}

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }


int check_ready(fr_ctx* c) {
  if (!c) return FR_ERR_ARG;
  if (c->ne <= 0) { snprintf(c->err, sizeof(c->err), "fr_set_mesh has not been called"); return FR_ERR_ARG; }
  return FR_OK;
}

// host copies of the small device scalars
int fetch(fr_ctx* c, int off, int count, cudaStream_t s) {
  FR_CUDA_CHECK(c, cudaMemcpyAsync(c->hsc + off, c->dsc + off, count * sizeof(double),
                                   cudaMemcpyDeviceToHost, s));
  FR_CUDA_CHECK(c, cudaStreamSynchronize(s));
  return FR_OK;
}

int norms_host(fr_ctx* c, const double* r, double* mass, double* all, cudaStream_t s) {
  constexpr int off = 4 * FR_MAX_RESTART;
  FR_TRY(frk::norms(c, r, c->dsc + off, s));
  FR_TRY(fetch(c, off, 2, s));
  *mass = std::sqrt(c->hsc[off]);
  *all = std::sqrt(c->hsc[off + 1]);
  if (!std::isfinite(*all)) { snprintf(c->err, sizeof(c->err), "non-finite residual norm"); return FR_ERR_NONFINITE; }
  return FR_OK;
}

// Classical Gram-Schmidt with one re-orthogonalisation against V[0..nv): projections of
// the first pass at dsc[0..nv), of the second at dsc[M..M+nv), ||w||^2 at dsc[2M]
// (M = FR_MAX_RESTART).  Vectors are processed in chunks of 32 per launch.
int cgs2(fr_ctx* c, int nv, double* w, cudaStream_t s) {
  constexpr int CH = 32, M = FR_MAX_RESTART;
  const size_t N = c->ndof;
  if (c->cfg.orthog == FR_ORTHO_CGS) {
    // one classical pass: projections at dsc[0..nv), the second set zero
    FR_CUDA_CHECK(c, cudaMemsetAsync(c->dsc + M, 0, nv * sizeof(double), s));
    for (int k0 = 0; k0 < nv; k0 += CH)
      FR_TRY(frk::dots(c, c->V + (size_t)k0 * N, std::min(CH, nv - k0), w, c->dsc + k0, s));
    for (int k0 = 0; k0 + CH < nv; k0 += CH)
      FR_TRY(frk::axpy(c, c->V + (size_t)k0 * N, CH, c->dsc + k0, w, s));
    const int last = ((nv - 1) / CH) * CH;
    return frk::axpy_norm(c, c->V + (size_t)last * N, nv - last, c->dsc + last, w, c->dsc + 2 * M, s);
  }
  if (nv <= CH) {
    FR_TRY(frk::dots(c, c->V, nv, w, c->dsc, s));
    FR_TRY(frk::axpy_dots(c, c->V, nv, c->dsc, w, c->dsc + M, s));
    return frk::axpy_norm(c, c->V, nv, c->dsc + M, w, c->dsc + 2 * M, s);
  }
  for (int k0 = 0; k0 < nv; k0 += CH)
    FR_TRY(frk::dots(c, c->V + (size_t)k0 * N, std::min(CH, nv - k0), w, c->dsc + k0, s));
  for (int k0 = 0; k0 < nv; k0 += CH)
    FR_TRY(frk::axpy(c, c->V + (size_t)k0 * N, std::min(CH, nv - k0), c->dsc + k0, w, s));
  for (int k0 = 0; k0 < nv; k0 += CH)
    FR_TRY(frk::dots(c, c->V + (size_t)k0 * N, std::min(CH, nv - k0), w, c->dsc + M + k0, s));
  for (int k0 = 0; k0 + CH < nv; k0 += CH)
    FR_TRY(frk::axpy(c, c->V + (size_t)k0 * N, CH, c->dsc + M + k0, w, s));
  const int last = ((nv - 1) / CH) * CH;
  return frk::axpy_norm(c, c->V + (size_t)last * N, nv - last, c->dsc + M + last, w, c->dsc + 2 * M, s);
}

// Restarted preconditioned GMRES(m), CGS2 Arnoldi, Givens rotations on the host.
// Left preconditioning (PETSc's default): Krylov space of B^-1 A, minimises
// ||B^-1 (b - A x)||, tolerance relative to ||B^-1 b||.  Right: Krylov space of A B^-1,
// x = B^-1 V y, minimises ||b - A x||, tolerance relative to ||b||.
// Layout of the device scalar area dsc (M = FR_MAX_RESTART): [0,M) first projections,
// [M,2M) second projections, [2M] squared norm, [3M,4M) Krylov coefficients y,
// [4M, 4M+2) norms.
// The Newton operator applied inside GMRES: the stored linearisation (default) or the
// dual-number JVP at q.
int op_apply(fr_ctx* c, const double* q, const double* x, double inv_dtau, double a0_dt,
             double* out, cudaStream_t s) {
  if (c->transposed) return frk::apply_linear(c, x, out, true, s);
  if (c->cfg.jvp_mode == FR_JVP_LINEARIZED) return frk::apply_linear(c, x, out, false, s);
  return frk::jvp(c, q, x, inv_dtau, a0_dt, out, s);
}

static int gmres_solve_impl(fr_ctx* c, const double* q, const double* b, double inv_dtau,
                            double a0_dt, double* x, int* iters, cudaStream_t s);

// GMRES (below), then the report of any device wait that ran out during it
int gmres_solve(fr_ctx* c, const double* q, const double* b, double inv_dtau, double a0_dt,
                double* x, int* iters, cudaStream_t s) {
  const int rc = gmres_solve_impl(c, q, b, inv_dtau, a0_dt, x, iters, s);
  const int wc = frk::check_device_waits(c, s);
  return wc != FR_OK ? wc : rc;
}

static int gmres_solve_impl(fr_ctx* c, const double* q, const double* b, double inv_dtau,
                            double a0_dt, double* x, int* iters, cudaStream_t s) {
  const size_t N = c->ndof;
  const int m = c->cfg.restart;
  const double tol = c->cfg.tol_res;
  const int maxit = c->cfg.maxit_lin;
  const bool left = c->cfg.gmres_side == FR_GMRES_LEFT;
  double* r = c->w_r;
  // the operator's terms go to the case table here, outside any captured chunk
  FR_TRY(frk::set_operator_terms(c, inv_dtau, a0_dt, s));
  if (m <= GmresState::LD) {
    // Device-resident Arnoldi (the per-case path with one case): iterations are queued in
    // chunks, one synchronisation per chunk reads the iteration count and stopping flag.
    std::vector<char> active(1, 1), failed(1, 0);
    std::vector<int> its;
    FR_TRY(frk::gmres_cases(c, q, b, x, inv_dtau, a0_dt, active, its, failed, s));
    if (failed[0]) { snprintf(c->err, sizeof(c->err), "GMRES: non-finite Krylov vector"); return FR_ERR_NONFINITE; }
    *iters = its[0];
    return FR_OK;
  }
  if (left) FR_TRY(frk::precond_apply(c, q, b, r, inv_dtau, a0_dt, s));
  else FR_CUDA_CHECK(c, cudaMemcpyAsync(r, b, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  double bm, bnorm;
  FR_TRY(norms_host(c, r, &bm, &bnorm, s));
  FR_CUDA_CHECK(c, cudaMemsetAsync(x, 0, N * sizeof(double), s));
  *iters = 0;
  if (bnorm == 0.0) return FR_OK;
  double beta = bnorm;
  int total = 0;
  std::vector<double> H((m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  while (true) {
    if (beta <= tol * bnorm) break;
    if (total >= maxit) break;
    FR_TRY(frk::scale(c, r, 1.0 / beta, c->V, s));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      double* Vj = c->V + (size_t)j * N;
      double* w = c->V + (size_t)(j + 1) * N;
      if (left) {
        FR_TRY(op_apply(c, q, Vj, inv_dtau, a0_dt, c->w_z, s));
        FR_TRY(frk::precond_apply(c, q, c->w_z, w, inv_dtau, a0_dt, s));
      } else {
        FR_TRY(frk::precond_apply(c, q, Vj, c->w_z, inv_dtau, a0_dt, s));
        FR_TRY(op_apply(c, q, c->w_z, inv_dtau, a0_dt, w, s));
      }
      FR_TRY(cgs2(c, j + 1, w, s));
      FR_CUDA_CHECK(c, cudaMemcpyAsync(c->hsc, c->dsc, (2 * FR_MAX_RESTART + 1) * sizeof(double),
                                       cudaMemcpyDeviceToHost, s));
      FR_CUDA_CHECK(c, cudaStreamSynchronize(s));
      for (int i = 0; i <= j; ++i) H[i * m + j] = c->hsc[i] + c->hsc[FR_MAX_RESTART + i];
      const double hn = std::sqrt(c->hsc[2 * FR_MAX_RESTART]);
      if (!std::isfinite(hn)) { snprintf(c->err, sizeof(c->err), "GMRES: non-finite Krylov vector"); return FR_ERR_NONFINITE; }
      H[(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
        H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
        H[i * m + j] = t;
      }
      const double den = std::hypot(H[j * m + j], H[(j + 1) * m + j]);
      cs[j] = H[j * m + j] / den;
      sn[j] = H[(j + 1) * m + j] / den;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++total;
      k = j + 1;
      if (hn > 0.0) FR_TRY(frk::scale(c, w, 1.0 / hn, w, s));
      if (std::fabs(g[j + 1]) <= tol * bnorm || total >= maxit || hn == 0.0) break;
    }
    for (int i = k - 1; i >= 0; --i) {
      double acc = g[i];
      for (int l = i + 1; l < k; ++l) acc -= H[i * m + l] * y[l];
      y[i] = acc / H[i * m + i];
    }
    std::memcpy(c->hsc + 3 * FR_MAX_RESTART, y.data(), k * sizeof(double));
    FR_CUDA_CHECK(c, cudaMemcpyAsync(c->dsc + 3 * FR_MAX_RESTART, c->hsc + 3 * FR_MAX_RESTART,
                                     k * sizeof(double), cudaMemcpyHostToDevice, s));
    FR_TRY(frk::lincomb(c, c->V, k, c->dsc + 3 * FR_MAX_RESTART, c->w_u, s));
    if (left) {
      FR_TRY(frk::axpby(c, 1.0, c->w_u, 1.0, x, s));
    } else {
      FR_TRY(frk::precond_apply(c, q, c->w_u, c->w_z, inv_dtau, a0_dt, s));
      FR_TRY(frk::axpby(c, 1.0, c->w_z, 1.0, x, s));
    }
    // residual of the restart: b - A x (left: preconditioned)
    FR_TRY(op_apply(c, q, x, inv_dtau, a0_dt, c->w_t, s));
    FR_TRY(frk::axpby(c, 1.0, b, -1.0, c->w_t, s));
    if (left) FR_TRY(frk::precond_apply(c, q, c->w_t, r, inv_dtau, a0_dt, s));
    else FR_CUDA_CHECK(c, cudaMemcpyAsync(r, c->w_t, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    double rm;
    FR_TRY(norms_host(c, r, &rm, &beta, s));
  }
  *iters = total;
  return FR_OK;
}

int newton_loop(fr_ctx* c, double* q, const double* qcn, const double* qcnm1, double a0,
                double a1, double a2, double dt, bool steady, fr_stats* st, cudaStream_t s) {
  fr_stats local;
  if (!st) st = &local;
  std::memset(st, 0, sizeof(*st));
  const int maxit = std::min(c->cfg.maxit_newton, FR_MAX_NEWTON);
  const double a0dt = steady ? 0.0 : a0 / dt;
  auto rhs = [&](double* out) -> int {
    if (steady) return frk::residual(c, q, out, nullptr, nullptr, 0, 0, 0, s);
    return frk::residual(c, q, out, qcn, a2 != 0.0 ? qcnm1 : nullptr, a0 / dt, a1 / dt, a2 / dt, s);
  };
  // pseudo-step residual in the spare vector after the Krylov basis (GMRES writes V[0..m],
  // w_r, w_z, w_t, w_u, and its solution into w_x)
  double* r = c->V + (size_t)(c->cfg.restart + 1) * c->ndof;
  FR_TRY(rhs(r));
  double rm, ra;
  FR_TRY(norms_host(c, r, &rm, &ra, s));
  const double res0 = rm;
  st->res_history[0] = rm;
  const bool ser = steady || c->cfg.ser_unsteady;
  double dtau = steady ? c->cfg.dtau0 : (c->cfg.ser_unsteady ? c->cfg.dtau0_unsteady : c->cfg.dtau_unsteady);
  st->dtau_history[0] = dtau;
  int m = 0;
  bool conv = false;
  for (m = 0; m < maxit; ++m) {
    if (rm <= c->cfg.tol_pseudo * res0) { conv = true; break; }
    const double inv_dtau = 1.0 / dtau;
    bool lin_done = false;   // a build from the local Jacobians leaves them stored at q
    bool build = false;
    if (ser || m % std::max(1, c->cfg.lag) == 0) {
      FR_TRY(frk::block_build(c, q, inv_dtau, a0dt, s));
      c->blocks_ready = 1;
      st->block_builds++;
      lin_done = c->cfg.block_mode == FR_BLOCK_LINEARIZED;
      build = true;
    }
    int its = 0;
    if (c->cfg.jvp_mode == FR_JVP_LINEARIZED && !lin_done) FR_TRY(frk::linearize(c, q, inv_dtau, a0dt, s));
    // the coarse operators are products of the operator GMRES applies at this q
    if (build) FR_TRY(frk::mg_build(c, q, inv_dtau, a0dt, s));
    FR_TRY(gmres_solve(c, q, r, inv_dtau, a0dt, c->w_x, &its, s));
    st->gmres_iterations[m] = its;
    const double prev = rm, prev_all = ra;
    FR_TRY(frk::axpby(c, 1.0, c->w_x, 1.0, q, s));
    FR_TRY(rhs(r));
    FR_TRY(norms_host(c, r, &rm, &ra, s));
    // backtracking: q = q_m + lambda dq while the full residual norm does not decrease
    double lambda = 1.0;
    for (int h = 0; h < c->cfg.line_search && !(ra < prev_all); ++h) {
      FR_TRY(frk::axpby(c, -0.5 * lambda, c->w_x, 1.0, q, s));
      lambda *= 0.5;
      FR_TRY(rhs(r));
      FR_TRY(norms_host(c, r, &rm, &ra, s));
      st->line_search_halvings++;
    }
    st->res_history[m + 1] = rm;
    if (ser) {
      dtau = std::max(c->cfg.dtau_min, std::min(c->cfg.dtau_max, dtau * std::pow(prev / rm, c->cfg.r_ser)));
    }
    st->dtau_history[m + 1] = dtau;
  }
  if (!conv && rm <= c->cfg.tol_pseudo * res0) conv = true;
  st->newton_iterations = m;
  st->converged = conv ? 1 : 0;
  return conv ? FR_OK : FR_ERR_NOT_CONVERGED;
}

const char* kKernelNames[KK_COUNT] = {
    "geometry", "trace", "face", "elem", "trace_jvp", "face_jvp", "elem_jvp", "block_jacobian",
    "block_factor", "block_apply", "krylov_reduce", "vector", "conservative", "linearize",
    "linear_apply", "linear_adjoint", "coarse"};

// Fold the recorded event pairs into the per-kind totals (synchronises on the events).
int prof_collect(fr_ctx* c) {
  for (const FrProfPair& p : c->prof.pairs) {
    FR_CUDA_CHECK(c, cudaEventSynchronize(p.b));
    float ms = 0.f;
    FR_CUDA_CHECK(c, cudaEventElapsedTime(&ms, p.a, p.b));
    c->prof.ms[p.kind] += ms;
    c->prof.n[p.kind] += 1;
  }
  c->prof.pairs.clear();
  c->prof.used = 0;
  return FR_OK;
}

}  // namespace

cudaEvent_t fr_prof_begin(fr_ctx* c, cudaStream_t s) {
  if (c->prof.used + 2 > c->prof.pool.size()) {
    if (c->prof.pool.size() >= (1u << 20)) prof_collect(c);  // bound the pool
    for (int k = 0; k < 256; ++k) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      c->prof.pool.push_back(e);
    }
  }
  cudaEvent_t e = c->prof.pool[c->prof.used++];
  cudaEventRecord(e, s);
  return e;
}

void fr_prof_end(fr_ctx* c, cudaStream_t s, cudaEvent_t begin, int kind) {
  if (c->prof.used + 1 > c->prof.pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    c->prof.pool.push_back(e);
  }
  cudaEvent_t e = c->prof.pool[c->prof.used++];
  cudaEventRecord(e, s);
  c->prof.pairs.push_back({begin, e, kind});
}

extern "C" {

int fr_profile(fr_ctx* c, int enable) {
  if (!c) return FR_ERR_ARG;
  FR_TRY(prof_collect(c));
  c->prof.on = enable != 0;
  return FR_OK;
}

int fr_profile_read(fr_ctx* c, double* ms, long long* counts, long long* launches, double* flops,
                    double* bytes, int reset) {
  if (!c) return FR_ERR_ARG;
  FR_TRY(prof_collect(c));
  for (int k = 0; k < KK_COUNT; ++k) {
    if (ms) ms[k] = c->prof.ms[k];
    if (counts) counts[k] = c->prof.n[k];
    if (launches) launches[k] = c->launches_by_kind[k];
    if (flops) flops[k] = c->alg_flops[k];
    if (bytes) bytes[k] = c->alg_bytes[k];
    if (reset) { c->prof.ms[k] = 0.0; c->prof.n[k] = 0; c->alg_flops[k] = 0.0; c->alg_bytes[k] = 0.0; }
  }
  return FR_OK;
}

const char* fr_profile_name(int kind) {
  return (kind >= 0 && kind < KK_COUNT) ? kKernelNames[kind] : "";
}

const char* fr_version(void) { return "fr-gb300 0.1 (sm_103a)"; }

void fr_default_config(fr_config* c) {
  std::memset(c, 0, sizeof(*c));
  c->p = 3;
  c->gamma = 1.4;
  c->prandtl = 0.72;
  c->mach = 0.05;
  c->re = 0.0;
  c->kappa = 1.0;
  c->eps_floor = 1e-8;
  c->prec_dtype = FR_PREC_FP64;
  c->restart = 30;
  c->maxit_lin = 100;
  c->maxit_newton = 20;
  c->lag = 2;
  c->tol_res = 1e-6;
  c->tol_pseudo = 1e-8;
  c->dtau0 = 0.01;
  c->dtau_min = 0.01;
  c->dtau_max = 1e20;
  c->r_ser = 2.0;
  c->dtau_unsteady = 1e20;
  c->gmres_side = FR_GMRES_LEFT;
  c->ser_unsteady = 0;
  c->dtau0_unsteady = 0.01;
  c->line_search = 0;
  c->jvp_mode = FR_JVP_LINEARIZED;
  c->graphs = 1;
  c->apply_accum = FR_ACCUM_DF64;
  c->tiles = 1;
  c->block_mode = FR_BLOCK_LINEARIZED;
  c->orthog = FR_ORTHO_CGS2;
  c->krylov_arith = FR_KRYLOV_FP64;
  c->precond = FR_PRECOND_BLOCK;
  c->mg_sweeps = 2;
  c->mg_omega = 0.7;
  c->mg_prec = FR_PREC_FP32;
  c->factor_tc = FR_FACTOR_SIMT;
  c->apply_bulk = 0;
  c->wait_spins = 0;
  c->arnoldi_fused = 0;
}

int fr_create(const fr_config* cfg, fr_ctx** out) {
  if (!cfg || !out) return FR_ERR_ARG;
  *out = nullptr;
  if (cfg->p < 1 || cfg->p > 4 || cfg->mach <= 0 || cfg->gamma <= 1.0 || cfg->restart < 1 ||
      cfg->restart > FR_MAX_RESTART || cfg->prec_dtype < 0 || cfg->prec_dtype > 2 ||
      (cfg->gmres_side != FR_GMRES_LEFT && cfg->gmres_side != FR_GMRES_RIGHT) ||
      (cfg->jvp_mode != FR_JVP_DUAL && cfg->jvp_mode != FR_JVP_LINEARIZED) ||
      (cfg->apply_accum != FR_ACCUM_FP32 && cfg->apply_accum != FR_ACCUM_DF64) ||
      cfg->tiles < 0 || cfg->tiles > 2 ||
      (cfg->block_mode != FR_BLOCK_LINEARIZED && cfg->block_mode != FR_BLOCK_DUAL) ||
      (cfg->orthog != FR_ORTHO_CGS2 && cfg->orthog != FR_ORTHO_CGS) ||
      (cfg->krylov_arith != FR_KRYLOV_FP64 && cfg->krylov_arith != FR_KRYLOV_DF64) ||
      (cfg->precond != FR_PRECOND_BLOCK && cfg->precond != FR_PRECOND_TWO_LEVEL) ||
      cfg->mg_sweeps < 1 || cfg->mg_sweeps > 2 || !(cfg->mg_omega > 0.0 && cfg->mg_omega <= 1.5) ||
      (cfg->mg_prec != FR_PREC_FP64 && cfg->mg_prec != FR_PREC_FP32) ||
      cfg->factor_tc < FR_FACTOR_SIMT || cfg->factor_tc > FR_FACTOR_TC_BF16X3 ||
      cfg->apply_bulk < 0 || cfg->apply_bulk == 1 || cfg->apply_bulk > 4 ||
      (cfg->arnoldi_fused != 0 && cfg->arnoldi_fused != 1 && cfg->arnoldi_fused != 2 &&
       cfg->arnoldi_fused != 4))
    return FR_ERR_ARG;
  fr_ctx* c = new fr_ctx();
  c->cfg = *cfg;
  c->p = cfg->p;
  c->n = cfg->p + 1;
  c->np2 = c->n * c->n;
  c->bsz = 4 * c->np2;
  c->ne = 0;
  c->err[0] = 0;
  c->basis = fr_make_basis(cfg->p);
  c->gas = fr_make_gas(*cfg);
  c->cp_h.gas = c->gas;
  c->cp_h.a0dt = c->cp_h.a1dt = c->cp_h.a2dt = 0.0;
  c->cp_h.inv_dtau = c->cp_h.a0_dt = 0.0;
  c->cp_h.off = 0;
  c->cp_h.e0 = 0;
  c->cp_h.sn = 0;
  c->cp_h.active = 1;
  if (cudaMalloc((void**)&c->dsc, (4 * FR_MAX_RESTART + 8) * sizeof(double)) != cudaSuccess ||
      cudaMallocHost((void**)&c->hsc, (4 * FR_MAX_RESTART + 8) * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&c->cp, sizeof(fr::CaseParams)) != cudaSuccess) {
    delete c;
    return FR_ERR_CUDA;
  }
  *out = c;
  return FR_OK;
}

void fr_destroy(fr_ctx* c) {
  if (!c) return;
  prof_collect(c);
  for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
  free_mesh(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->dsc) cudaFree(c->dsc);
  if (c->hsc) cudaFreeHost(c->hsc);
  if (c->cp) cudaFree(c->cp);
  delete c;
}

int fr_set_mesh(fr_ctx* c, int nx, int ny, int px, int py) {
  if (!c) return FR_ERR_ARG;
  if (nx < 2 || ny < 2 || px != 1 || py != 1) {
    snprintf(c->err, sizeof(c->err), "fr_set_mesh: need nx, ny >= 2 and periodic_x = periodic_y = 1");
    return FR_ERR_ARG;
  }
  return fr_setup_cases(c, 1, &nx, &ny, &c->cp_h);
}

int fr_wall_force(fr_ctx* c, const double* q, double* force_h, void* s) {
  FR_TRY(check_ready(c));
  if (!q || !force_h) return FR_ERR_ARG;
  if (!c->bounded || (c->bc_below != FR_BC_WALL && c->bc_above != FR_BC_WALL)) {
    snprintf(c->err, sizeof(c->err), "fr_wall_force: the mesh has no wall faces");
    return FR_ERR_ARG;
  }
  return frk::wall_force(c, q, force_h, S(s));
}

int fr_set_mesh_bounded(fr_ctx* c, int nx, int ny, int bc_below, int bc_above, const double* q_inf_h) {
  if (!c) return FR_ERR_ARG;
  const bool kinds_ok = (bc_below == FR_BC_WALL || bc_below == FR_BC_FARFIELD) &&
                        (bc_above == FR_BC_WALL || bc_above == FR_BC_FARFIELD);
  const bool need_qinf = bc_below == FR_BC_FARFIELD || bc_above == FR_BC_FARFIELD;
  if (nx < 2 || ny < 1 || !kinds_ok || (need_qinf && !q_inf_h)) {
    snprintf(c->err, sizeof(c->err), "fr_set_mesh_bounded: need nx >= 2, ny >= 1, boundary kinds "
             "FR_BC_WALL / FR_BC_FARFIELD and q_inf for a far field");
    return FR_ERR_ARG;
  }
  if (need_qinf && !(q_inf_h[0] > 0.0 && q_inf_h[3] > 0.0)) {
    snprintf(c->err, sizeof(c->err), "fr_set_mesh_bounded: q_inf needs p > 0 and T > 0");
    return FR_ERR_ARG;
  }
  for (int k = 0; k < 4; ++k) c->cp_h.qinf[k] = need_qinf ? q_inf_h[k] : 0.0;
  FR_TRY(fr_setup_cases(c, 1, &nx, &ny, &c->cp_h));
  c->bounded = 1;
  c->bc_below = bc_below;
  c->bc_above = bc_above;
  const size_t nb = (size_t)nx * 4 * c->n;
  FR_TRY(dev_alloc(c, &c->fnb, nb));
  FR_TRY(dev_alloc(c, &c->fnb_d, nb));
  FR_TRY(dev_alloc(c, &c->qcb, nb));
  FR_TRY(dev_alloc(c, &c->qcb_d, nb));
  // local Jacobians of the boundary faces below row 0 (those above the last row are owned
  // faces of the stored face map)
  FR_TRY(dev_alloc(c, &c->JFQb, (size_t)nx * c->n * 16));
  FR_TRY(dev_alloc(c, &c->JFGb, (size_t)nx * c->n * 32));
  FR_TRY(frk::mark_bounds(c, nx, ny, bc_below, bc_above, 0));
  FR_CUDA_CHECK(c, cudaStreamSynchronize(0));
  // the coarse hierarchy again, now without the wrap in eta
  return frk::mg_setup(c);
}

}  // extern "C"

int fr_setup_cases(fr_ctx* c, int ncases, const int* nxs, const int* nys,
                   const fr::CaseParams* params) {
  free_mesh(c);
  long long ne_total = 0;
  for (int k = 0; k < ncases; ++k) ne_total += (long long)nxs[k] * nys[k];
  if (ncases < 1 || ne_total * c->np2 * 4 > (1LL << 31) - 1) {
    snprintf(c->err, sizeof(c->err), "setup: %d cases, %lld elements", ncases, ne_total);
    return FR_ERR_ARG;
  }
  c->nx = nxs[0]; c->ny = nys[0]; c->ne = (int)ne_total;
  c->ncases = ncases;
  c->cps.assign(params, params + ncases);
  FR_TRY(dev_alloc(c, &c->nbr, (size_t)4 * c->ne));
  FR_TRY(dev_alloc(c, &c->ecase, (size_t)c->ne));
  FR_TRY(dev_alloc(c, &c->cp, (size_t)ncases));
  c->mesh.nbr = c->nbr;
  c->mesh.ecase = c->ecase;
  c->mesh.cp = c->cp;
  c->mesh.ne = c->ne;
  c->mesh.viscous = c->gas.viscous;
  // cases in order: elements [e0, e0 + nx ny), states contiguous from off
  long long e0 = 0;
  for (int k = 0; k < ncases; ++k) {
    fr::CaseParams& p = c->cps[k];
    p.e0 = (int)e0;
    p.off = 4 * e0 * c->np2;
    p.sn = nxs[k] * nys[k] * c->np2;
    p.nx = nxs[k];
    p.ny = nys[k];
    FR_TRY(frk::fill_topology(c, nxs[k], nys[k], (int)e0, k, 0));
    e0 += (long long)nxs[k] * nys[k];
  }
  c->cp_h = c->cps[0];
  FR_CUDA_CHECK(c, cudaMemcpy(c->cp, c->cps.data(), ncases * sizeof(fr::CaseParams),
                              cudaMemcpyHostToDevice));
  FR_CUDA_CHECK(c, cudaStreamSynchronize(0));
  const size_t ne = c->ne, n = c->n, np2 = c->np2, bs = c->bsz;
  c->ndof = 4 * ne * np2;
  // reduction grid: at least 4 pairs of entries per thread (256 threads), one to four
  // blocks per SM, so that the per-block reduction stays small against the streaming
  c->red_blocks = (int)std::max<size_t>(152, std::min<size_t>(4 * 152, c->ndof / 2 / (256 * 4)));
  FR_TRY(dev_alloc(c, &c->gs, (size_t)fr::GS_COUNT * ne * np2));
  FR_TRY(dev_alloc(c, &c->gf, (size_t)fr::GF_COUNT * ne * 4 * n));
  FR_TRY(dev_alloc(c, &c->tq, ne * 16 * n));
  FR_TRY(dev_alloc(c, &c->tq_d, ne * 16 * n));
  FR_TRY(dev_alloc(c, &c->tg, ne * 32 * n));
  FR_TRY(dev_alloc(c, &c->tg_d, ne * 32 * n));
  FR_TRY(dev_alloc(c, &c->gl, 8 * ne * np2));
  FR_TRY(dev_alloc(c, &c->gl_d, 8 * ne * np2));
  FR_TRY(dev_alloc(c, &c->fn, ne * 8 * n));
  FR_TRY(dev_alloc(c, &c->fn_d, ne * 8 * n));
  FR_TRY(dev_alloc(c, &c->qcm, ne * 8 * n));
  FR_TRY(dev_alloc(c, &c->qcm_d, ne * 8 * n));
  FR_TRY(dev_alloc(c, &c->B64, ne * bs * bs));
  const size_t esz = c->cfg.prec_dtype == FR_PREC_FP64 ? 8 : c->cfg.prec_dtype == FR_PREC_FP32 ? 4 : 2;
  FR_CUDA_CHECK(c, cudaMalloc(&c->Binv, ne * bs * bs * esz));
  FR_TRY(dev_alloc(c, &c->Dr, ne * bs));
  FR_TRY(dev_alloc(c, &c->Dc, ne * bs));
  FR_TRY(dev_alloc(c, &c->info, ne));
  // Krylov basis V[0..m] plus one extra vector holding the pseudo-step residual
  FR_TRY(dev_alloc(c, &c->V, (size_t)(c->cfg.restart + 2) * c->ndof));
  FR_TRY(dev_alloc(c, &c->w_r, c->ndof));
  FR_TRY(dev_alloc(c, &c->w_z, c->ndof));
  FR_TRY(dev_alloc(c, &c->w_x, c->ndof));
  FR_TRY(dev_alloc(c, &c->w_t, c->ndof));
  FR_TRY(dev_alloc(c, &c->w_u, c->ndof));
  FR_TRY(dev_alloc(c, &c->red, (size_t)32 * c->red_blocks));
  const size_t nfp = ne * 2 * n;
  FR_TRY(dev_alloc(c, &c->JFQ, 32 * nfp));
  FR_TRY(dev_alloc(c, &c->JFG, 64 * nfp));
  FR_TRY(dev_alloc(c, &c->JP, 32 * ne * np2));
  FR_TRY(dev_alloc(c, &c->JG, 64 * ne * np2));
  FR_TRY(dev_alloc(c, &c->PP, 16 * ne * np2));
  FR_TRY(dev_alloc(c, &c->adj_q, c->ndof));
  FR_TRY(dev_alloc(c, &c->adj_fn, ne * 16 * n));
  FR_TRY(dev_alloc(c, &c->adj_qc, ne * 16 * n));
  FR_TRY(dev_alloc(c, &c->ticket, 1));
  FR_CUDA_CHECK(c, cudaMemset(c->ticket, 0, sizeof(unsigned int)));
  FR_TRY(dev_alloc(c, &c->dev_err, 1));
  FR_CUDA_CHECK(c, cudaMemset(c->dev_err, 0, sizeof(int)));
  // per-case vector partition, GMRES states and staging (used by every context)
  FR_TRY(frk::batch_setup(c));
  // coarse hierarchy of the two-level preconditioner (nothing unless configured)
  FR_TRY(frk::mg_setup(c));
  // tile shapes of the point-parallel kernels (timed on these buffers unless forced)
  return frk::autotune_tiles(c);
}

extern "C" {

int fr_update_mesh(fr_ctx* c, const double* corners, const double* vel, void* s) {
  FR_TRY(check_ready(c));
  if (!corners || !vel) return FR_ERR_ARG;
  return frk::geometry(c, corners, vel, S(s));
}

int fr_residual(fr_ctx* c, const double* q, double* R, void* s) {
  FR_TRY(check_ready(c));
  return frk::residual(c, q, R, nullptr, nullptr, 0, 0, 0, S(s));
}

int fr_bdf_rhs(fr_ctx* c, const double* q, const double* qcn, const double* qcnm1, double a0,
               double a1, double a2, double dt, double* r, void* s) {
  FR_TRY(check_ready(c));
  if (!qcn || dt <= 0 || (a2 != 0.0 && !qcnm1)) return FR_ERR_ARG;
  return frk::residual(c, q, r, qcn, a2 != 0.0 ? qcnm1 : nullptr, a0 / dt, a1 / dt, a2 / dt, S(s));
}

int fr_conservative(fr_ctx* c, const double* q, double* qc, void* s) {
  FR_TRY(check_ready(c));
  return frk::conservative(c, q, qc, S(s));
}

int fr_jvp(fr_ctx* c, const double* q, const double* v, double inv_dtau, double a0_dt, double* Av,
           void* s) {
  FR_TRY(check_ready(c));
  return frk::jvp(c, q, v, inv_dtau, a0_dt, Av, S(s));
}

int fr_linearize(fr_ctx* c, const double* q, double inv_dtau, double a0_dt, void* s) {
  FR_TRY(check_ready(c));
  if (!q) return FR_ERR_ARG;
  return frk::linearize(c, q, inv_dtau, a0_dt, S(s));
}

int fr_apply_linear(fr_ctx* c, const double* v, double* out, int transpose, void* s) {
  FR_TRY(check_ready(c));
  if (!v || !out) return FR_ERR_ARG;
  return frk::apply_linear(c, v, out, transpose != 0, S(s));
}

int fr_vjp(fr_ctx* c, const double* q, const double* w, double inv_dtau, double a0_dt, double* out,
           void* s) {
  FR_TRY(check_ready(c));
  if (!q || !w || !out) return FR_ERR_ARG;
  FR_TRY(frk::linearize(c, q, inv_dtau, a0_dt, S(s)));
  return frk::apply_linear(c, w, out, true, S(s));
}

int fr_precond_build(fr_ctx* c, const double* q, double inv_dtau, double a0_dt, void* s) {
  FR_TRY(check_ready(c));
  FR_TRY(frk::block_build(c, q, inv_dtau, a0_dt, S(s)));
  c->blocks_ready = 1;
  if (c->cfg.precond == FR_PRECOND_TWO_LEVEL) {
    if (c->cfg.jvp_mode == FR_JVP_LINEARIZED && c->cfg.block_mode != FR_BLOCK_LINEARIZED)
      FR_TRY(frk::linearize(c, q, inv_dtau, a0_dt, S(s)));
    FR_TRY(frk::mg_build(c, q, inv_dtau, a0_dt, S(s)));
  }
  return FR_OK;
}

int fr_precond_blocks(fr_ctx* c, double* B, void* s) {
  FR_TRY(check_ready(c));
  if (!c->blocks_ready) { snprintf(c->err, sizeof(c->err), "no preconditioner built"); return FR_ERR_ARG; }
  FR_CUDA_CHECK(c, cudaMemcpyAsync(B, c->B64, (size_t)c->ne * c->bsz * c->bsz * sizeof(double),
                                   cudaMemcpyDeviceToDevice, S(s)));
  return FR_OK;
}

int fr_precond_apply(fr_ctx* c, const double* r, double* z, void* s) {
  FR_TRY(check_ready(c));
  if (!c->blocks_ready) { snprintf(c->err, sizeof(c->err), "no preconditioner built"); return FR_ERR_ARG; }
  FR_TRY(frk::precond_apply(c, c->mg_q, r, z, c->mg_inv_dtau, c->mg_a0_dt, S(s)));
  return frk::check_device_waits(c, S(s));
}

int fr_gmres(fr_ctx* c, const double* q, const double* b, double inv_dtau, double a0_dt, double* x,
             int* iters, void* s) {
  FR_TRY(check_ready(c));
  if (!c->blocks_ready) { snprintf(c->err, sizeof(c->err), "no preconditioner built"); return FR_ERR_ARG; }
  if (c->cfg.jvp_mode == FR_JVP_LINEARIZED) FR_TRY(frk::linearize(c, q, inv_dtau, a0_dt, S(s)));
  int its = 0;
  FR_TRY(gmres_solve(c, q, b, inv_dtau, a0_dt, x, &its, S(s)));
  if (iters) *iters = its;
  return FR_OK;
}

int fr_adjoint_solve(fr_ctx* c, const double* q, const double* g, double inv_dtau, double a0_dt,
                     double* lam, int* iters, void* s) {
  FR_TRY(check_ready(c));
  if (!q || !g || !lam) return FR_ERR_ARG;
  if (c->ncases != 1) { snprintf(c->err, sizeof(c->err), "fr_adjoint_solve: single-case contexts only"); return FR_ERR_ARG; }
  // the element blocks at q (applied transposed), the operator's local Jacobians at q and,
  // with the two-level preconditioner, its hierarchy at q and the transposed hierarchy
  FR_TRY(frk::block_build(c, q, inv_dtau, a0_dt, S(s)));
  c->blocks_ready = 1;
  if (c->cfg.block_mode != FR_BLOCK_LINEARIZED) FR_TRY(frk::linearize(c, q, inv_dtau, a0_dt, S(s)));
  if (c->cfg.precond == FR_PRECOND_TWO_LEVEL) {
    FR_TRY(frk::mg_build(c, q, inv_dtau, a0_dt, S(s)));
    FR_TRY(frk::mg_transpose(c, S(s)));
  }
  c->transposed = 1;
  int its = 0;
  const int rc = gmres_solve(c, q, g, inv_dtau, a0_dt, lam, &its, S(s));
  c->transposed = 0;
  if (iters) *iters = its;
  return rc;
}

int fr_precond_apply_transposed(fr_ctx* c, const double* r, double* z, void* s) {
  FR_TRY(check_ready(c));
  if (!r || !z) return FR_ERR_ARG;
  if (!c->blocks_ready) { snprintf(c->err, sizeof(c->err), "no preconditioner built"); return FR_ERR_ARG; }
  if (c->cfg.precond == FR_PRECOND_TWO_LEVEL && !c->mg_t_ready) FR_TRY(frk::mg_transpose(c, S(s)));
  c->transposed = 1;
  const int rc = frk::precond_apply(c, c->mg_q, r, z, c->mg_inv_dtau, c->mg_a0_dt, S(s));
  c->transposed = 0;
  FR_TRY(rc);
  return frk::check_device_waits(c, S(s));
}

int fr_wall_force_vjp(fr_ctx* c, const double* q, double wx, double wy, double alpha, double beta,
                      double* out, void* s) {
  FR_TRY(check_ready(c));
  if (!q || !out) return FR_ERR_ARG;
  if (!c->bounded || (c->bc_below != FR_BC_WALL && c->bc_above != FR_BC_WALL)) {
    snprintf(c->err, sizeof(c->err), "fr_wall_force_vjp: the mesh has no wall faces");
    return FR_ERR_ARG;
  }
  return frk::wall_force_vjp(c, q, wx, wy, alpha, beta, out, S(s));
}

int fr_conservative_vjp(fr_ctx* c, const double* q, const double* w, double alpha, double beta,
                        double* out, void* s) {
  FR_TRY(check_ready(c));
  if (!q || !w || !out) return FR_ERR_ARG;
  return frk::conservative_vjp(c, q, w, alpha, beta, out, S(s));
}

int fr_conservative_dmach(fr_ctx* c, const double* q, const double* w, double* out_h, void* s) {
  FR_TRY(check_ready(c));
  if (!q || !w || !out_h) return FR_ERR_ARG;
  return frk::conservative_dmach(c, q, w, out_h, S(s));
}

int fr_inject_barrier_offset(fr_ctx* c, long long n) {
  FR_TRY(check_ready(c));
  if (c->bw.fz_pt == 0 || !c->bw.fz_arrive || n < 0) return FR_ERR_ARG;
  std::vector<unsigned long long> h(c->ncases);
  FR_CUDA_CHECK(c, cudaDeviceSynchronize());
  FR_CUDA_CHECK(c, cudaMemcpy(h.data(), c->bw.fz_arrive, h.size() * sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost));
  for (unsigned long long& v : h) v += (unsigned long long)n;
  FR_CUDA_CHECK(c, cudaMemcpy(c->bw.fz_arrive, h.data(), h.size() * sizeof(unsigned long long),
                              cudaMemcpyHostToDevice));
  return FR_OK;
}

int fr_bdf2_step(fr_ctx* c, double* q, const double* qcn, const double* qcnm1, double a0, double a1,
                 double a2, double dt, fr_stats* st, void* s) {
  FR_TRY(check_ready(c));
  if (!q || !qcn || dt <= 0 || (a2 != 0.0 && !qcnm1)) return FR_ERR_ARG;
  return newton_loop(c, q, qcn, qcnm1, a0, a1, a2, dt, false, st, S(s));
}

int fr_ptc_solve(fr_ctx* c, double* q, fr_stats* st, void* s) {
  FR_TRY(check_ready(c));
  if (!q) return FR_ERR_ARG;
  return newton_loop(c, q, nullptr, nullptr, 0, 0, 0, 1.0, true, st, S(s));
}

int fr_residual_norms(fr_ctx* c, const double* r, double* mass, double* all, void* s) {
  FR_TRY(check_ready(c));
  double m, a;
  FR_TRY(norms_host(c, r, &m, &a, S(s)));
  if (mass) *mass = m;
  if (all) *all = a;
  return FR_OK;
}

size_t fr_num_dof(const fr_ctx* c) { return c ? c->ndof : 0; }
int fr_tiles(const fr_ctx* c, int* k) {
  if (!c || !k) return FR_ERR_ARG;
  k[0] = c->tile.trace; k[1] = c->tile.elem; k[2] = c->tile.trace_d; k[3] = c->tile.elem_d;
  k[4] = c->tile.lin_elem;
  return FR_OK;
}
int fr_block_size(const fr_ctx* c) { return c ? c->bsz : 0; }
long long fr_kernel_launches(const fr_ctx* c) { return c ? c->launches : 0; }
const char* fr_last_error(const fr_ctx* c) { return c ? c->err : "null context"; }

}  // extern "C"
