// fr_batch.cu -- many independent cases advanced together: the pseudo-time Newton loop
// and restarted GMRES of Sec. 3.2 run per case, in lock step, with each kernel launched
// once over all cases of a group (equal degree and viscous switch).
//
// Within a group the element kernels read each case's gas and time/operator terms from
// the case table, and the vector kernels reduce per case (fr_krylov.cu, batched forms).
// A case whose Newton loop has converged gets a zero update and no GMRES iterations; a
// case whose GMRES cycle has stopped is skipped by the Arnoldi passes.  Cases never
// interact: their elements are not neighbours and every reduction is per case.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <thread>
#include <vector>
#include "fr_internal.h"

namespace {

constexpr int kBDS = 4 * GmresState::LD;   // per-case scalar stride of bw.dsc
constexpr int kNormOff = 3 * GmresState::LD;

struct Group {
  fr_ctx* c = nullptr;
  std::vector<int> cases;     // batch indices in group order
  size_t dof_off = 0, elem_off = 0;
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
};

}  // namespace

struct fr_batch {
  fr_config cfg;
  int device = 0;
  std::vector<fr_case> cases;
  std::vector<int> group_of;
  std::vector<size_t> dof_off, ndof, elem_off, nelem;
  std::vector<Group> groups;
  size_t ndof_total = 0, ne_total = 0;
  char err[512];
};

namespace frk {

// Per-case continuity-row and full 2-norms of r (synchronises).  A case with a
// non-finite norm is reported in bad[] (norms set to +inf).
int case_norms(fr_ctx* c, const double* r, std::vector<double>& mass, std::vector<double>& all,
               std::vector<char>& bad, cudaStream_t s) {
  const int nc = c->ncases;
  FR_TRY(frk::bk_norms(c, r, s));
  FR_CUDA_CHECK(c, cudaMemcpy2DAsync(c->bw.hsc, 2 * sizeof(double), c->bw.dsc + kNormOff,
                                     kBDS * sizeof(double), 2 * sizeof(double), nc,
                                     cudaMemcpyDeviceToHost, s));
  FR_CUDA_CHECK(c, cudaStreamSynchronize(s));
  mass.resize(nc);
  all.resize(nc);
  bad.assign(nc, 0);
  for (int k = 0; k < nc; ++k) {
    mass[k] = std::sqrt(c->bw.hsc[2 * k]);
    all[k] = std::sqrt(c->bw.hsc[2 * k + 1]);
    if (!std::isfinite(all[k])) {
      bad[k] = 1;
      mass[k] = all[k] = INFINITY;
    }
  }
  return FR_OK;
}

// Per-case coefficients to the device (pinned staging, guarded like the case table).
static int upload_coef(fr_ctx* c, const std::vector<double>& a, cudaStream_t s) {
  BatchWork& b = c->bw;
  FR_CUDA_CHECK(c, cudaEventSynchronize(b.staged));
  std::memcpy(b.coef_h, a.data(), c->ncases * sizeof(double));
  FR_CUDA_CHECK(c, cudaMemcpyAsync(b.coef, b.coef_h, c->ncases * sizeof(double),
                                   cudaMemcpyHostToDevice, s));
  FR_CUDA_CHECK(c, cudaEventRecord(b.staged, s));
  return FR_OK;
}

// The header of every case's GMRES state (the Hessenberg matrix needs no initial value).
static int upload_gmres(fr_ctx* c, cudaStream_t s) {
  BatchWork& b = c->bw;
  FR_CUDA_CHECK(c, cudaMemcpy2DAsync(b.gst, sizeof(GmresState), b.gst_h, sizeof(GmresState),
                                     offsetof(GmresState, H), c->ncases, cudaMemcpyHostToDevice, s));
  FR_CUDA_CHECK(c, cudaEventRecord(b.staged, s));
  return FR_OK;
}

static int op_apply(fr_ctx* c, const double* q, const double* x, double inv_dtau, double a0_dt,
                    double* out, cudaStream_t s) {
  if (c->transposed) return frk::apply_linear(c, x, out, true, s);
  if (c->cfg.jvp_mode == FR_JVP_LINEARIZED) return frk::apply_linear(c, x, out, false, s);
  return frk::jvp(c, q, x, inv_dtau, a0_dt, out, s);
}

// Batched restarted GMRES(m <= 128): every active case solves its own A_k x_k = b_k with
// its own Krylov space, tolerance and iteration limit; x is zero for inactive cases.
int gmres_cases(fr_ctx* c, const double* q, const double* b, double* x, double inv_dtau,
                double a0_dt, const std::vector<char>& active, std::vector<int>& iters,
                std::vector<char>& failed, cudaStream_t s) {
  const int nc = c->ncases;
  const size_t N = c->ndof;
  const int m = c->cfg.restart;
  const double tol = c->cfg.tol_res;
  const int maxit = c->cfg.maxit_lin;
  const bool left = c->cfg.gmres_side == FR_GMRES_LEFT;
  double* r = c->w_r;
  double* tmp = c->w_u;
  double* w = c->w_t;
  if (left) FR_TRY(frk::precond_apply(c, q, b, r, inv_dtau, a0_dt, s));
  else FR_CUDA_CHECK(c, cudaMemcpyAsync(r, b, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  std::vector<double> rm, bnorm, beta;
  std::vector<char> bad;
  FR_TRY(case_norms(c, r, rm, bnorm, bad, s));
  FR_CUDA_CHECK(c, cudaMemsetAsync(x, 0, N * sizeof(double), s));
  beta = bnorm;
  std::vector<int> total(nc, 0);
  iters.assign(nc, 0);
  for (int k = 0; k < nc; ++k)
    if (active[k] && bad[k]) failed[k] = 1;
  constexpr int kChunk = 10;
  while (true) {
    std::vector<char> cyc(nc, 0);
    int jmax_all = 0;
    FR_CUDA_CHECK(c, cudaEventSynchronize(c->bw.staged));
    for (int k = 0; k < nc; ++k) {
      cyc[k] = active[k] && !failed[k] && bnorm[k] > 0.0 && beta[k] > tol * bnorm[k] &&
               total[k] < maxit;
      GmresState& h = c->bw.gst_h[k];
      std::memset(&h, 0, offsetof(GmresState, H));
      if (cyc[k]) {
        h.g[0] = beta[k];
        h.tol = tol * bnorm[k];
        h.jmax = std::min(m, maxit - total[k]);
        h.inv_hn = 1.0 / beta[k];
        jmax_all = std::max(jmax_all, h.jmax);
      } else {
        h.done = 1;
      }
    }
    if (jmax_all == 0) break;
    FR_TRY(upload_gmres(c, s));
    FR_TRY(frk::bk_init(c, r, tmp, s));
    int issued = 0;
    while (true) {
      const int nchunk = std::min(kChunk, jmax_all - issued);
      const int j0 = issued;
      auto issue = [&](cudaStream_t cs) -> int {
        for (int it = 0; it < nchunk; ++it) {
          if (left) {
            FR_TRY(op_apply(c, q, tmp, inv_dtau, a0_dt, c->w_z, cs));
            FR_TRY(frk::precond_apply(c, q, c->w_z, w, inv_dtau, a0_dt, cs));
          } else {
            FR_TRY(frk::precond_apply(c, q, tmp, c->w_z, inv_dtau, a0_dt, cs));
            FR_TRY(op_apply(c, q, c->w_z, inv_dtau, a0_dt, w, cs));
          }
          FR_TRY(frk::bk_orthogonalize(c, w, tmp, j0 + it + 1, cs));
        }
        return FR_OK;
      };
      const bool dual = c->cfg.jvp_mode == FR_JVP_DUAL && !c->transposed;
      FR_TRY(gm_chunk(c, j0, nchunk, 4 + (left ? 2 : 0) + (dual ? 1 : 0) + (c->transposed ? 8 : 0),
                      dual ? q : nullptr, issue, s));
      issued += nchunk;
      FR_TRY(frk::bk_status(c, s));
      FR_CUDA_CHECK(c, cudaStreamSynchronize(s));
      if (c->bw.status_h[nc].x) {
        // a bounded wait ran out: the cycle's state is not to be trusted
        snprintf(c->err, sizeof(c->err), "a bounded device wait ran out of its budget (wait_spins)");
        return FR_ERR_TIMEOUT;
      }
      bool all_done = true;
      for (int k = 0; k < nc; ++k) {
        const int4 st = c->bw.status_h[k];
        if (st.w) failed[k] = 1;
        if (cyc[k] && !st.z && st.x < st.y) all_done = false;
      }
      if (all_done || issued >= jmax_all) break;
    }
    for (int k = 0; k < nc; ++k)
      if (cyc[k]) total[k] += c->bw.status_h[k].x;
    FR_TRY(frk::bk_finish(c, c->w_u, s));
    if (left) {
      FR_TRY(frk::axpby(c, 1.0, c->w_u, 1.0, x, s));   // u = 0 for cases that did not iterate
    } else {
      // B^-1 u, added only for the cases that iterated (the block apply skips the elements
      // of stopped cases, whose entries of w_z are stale)
      FR_TRY(frk::precond_apply(c, q, c->w_u, c->w_z, inv_dtau, a0_dt, s));
      std::vector<double> one(nc);
      for (int k = 0; k < nc; ++k) one[k] = cyc[k] ? 1.0 : 0.0;
      FR_TRY(upload_coef(c, one, s));
      FR_TRY(frk::bk_axpy_case(c, c->bw.coef, c->w_z, x, s));
    }
    FR_TRY(op_apply(c, q, x, inv_dtau, a0_dt, c->w_t, s));
    FR_TRY(frk::axpby(c, 1.0, b, -1.0, c->w_t, s));
    if (left) FR_TRY(frk::precond_apply(c, q, c->w_t, r, inv_dtau, a0_dt, s));
    else FR_CUDA_CHECK(c, cudaMemcpyAsync(r, c->w_t, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    FR_TRY(case_norms(c, r, rm, beta, bad, s));
    for (int k = 0; k < nc; ++k)
      if (cyc[k] && bad[k]) failed[k] = 1;
  }
  iters = total;
  return FR_OK;
}

}  // namespace frk

namespace {

using frk::case_norms;
using frk::upload_coef;

// The pseudo-time Newton loop of Sec. 3.2 for every case of a group, in lock step.
// a[k] = {a0, a1, a2, dt} of case k (unsteady) or unused (steady).
int batch_newton(fr_ctx* c, double* q, const double* qcn, const double* qcnm1,
                 const std::vector<std::array<double, 4>>* a, bool steady, fr_stats* const* st,
                 cudaStream_t s) {
  const int nc = c->ncases;
  const fr_config& cfg = c->cfg;
  const int maxit = std::min(cfg.maxit_newton, FR_MAX_NEWTON);
  std::vector<fr_stats> local(nc);
  std::vector<fr_stats*> S(nc);
  for (int k = 0; k < nc; ++k) {
    S[k] = st[k] ? st[k] : &local[k];
    std::memset(S[k], 0, sizeof(fr_stats));
  }
  std::vector<double> a0dt(nc, 0.0);
  bool any_bdf2 = false;
  for (int k = 0; k < nc; ++k) {
    fr::CaseParams& p = c->cps[k];
    if (steady) {
      p.a0dt = p.a1dt = p.a2dt = 0.0;
    } else {
      const auto& ak = (*a)[k];
      p.a0dt = ak[0] / ak[3];
      p.a1dt = ak[1] / ak[3];
      p.a2dt = ak[2] / ak[3];
      a0dt[k] = p.a0dt;
      any_bdf2 = any_bdf2 || ak[2] != 0.0;
    }
    p.inv_dtau = 0.0;
    p.a0_dt = a0dt[k];
    p.active = 1;
  }
  FR_TRY(frk::upload_cases(c, s));
  // every case active again on return, whatever the exit path
  struct Restore {
    fr_ctx* c;
    cudaStream_t s;
    ~Restore() {
      for (fr::CaseParams& p : c->cps) p.active = 1;
      frk::upload_cases(c, s);
    }
  } restore{c, s};
  auto rhs = [&](double* out) -> int {
    if (steady) return frk::residual(c, q, out, nullptr, nullptr, 0, 0, 0, s);
    return frk::residual(c, q, out, qcn, any_bdf2 ? qcnm1 : nullptr, 0, 0, 0, s);
  };
  double* r = c->V + (size_t)(cfg.restart + 1) * c->ndof;
  FR_TRY(rhs(r));
  std::vector<double> rm, ra, res0;
  std::vector<char> bad, failed(nc, 0), conv(nc, 0), active(nc, 0);
  FR_TRY(case_norms(c, r, rm, ra, bad, s));
  res0 = rm;
  const bool ser = steady || cfg.ser_unsteady;
  const double dtau_init = steady ? cfg.dtau0 : (cfg.ser_unsteady ? cfg.dtau0_unsteady : cfg.dtau_unsteady);
  std::vector<double> dtau(nc, dtau_init);
  std::vector<int> mk(nc, 0), its;
  for (int k = 0; k < nc; ++k) {
    if (bad[k]) failed[k] = 1;
    S[k]->res_history[0] = rm[k];
    S[k]->dtau_history[0] = dtau[k];
  }
  std::vector<double> coef(nc, 0.0), lambda(nc, 1.0), prev(nc), prev_all(nc);
  for (int m = 0; m < maxit; ++m) {
    int nact = 0;
    for (int k = 0; k < nc; ++k) {
      if (!failed[k] && rm[k] <= cfg.tol_pseudo * res0[k]) conv[k] = 1;
      active[k] = !conv[k] && !failed[k];
      nact += active[k];
    }
    if (nact == 0) break;
    for (int k = 0; k < nc; ++k) {
      c->cps[k].inv_dtau = 1.0 / dtau[k];
      c->cps[k].a0_dt = a0dt[k];
      c->cps[k].active = active[k];   // the kernels skip the elements of stopped cases
    }
    FR_TRY(frk::upload_cases(c, s));
    bool lin_done = false;   // a build from the local Jacobians leaves them stored at q
    bool build = false;
    if (ser || m % std::max(1, cfg.lag) == 0) {
      FR_TRY(frk::block_build(c, q, 0.0, 0.0, s));
      c->blocks_ready = 1;
      for (int k = 0; k < nc; ++k) S[k]->block_builds += active[k];
      lin_done = cfg.block_mode == FR_BLOCK_LINEARIZED;
      build = true;
    }
    if (cfg.jvp_mode == FR_JVP_LINEARIZED && !lin_done) FR_TRY(frk::linearize(c, q, 0.0, 0.0, s));
    if (build) FR_TRY(frk::mg_build(c, q, 0.0, 0.0, s));
    FR_TRY(frk::gmres_cases(c, q, r, c->w_x, 0.0, 0.0, active, its, failed, s));
    FR_TRY(frk::check_device_waits(c, s));
    for (int k = 0; k < nc; ++k) {
      if (active[k]) S[k]->gmres_iterations[mk[k]] = its[k];
      prev[k] = rm[k];
      prev_all[k] = ra[k];
      lambda[k] = 1.0;
    }
    FR_TRY(frk::axpby(c, 1.0, c->w_x, 1.0, q, s));
    FR_TRY(rhs(r));
    FR_TRY(case_norms(c, r, rm, ra, bad, s));
    for (int h = 0; h < cfg.line_search; ++h) {
      int need = 0;
      for (int k = 0; k < nc; ++k) {
        const bool nk = active[k] && !failed[k] && !(ra[k] < prev_all[k]);
        coef[k] = nk ? -0.5 * lambda[k] : 0.0;
        if (nk) {
          lambda[k] *= 0.5;
          S[k]->line_search_halvings++;
          ++need;
        }
      }
      if (need == 0) break;
      FR_TRY(upload_coef(c, coef, s));
      FR_TRY(frk::bk_axpy_case(c, c->bw.coef, c->w_x, q, s));
      FR_TRY(rhs(r));
      FR_TRY(case_norms(c, r, rm, ra, bad, s));
    }
    for (int k = 0; k < nc; ++k) {
      if (!active[k]) continue;
      if (bad[k]) failed[k] = 1;
      S[k]->res_history[mk[k] + 1] = rm[k];
      if (ser && !failed[k])
        dtau[k] = std::max(cfg.dtau_min, std::min(cfg.dtau_max, dtau[k] * std::pow(prev[k] / rm[k], cfg.r_ser)));
      S[k]->dtau_history[mk[k] + 1] = dtau[k];
      mk[k]++;
    }
  }
  bool all_conv = true, any_failed = false;
  for (int k = 0; k < nc; ++k) {
    if (!failed[k] && rm[k] <= cfg.tol_pseudo * res0[k]) conv[k] = 1;
    S[k]->newton_iterations = mk[k];
    S[k]->converged = conv[k] && !failed[k];
    all_conv = all_conv && S[k]->converged;
    any_failed = any_failed || failed[k];
  }
  if (any_failed) {
    snprintf(c->err, sizeof(c->err), "non-finite values in some case of the batch");
    return FR_ERR_NONFINITE;
  }
  return all_conv ? FR_OK : FR_ERR_NOT_CONVERGED;
}

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int batch_check(fr_batch* b) {
  if (!b) return FR_ERR_ARG;
  if (b->groups.empty()) { snprintf(b->err, sizeof(b->err), "empty batch"); return FR_ERR_ARG; }
  return FR_OK;
}

// Runs fn(group) for every group, each on its own stream and host thread, after the
// caller's stream; the caller's stream then waits for all groups.  Returns the first
// error (a group's message is copied into the batch's).
template <class F>
int run_groups(fr_batch* b, cudaStream_t caller, F fn) {
  cudaEvent_t start;
  if (cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess) return FR_ERR_CUDA;
  cudaEventRecord(start, caller);
  const int ng = (int)b->groups.size();
  std::vector<int> rc(ng, FR_OK);
  auto body = [&](int g) {
    cudaSetDevice(b->device);
    Group& G = b->groups[g];
    cudaStreamWaitEvent(G.s, start, 0);
    rc[g] = fn(G);
    cudaEventRecord(G.ev, G.s);
  };
  if (ng == 1) {
    body(0);
  } else {
    std::vector<std::thread> th;
    for (int g = 0; g < ng; ++g) th.emplace_back(body, g);
    for (auto& t : th) t.join();
  }
  for (int g = 0; g < ng; ++g) cudaStreamWaitEvent(caller, b->groups[g].ev, 0);
  cudaEventDestroy(start);
  int out = FR_OK;
  for (int g = 0; g < ng; ++g) {
    if (rc[g] == FR_OK) continue;
    // a hard error outranks a non-converged case
    if (out == FR_OK || out == FR_ERR_NOT_CONVERGED) {
      out = rc[g];
      snprintf(b->err, sizeof(b->err), "group %d: %s", g, b->groups[g].c->err);
    }
  }
  return out;
}

}  // namespace

extern "C" {

int fr_batch_create(const fr_config* cfg, const fr_case* cases, int ncases, fr_batch** out) {
  if (!out) return FR_ERR_ARG;
  *out = nullptr;
  if (!cfg || !cases || ncases < 1 || cfg->restart < 1 || cfg->restart > GmresState::LD)
    return FR_ERR_ARG;
  for (int k = 0; k < ncases; ++k) {
    const fr_case& q = cases[k];
    if (q.p < 1 || q.p > 4 || q.nx < 2 || q.ny < 2 || !(q.mach > 0.0) || !std::isfinite(q.re) ||
        !(q.kappa >= 0.0))
      return FR_ERR_ARG;
  }
  fr_batch* b = new fr_batch();
  b->cfg = *cfg;
  b->err[0] = 0;
  cudaGetDevice(&b->device);
  b->cases.assign(cases, cases + ncases);
  b->group_of.assign(ncases, -1);
  // groups by (degree, viscous switch), in order of first appearance
  std::vector<std::pair<int, int>> keys;
  for (int k = 0; k < ncases; ++k) {
    const std::pair<int, int> key(cases[k].p, cases[k].re > 0.0 ? 1 : 0);
    auto it = std::find(keys.begin(), keys.end(), key);
    if (it == keys.end()) { keys.push_back(key); it = keys.end() - 1; }
    b->group_of[k] = (int)(it - keys.begin());
  }
  b->groups.resize(keys.size());
  b->dof_off.assign(ncases, 0);
  b->ndof.assign(ncases, 0);
  b->elem_off.assign(ncases, 0);
  b->nelem.assign(ncases, 0);
  size_t dof = 0, el = 0;
  int rc = FR_OK;
  for (size_t g = 0; g < keys.size() && rc == FR_OK; ++g) {
    Group& G = b->groups[g];
    G.dof_off = dof;
    G.elem_off = el;
    std::vector<int> nxs, nys;
    std::vector<fr::CaseParams> params;
    for (int k = 0; k < ncases; ++k) {
      if (b->group_of[k] != (int)g) continue;
      const fr_case& q = cases[k];
      const size_t n = q.p + 1, ne = (size_t)q.nx * q.ny;
      G.cases.push_back(k);
      b->dof_off[k] = dof;
      b->ndof[k] = 4 * ne * n * n;
      b->elem_off[k] = el;
      b->nelem[k] = ne;
      dof += b->ndof[k];
      el += ne;
      nxs.push_back(q.nx);
      nys.push_back(q.ny);
      fr_config ck = *cfg;
      ck.p = q.p;
      ck.mach = q.mach;
      ck.re = q.re;
      ck.kappa = q.kappa;
      fr::CaseParams cp;
      std::memset(&cp, 0, sizeof(cp));
      cp.gas = fr_make_gas(ck);
      cp.active = 1;
      params.push_back(cp);
    }
    fr_config gc = *cfg;
    const fr_case& first = cases[G.cases[0]];
    gc.p = first.p;
    gc.mach = first.mach;
    gc.re = first.re;
    gc.kappa = first.kappa;
    rc = fr_create(&gc, &G.c);
    if (rc != FR_OK) break;
    G.c->external_terms = true;
    rc = fr_setup_cases(G.c, (int)G.cases.size(), nxs.data(), nys.data(), params.data());
    if (rc == FR_OK && (cudaStreamCreateWithFlags(&G.s, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaEventCreateWithFlags(&G.ev, cudaEventDisableTiming) != cudaSuccess))
      rc = FR_ERR_CUDA;
  }
  b->ndof_total = dof;
  b->ne_total = el;
  if (rc != FR_OK) {
    fr_batch_destroy(b);
    return rc;
  }
  *out = b;
  return FR_OK;
}

void fr_batch_destroy(fr_batch* b) {
  if (!b) return;
  for (Group& G : b->groups) {
    if (G.s) cudaStreamSynchronize(G.s);
    if (G.c) fr_destroy(G.c);
    if (G.s) cudaStreamDestroy(G.s);
    if (G.ev) cudaEventDestroy(G.ev);
  }
  delete b;
}

int fr_batch_case_info(const fr_batch* b, int k, size_t* dof_offset, size_t* ndof,
                       size_t* elem_offset, size_t* nelem) {
  if (!b || k < 0 || k >= (int)b->cases.size()) return FR_ERR_ARG;
  if (dof_offset) *dof_offset = b->dof_off[k];
  if (ndof) *ndof = b->ndof[k];
  if (elem_offset) *elem_offset = b->elem_off[k];
  if (nelem) *nelem = b->nelem[k];
  return FR_OK;
}

size_t fr_batch_num_dof(const fr_batch* b) { return b ? b->ndof_total : 0; }
size_t fr_batch_num_elements(const fr_batch* b) { return b ? b->ne_total : 0; }
int fr_batch_num_groups(const fr_batch* b) { return b ? (int)b->groups.size() : 0; }

int fr_batch_update_mesh(fr_batch* b, const double* corners, const double* vel, void* s) {
  FR_TRY(batch_check(b));
  if (!corners || !vel) return FR_ERR_ARG;
  return run_groups(b, S(s), [&](Group& G) {
    return frk::geometry(G.c, corners + 8 * G.elem_off, vel + 8 * G.elem_off, G.s);
  });
}

int fr_batch_residual(fr_batch* b, const double* q, double* R, void* s) {
  FR_TRY(batch_check(b));
  if (!q || !R) return FR_ERR_ARG;
  return run_groups(b, S(s), [&](Group& G) {
    for (fr::CaseParams& p : G.c->cps) p.a0dt = p.a1dt = p.a2dt = 0.0;
    FR_TRY(frk::upload_cases(G.c, G.s));
    return frk::residual(G.c, q + G.dof_off, R + G.dof_off, nullptr, nullptr, 0, 0, 0, G.s);
  });
}

int fr_batch_conservative(fr_batch* b, const double* q, double* qc, void* s) {
  FR_TRY(batch_check(b));
  if (!q || !qc) return FR_ERR_ARG;
  return run_groups(b, S(s), [&](Group& G) {
    return frk::conservative(G.c, q + G.dof_off, qc + G.dof_off, G.s);
  });
}

int fr_batch_bdf2_step(fr_batch* b, double* q, const double* qcn, const double* qcnm1,
                       const double* coef, fr_stats* stats, void* s) {
  FR_TRY(batch_check(b));
  if (!q || !qcn || !coef) return FR_ERR_ARG;
  const int nc = (int)b->cases.size();
  for (int k = 0; k < nc; ++k) {
    const double* a = coef + 4 * k;
    if (!(a[3] > 0.0) || (a[2] != 0.0 && !qcnm1)) return FR_ERR_ARG;
  }
  return run_groups(b, S(s), [&](Group& G) {
    const int n = (int)G.cases.size();
    std::vector<std::array<double, 4>> a(n);
    std::vector<fr_stats*> st(n);
    for (int i = 0; i < n; ++i) {
      const int k = G.cases[i];
      for (int j = 0; j < 4; ++j) a[i][j] = coef[4 * k + j];
      st[i] = stats ? stats + k : nullptr;
    }
    return batch_newton(G.c, q + G.dof_off, qcn + G.dof_off, qcnm1 ? qcnm1 + G.dof_off : nullptr,
                        &a, false, st.data(), G.s);
  });
}

int fr_batch_ptc_solve(fr_batch* b, double* q, fr_stats* stats, void* s) {
  FR_TRY(batch_check(b));
  if (!q) return FR_ERR_ARG;
  return run_groups(b, S(s), [&](Group& G) {
    const int n = (int)G.cases.size();
    std::vector<fr_stats*> st(n);
    for (int i = 0; i < n; ++i) st[i] = stats ? stats + G.cases[i] : nullptr;
    return batch_newton(G.c, q + G.dof_off, nullptr, nullptr, nullptr, true, st.data(), G.s);
  });
}

int fr_batch_profile(fr_batch* b, int enable) {
  FR_TRY(batch_check(b));
  for (Group& G : b->groups) FR_TRY(fr_profile(G.c, enable));
  return FR_OK;
}

int fr_batch_profile_read(fr_batch* b, double* ms, long long* counts, long long* launches,
                          double* flops, double* bytes, int reset) {
  FR_TRY(batch_check(b));
  double m[FR_PROF_KINDS], f[FR_PROF_KINDS], by[FR_PROF_KINDS];
  long long n[FR_PROF_KINDS], l[FR_PROF_KINDS];
  for (int k = 0; k < FR_PROF_KINDS; ++k) {
    if (ms) ms[k] = 0.0;
    if (counts) counts[k] = 0;
    if (launches) launches[k] = 0;
    if (flops) flops[k] = 0.0;
    if (bytes) bytes[k] = 0.0;
  }
  for (Group& G : b->groups) {
    FR_TRY(fr_profile_read(G.c, m, n, l, f, by, reset));
    for (int k = 0; k < FR_PROF_KINDS; ++k) {
      if (ms) ms[k] += m[k];
      if (counts) counts[k] += n[k];
      if (launches) launches[k] += l[k];
      if (flops) flops[k] += f[k];
      if (bytes) bytes[k] += by[k];
    }
  }
  return FR_OK;
}

long long fr_batch_kernel_launches(const fr_batch* b) {
  if (!b) return 0;
  long long n = 0;
  for (const Group& G : b->groups) n += fr_kernel_launches(G.c);
  return n;
}

const char* fr_batch_last_error(const fr_batch* b) { return b ? b->err : "null batch"; }

}  // extern "C"
