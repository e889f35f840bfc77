/*
 * fr.h -- C ABI of the GB300 preconditioned FR/CPR implicit hot path
 * (Wang & Yu, "An Implicit High-Order Preconditioned Flux Reconstruction Method for
 * Low-Mach-Number Flow Simulation with Dynamic Meshes", arXiv 1903.06304).
 *
 * Problem statement (Sec. 3.2): given a mesh with grid velocities at time t, the
 * primitive state q^p = (p, u, v, T) and the BDF2 history q^c,n, q^c,n-1, evaluate the
 * residual R(q^p), the Newton operator A = Gamma/dtau + (a0/dt) M - dR/dq^p applied to
 * vectors, an element block-Jacobi preconditioner, and advance one BDF2 step by
 * Newton-GMRES (Eq. unsteady_pre_discretized_3) or one steady PTC solve (Eqs.
 * steady_pre_discretized_1, SER).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Element e = j*nx + i on a structured nx-by-ny quad mesh, periodic in both
 *   directions (fr_set_mesh) or in xi only with boundary faces below row 0 and above
 *   row ny-1 (fr_set_mesh_bounded); corners per element in the order (xi,eta) =
 *   (-1,-1), (1,-1), (1,1), (-1,1).
 * - Solution vectors (q^p, R, v, A v, q^c histories) are FP64, structure of arrays
 *   [4][Ne][n][n] with n = p+1: variable, element, eta index j, xi index i.
 *   Their length is fr_num_dof().  The caller owns them (device memory).
 * - Element blocks use the local index d = var*n*n + j*n + i.
 * - Pointers suffixed _d are device pointers, _h host pointers.  Every call that takes
 *   a stream enqueues asynchronously on it unless stated; calls that return host
 *   statistics synchronise the stream.
 * - The library owns its workspace, allocated by fr_create / fr_set_mesh.  Hot calls
 *   (residual, jvp, precond, steps) allocate nothing.
 * - Return value: FR_OK or a negative FR_ERR_* code; fr_last_error() gives the text.
 *   Calls never abort the process.  A context is not thread safe.
 */
#ifndef FR_H
#define FR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FR_OK 0
#define FR_ERR_ARG (-1)           /* invalid argument or call order */
#define FR_ERR_CUDA (-2)          /* a CUDA runtime call failed */
#define FR_ERR_NONFINITE (-3)     /* NaN/Inf met in a norm */
#define FR_ERR_NOT_CONVERGED (-4) /* Newton loop hit maxit (stats still filled) */
#define FR_ERR_TIMEOUT (-5)       /* a bounded device wait expired */

#define FR_PREC_FP64 0
#define FR_PREC_FP32 1
#define FR_PREC_BF16 2

typedef struct fr_ctx fr_ctx;

/* Physical and solver parameters.
 * gamma, Pr: Sec. 2.1 (1.4, 0.72); mu = 1.
 * mach: reference Mach number Ma_ref = Ma_inf of the nondimensionalisation (Sec. 2.1).
 * re: Re_ref (Eq. diffusion); re <= 0 turns the viscous flux off (Euler).
 * kappa: cut-off factor of Eqs. eps_nonmove / eps_move; eps_floor: lower bound of eps.
 * prec_dtype: FR_PREC_* storage/factorisation precision of the element blocks.
 * restart: GMRES Krylov dimension (1..FR_MAX_RESTART); maxit_lin: GMRES iteration cap;
 * tol_res: GMRES tolerance relative to ||b|| (Sec. 4);
 * maxit_newton, tol_pseudo: pseudo-time loop cap and Res_m/Res_0 target (Sec. 4);
 * lag: rebuild the blocks every `lag` pseudo-iterations (2 unsteady, 1 steady, Sec. 4);
 * dtau0, dtau_min, dtau_max, r_ser: SER law (Eq. SER) for steady PTC;
 * dtau_unsteady: the fixed pseudo step of BDF2 runs (1e20 in Sec. 3.2);
 * ser_unsteady: if nonzero, BDF2 pseudo-loops start at dtau0_unsteady and adapt dtau by
 * the SER law (Eq. SER, same dtau_min/dtau_max/r_ser) instead of the fixed step, with the
 * blocks rebuilt at every pseudo-iteration (pseudo-transient continuation);
 * jvp_mode: how GMRES applies the Newton operator: FR_JVP_LINEARIZED (default) stores
 * the local Jacobians once per Newton iteration (fr_linearize) and applies them, or
 * FR_JVP_DUAL re-evaluates the residual over dual numbers for every product (fr_jvp);
 * both are exact and agree to rounding;
 * line_search: 0 = plain Newton updates (the paper); k > 0 = backtracking: the update
 * q + lambda dq is tried with lambda = 1, 1/2, ..., 2^-k and the first lambda that lowers
 * the full 2-norm of the pseudo-step residual is kept (the last one otherwise);
 * gmres_side: FR_GMRES_LEFT (PETSc's default, the paper's solver: Krylov space of B^-1 A,
 * tol_res relative to ||B^-1 b||) or FR_GMRES_RIGHT (Krylov space of A B^-1, tol_res
 * relative to ||b||);
 * apply_accum: arithmetic of the block apply with FP32/BF16-stored inverses:
 * FR_ACCUM_DF64 (default) carries the input and the sums as FP32 pairs with error-free
 * transformations (about 2^-44 relative), so the preconditioner is linear to near FP64
 * round-off while it runs on the FP32 pipe; FR_ACCUM_FP32 rounds the input and
 * accumulates in plain FP32 (a state-dependent perturbation with which GMRES can stall
 * on stiff cases);
 * orthog: Arnoldi orthogonalisation: FR_ORTHO_CGS2 (default) classical Gram-Schmidt with
 * one re-orthogonalisation; FR_ORTHO_CGS a single classical pass (PETSc's default
 * refinement setting, "never"), about half the Arnoldi work;
 * krylov_arith: arithmetic of the device-resident Arnoldi cycle (restart <= 128):
 * FR_KRYLOV_FP64 (default) keeps the basis in FP64 and runs the Gram-Schmidt products on
 * the FP64 pipe; FR_KRYLOV_DF64 stores each basis entry as an FP32 pair (hi, lo) in the
 * same 8 bytes and runs the products, sums and updates as double-float on the FP32 pipe
 * (about 2^-48 relative, against 2^-53): w, the operator input, the Hessenberg matrix
 * and the solution stay FP64.  Restarts above 128 always use FP64;
 * block_mode: how the element blocks are formed, both exact: FR_BLOCK_LINEARIZED
 * (default) composes them from the stored local Jacobians (fr_linearize, done by the
 * build), FR_BLOCK_DUAL differentiates each element's residual by dual numbers;
 * tiles: elements per CTA of the point-parallel kernels, K x floor(128 / (p+1)^2) with
 * K = 1 (default) or 2; 0 lets fr_set_mesh time both for each kernel on the context's
 * own sizes and keep the faster.  The two shapes compute the same operations per point
 * but are compiled separately, and their results agree to rounding (about 1e-14
 * relative), not bit for bit; a timed choice can therefore differ between runs;
 * graphs: if nonzero (default) and restart <= 128, GMRES iterations are issued in chunks of
 * up to 10 whose kernel launches are captured once into a CUDA graph and replayed (same
 * results; fewer launch overheads); ignored while fr_profile timing is on;
 * precond: FR_PRECOND_BLOCK (default) element block Jacobi; FR_PRECOND_TWO_LEVEL adds a
 * coarse correction before the block-Jacobi step (not in the paper, whose per-process
 * ILU(0) of Sec. 4 this replaces: element blocks alone stall once the preconditioned
 * dissipation's pressure coupling, growing as p^2/h, dominates the BDF2 term
 * gamma M^2 a0/dt).  With r the vector to precondition and A the Newton operator GMRES
 * applies, M^-1 r = z0 + B^-1 (r - A z0), z0 = P V(P^T r): P maps per element and
 * variable the three coefficients of c0 + c1 xi + c2 eta (reference coordinates) to the
 * solution points, and V is one multigrid V-cycle on the Galerkin operator P^T A P,
 * agglomerating 2 x 2 cells per level within each case down to at most 4 cells, which are
 * solved exactly; on each other level mg_sweeps (1 or 2) damped block-Jacobi sweeps
 * (12 x 12 blocks, damping mg_omega) before and after the correction (defaults 2, 0.7).  The
 * coarse operators are rebuilt with the blocks (every `lag` Newton iterations) by
 * coloured products of A with the P1 functions of the elements.  mg_prec: storage and
 * sweep arithmetic of the coarse levels, FR_PREC_FP32 (default) or FR_PREC_FP64 (the
 * builds and the transfers to and from the solution points are FP64 either way); B^-1 in
 * the configured block precision;
 * factor_tc: how the element blocks are inverted: FR_FACTOR_SIMT (default) Gauss-Jordan
 * with partial pivoting in FP32 (FP64 for FP64 blocks) on the SIMT pipe;
 * FR_FACTOR_TC_BF16 blocked Gauss-Jordan on [B | I] in FP32 shared memory whose rank-16
 * panel updates run on the tensor cores with BF16 operands and FP32 accumulation (a
 * mixed-precision factorisation: about 2^-9 relative per update, which the outer FP64
 * Krylov iteration absorbs); FR_FACTOR_TC_BF16X3 the same with every operand split
 * into two BF16 numbers and three products per update (about 2^-16 relative).  Panel
 * pivoting and elimination stay FP32 SIMT; the inverse is stored in prec_dtype.  On a periodic mesh with a very
 * large dtau and no time term (a0_dt = 0) the constant states make the coarsest operator
 * singular: use it for BDF2 steps (a0_dt > 0) or on bounded meshes;
 * apply_bulk: 0 (default) applies the blocks with one thread block per element;
 * k = 2, 3 or 4 runs the block apply (and the two-level smoothing step) as a persistent
 * kernel whose blocks stream each element's stored inverse into a k-slab shared ring by
 * bulk asynchronous copies, k - 1 elements in flight behind the one being computed (where
 * k slabs fit in shared memory; the transposed apply always uses one block per element);
 * wait_spins: budget of the device's bounded waits on those copies: 0 = the default
 * (4,194,304 potentially blocking tries), k > 0 = k tries, k < 0 = one non-blocking test
 * (a diagnostic setting under which a wait all but surely runs out).  A wait that runs
 * out makes the call that launched it return FR_ERR_TIMEOUT after the block has waited,
 * again bounded, for its copies in flight; the context stays usable;
 * arnoldi_fused: 0 (default) runs each Arnoldi step of the device-resident GMRES cycle as
 * split passes (V^T w; w -= V h1 with V^T w; w -= V h2 with ||w|| and the Givens update;
 * the scaled store); 1 runs the whole step in one launch of 512-thread blocks, each
 * keeping a part of w in registers, the blocks of a case meeting at bounded barriers for
 * the three reductions (the smallest part size with one block per SM, else the smallest
 * whose blocks the GPU holds at once; 2 or 4 force 2 or 4 pairs of entries per thread).
 * Where no part size fits (vectors above about 0.6 M pairs of entries) or the basis is
 * double-float, the split passes run.  Its barrier waits use the wait_spins budget: a
 * wait that runs out ends the solve with FR_ERR_TIMEOUT and the context stays usable. */
#define FR_MAX_RESTART 256
#define FR_JVP_DUAL 0
#define FR_JVP_LINEARIZED 1
#define FR_GMRES_LEFT 0
#define FR_GMRES_RIGHT 1
#define FR_ACCUM_FP32 0
#define FR_ACCUM_DF64 1
#define FR_BLOCK_LINEARIZED 0
#define FR_BLOCK_DUAL 1
#define FR_ORTHO_CGS2 0
#define FR_ORTHO_CGS 1
#define FR_KRYLOV_FP64 0
#define FR_KRYLOV_DF64 1
#define FR_BC_WALL 1
#define FR_BC_FARFIELD 2
#define FR_PRECOND_BLOCK 0
#define FR_PRECOND_TWO_LEVEL 1
#define FR_FACTOR_SIMT 0
#define FR_FACTOR_TC_BF16 1
#define FR_FACTOR_TC_BF16X3 2
typedef struct fr_config {
  int p;
  double gamma, prandtl, mach, re, kappa, eps_floor;
  int prec_dtype;
  int restart, maxit_lin, maxit_newton, lag;
  double tol_res, tol_pseudo;
  double dtau0, dtau_min, dtau_max, r_ser, dtau_unsteady;
  int gmres_side;
  int ser_unsteady;
  double dtau0_unsteady;
  int line_search;
  int jvp_mode;
  int graphs;
  int apply_accum;
  int tiles;
  int block_mode;
  int orthog;
  int krylov_arith;
  int precond;
  int mg_sweeps;
  double mg_omega;
  int mg_prec;
  int factor_tc;
  int apply_bulk;
  long long wait_spins;
  int arnoldi_fused;
} fr_config;

/* Statistics of one fr_bdf2_step / fr_ptc_solve (host memory, filled on return).
 * res_history[m] = Res_m (2-norm of the continuity row of the pseudo-step residual,
 * Sec. 3.2), m = 0..newton_iterations; gmres_iterations[m] per Newton step. */
#define FR_MAX_NEWTON 64
typedef struct fr_stats {
  int newton_iterations;
  int converged;
  int line_search_halvings;
  int gmres_iterations[FR_MAX_NEWTON];
  double res_history[FR_MAX_NEWTON + 1];
  double dtau_history[FR_MAX_NEWTON + 1];
  int block_builds;
} fr_stats;

/* Fill *cfg with the paper's defaults (gamma 1.4, Pr 0.72, kappa 1, GMRES(30), tol_res
 * 1e-6, tol_pseudo 1e-8, lag 2, SER 0.01/0.01/1e20/2, dtau_unsteady 1e20, FP64 blocks,
 * left preconditioning). */
void fr_default_config(fr_config* cfg);

/* Create a context for polynomial degree cfg->p (1..4) on the current CUDA device.
 * Computes the Gauss points, Lagrange derivative/extrapolation rows and Radau
 * correction derivatives (Sec. 3.1).  *out receives the context.  FR_ERR_ARG on a bad
 * config, FR_ERR_CUDA on a failed allocation. */
int fr_create(const fr_config* cfg, fr_ctx** out);
void fr_destroy(fr_ctx* ctx);

/* Mesh topology: nx-by-ny elements, periodic in both directions (periodic_x,
 * periodic_y must be 1).  Allocates all per-mesh workspace (geometry, traces, Krylov
 * basis, blocks).  Must be called before any compute call; may be called again to
 * resize. */
int fr_set_mesh(fr_ctx* ctx, int nx, int ny, int periodic_x, int periodic_y);

/* Mesh topology periodic in xi and bounded in eta (Sec. 3.3 boundary conditions), e.g.
 * an O-grid around a body: element e = j*nx + i, i around the body (periodic), the faces
 * below row 0 of kind bc_below and above row ny-1 of kind bc_above, each FR_BC_WALL (an
 * adiabatic no-slip wall moving with the grid: boundary state (p^-, v_g, T^-), dT/dn = 0)
 * or FR_BC_FARFIELD (boundary state q_inf, through the approximate Riemann solver).
 * q_inf_h: host array of 4 doubles, the far-field primitive state (p, u, v, T), p, T > 0;
 * required when a side is a far field, may be NULL otherwise; copied.  Boundary faces
 * take the interior trace's local gradient with the full one-sided BR2 lift of
 * q_b - q^- (times the face penalty 2; the boundary state is also q^com).  Allocates like fr_set_mesh plus 4
 * arrays of nx*4*(p+1) doubles and the boundary faces' local Jacobians (48 nx (p+1)
 * doubles).  Every operator mode works on a bounded mesh: the stored linearisation
 * holds the boundary map's Jacobian in (q^-, grad q^-) at each boundary flux point, and
 * the common solution there varies as D_b q^- (D_b = diag(1, 0, 0, 1) at a wall, 0 at a
 * far field), so fr_linearize, fr_apply_linear (both ways), fr_vjp and the linearised
 * element blocks include the boundary faces.  FR_ERR_ARG for nx < 2, ny < 1, an unknown
 * kind or a missing / non-positive q_inf. */
int fr_set_mesh_bounded(fr_ctx* ctx, int nx, int ny, int bc_below, int bc_above,
                        const double* q_inf_h);

/* Force of the fluid on the wall faces of a bounded mesh (the numerator of the force
 * coefficients of Sec. 4, per unit span): F = sum over wall faces of the integral of
 * -(p - p_inf) n + tau . n, with n the unit normal out of the body, p_inf = 1/(gamma M^2),
 * the pressure of the interior trace and the viscous stress of the wall's common
 * gradient (the same as in the wall's viscous flux), Gauss quadrature on the flux
 * points.  q_d: device state vector; force_h: host array receiving (F_x, F_y);
 * deterministic.  C_d = F_x / (rho_inf U_inf^2 c / 2) for a free stream along +x, C_l
 * likewise with F_y, C_t = -C_d.  Synchronises the stream.  FR_ERR_ARG if the mesh has
 * no wall faces. */
int fr_wall_force(fr_ctx* ctx, const double* q_d, double* force_h, void* stream);

/* Update geometry at the current time (Sec. 2.3): corners_d and corner_vel_d are
 * device [Ne][4][2] FP64 (corner coordinates and their grid velocities); the library
 * evaluates |J|, |J| grad(xi), |J| grad(eta), v_g and |J| xi_t, |J| eta_t at solution and
 * flux points of the bilinear map, plus the interpolant divergence of (|J| xi_t,
 * |J| eta_t).  Static meshes pass zero velocities once. */
int fr_update_mesh(fr_ctx* ctx, const double* corners_d, const double* corner_vel_d,
                   void* stream);

/* R(q^p) of Sec. 3.1 (Eq. cpr_ns in its computational-domain form Eq.
 * unsteady_pre_mov_cdomain_GCL): R_d[4][Ne][n][n] = -(1/|J|)(dF/dxi + dG/deta -
 * q^c div(|J| xi_t, |J| eta_t)) with FR correction by Radau g_L, g_R, preconditioned
 * Rusanov (Eq. Rosanov) and BR2 viscous common fluxes (face gradient: the mean of the
 * two local gradients plus twice the mean of the two lifted jumps, a face penalty of 2;
 * the corrected gradient at the solution points adds the lifted jumps once). */
int fr_residual(fr_ctx* ctx, const double* qp_d, double* R_d, void* stream);

/* Pseudo-step right-hand side of Eq. unsteady_pre_discretized_3:
 * r = -(a0 q^c(q^p) + a1 qc_n + a2 qc_nm1)/dt + R(q^p).  a = (1.5, -2, 0.5) for BDF2,
 * (1, -1, 0) for BDF1; qc_nm1_d may be NULL when a2 == 0. */
int fr_bdf_rhs(fr_ctx* ctx, const double* qp_d, const double* qc_n_d, const double* qc_nm1_d,
               double a0, double a1, double a2, double dt, double* r_d, void* stream);

/* q^c(q^p) pointwise (Sec. 2.1): (rho, rho u, rho v, E) into qc_d[4][Ne][n][n]. */
int fr_conservative(fr_ctx* ctx, const double* qp_d, double* qc_d, void* stream);

/* Newton operator applied to a vector (forward-mode, exact):
 * Av = (1/dtau) Gamma(q) v + a0_dt M(q) v - (dR/dq^p)(q) v, Eq. unsteady_pre_discretized_3
 * (a0_dt = a0/dt; a0_dt = 0 gives the steady Eq. steady_pre_discretized_1).
 * Pass inv_dtau = a0_dt = 0 for the plain Jacobian action -(dR/dq) v. */
int fr_jvp(fr_ctx* ctx, const double* qp_d, const double* v_d, double inv_dtau, double a0_dt,
           double* Av_d, void* stream);

/* Store the Newton operator's local Jacobians at q (forward mode, one dual direction per
 * local input): the face map (q-, q+, grad q-, grad q+) -> F^num at every owned flux
 * point, the point map (q, corrected grad q) -> (F, G) at every solution point, and the
 * point matrix Gamma/dtau + a0_dt M - (1/|J|) div(|J| xi_t, |J| eta_t) M.  The linear maps
 * (gradients, traces, liftings, corrected divergence) are fixed by basis and geometry.
 * Overwrites the previous linearisation. */
int fr_linearize(fr_ctx* ctx, const double* qp_d, double inv_dtau, double a0_dt, void* stream);
/* out = A v (transpose = 0) or A^T v (transpose = 1) with the stored linearisation; A as
 * in fr_jvp.  FR_ERR_ARG if fr_linearize has not been called. */
int fr_apply_linear(fr_ctx* ctx, const double* v_d, double* out_d, int transpose, void* stream);
/* Reverse-mode product (the adjoint of fr_jvp): out = A^T w at state q, i.e.
 * (Gamma/dtau + a0_dt M)^T w - (dR/dq^p)^T w; inv_dtau = a0_dt = 0 gives -(dR/dq)^T w.
 * Linearises at q (overwriting the stored linearisation) and applies the transposed
 * factors in reverse order (elements, faces, traces); no face state is stored beyond
 * the local Jacobians. */
int fr_vjp(fr_ctx* ctx, const double* qp_d, const double* w_d, double inv_dtau, double a0_dt,
           double* out_d, void* stream);

/* Build the element block-Jacobi preconditioner at q (Sec. 4 parallel setting, element
 * blocks replacing per-process ILU(0)):
 * B_e = Gamma_e/dtau + a0_dt M_e - dR_e/dq_e (neighbours frozen), then factor it in the
 * configured precision (FP64, FP32 or BF16 storage of the FP32 inverse). */
int fr_precond_build(fr_ctx* ctx, const double* qp_d, double inv_dtau, double a0_dt,
                     void* stream);
/* Copy the unfactored FP64 blocks of the last build to B_d[Ne][b][b] (b = 4 n^2). */
int fr_precond_blocks(fr_ctx* ctx, double* B_d, void* stream);
/* z = M^-1 r with the configured preconditioner (FP64 in and out): z_e = B_e^-1 r_e for
 * every element, or the two-level map.  Synchronises the stream (a bounded device wait
 * that ran out returns FR_ERR_TIMEOUT). */
int fr_precond_apply(fr_ctx* ctx, const double* r_d, double* z_d, void* stream);

/* Restarted block-Jacobi-preconditioned GMRES(m) with CGS2 (Sec. 3.2, PETSc's solver
 * replaced; left or right preconditioning per cfg.gmres_side): solve A x = b at state q
 * with the blocks of the last build; x_d receives the solution (zero initial guess).
 * *iters (host) receives the iteration count.  Synchronises the stream. */
int fr_gmres(fr_ctx* ctx, const double* qp_d, const double* b_d, double inv_dtau, double a0_dt,
             double* x_d, int* iters, void* stream);

/* One physical BDF2 step (Eq. unsteady_pre_discretized_3) by the pseudo-time Newton loop:
 * qp_d holds q^n on entry (initial guess) and q^n+1 on return; qc_n_d, qc_nm1_d are the
 * conservative histories; coefficients a0,a1,a2 as in fr_bdf_rhs.  stats (host) is
 * filled.  Synchronises.  FR_ERR_NOT_CONVERGED if maxit_newton is reached. */
int fr_bdf2_step(fr_ctx* ctx, double* qp_d, const double* qc_n_d, const double* qc_nm1_d,
                 double a0, double a1, double a2, double dt, fr_stats* stats, void* stream);

/* Steady pseudo-transient continuation with SER (Eqs. steady_pre_discretized_1, SER):
 * qp_d updated in place.  Synchronises. */
int fr_ptc_solve(fr_ctx* ctx, double* qp_d, fr_stats* stats, void* stream);

/* Continuity-row 2-norm ||r[0]|| (Res_m of Sec. 3.2) and full 2-norm of a vector,
 * written to host *res_mass, *res_all.  Synchronises. */
int fr_residual_norms(fr_ctx* ctx, const double* r_d, double* res_mass, double* res_all,
                      void* stream);

/* Instrumentation (no counterpart in the paper).  While enabled, every kernel launch
 * is bracketed by a pair of CUDA events on its own stream; fr_profile_read
 * synchronises on them and returns, per kernel class k < FR_PROF_KINDS, the summed
 * device milliseconds ms[k], the timed launch counts counts[k], the total launches
 * launches[k] since creation, and the algorithmic flops[k] and DRAM bytes[k] of the
 * launches issued since the last reset (both counted whether or not timing is on);
 * reset != 0 clears the timing and the algorithmic totals.  Any output pointer may be
 * NULL.  fr_profile_name(k) names class k. */
#define FR_PROF_KINDS 17
int fr_profile(fr_ctx* ctx, int enable);
int fr_profile_read(fr_ctx* ctx, double* ms, long long* counts, long long* launches, double* flops,
                    double* bytes, int reset);
const char* fr_profile_name(int kind);

/* Residual without any allocation (no counterpart in the paper: a deployment variant of
 * fr_residual).  For callers that cannot call cudaMalloc -- code running while a CUDA
 * graph is being captured, code under an allocator or memory pool that forbids outside
 * allocations, an embedding runtime that owns all device memory -- and so cannot create
 * a context.  Computes the geometry of the bilinear mesh from corners_d / corner_vel_d
 * (device [Ne][4][2]) and then R(q^p) exactly as fr_update_mesh + fr_residual do, with
 * the configuration *cfg (host; only p, gamma, prandtl, mach, re, kappa, eps_floor are
 * read), on a periodic nx-by-ny mesh; qp_d, R_d are device [4][Ne][n][n].
 * Scratch: a file-scope 32 MiB device array that every GPU which loads the library
 * holds until the process exits.  The mesh must fit in it:
 *   Ne * ((19 n^2 + 84 n) * 8 + 20) bytes plus the case parameters (each of 9
 *   sub-arrays rounded up to 256 bytes) <= 32 MiB, i.e. Ne <= 17015 at p = 1, 9857 at
 *   p = 2, 6528 at p = 3 (64x64 fits), 4673 at p = 4;
 * larger meshes return FR_ERR_ARG before any GPU work.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress, once per device, with that device
 * current): make that first call before any stream capture.  Every call writes each
 * scratch entry it later reads, so nothing needs clearing, but all calls share the one
 * array: calls that overlap on the GPU (other streams, other threads) race and must be
 * serialised by the caller.  The looked-up address is kept for the life of the process:
 * after cudaDeviceReset on a device the library must be reloaded (a new process) before
 * this entry point is used on that device again.  Asynchronous on `stream`; returns
 * FR_OK, FR_ERR_ARG or FR_ERR_CUDA (no error text: there is no context); a CUDA error
 * already pending when the call starts returns FR_ERR_CUDA before any launch and is left
 * pending for its owner. */
int fr_residual_noalloc(const fr_config* cfg, int nx, int ny, const double* corners_d,
                        const double* corner_vel_d, const double* qp_d, double* R_d,
                        void* stream);

/* Parameter sensitivities of the residual contracted with a weight vector (the paper does
 * not differentiate its solver; this is the parameter part of a discrete adjoint, e.g.
 * for sensitivities of forces to the Mach number or to a prescribed mesh motion).  At
 * state qp_d, for the mesh given again by corners_d / corner_vel_d (device [Ne][4][2], as
 * passed to fr_update_mesh) and weights w_d (device, state layout):
 *   *dmach (host)        = w . dR/dM_inf  (the gas constants R = 1/(gamma M^2),
 *                           C_p = 1/((gamma-1) M^2), k = mu C_p/Pr and the cut-off kappa M_inf
 *                           all move with M_inf, Sec. 2.1 and Eq. eps_move);
 *   dcorners_d[e][a][c]  = w . dR/d(coordinate c of corner a of element e);
 *   dvel_d[e][a][c]      = w . dR/d(velocity component c of corner a of element e).
 * A node shared by several elements appears once per element: its sensitivity is the sum
 * over its copies.  Any of dmach, dcorners_d, dvel_d may be NULL (skipped).  Exact
 * forward mode over colour classes of elements (9 to 25 classes, 8 directions each for
 * corners and again for velocities).  Single-case contexts, periodic or bounded (a far
 * field's q_inf is held fixed in dmach; fr_param_jvp takes its tangent).  Synchronises
 * when dmach is requested; otherwise asynchronous on stream. */
int fr_param_vjp(fr_ctx* ctx, const double* qp_d, const double* w_d, const double* corners_d,
                 const double* corner_vel_d, double* dmach, double* dcorners_d, double* dvel_d,
                 void* stream);

/* Directional derivative of the residual and of the wall force along one parameter
 * direction at a fixed state (the forward counterpart of fr_param_vjp, for a few
 * parameters such as a plunge amplitude and the Mach number): corners_d / corner_vel_d
 * give the mesh again (as passed to fr_update_mesh), dcorners_d / dvel_d (device
 * [Ne][4][2], either may be NULL = zero) the direction of the corners and of their
 * velocities, dmach the Mach tangent (moving R, C_p, k and kappa M_inf as in fr_param_vjp)
 * and dqinf_h (host, 4 doubles, may be NULL = zero) the tangent of the far-field state.
 *   *wdR_h (host, may be NULL)   = w . R'   (w_d device, state layout; needed if wdR_h);
 *   dforce_h[0..1] (host, may be NULL) = (F_x', F_y') of fr_wall_force (needs a wall).
 * Exact forward mode (dual-number geometry, gas and boundary states), bounded or periodic
 * single-case meshes.  Synchronises the stream. */
int fr_param_jvp(fr_ctx* ctx, const double* qp_d, const double* w_d, const double* corners_d,
                 const double* corner_vel_d, const double* dcorners_d, const double* dvel_d,
                 double dmach, const double* dqinf_h, double* wdR_h, double* dforce_h,
                 void* stream);

/* ---------------------------------------------------------------- discrete adjoint
 * Building blocks of the reverse sweep of the BDF2 march (Sec. 3.2) for force objectives
 * (Sec. 4), e.g. the mean thrust coefficient J = (1/K) sum_n -2 F_x(q^n) of a plunging
 * airfoil (Sec. 4.4).  With G^n(q^n, q^{n-1}, q^{n-2}) = R(q^n) - (a0 q^c(q^n) +
 * a1 q^c(q^{n-1}) + a2 q^c(q^{n-2}))/dt the step equations, the adjoint states solve, for
 * n = K .. 1 with the mesh of t^n set,
 *   (dG^n/dq^n)^T lam^n = -dJ/dq^n + (a1^{n+1}/dt) Mq(q^n)^T lam^{n+1}
 *                                   + (a2^{n+2}/dt) Mq(q^n)^T lam^{n+2},
 * Mq = dq^c/dq^p, and dJ/dtheta = dJ/dtheta|_q + sum_n lam^n . dG^n/dtheta|_q.  Since
 * dG^n/dq^n = -A(inv_dtau = 0, a0_dt = a0/dt) (the Newton operator of fr_jvp), a step is
 * fr_wall_force_vjp and fr_conservative_vjp into g, then fr_adjoint_solve of A^T lam = -g;
 * the parameter part is fr_param_jvp (R' and F') and fr_conservative_dmach. */

/* Solve A^T lam = g at state q, A the Newton operator at (inv_dtau, a0_dt) as in fr_gmres:
 * builds the element blocks and the stored linearisation at q, then restarted GMRES with
 * the configured side, restart and tolerance on A^T, preconditioned by the transposed
 * element blocks B_e^-T, or with FR_PRECOND_TWO_LEVEL by the transposed two-level map
 * M^-T r = u + P V'(P^T r - (A P)^T u), u = B^-T r, V' the V-cycle on the transposed coarse
 * operators (those of A^T).
 * lam_d receives the solution (zero initial guess), *iters (host, may be NULL) the
 * iteration count.  Single-case contexts.  Synchronises the stream. */
int fr_adjoint_solve(fr_ctx* ctx, const double* qp_d, const double* g_d, double inv_dtau,
                     double a0_dt, double* lam_d, int* iters, void* stream);
/* z = M^-T r with the preconditioner of the last build (the transpose of
 * fr_precond_apply's map: <y, M^-1 x> = <M^-T y, x>).  Synchronises the stream. */
int fr_precond_apply_transposed(fr_ctx* ctx, const double* r_d, double* z_d, void* stream);
/* out = beta out + alpha d(wx F_x + wy F_y)/dq at q (F of fr_wall_force): the weighted
 * tractions differentiated in the wall faces' traces and local gradients (forward mode)
 * and mapped back by the transposed traces and gradients.  beta = 0 ignores out's
 * contents.  FR_ERR_ARG if the mesh has no wall faces. */
int fr_wall_force_vjp(fr_ctx* ctx, const double* qp_d, double wx, double wy, double alpha,
                      double beta, double* out_d, void* stream);
/* out = beta out + alpha (dq^c/dq^p)(q)^T w, pointwise (the conservative map of Sec. 2.1);
 * beta = 0 ignores out's contents. */
int fr_conservative_vjp(fr_ctx* ctx, const double* qp_d, const double* w_d, double alpha,
                        double beta, double* out_d, void* stream);
/* *out_h (host) = sum of w . dq^c/dM_inf at fixed q^p (rho = p/(R T), R = 1/(gamma M^2)).
 * Synchronises the stream. */
int fr_conservative_dmach(fr_ctx* ctx, const double* qp_d, const double* w_d, double* out_h,
                          void* stream);

/* Failure injection on the host, for tests of the bounded waits (arnoldi_fused): adds n
 * arrivals to every case's barrier counter of the fused Arnoldi step, so that the next
 * barrier of a case with two or more blocks cannot complete for one of its blocks; that
 * block's wait runs out (wait_spins), the solve returns FR_ERR_TIMEOUT and the counters
 * are reset.  Synchronises the device.  FR_ERR_ARG when the fused step is not in use. */
int fr_inject_barrier_offset(fr_ctx* ctx, long long n);

/* ---------------------------------------------------------------- batches
 * Many independent problems solved together (the paper solves one at a time; Sec. 3.2's
 * loop is applied to each case).  Cases may differ in polynomial degree, mesh size and
 * gas (Mach, Reynolds, kappa); gamma, Pr, eps_floor and every solver setting come from
 * the batch's fr_config.  Cases of equal degree and equal viscous switch form a group;
 * every kernel of a group runs over all of the group's elements in one launch, with
 * per-case parameters, per-case reductions, per-case GMRES state and a per-case Newton
 * loop (a case stops iterating when it converges; the group stops when all have).
 * Groups run concurrently, each on its own stream and host thread.
 *
 * Layout: a batch state vector (device, FP64) is the concatenation of the cases' states,
 * each in the single-case layout [4][Ne_k][n_k][n_k]; fr_batch_case_info gives case k's
 * offset and length (the cases of one group are adjacent, so offsets follow the group
 * order, not the case order).  Corner arrays concatenate [Ne_k][4][2] blocks at the
 * element offsets.  The restart length must be <= 128 (device-resident Arnoldi). */
typedef struct fr_case {
  int p;                    /* polynomial degree 1..4 */
  int nx, ny;               /* doubly periodic box of nx x ny elements (>= 2 each) */
  double mach, re, kappa;   /* free-stream Mach, Reynolds (<= 0: Euler), eps factor */
} fr_case;
typedef struct fr_batch fr_batch;

/* Create a batch of ncases cases on the current device (host arrays; copied).
 * FR_ERR_ARG on a bad case or config (*out stays NULL), FR_ERR_CUDA on allocation. */
int fr_batch_create(const fr_config* cfg, const fr_case* cases, int ncases, fr_batch** out);
void fr_batch_destroy(fr_batch* b);
/* Case k's DOF offset and length in batch vectors, element offset and count. */
int fr_batch_case_info(const fr_batch* b, int k, size_t* dof_offset, size_t* ndof,
                       size_t* elem_offset, size_t* nelem);
size_t fr_batch_num_dof(const fr_batch* b);
size_t fr_batch_num_elements(const fr_batch* b);
int fr_batch_num_groups(const fr_batch* b);
/* Geometry of every case from concatenated corners / corner velocities (device). */
int fr_batch_update_mesh(fr_batch* b, const double* corners_d, const double* corner_vel_d,
                         void* stream);
/* R(q^p) of every case (as fr_residual), and the conservative variables (as
 * fr_conservative).  Asynchronous on stream. */
int fr_batch_residual(fr_batch* b, const double* qp_d, double* R_d, void* stream);
int fr_batch_conservative(fr_batch* b, const double* qp_d, double* qc_d, void* stream);
/* One BDF2 step of every case (as fr_bdf2_step): coef (host [ncases][4]) holds case k's
 * a0, a1, a2, dt; a2 = 0 makes it a BDF1 step and qc_nm1_d is then not read for it
 * (qc_nm1_d may be NULL if every a2 is 0).  stats (host [ncases], may be NULL) is filled
 * per case.  Synchronises.  FR_ERR_NOT_CONVERGED if some case reached maxit_newton,
 * FR_ERR_NONFINITE if some case produced a non-finite value (other cases are still
 * advanced: cases never interact). */
int fr_batch_bdf2_step(fr_batch* b, double* qp_d, const double* qc_n_d, const double* qc_nm1_d,
                       const double* coef, fr_stats* stats, void* stream);
/* Steady PTC with SER for every case (as fr_ptc_solve). */
int fr_batch_ptc_solve(fr_batch* b, double* qp_d, fr_stats* stats, void* stream);
/* Instrumentation summed over the groups (as fr_profile / fr_profile_read). */
int fr_batch_profile(fr_batch* b, int enable);
int fr_batch_profile_read(fr_batch* b, double* ms, long long* counts, long long* launches,
                          double* flops, double* bytes, int reset);
long long fr_batch_kernel_launches(const fr_batch* b);
const char* fr_batch_last_error(const fr_batch* b);

/* Sizes: number of FP64 entries of a solution vector, block size b. */
size_t fr_num_dof(const fr_ctx* ctx);
int fr_block_size(const fr_ctx* ctx);
/* The tile shapes in use (K of each point-parallel kernel: residual trace, residual
 * element pass, JVP trace, JVP element pass, linearised-operator element pass) into
 * k[0..4] (host). */
int fr_tiles(const fr_ctx* ctx, int* k);
/* Number of kernels this context has launched since creation (device work items). */
long long fr_kernel_launches(const fr_ctx* ctx);

const char* fr_last_error(const fr_ctx* ctx);
const char* fr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FR_H */
