/* nlmg.h - C ABI of the GB300 FAS multigrid library for heterogeneous nonlinear diffusion.
 *
 * Method: Lee, Hamon, Castelletto, Vassilevski, White, "Nonlinear multigrid based on local spectral coarsening for
 * heterogeneous diffusion problems". Problem (Sec. 2): div(-K0(x) kappa(p) grad p) = f with Dirichlet / Neumann
 * data, discretised by cell-centred TPFA finite volumes (eqs. TPFA_flux, half-transmissibility, FV_matrix); solved by
 * FAS V-cycles (Algorithm 2) with backtracking (Algorithm 1) on a hierarchy built by local spectral coarsening
 * (Sec. 3.1, App. A) whose coarse operators use one coefficient per aggregate (eq. structure, Prop. 1).
 *
 * Conventions (all calls):
 *   - every pointer argument is a HOST pointer unless the name ends in _dev (device pointer on the context's
 *     device); host arrays are read or written during the call only and stay owned by the caller;
 *   - the context owns all device memory it allocates; nothing is thrown across the ABI; every call returns a
 *     status and, on error, nlmg_last_error(ctx) describes it;
 *   - indices are int32, values float64 (IEEE binary64). Cells 0..n_cells-1, faces 0..n_faces-1;
 *   - a context is used by one host thread at a time; its device work runs on the context's own CUDA stream.
 */
#ifndef NLMG_H
#define NLMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nlmg_ctx nlmg_ctx;

typedef enum {
  NLMG_OK = 0,
  NLMG_EINVAL = 1,        /* invalid argument or mesh */
  NLMG_ENOMEM = 2,        /* device allocation failed */
  NLMG_ENOCONV = 3,       /* tolerance not reached within max_cycles (best iterate still written) */
  NLMG_EDIVERGED = 4,     /* NaN/Inf residual */
  NLMG_ETIMEOUT = 5,
  NLMG_ECUDA = 6,         /* CUDA runtime error */
  NLMG_EUNSUPPORTED = 7
} nlmg_status;

/* kappa(p) multiplying K0 (eq. kappa): NLMG_KAPPA_EXP is exp(a p) (eq. permeability_pressure_relationship);
 * NLMG_KAPPA_INV1P2 is 1 / (1 + p^2) (a is ignored). */
typedef enum { NLMG_KAPPA_EXP = 0, NLMG_KAPPA_INV1P2 = 1 } nlmg_kappa_kind;
typedef struct {
  int32_t kind;
  double a;
} nlmg_kappa;

/* Face boundary tags. */
enum { NLMG_FACE_INTERIOR = 0, NLMG_FACE_DIRICHLET = 1, NLMG_FACE_NEUMANN = 2 };

/* The cell graph of Sec. 2.1. face_cells[2f] = K, face_cells[2f+1] = L with K < L for an interior face and L = -1 for
 * a boundary face; half_trans[2f + i] is the geometric half transmissibility Ups_bar of eq. half-transmissibility of
 * cell K (i = 0) and L (i = 1, ignored on boundary faces); face_bc[f] is a NLMG_FACE_* tag; face_area[f] = |eps|;
 * cell_volume[K] = |tau_K|. The flux of face f is oriented out of K. */
typedef struct {
  int32_t n_cells;
  const double* cell_volume;
  int32_t n_faces;
  const int32_t* face_cells;
  const double* half_trans;
  const uint8_t* face_bc;
  const double* face_area;
} nlmg_mesh;

/* Smoother on level 0: a Picard step (Sec. 3.3.1), nu nonlinear Jacobi sweeps, or Picard steps followed by Newton
 * steps (Sec. 3.3.2) once the residual is below newton_switch times the initial one. */
enum { NLMG_SMOOTH_PICARD = 0, NLMG_SMOOTH_JACOBI = 1, NLMG_SMOOTH_PICARD_NEWTON = 2 };

typedef struct {
  int32_t n_levels;          /* hierarchy levels including the fine one (1..8) */
  int32_t agg_size[8];       /* target aggregate size of coarsening step l -> l+1 */
  int32_t modes[8];          /* spectral pressure modes per aggregate of step l -> l+1 */
  int32_t smoother;          /* NLMG_SMOOTH_* for level 0; coarse levels always take a Picard step */
  int32_t nu_pre, nu_post;   /* Jacobi sweeps per smoothing step (Jacobi smoother only) */
  double omega;              /* Jacobi damping */
  int32_t bt_nmax;           /* Algorithm 1: maximum halvings (paper: 4) */
  double bt_theta;           /* Algorithm 1: theta (paper: 0.9) */
  double dp_clamp;           /* Sec. 4.1 pressure-change clamp; <= 0 disables */
  int32_t coarsest_steps;    /* Picard steps on the coarsest level (paper: <= 10) */
  double coarsest_tol;       /* the coarsest level counts as converged once its residual is <= coarsest_tol times
                                its value on entry (or <= the absolute tolerance of the solve); <= 0: the relative
                                tolerance of the solve */
  double lin_tol;            /* relative tolerance of the level-0 CG solves inside Picard steps (default 1e-2) */
  int32_t lin_maxit;         /* iteration cap of the CG solves */
  double coarse_lin_tol;     /* relative tolerance of the coarse-level (hybridized) CG solves (default 1e-1) */
  int32_t lin_precision;     /* 0: level-0 CG in FP64; 1: level-0 CG vectors and matrix in FP32 (tolerance floored
                                at 1e-6), inside the FP64 nonlinear iteration; the coarse levels' hybridized CG and
                                the Newton steps' BiCGStab stay FP64. With lin_precond = 1 the V-cycle is FP32 and the
                                Krylov iteration FP64 whatever this is, and 2 stores the V-cycle's transfers P in BF16
                                (FP32 accumulation; the Galerkin operators use the same rounded P) */
  int32_t setup_threads;     /* host threads for the setup (0 = all) */
  int32_t max_sms;           /* SMs the persistent solver kernels of a context may use (0 = all): contexts that
                                solve concurrently (nlmg_solve_many, the request loop) can then run side by side.
                                The grid, and with it the reduction order, follows from it: results are bitwise
                                reproducible for a given max_sms */
  double newton_switch;      /* NLMG_SMOOTH_PICARD_NEWTON: a level-0 smoothing step at p_k is a Newton step (exact
                                Jacobian, persistent FP64 BiCGStab to newton_lin_tol, clamp, Algorithm 1) once
                                ||R(p_k)|| <= newton_switch ||R(p_0)||, a Picard step before (default 1e-3; >= 0).
                                A Newton step that does not halve the residual returns the rest of the solve to
                                Picard steps (cleared by the next solve and by nlmg_set_options; consecutive
                                nlmg_vcycle calls carry it) */
  double newton_lin_tol;     /* relative tolerance of the BiCGStab solves of the Newton steps (default 1e-2) */
  double coarsest_lin_tol;   /* the same on the coarsest level (default 2e-1; <= 0: coarse_lin_tol) */
  int32_t flux_modes[8];     /* m_f of step l -> l+1: flux unknowns per coarse interface at most (1..8, default 1).
                                1 keeps sigma^PV alone; above 1 the traces of eq. definition-traces from both
                                aggregates' pressure modes are projected off the net flux, and the leading left
                                singular vectors (value > 1e-8 on unit-norm traces) are added beside sigma^PV, each
                                extended into both aggregates (App. A.2). A hierarchy option, fixed at setup */
  int32_t cascadic;          /* 1: nlmg_solve starts its FAS cycles from the nonlinear cascadic iterate (Sec. 4.2):
                                the coarse problems of Algorithm 2 are formed top-down at the initial iterate without
                                smoothing; then, from the coarsest level up, each is solved by up to coarsest_steps
                                Picard steps (stopping like the coarsest solve) from the point its finer level
                                projected, and its correction is carried to the finer level with Algorithm 1; the
                                level-0 correction too. The report's history then holds the residual after it as its
                                second entry (not counted as a cycle). 0 (default): plain FAS cycles */
  int32_t lin_precond;       /* preconditioner of the level-0 Krylov solves (the Picard steps' CG and the Newton
                                steps' BiCGStab; Sec. 3.4 uses AMG there): 0 (default) Jacobi, in the persistent
                                kernels; 1 one V-cycle of a linear multigrid on the hierarchy's pressure spaces
                                (Galerkin operators P^T A P, Chebyshev smoothing, dense coarsest solve; FP32 inside
                                the FP64 Krylov iteration, run as CUDA graphs with a device-side loop). A hierarchy
                                option when set at setup: the setup then coarsens beyond n_levels, for the
                                preconditioner only, until the coarsest level has at most 128 pressure unknowns (the
                                FAS cycles still use n_levels levels); a context set up with 0 cannot switch to 1 */
  int32_t mg_row_cells;      /* multigrid preconditioner (lin_precond = 1): block levels with at least this many cells
                                run their smoothing steps and residuals one thread per cell component (vector loads
                                of the block rows, every lane busy: for large levels, bandwidth bound); smaller levels
                                one warp per cell (shorter dependent chains: for small, latency-bound levels). Only
                                the order of the sums differs. Default 16384; 0: every level row-parallel; >= 0 */
  int32_t reserved[2];
} nlmg_options;

typedef struct {
  int32_t cycles;            /* V-cycles (or Picard iterations for nlmg_solve_picard) */
  int32_t early_exit;        /* last cycle stopped after pre-smoothing */
  double res0, res;          /* ||R(p_0)||_2, ||R(p_final)||_2 */
  double solve_ms;           /* device wall time of the solve */
  int64_t fine_evals;        /* fine residual evaluations */
  int64_t lin_iters;         /* PCG iterations, all levels */
  int64_t kernel_launches;   /* CUDA kernels launched by the solve */
  int64_t lin_iters_level[8];/* PCG iterations per level */
  int32_t tol_tightened;     /* times the inner tolerances were divided by 100 after a cycle that stalled */
  int32_t newton_steps;      /* level-0 Newton smoothing steps (NLMG_SMOOTH_PICARD_NEWTON) */
  int32_t history_len;
  double history[64];        /* ||R|| after each cycle (first entry = res0) */
} nlmg_report;

typedef struct {
  int32_t n_cells, n_flux, n_p, n_lambda;
  int32_t eig_host;   /* level >= 1: local eigenproblems of its coarsening solved on the host although a batched GPU
                         solve was used (the GPU result of that matrix was not finite) */
} nlmg_level_info;

/* Fills *opt with the paper's constants (n_max = 4, theta = 0.9, <= 10 coarsest steps) and library defaults. */
void nlmg_default_options(nlmg_options* opt);

/* Builds the hierarchy (host C++: aggregation, spectral bases, coarse flux space, static local matrices;
 * App. A-C) and uploads it and the mesh to the current CUDA device. *out receives a new context, to be released
 * with nlmg_destroy. Errors: NLMG_EINVAL (bad mesh/options), NLMG_ENOMEM, NLMG_ECUDA, NLMG_EUNSUPPORTED (a coarse
 * cell with more than 128 local flux unknowns or more than 8 pressure modes). */
nlmg_status nlmg_setup(const nlmg_mesh* mesh, const nlmg_kappa* kappa, const nlmg_options* opt, nlmg_ctx** out);

/* Host-only variant of nlmg_setup: builds the same hierarchy without touching any CUDA device. The context then
 * serves the hierarchy export calls below (nlmg_level_info_get, nlmg_get_aggregates, nlmg_get_transfer_dense)
 * and nothing else; every device call on it returns NLMG_EINVAL. */
nlmg_status nlmg_setup_host(const nlmg_mesh* mesh, const nlmg_kappa* kappa, const nlmg_options* opt,
                            nlmg_ctx** out);

/* A second context on the hierarchy of `base` (a context made by nlmg_setup). The hierarchy is built from the
 * reference operator at kappa = 1 (the local eigenproblems of App. A use the linear reference operator), so it does
 * not depend on the nonlinearity's parameter, the right-hand side or the boundary data: the new context shares the
 * read-only device copy of the mesh and hierarchy with `base` (no second setup, no second copy) and owns only its
 * work buffers and CUDA stream, so that solves on different contexts of one hierarchy may run concurrently from
 * different host threads. `kappa` may be NULL (base's nonlinearity) or name another kind / parameter. The solver
 * options are base's. The shared data are freed with the last context that refers to them; each context is
 * destroyed with nlmg_destroy. Errors: NLMG_EINVAL (NULL base or out, host-only base), NLMG_ENOMEM / NLMG_ECUDA. */
nlmg_status nlmg_instance(const nlmg_ctx* base, const nlmg_kappa* kappa, nlmg_ctx** out);

/* Launch-shape autotuner for concurrent solves: times nlmg_solve_many of the n_streams given rows
 * (f_cell[n_streams][n_cells], g_face[n_streams][n_faces], host buffers) on n_streams streams with the persistent
 * kernels of every context capped at each of the SM shares {all, 1/2, 1/4, 1/8 of the SMs}, after one untimed run,
 * and returns the fastest as *best_max_sms (an SM count; the full count for all of them); solves_per_s (NULL or 4
 * entries) receives the measured throughput of each candidate. Not a step of the paper's method. The context's options are left as they were:
 * set max_sms to the result (nlmg_set_options) to use it. Which candidate wins depends on the problem size (small
 * solves are latency bound and run best side by side on a share of the GPU, large ones fill it) and on timing
 * noise, so the result may differ from run to run; a fixed max_sms keeps results bitwise reproducible. */
nlmg_status nlmg_tune_sm_share(nlmg_ctx* ctx, int32_t n_streams, const double* f_cell, const double* g_face,
                               int32_t* best_max_sms, double* solves_per_s);

/* Replaces the solver options of ctx (smoother, backtracking, clamp, coarsest steps, inner tolerances, precision)
 * for the following solves. The hierarchy options (n_levels, agg_size, modes) must equal those ctx was set up with
 * (NLMG_EINVAL otherwise); setup_threads is ignored. */
nlmg_status nlmg_set_options(nlmg_ctx* ctx, const nlmg_options* opt);

/* n_rhs independent FAS solves on the hierarchy of ctx (several right-hand sides and boundary data on one mesh):
 * f_cell[n_rhs][n_cells], g_face[n_rhs][n_faces], x0[n_rhs][n_cells] (NULL = all zero) and p_out[n_rhs][n_cells]
 * are host buffers, row r being right-hand side r. The solves run on up to n_streams contexts of the same hierarchy
 * (ctx and n_streams - 1 instances made by nlmg_instance on first use and kept by ctx), each on its own stream and
 * host thread; n_streams <= 0 picks 8. Unless ctx's max_sms is set, the persistent kernels of each context then
 * use max_sms = SMs / min(n_streams, 4), so that several run side by side. Every row is bitwise the solve that
 * nlmg_solve returns for it on a context with that max_sms (each context owns its buffers, every reduction has a
 * fixed order, and the share depends on n_streams only, not on the load). rep (NULL or n_rhs entries) and status (NULL or
 * n_rhs entries) receive each row's report and status. Returns NLMG_OK if every row converged, else the first
 * failing row's status (its message is then ctx's last error). */
nlmg_status nlmg_solve_many(nlmg_ctx* ctx, int32_t n_rhs, const double* f_cell, const double* g_face,
                            const double* x0, double tol_rel, double tol_abs, int32_t max_cycles, int32_t n_streams,
                            double* p_out, nlmg_report* rep, int32_t* status);

/* nlmg_solve_many on device-resident rows: f_dev[n_rhs][n_cells], g_dev[n_rhs][n_faces], x0_dev (NULL = all zero)
 * and p_dev[n_rhs][n_cells] are device pointers on the context's device, complete before the call (each instance
 * reads its rows on its own stream); every row is bitwise the nlmg_solve_device result on a context with the same SM
 * share. rep and status are host arrays as for nlmg_solve_many. */
nlmg_status nlmg_solve_many_device(nlmg_ctx* ctx, int32_t n_rhs, const double* f_dev, const double* g_dev,
                                   const double* x0_dev, double tol_rel, double tol_abs, int32_t max_cycles,
                                   int32_t n_streams, double* p_dev, nlmg_report* rep, int32_t* status);

/* Sets the problem data: f_cell[n_cells] (source density f|_K) and g_face[n_faces] (Dirichlet pressure or Neumann
 * flux density per boundary face, ignored on interior faces). [f]_K = |tau_K| f_K + sum_Neumann |eps| g_N
 * (definitions under eq. FV_matrix). */
nlmg_status nlmg_set_data(nlmg_ctx* ctx, const double* f_cell, const double* g_face);

/* FAS solve (Algorithm 2 cycles from level 0) from x0[n_cells] (NULL = 0) until ||R|| <= tol_rel ||R(x0)|| or
 * ||R|| <= tol_abs (Sec. 4), at most max_cycles cycles; p_out[n_cells]. Host buffers: data are copied in and the
 * solution out inside the call. Returns NLMG_ENOCONV if the tolerance was not met (p_out holds the last iterate). */
nlmg_status nlmg_solve(nlmg_ctx* ctx, const double* f_cell, const double* g_face, const double* x0, double tol_rel,
                       double tol_abs, int32_t max_cycles, double* p_out, nlmg_report* rep);

/* Same on device-resident buffers (f_dev[n_cells], g_dev[n_faces], x0_dev may be NULL, p_dev[n_cells] output). */
nlmg_status nlmg_solve_device(nlmg_ctx* ctx, const double* f_dev, const double* g_dev, const double* x0_dev,
                              double tol_rel, double tol_abs, int32_t max_cycles, double* p_dev, nlmg_report* rep);

/* Single-level Picard baseline (Sec. 2.2): frozen-coefficient TPFA solves (PCG) + clamp + Algorithm 1. Host buffers;
 * max_cycles bounds the Picard iterations. */
nlmg_status nlmg_solve_picard(nlmg_ctx* ctx, const double* f_cell, const double* g_face, const double* x0,
                              double tol_rel, double tol_abs, int32_t max_cycles, double* p_out, nlmg_report* rep);

/* Single-level Newton baseline (Sec. 2.2; linearisation of Sec. 3.3.2 on level 0): the exact Jacobian of the TPFA
 * residual (assembled on the device in the SELL layout), restarted GMRES(30) with Jacobi right preconditioning to
 * lin_tol, then the clamp and Algorithm 1. Host buffers; max_cycles bounds the Newton iterations. */
nlmg_status nlmg_solve_newton(nlmg_ctx* ctx, const double* f_cell, const double* g_face, const double* x0,
                              double tol_rel, double tol_abs, int32_t max_cycles, double* p_out, nlmg_report* rep);

/* ---- single steps of the path, for parity tests (host buffers; problem data from nlmg_set_data) ------------ */

/* R(p) (reduced TPFA residual, net outgoing flux minus [f]) at p[n_cells] -> r_out[n_cells]. */
nlmg_status nlmg_fine_residual(nlmg_ctx* ctx, const double* p, double* r_out);

/* TPFA fluxes on the level-0 flux unknowns (interior + Dirichlet faces in face order) -> sigma_out[n_flux(0)]. */
nlmg_status nlmg_fine_flux(nlmg_ctx* ctx, const double* p, double* sigma_out);

/* A^l(x) = [M^l(Pi~ p) sigma + D^T p ; D sigma] (eq. structure) on a coarse level l >= 1; x = [sigma; p] of length
 * n_flux(l) + n_p(l) -> out (same length). */
nlmg_status nlmg_level_apply(nlmg_ctx* ctx, int32_t level, const double* x, double* out);

/* Intergrid transfers between level l and l+1 (Sec. 3.1): op 0 = projection Q x, 1 = restriction P^T r,
 * 2 = prolongation P e. Vectors are [sigma; p]; on level 0 they hold p only, and the projection takes p and uses the
 * TPFA fluxes of p (the data of nlmg_set_data) for the flux part. */
enum { NLMG_PROJECT = 0, NLMG_RESTRICT = 1, NLMG_PROLONG = 2 };
nlmg_status nlmg_transfer(nlmg_ctx* ctx, int32_t level, int32_t op, const double* in, double* out);

/* The Picard update on level l: dx solving the frozen-coefficient system of eq. picardian_system,
 * A_frozen(x) dx = b - A(x) (level 0: A(kappa(p)) dp = -R(p), b ignored), with the kernels the solves run: level 0 by
 * the persistent Jacobi-preconditioned CG to lin_tol (the variant follows from lin_tol, lin_precision and max_sms as
 * in a solve); level l >= 1 by one launch of the fused coarse step, whose hybridized CG (Sec. 3.4) runs to
 * coarse_lin_tol (coarsest_lin_tol on the coarsest level). Every Krylov solve stops after at most lin_maxit
 * iterations; *iters (may be NULL) receives the iterations taken. */
nlmg_status nlmg_picard_update(nlmg_ctx* ctx, int32_t level, const double* x, const double* b, double* dx_out,
                               int32_t* iters);

/* One application z = B r of the multigrid preconditioner of the level-0 Krylov solves (lin_precond = 1; the
 * paper's Sec. 3.4 preconditions them with AMG) for the frozen TPFA matrix A(kappa(p)): one V-cycle on the
 * hierarchy's pressure spaces with Galerkin operators A_{l+1} = P_l^T A_l P_l, Chebyshev smoothing preconditioned by
 * the (block) diagonal and a dense coarsest solve, in FP32. p, r, z_out are host arrays of n_cells. Errors:
 * NLMG_EINVAL (context not set up with lin_precond = 1, no data). */
nlmg_status nlmg_precond_apply(nlmg_ctx* ctx, const double* p, const double* r, double* z_out);

/* The level-0 Newton update (Sec. 3.3.2 in the reduced form): dx solving J(p) dx = -R(p) with the exact Jacobian of
 * the TPFA residual, by the persistent FP64 BiCGStab of the Picard-then-Newton smoother to newton_lin_tol (relative,
 * on the Jacobi-scaled residual). p and dx_out are host arrays of n_cells; *iters (may be NULL) receives the iterations. */
nlmg_status nlmg_newton_update(nlmg_ctx* ctx, const double* p, double* dx_out, int32_t* iters);

/* One FAS cycle from level 0 (Algorithm 2) from p_in; r0 is the reference ||R(p_0)|| for the early exit. */
nlmg_status nlmg_vcycle(nlmg_ctx* ctx, const double* p_in, double r0, double* p_out, double* res_out,
                        int32_t* early_exit);

/* ---- hierarchy export, for tests -------------------------------------------------------------------------- */
nlmg_status nlmg_level_info_get(nlmg_ctx* ctx, int32_t level, nlmg_level_info* out);
/* Aggregates of coarsening step l -> l+1: agg_of[n_cells(l)]; m_out[n_cells(l+1)] modes per aggregate. */
nlmg_status nlmg_get_aggregates(nlmg_ctx* ctx, int32_t level, int32_t* agg_of, int32_t* m_out);
/* Dense export of a transfer matrix of step l -> l+1: which 0 = P_p (n_p(l) x n_p(l+1)), 1 = P_sigma
 * (n_flux(l) x n_flux(l+1)), 2 = Q_sigma (n_flux(l+1) x n_flux(l)); row-major into dense (caller-sized). */
nlmg_status nlmg_get_transfer_dense(nlmg_ctx* ctx, int32_t level, int32_t which, double* dense);

/* ---- request loop (continuous batching of independent solves) -------------------------------------------- */
/* Not a step of the paper's method: a serving layer over the calls above. Requests are queued on submit and taken in
 * arrival order by up to max_inflight worker threads as soon as their estimated device memory fits in
 * mem_budget_bytes; each request gets its own context (hierarchy built with setup_threads_per_request host threads)
 * and CUDA stream, so requests that arrive while others run are admitted as slots and memory free up and their GPU
 * work overlaps. Hierarchies stay on the device after their request: up to hierarchy_cache of them are kept (least
 * recently used evicted first, also when the memory budget needs room), and a later request whose mesh arrays and
 * hierarchy options (n_levels, agg_size, modes) are identical runs on an nlmg_instance of the kept hierarchy instead
 * of a new setup, whatever its nonlinearity parameter, data and solver options. Unless a request sets max_sms, its
 * persistent kernels use SMs / min(max_inflight, 4) of them (a share fixed by the server options, not by the load).
 * A request's result is the same alone and in any mix and with or without reuse (each context owns its buffers,
 * every reduction has a fixed order and the setup is deterministic). All pointers are host pointers, copied at
 * submit. */
typedef struct nlmg_server nlmg_server;
typedef struct {
  int32_t max_inflight;
  size_t mem_budget_bytes;
  int32_t setup_threads_per_request;
  int32_t hierarchy_cache;   /* hierarchies kept for reuse (0 = none) */
} nlmg_server_options;
typedef struct {
  double queue_ms, setup_ms, solve_ms, latency_ms;   /* latency = submit -> result ready */
  int32_t hierarchy_reused;                          /* 1 if the request ran on a kept hierarchy */
} nlmg_request_times;
void nlmg_server_default_options(nlmg_server_options* opt);
/* The device memory the request loop reserves for a request on this mesh before admitting it (the estimate its
 * admission compares with mem_budget_bytes): a fixed 4 MiB plus 2,000 bytes per cell and 200 per face. It is meant to
 * cover the shared and own device bytes a context holds after a solve (nlmg_device_bytes). Errors: NLMG_EINVAL. */
nlmg_status nlmg_server_request_bytes(const nlmg_mesh* mesh, size_t* bytes);
/* Uses the calling thread's current CUDA device. */
nlmg_status nlmg_server_create(const nlmg_server_options* opt, nlmg_server** out);
/* Returns NLMG_ENOMEM if the request alone exceeds the memory budget. *ticket identifies the request. */
nlmg_status nlmg_server_submit(nlmg_server* srv, const nlmg_mesh* mesh, const nlmg_kappa* kappa,
                               const nlmg_options* opt, const double* f_cell, const double* g_face, double tol_rel,
                               double tol_abs, int32_t max_cycles, uint64_t* ticket);
/* Waits up to wait_ms (0: no wait) for the request; NLMG_ETIMEOUT if it is not done yet. Once a result is returned
 * (p_out[n_cells], rep, times; each may be NULL) the ticket is released. Returns the request's solve status. */
nlmg_status nlmg_server_poll(nlmg_server* srv, uint64_t ticket, int32_t wait_ms, double* p_out, nlmg_report* rep,
                             nlmg_request_times* times);
/* Finishes the queued requests, joins the workers and frees the server. */
void nlmg_server_destroy(nlmg_server* srv);

/* ---- measurement ----------------------------------------------------------------------------------------- */
/* Enables (1) or disables (0) CUDA-event timing of the hot kernels on the context stream and clears the counters.
 * Kernel ids: 0 = persistent fine CG solve (kp_fine_cg*), 1 = persistent coarse Picard step (kp_coarse_step:
 * coarse operator evaluations, hybridized CG, clamp and Algorithm 1 in one launch; also for nlmg_picard_update)
 * on the levels between the finest and the coarsest, 2 = fine TPFA residual (k_residual), 3 = persistent fine
 * BiCGStab of the Newton smoothing steps (kp_fine_bicgstab), 4 = kp_coarse_step on the coarsest level (the whole
 * coarsest solve in one launch), 5 = a level-0 CG solve preconditioned by the multigrid V-cycle (lin_precond = 1:
 * its graph launches), 6 = the same for a Newton step's BiCGStab, 7 = the multigrid setup of one such solve (FP32
 * fine values, Galerkin operators, block inverses, coarsest inverse). */
nlmg_status nlmg_profile(nlmg_ctx* ctx, int32_t enable);
/* Launch count, summed event time, algorithmic bytes per launch (each streamed array counted once; the gathered
 * neighbour values counted once) and arithmetic per launch (FMA = 2 flops; every kernel but 2) of a profiled kernel
 * since nlmg_profile(ctx, 1). Any output pointer may be NULL. */
nlmg_status nlmg_profile_read(nlmg_ctx* ctx, int32_t kernel, int64_t* launches, double* total_ms,
                              double* bytes_per_launch, double* flops_per_launch);

/* ---- allocation-free call ------------------------------------------------------------------------------- */
/* R(p) into r_dev[n_cells] and ||R(p)||_2^2 into *norm2_dev, for callers that cannot allocate device memory when
 * they call: an application whose caching allocator already holds the device memory it may use (a cudaMalloc
 * there fails or forces the pool to give memory back), code under a fixed device-memory budget, and loops that must
 * not stall other streams (cudaFree, and often cudaMalloc, synchronize the device). It allocates nothing: the
 * per-cell kappa values and the reduction partial sums live in one fixed device array of this library (about
 * 8.1 MiB, held on every device that loads the library until the process exits), and p_dev, r_dev, norm2_dev are
 * caller-owned device pointers. It computes exactly what nlmg_fine_residual computes, with the same kernels, on the
 * context's mesh and the context's current problem data: those of the last nlmg_set_data, or of the last solve
 * call that took data (nlmg_solve, nlmg_solve_device, nlmg_solve_picard, nlmg_solve_newton), which must have
 * completed. The paper has no counterpart: this is a library-interface addition.
 *   - stream: a cudaStream_t given as void* (NULL = legacy default stream); the work is only enqueued there.
 *   - meshes of more than 1,048,576 cells are rejected with NLMG_EINVAL.
 *   - the first call on a device resolves the array's device address (cudaGetSymbolAddress, checked), so make that
 *     first call before any stream capture.
 *   - every call reuses the same array, which keeps the last call's contents (the reduction's arrival counter is
 *     zeroed on the given stream by every call); calls that overlap on the GPU (on different streams, or from
 *     different contexts on the same device) race on it and must be serialized. */
nlmg_status nlmg_fine_residual_noalloc(nlmg_ctx* ctx, const double* p_dev, double* r_dev, double* norm2_dev,
                                       void* stream);

/* Device memory held by ctx: *shared_bytes by the hierarchy and mesh copies it shares with its instances,
 * *own_bytes by its own work buffers (the level-0 Newton and GMRES buffers are allocated by the first call that needs
 * them). Either pointer may be NULL. Not a step of the paper's method. */
nlmg_status nlmg_device_bytes(const nlmg_ctx* ctx, size_t* shared_bytes, size_t* own_bytes);

/* Failure detection, without a GPU fault (not a step of the paper's method). Every grid-wide wait of the persistent
 * kernels is bounded: a block that has polled the barrier spin_limit times (about 2 s in the solver kernels) records
 * an error and every block leaves, so a solve returns NLMG_ETIMEOUT instead of hanging. This call runs that barrier
 * alone on the context's stream, in a cooperative launch of min(blocks, co-resident) blocks of which block
 * absent_block (< 0: none) leaves without arriving, with the given spin limit (1024 .. 2^26 polls of ~32 ns sleeps).
 * Returns NLMG_ETIMEOUT when a wait gave up (the expected outcome with an absent block), NLMG_OK when every block
 * passed; *passed (may be NULL) receives the number of blocks whose wait completed. The context stays usable.
 * Errors: NLMG_EINVAL (bad arguments, host-only context), NLMG_ECUDA. */
nlmg_status nlmg_check_grid_barrier(nlmg_ctx* ctx, int32_t blocks, int32_t absent_block, int64_t spin_limit,
                                    int32_t* passed);

/* FP64 fused multiply-add throughput of the current device in GFLOP/s (an FMA counts 2), measured with a synthetic
 * kernel of independent FMA chains; the denominator of the FP64-arithmetic roofline. */
nlmg_status nlmg_measure_fp64(double* gflops);

/* The message of the context's last failed call; with ctx = NULL, that of the calling thread's last failed
 * nlmg_setup / nlmg_setup_host (whose context was freed). */
const char* nlmg_last_error(const nlmg_ctx* ctx);
void nlmg_destroy(nlmg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
