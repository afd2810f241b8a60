/*
 * stc.h -- C ABI of libstc: keyframe smoke control by spacetime multigrid on one
 * GPU (Pan & Manocha, "Efficient Optimal Control of Smoke using Spacetime
 * Multigrid", arXiv 1608.01102).
 *
 * The library solves the control problem of Eq. opt: find forces u_0..u_{N-1}
 * on a 2D or 3D staggered grid so that the density rho_i advected by the implicit
 * Navier-Stokes velocity v_i (Eq. NSA, NSB, Conv) matches keyframes rho*_i,
 * with force regularisation r.  It runs the paper's ADMM loop (Alg. 3): the
 * advection-optimisation fixed point (Alg. 1) and the Navier-Stokes
 * optimisation solved by STFAS V-cycles (Alg. 2) with the temporally augmented
 * SCGS smoother (Eq. HESS).
 *
 * Conventions (all entry points):
 *  - Grid: nx x ny cells on [0, nx h] x [0, ny h], h = 1/nx, closed box (all
 *    wall-normal velocities are zero).  Centre fields are [ny][nx], i fastest.
 *    Face fields are all x-faces [ny][nx+1] then all y-faces [ny+1][nx], i
 *    fastest; wall faces are stored and are zero.  A time-dependent field is
 *    a contiguous sequence of such slabs (v: N+1 slabs, u: N slabs, ...).
 *    A 3D grid (stc_params.nz >= 2) adds a third axis: cells [nz][ny][nx],
 *    faces x [nz][ny][nx+1], y [nz][ny+1][nx], z [nz+1][ny][nx].
 *  - Host arrays are double precision and owned by the caller; the library
 *    copies every input and never keeps a host pointer.  A length argument
 *    that does not match the field returns STC_ERR_INVALID_ARG and writes
 *    nothing.
 *  - Device precision follows stc_params.precision: 0 = fp32 state with fp64
 *    reductions and an fp64 coarsest STFAS level; 1 = fp64 everywhere.
 *  - All work is enqueued on the CUDA stream given at creation (NULL = the
 *    legacy default stream); calls that return numbers synchronise it.
 *  - No exception crosses the ABI.  A CUDA error returns STC_ERR_CUDA and
 *    leaves the problem unusable.  stc_last_error() gives a thread-local
 *    message for the last failing call.
 *  - A problem must not be used from two host threads at once.
 */
#ifndef STC_H
#define STC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  STC_OK = 0,
  STC_ERR_INVALID_ARG = 1,
  STC_ERR_OOM = 2,
  STC_ERR_CUDA = 3,
  STC_ERR_NOT_CONVERGED = 4,
  STC_ERR_DIVERGED = 5, /* Taylor order above taylor_kmax, or a non-finite norm */
  STC_ERR_UNSUPPORTED = 6,
  STC_ERR_BUSY = 7      /* the object is in use (a running serving request) */
} stc_status;

typedef struct stc_problem stc_problem; /* opaque; owns all of its device memory */

/* Parameters.  Defaults (stc_default_params) follow the paper's Table 2 where it
 * gives a value and the readings stated beside each field otherwise. */
typedef struct {
  int nx, ny;           /* cells per axis (2D); h = 1/nx                          */
  int num_steps;        /* N timesteps (Sec. 3)                                    */
  double dt;            /* timestep                                                */
  double r;             /* force regularisation (Eq. opt)                          */
  double K;             /* ADMM penalty (Eq. optAdmm); changes the rate, not the solution; default 1 */
  double beta;          /* multiplier step lambda += K beta (v - v*) (Alg. 3), default 1 */
  int precision;        /* 0 = fp32 state + fp64 reductions/coarsest, 1 = fp64 */
  int ao_iters;         /* Alg. 1 forward/backward pairs per ADMM iteration (Table 2: 2) */
  int pre, post;        /* V-cycle smoothing sweeps (Alg. 2: 2, 2)                 */
  int coarse_sweeps;    /* smoothing sweeps on the coarsest level (Alg. 2: 10)     */
  int coarsest_n;       /* stop coarsening below this many cells per axis (4)      */
  double taylor_tol;    /* Taylor truncation, relative to max|rho_0| (Sec. 3.1: 1e-5) */
  int taylor_kmax;      /* Taylor order limit; exceeding it is STC_ERR_DIVERGED (64) */
  double eps_stfas;     /* NSO stop: ||f||_inf <= eps_stfas * ||f||_inf at the first NSO (1e-5) */
  double eps_admm;      /* ADMM stop on max_i ||rho_i - rho_i^last||_inf (Alg. 3); <0: max|rho_0|/100 */
  int max_vcycles;      /* V-cycle cap per NSO solve (20)                          */
  int metric_levels;    /* Gaussian filters in C_i (Sec. 4.1); 0 gives C_i = c_i I  */
  double metric_sigma0; /* std-dev of the first filter in cells (1)                */
  double scgs_omega;    /* SCGS under-relaxation (0.8)                             */
  double lm_shift;      /* Levenberg-Marquardt shift of the smoother's v blocks; <0: 1/dt^2 */
  int poisson_vcycles;  /* multigrid cycles per projection Q (8) where Q runs as a
                           multigrid: 3D, and 2D fields too large for one CTA's
                           shared memory.  Other 2D fields are projected exactly
                           (DCT-II diagonalisation of the Neumann Laplacian). */
  int self_advection;   /* 1 (default); 0 drops Adv (linear saddle problem, tests only) */
  int ao_halvings;      /* Sec. 5 safeguard of Alg. 1: v* moves to v* + a (y - v*) with
                           a = 1, 1/2, ... (at most this many halvings) until the AO
                           objective of Eq. PO does not increase; -1 = plain Alg. 1 (8) */
  int cgc_guard;        /* 1 (default): a V-cycle keeps a level's coarse-grid correction
                           only if it does not raise that level's ||res - f||_2 */
  int lm_adapt;         /* 1 (default): Sec. 5's Levenberg-Marquardt safeguard in stc_solve's
                           NSO loop: a V-cycle that raises ||f||_inf is undone and lm_shift
                           quadrupled (at most 4096x its default; a cycle undone there ends
                           the NSO solve); each NSO solve starts by halving it back toward
                           its default */
  double al_threshold;  /* Sec. 5 augmented-Lagrangian fallback in stc_solve: the multiplier
                           update is applied only when the objective of Eq. opt fell by at
                           most al_threshold * |J| since the previous ADMM iteration; < 0
                           (default) applies it every iteration (the plain Alg. 3) */
  int time_coarsen;     /* 0 (default, the paper: STFAS coarsens in space only); 1: every
                           level whose N is even hands the next one N/2 steps of 2 dt
                           (point fields: full weighting / linear interpolation in time,
                           interval fields: pair means / piecewise constant) */
  int nz;               /* 0 (default): the 2D grid nx x ny.  >= 2: the 3D grid nx x ny x nz
                           (Sec. 3.1 with a third axis; h = 1/nx).  3D layouts: cells
                           [nz][ny][nx]; faces = x-faces [nz][ny][nx+1], then y-faces
                           [nz][ny+1][nx], then z-faces [nz+1][ny][nx]; the hierarchy
                           halves all three axes; SCGS blocks are 7x7 (6 faces + pressure)
                           with 8 parity colours.  1 is invalid. */
  int boundary;         /* 0 (default): the closed box (wall faces are not unknowns).
                           1: periodic in every axis (3D only; nx, ny, nz even, so the
                           parity colours of SCGS stay independent across the wrap).
                           Face layouts keep n + 1 slots per axis; slot n is not a face
                           and reads as zero; neighbour indices, QUICK stencils, the
                           metric filters and the transfers wrap. */
  int scgs_cta_cells;   /* 2D smoother kernel choice, results unchanged: a colour of at
                           most this many cells runs one CTA per cell (each block step of
                           the cyclic reduction split over the CTA's threads; short
                           dependency chains for the coarse levels), a larger one a warp
                           per cell.  0: always a warp per cell.  -1 (default): 256 for
                           fp32 solves, every colour for fp64 solves (the faster choice
                           measured on GB300 for each solve type). */
  int ao_trials;        /* AO blend (Sec. 5), 2D: blend factors 2^-h tried at once, each
                           on its own stream with its own trajectory buffers (1..8; 1 =
                           one at a time; 3D always one at a time).  The accepted factor
                           is the first that does not raise the objective, exactly as
                           in the one-at-a-time search.  Default 4. */
  int k_adapt;          /* 0 (default): the ADMM penalty K stays fixed (Alg. 3 with Table 2's
                           constant K).  1: stc_solve balances it (residual balancing, not in
                           the paper): after each multiplier update, with r_p = ||v - v*|| and
                           r_d = K ||v - v_prev|| over steps 1..N-1, K doubles when r_p > 10 r_d
                           and halves when r_d > 10 r_p, within 2^+-10 of its value at the
                           start of the solve.  The fixed point does not depend on K; the
                           adapted K stays in the problem after the solve (report.K_final). */
} stc_params;

typedef struct {
  int admm_iters;      /* ADMM iterations run                                  */
  int vcycles;         /* V-cycles run in total                                */
  double kkt_rel;      /* ||g(v)|| / ||g(v_start)|| at exit                    */
  double kkt_abs;      /* ||g(v)||                                             */
  double f_inf;        /* NSO residual ||f||_inf at exit                       */
  double drho;         /* last max_i ||rho_i - rho_i^last||_inf                */
  double seconds;      /* wall time of the solve                               */
  double seconds_to_1e4; /* time at which kkt_rel first reached 1e-4 (<0: never) */
  int rejected_vcycles; /* V-cycles undone by the LM safeguard (counted in vcycles) */
  double lm_shift;      /* the smoother's LM shift at exit                      */
  int density_stop_iter;      /* first ADMM iteration (1-based) at which Alg. 3's density
                                 test max_i ||rho_i - rho_i^last||_inf < max|rho_0|/100
                                 held, whatever eps_admm is (0: never)          */
  double seconds_to_density_stop; /* wall time at that iteration (<0: never)    */
  double objective;     /* J(v) of Eq. opt at exit (misfit + r/2 ||u||^2)        */
  int lambda_updates;   /* multiplier updates applied (fewer than admm_iters under
                           the AL fallback)                                       */
  double seconds_to_1e2; /* times at which kkt_rel first reached 1e-2, 1e-3, 1e-6 */
  double seconds_to_1e3; /* (<0: never)                                           */
  double seconds_to_1e6;
  double K_final;       /* the ADMM penalty at exit (differs from params.K when it
                           adapts, stc_params.k_adapt)                            */
} stc_report;

/* Field identifiers for stc_get_field / stc_set_field (level 0 = finest grid). */
typedef enum {
  STC_FIELD_V = 0,      /* velocity v_i, i = 0..N           (N+1) x faces  (level l) */
  STC_FIELD_PBAR = 1,   /* multiplier pbar_i, i = 0..N      (N+1) x cells  (level l) */
  STC_FIELD_U = 2,      /* force u_i, i = 0..N-1            N x faces      (level l) */
  STC_FIELD_P = 3,      /* pressure p_{i+1}, i = 0..N-1     N x cells      (level l) */
  STC_FIELD_RES_V = 4,  /* residual buffer, rows 1..4 of f  same shapes as V, PBAR, U, P */
  STC_FIELD_RES_PBAR = 5,
  STC_FIELD_RES_U = 6,
  STC_FIELD_RES_P = 7,
  STC_FIELD_Z = 8,      /* NSO target z_i = v*_i - lambda_i/K  N x faces (level l) */
  STC_FIELD_VSTAR = 9,  /* slack velocity v*_i, i = 0..N-1  N x faces      */
  STC_FIELD_LAMBDA = 10,/* ADMM multiplier lambda_i          N x faces      */
  STC_FIELD_RHO = 11,   /* density rho_i, i = 0..N           (N+1) x cells  */
  STC_FIELD_MU = 12,    /* adjoint mu_i, i = 0..N-1          N x cells      */
  STC_FIELD_W = 13,     /* AO target w_i = v_i + lambda_i/K  N x faces      */
  STC_FIELD_Y = 14,     /* adjoint-sweep output, see stc_adjoint  N x faces  */
  STC_FIELD_KKT_U = 15, /* u_i(v) of the KKT metric          N x faces      */
  STC_FIELD_KKT_G = 16, /* reduced gradient g_i(v)           (N+1) x faces  */
  STC_FIELD_MTERM = 17, /* C_i (rho_i - rho*_i)              (N+1) x cells  */
  STC_FIELD_RES_IN_V = 18, /* FAS right-hand side res^h of level l (V, PBAR, U, P shapes) */
  STC_FIELD_RES_IN_PBAR = 19,
  STC_FIELD_RES_IN_U = 20,
  STC_FIELD_RES_IN_P = 21,
  STC_FIELD_XOLD_V = 22,   /* copy of R x^h kept for the FAS correction (level l >= 1) */
  STC_FIELD_XOLD_PBAR = 23,
  STC_FIELD_XOLD_U = 24,
  STC_FIELD_XOLD_P = 25,
  /* forward simulation and its adjoint (stc_simulate, stc_simulate_adjoint) */
  STC_FIELD_SIM_GRAD_RHO = 26, /* input dL/d rho_i, i = 0..N (fp64)  (N+1) x cells */
  STC_FIELD_SIM_GRAD_U = 27,   /* output dL/d u_i, i = 0..N-1      N x faces      */
  STC_FIELD_SIM_ADJ_V0 = 28,   /* output dL/d v_0                  1 x faces      */
  STC_FIELD_SIM_ADJ_RHO0 = 29, /* output dL/d rho_0 (with_step0)   1 x cells      */
  STC_FIELD_SIM_ADJ_VN = 30    /* input dL/d v_N (zero unless set) 1 x faces      */
} stc_field;

/* Fill *p with the defaults for an nx x ny grid with N steps, dt = 1/N. */
void stc_default_params(stc_params* p, int nx, int ny, int num_steps);

/* Create a problem (Sec. 3: initial density rho_0 and initial velocity v_0,
 * which is fixed).  rho0: nx*ny doubles; v0: face array or NULL for zero.
 * cuda_stream: a cudaStream_t, or NULL.  Allocates all device memory of the
 * problem (state of every level, AO/KKT buffers, scratch).  Errors:
 * INVALID_ARG (bad sizes/params), UNSUPPORTED (grid beyond the kernels'
 * on-chip limits: 2D, nx*ceil(ny/8) <= 4096, projection levels fit in shared
 * memory), OOM, CUDA. */
stc_status stc_create_problem(const stc_params* params, const double* rho0, const double* v0,
                              void* cuda_stream, stc_problem** out);

/* Keyframes (Eq. opt: c_i ||rho_i - rho*_i||^2 with c_i replaced by the metric
 * C_i of Sec. 4.1).  steps: count step indices in 1..N; rho_star: count x
 * cells; c: count weights or NULL for 1.  Replaces earlier keyframes. */
stc_status stc_set_keyframes(stc_problem* p, int count, const int* steps, const double* rho_star,
                             const double* c);

/* ncycles STFAS V-cycles (Alg. 2) on the NSO system f = 0 with the current
 * state and target z, each followed by removal of the pressures' means.
 * nso_res_inf (may be NULL) receives ||f||_inf after the last cycle. */
stc_status stc_vcycle(stc_problem* p, int ncycles, double* nso_res_inf);

/* The ADMM outer loop (Alg. 3) from v_i = 0 (i >= 1), lambda = 0: each
 * iteration runs the AO fixed point (cold on the first iteration, warm-started
 * from the previous v* afterwards), at least one V-cycle and then V-cycles
 * until ||f||_inf <= eps_stfas * ||f||_inf of the first NSO (or max_vcycles),
 * the KKT metric and the multiplier update.  Stops when the relative KKT
 * residual ||g(v)||/||g(v_start)|| <= kkt_rel_tol, or on the paper's
 * density-change test, or after max_admm iterations (then
 * STC_ERR_NOT_CONVERGED, with the state kept).  report may be NULL. */
stc_status stc_solve(stc_problem* p, double kkt_rel_tol, int max_admm, stc_report* report);

/* ---- the ADMM loop as resumable phases, and batched NSO V-cycles ---------- */

/* stc_solve (Alg. 3) split into the phases a serving loop interleaves across
 * problems.  stc_solve_begin resets the state and evaluates the KKT
 * denominator at v = 0 (as stc_solve does).  Then, per ADMM iteration:
 * phase 0 -- stc_solve_head runs Alg. 1 and starts the NSO solve; phase 1 --
 * NSO V-cycles under the LM safeguard of Sec. 5 (stc_batch_nso_cycle; one per
 * call) while *wants_cycle of stc_solve_phase is 1, i.e. until ||f||_inf <=
 * eps_stfas times the first NSO's norm, max_vcycles, or a cycle undone at the
 * largest shift (at least one cycle per iteration); then stc_solve_tail
 * (KKT metric, multiplier update, penalty balancing, stopping tests) leads to
 * phase 0 again or to phase 2 (finished).  stc_solve_report gives the report
 * so far and whether a stopping test held.  A phase call out of turn returns
 * STC_ERR_INVALID_ARG.  Running the phases in this order is stc_solve. */
stc_status stc_solve_begin(stc_problem* p, double kkt_rel_tol, int max_admm);
stc_status stc_solve_phase(const stc_problem* p, int* phase, int* wants_cycle);
stc_status stc_solve_head(stc_problem* p);
stc_status stc_solve_tail(stc_problem* p);
stc_status stc_solve_report(const stc_problem* p, stc_report* report, int* converged);

/* A batch runs the NSO V-cycles of many problems as ONE CUDA graph launch on
 * its stream: each problem's captured V-cycle graph (Alg. 2) is a child node,
 * the children independent, so their kernels overlap on the device.  The
 * instantiated batch graph is kept and reused while the set of problems (and
 * their captured graphs) stays the same.  stc_batch_nso_cycle: every problem
 * of probs[0..n) whose solve is in phase 1 and wants a cycle gets one V-cycle
 * in the launch; afterwards each reads its ||f||_inf and takes the LM
 * decision (Sec. 5).  *cycled (may be NULL) = problems cycled; status (n
 * entries, may be NULL) receives each problem's outcome (a failing problem
 * does not stop the others).  The problems' streams are synchronised before
 * the launch and the batch stream after it.  All problems must live on the
 * current device. */
typedef struct stc_batch stc_batch;
stc_status stc_batch_create(void* cuda_stream, stc_batch** out);
stc_status stc_batch_nso_cycle(stc_batch* b, stc_problem* const* probs, int n, int* cycled, stc_status* status);
stc_status stc_batch_destroy(stc_batch* b);

/* Per-iteration record of the last stc_solve on this problem: for ADMM
 * iteration k (0-based), out[3k] = kkt_rel after it, out[3k+1] = seconds since
 * the solve started, out[3k+2] = the penalty K it used.  Writes min(len,
 * 3 count) values; *count (may be NULL) = iterations recorded (0 before any
 * solve).  Host data only; no device work.  STC_ERR_INVALID_ARG for a null
 * problem, or a null out with len > 0. */
stc_status stc_solve_history(const stc_problem* p, double* out, size_t len, int* count);

/* Results.  len must equal the field size: u N x faces, rho (N+1) x cells,
 * v (N+1) x faces. */
stc_status stc_get_forces(const stc_problem* p, double* u, size_t len);
stc_status stc_get_density(const stc_problem* p, double* rho, size_t len);
stc_status stc_get_velocity(const stc_problem* p, double* v, size_t len);

stc_status stc_destroy_problem(stc_problem* p);
const char* stc_last_error(void);

/* ---- step-level entry points: each runs one row of the hot path ---------- */

/* Copy a field of level `level` to / from the host (sizes as listed in
 * stc_field; level must be 0 for fields that exist on the finest grid only). */
stc_status stc_get_field(const stc_problem* p, int field, int level, double* out, size_t len);
stc_status stc_set_field(stc_problem* p, int field, int level, const double* in, size_t len);
/* Number of levels, and the cells per axis of one level. */
stc_status stc_level_info(const stc_problem* p, int* nlevels, int level, int* nx, int* ny);
/* Cells per axis of one level, nz = 0 on a 2D grid.  Outputs may be NULL. */
stc_status stc_level_dims(const stc_problem* p, int level, int* nx, int* ny, int* nz);

/* ---- forward simulation with a given control, and its adjoint -------------
 * The full-resimulation path of Sec. 5 and Appendix A: from v_0 (STC_FIELD_V
 * slab 0) and rho_0 (STC_FIELD_RHO slab 0) under the forces u_i (STC_FIELD_U),
 * stc_simulate solves each implicit step of Eq. NSA/NSB,
 *   (v_{i+1} - v_i)/dt + Adv(v_{i+1}) - u_i + grad p = 0,  div v_{i+1} = 0,
 * by the Picard iteration v <- Q[v_i + dt (u_i - Adv(v))] until the change is
 * at most picard_tol * max|v|, or has stopped halving after 8 iterations within
 * 100 picard_tol * max|v| (the rounding floor of fp32), STC_ERR_NOT_CONVERGED
 * after max_iter; writes
 * v_1..v_N, then advects rho_1..rho_N with v_0..v_{N-1} (Eq. Conv; Taylor
 * orders as stc_advect).  iters (may be NULL): Picard iterations in total.
 * The buffers of both calls are allocated at the first call (not counted by
 * stc_problem_bytes).  Q is exact to rounding where the 2D DCT projection
 * applies; the multigrid projection (3D, large 2D fields) makes it exact to
 * its truncation (~1e-7 relative in fp32, ~1e-9 in fp64 after 8 cycles). */
stc_status stc_simulate(stc_problem* p, double picard_tol, int max_iter, int* iters);
/* Adjoint of stc_simulate's map (u, v_0, rho_0) -> (rho_0..rho_N, v_N) at its last
 * trajectory: given dL/d rho_i in STC_FIELD_SIM_GRAD_RHO and dL/d v_N in
 * STC_FIELD_SIM_ADJ_VN, writes dL/d u_i to STC_FIELD_SIM_GRAD_U and dL/d v_0 to
 * STC_FIELD_SIM_ADJ_V0 (through the velocity chain and, with with_step0, the
 * density of step 0); with with_step0 also the total dL/d rho_0 (its direct
 * term SIM_GRAD_RHO slab 0 included) to STC_FIELD_SIM_ADJ_RHO0, else zero there.  The density part is the
 * backward sweep of stc_adjoint (it overwrites STC_FIELD_MTERM and MU); the
 * velocity part the transposed step z <- Q[a - dt dAdv(v_{i+1})^T z],
 * dL/d u_i = dt z, a <- dL/d v_i|density + z, until the change is at most
 * picard_tol * max|z|.  iters: iterations in total. */
stc_status stc_simulate_adjoint(stc_problem* p, double picard_tol, int max_iter, int with_step0, int* iters);
/* Device-to-device copy between a field and a caller's device buffer of len
 * elements (fp64 if buffer_is_double, else fp32), converting to the field's
 * type and multiplying by scale; to_field = 1 writes the field, 0 reads it.
 * Enqueued on the problem's stream (no synchronisation). */
stc_status stc_copy_field_device(stc_problem* p, int field, int level, void* buffer, size_t len,
                                 int buffer_is_double, int to_field, double scale);
/* Timesteps N_l and timestep dt_l of level `level` (they differ from the
 * finest level's only with stc_params.time_coarsen).  Either output may be NULL. */
stc_status stc_level_steps(const stc_problem* p, int level, int* num_steps, double* dt);

/* Forward density sweep (Eq. Conv, Eq. Adv): rho_{i+1} = A[rho_i, w_i] with
 * w = v* (source STC_FIELD_VSTAR) or w = v (STC_FIELD_V); writes STC_FIELD_RHO
 * and the Taylor orders (read with stc_get_taylor_orders). */
stc_status stc_advect(stc_problem* p, int source_field);
stc_status stc_get_taylor_orders(const stc_problem* p, int* K, size_t len);

/* Keyframe metric terms C_i (rho_i - rho*_i) of the current STC_FIELD_RHO into
 * STC_FIELD_MTERM (zero at steps without a keyframe). */
stc_status stc_metric_terms(stc_problem* p);

/* Backward adjoint sweep of Alg. 1 / Eq. KKTPO for the velocity of the last
 * stc_advect (source_field as there), using STC_FIELD_RHO, the Taylor orders
 * and STC_FIELD_MTERM: mu_{i-1} = (dA_i/drho)^T mu_i - C_i(rho_i - rho*_i) into
 * STC_FIELD_MU, and Y_i = alpha W_i + beta (dA[rho_i, w_i]/dw_i)^T mu_i,
 * i = 1..N-1, into STC_FIELD_Y. */
stc_status stc_adjoint(stc_problem* p, int source_field, double alpha, double beta);

/* Solenoidal projection Q (Eq. KKTPO) in place on slabs [first, first+count)
 * of a face field of the finest level (V, U, VSTAR, Y, W, KKT_U, KKT_G, Z):
 * Q v = v - G phi, (D G) phi = D v.  Exact (DCT) for 2D fields that fit on
 * chip, else poisson_vcycles multigrid cycles (Sec. 4.1's solver). */
stc_status stc_project(stc_problem* p, int field, int first, int count);

/* One AO solve (Alg. 1): w = v + lambda/K; v* = w (warm_start = 0) or the
 * current v* is kept (warm_start != 0, how stc_solve continues the fixed-point
 * iteration after its first ADMM iteration); then `iters` passes, each a
 * backward sweep and projection y = Q(w + (dA/dv*)^T mu / K) followed, when
 * ao_halvings >= 0, by Sec. 5's blend v* <- v* + a (y - v*) with the first
 * a in 1, 1/2, ..., 2^-ao_halvings whose forward sweep does not raise the AO
 * objective (fp64, read back per trial; if none does, v* stays and the pass
 * loop ends); then z = v* - lambda/K on every level.  Afterwards
 * STC_FIELD_RHO and the Taylor orders are those of a forward sweep at the
 * final v*. */
stc_status stc_ao(stc_problem* p, int iters, int warm_start);
/* Halvings taken by each pass of the last stc_ao (-1: every trial rejected;
 * 0 for every pass of the plain form).  *count = passes run; at most `len`
 * are written. */
stc_status stc_ao_trace(const stc_problem* p, int* halvings, size_t len, int* count);
/* The NSO solve of Alg. 3's inner loop on the current targets: at least one
 * V-cycle, then V-cycles until ||f||_inf <= f_target or max_cycles, each under
 * the LM safeguard when stc_params.lm_adapt is set (the smoother's shift is
 * first halved back toward its default; a cycle that raises ||f||_inf is
 * undone and the shift quadrupled).  Outputs (may be NULL): cycles run,
 * including undone ones, and the final ||f||_inf. */
stc_status stc_nso_solve(stc_problem* p, double f_target, int max_cycles, int* cycles, double* f_inf);
/* The smoother's current LM shift and the V-cycles undone by the safeguard
 * since the problem was created or stc_solve last started. */
stc_status stc_lm_info(const stc_problem* p, double* lm_shift, int* rejected);
/* z = v* - lambda/K on the finest level, restricted to every coarser level. */
stc_status stc_prepare_targets(stc_problem* p);

/* NSO residual (Eq. KKTAO) of level `level`: RES fields = f(x) - res^h
 * (res^h = 0 on the finest level); *inf (may be NULL) = its max-norm. */
stc_status stc_nso_residual(stc_problem* p, int level, double* inf);

/* `sweeps` SCGS sweeps (Sec. 4.3, Eq. HESS) on level `level` for f = res^h. */
stc_status stc_smooth(stc_problem* p, int level, int sweeps);

/* FAS transfers of Alg. 2 between level l and l+1: x^{2h} = R x^h (also kept
 * as XOLD), and x^h += P(x^{2h} - XOLD^{2h}). */
stc_status stc_restrict(stc_problem* p, int level);
stc_status stc_prolong_correct(stc_problem* p, int level);

/* Reduced gradient of the KKT metric at the current v: g_i = Q[r(-u_i/dt +
 * (I/dt + dAdv(v_i))^T u_{i-1}) - (dA[rho_i, v_i]/dv_i)^T mu_i] (Appendix A)
 * into STC_FIELD_KKT_G; *norm = ||g||_2 (fp64). */
stc_status stc_kkt_residual(stc_problem* p, double* norm);

/* lambda_i += K beta (v_i - v*_i) (Alg. 3) and *drho = max_i ||rho_i - rho_i^last||_inf,
 * then rho^last = rho. */
stc_status stc_admm_update(stc_problem* p, double* drho);

/* Sets the ADMM penalty K (Eq. optAdmm) and the multiplier step beta (Alg. 3)
 * of an existing problem, for the iterations that follow (K > 0, beta > 0,
 * else STC_ERR_INVALID_ARG and nothing changes).  The multiplier lambda is kept
 * unscaled, so the scaled target z = v* - lambda/K and the AO centre
 * w = v + lambda/K follow the new K; the NSO's K/r of every level changes and
 * the V-cycle graph is captured again at the next V-cycle.  K changes the path
 * of the iteration, not its fixed point (Sec. 4).  Synchronises the stream. */
stc_status stc_set_penalty(stc_problem* p, double K, double beta);

/* ---- instrumentation ------------------------------------------------------ */

/* Number of kernel launches this problem has enqueued since creation (a V-cycle
 * graph replay counts each kernel node it runs). */
stc_status stc_launch_count(const stc_problem* p, long long* launches);

/* enable != 0: the first V-cycle of every stc_vcycle call runs a second
 * V-cycle graph with a CUDA event pair around every finest-level SCGS colour
 * launch and every finest-level colour residual launch (the two largest
 * kernels), recorded on the stream that runs them (the other cycles run the
 * plain graph, so the events perturb one cycle per call).
 * stc_kernel_timing_of(kind) then returns the summed device time (ms) and the
 * number of timed launches of kind 0 (SCGS colour) or 1 (colour residual)
 * since the last enable; stc_kernel_timing is kind 0.  Another kind is
 * STC_ERR_INVALID_ARG.  enable = 0 drops the timed graph. */
stc_status stc_set_kernel_timing(stc_problem* p, int enable);
stc_status stc_kernel_timing(const stc_problem* p, double* total_ms, long long* launches);
stc_status stc_kernel_timing_of(const stc_problem* p, int kind, double* total_ms, long long* launches);

/* FP32 fused multiply-add throughput of the current device, measured: four
 * timed launches of a kernel that keeps every SM busy with independent FMA
 * chains (four waves of the resident CTAs), the best of the last three, in
 * GFLOP/s (2 flops per FMA) into *gflops.  The ALU-side roofline denominator
 * of the SCGS smoother (its dense block arithmetic, Eq. HESS).  Runs on
 * cuda_stream (NULL = legacy default stream) and synchronises it;
 * STC_ERR_INVALID_ARG for a null gflops, STC_ERR_CUDA on a CUDA error. */
stc_status stc_measure_fp32_peak(void* cuda_stream, double* gflops);

/* Device memory held by the problem, in bytes. */
stc_status stc_memory_bytes(const stc_problem* p, size_t* bytes);
/* Device bytes stc_create_problem(params) followed by stc_set_keyframes with
 * nkeys keyframes would allocate -- the number stc_memory_bytes reports for
 * that problem -- computed on the host without a device (the serving
 * admission size).  STC_ERR_INVALID_ARG for parameters stc_create_problem
 * rejects. */
stc_status stc_problem_bytes(const stc_params* params, int nkeys, size_t* bytes);
/* The tables of the exact 2D projection (host arithmetic, no device): for the
 * closed nx x ny box with h = 1/nx, out receives, in order, the orthonormal
 * DCT-II matrices C_x (nx x nx, C[k][i] = s_k cos(pi k (2i+1) / 2n), s_0 =
 * sqrt(1/n), s_k = sqrt(2/n)), C_x^T, C_y (ny x ny), C_y^T, then 1/lam
 * (ny x nx, row ky, column kx; lam = -(4/h^2)(sin^2(pi kx/2nx) +
 * sin^2(pi ky/2ny)), 1/lam_00 = 0), row-major fp64: 2 nx^2 + 2 ny^2 + nx ny
 * values.  The library rounds them to the state type.  STC_ERR_INVALID_ARG
 * for nx or ny < 1, a null out, or len smaller than that count. */
stc_status stc_dct_tables(int nx, int ny, double* out, size_t len);

/* ---- allocation-free entry point ------------------------------------------- */

/* The backward adjoint sweep of stc_adjoint on caller-owned device arrays,
 * allocating nothing.  The paper has no counterpart: this exists for callers
 * that cannot allocate device memory when they run the sweep -- a process that
 * reserves its whole device-memory budget up front in its own pool (so a later
 * cudaMalloc fails or is forbidden), or a latency-critical caller that cannot
 * afford cudaMalloc's implicit device synchronisation.
 *
 * fp32 arrays on the device, layouts as the fields of the same names:
 * vel = the advecting velocity (N face slabs), rho = densities (N+1 cell
 * slabs), K = the Taylor orders of the forward sweep (N ints), mterm =
 * C_i (rho_i - rho*_i) (N+1 cell slabs, fp64), mu = output adjoint (N cell
 * slabs), base = N face slabs or NULL, out = output face slabs: slab i =
 * alpha base_i + beta (dA[rho_i, vel_i]/dvel_i)^T mu_i for i = 1..N-1 (slab 0
 * is not written).  Enqueued on cuda_stream (NULL = legacy default stream);
 * the call then reads the sweep's error word back on that stream and returns
 * once the sweep has finished: a Taylor order in K outside 1..taylor_kmax
 * (orders from a forward sweep run with a larger taylor_kmax) returns
 * STC_ERR_DIVERGED, and mu / out are then not the adjoint.
 *
 * Scratch: the sweep's Taylor powers live in one library-wide device array of
 * 1,048,576 floats (4 MiB, plus 64 words holding the error word) that every
 * GPU loading the library holds until the process exits.  taylor_kmax * nx *
 * ny above that returns STC_ERR_INVALID_ARG with a message.  Every call
 * shares the array and it keeps the last call's contents (the powers need not
 * start at zero; each call clears the error word), so calls that overlap on
 * the GPU race: serialise them.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current and
 * caches it for the process; that lookup may load the library's device code
 * (CUDA loads modules lazily), which is when the 4 MiB array is placed on the
 * device, so make the first call -- or any earlier use of the library on that
 * device -- before reserving the rest of the device memory in a pool, and
 * before any stream capture.  The cached address does not survive
 * cudaDeviceReset: do not use this entry point on a device after resetting
 * it.  No cudaMalloc, cudaFree or allocating library routine is called. */
stc_status stc_adjoint_sweep_noalloc(int nx, int ny, int num_steps, double dt, int taylor_kmax,
                                     const float* vel, const float* rho, const int* K, const double* mterm,
                                     float* mu, const float* base, double alpha, double beta, float* out,
                                     void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* STC_H */
