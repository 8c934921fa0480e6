/*
 * sim.h -- C ABI of the GB300 fully implicit reservoir Newton step.
 *
 * Method (arXiv:1606.00548): oil-water (Eq. 5) and three-component black-oil
 * (Eq. 3-4) mass conservation with Darcy flux (Eq. 1-2), BHP-controlled
 * Peaceman wells (Eq. 6-7), backward Euler (Eq. 10) and cell-centred
 * two-point transmissibilities (Eq. 11) on a structured 7-point grid,
 * solved by inexact Newton (Algorithm 1) whose linear systems (Eq. 16) are
 * solved by CPR-preconditioned FGMRES (Sec. 2.4.2: quasi-IMPES decoupling,
 * AMG on the pressure block, block ILU(0) / block-Jacobi second stage).
 *
 * Conventions
 *   - cell index i = ix + nx*(iy + ny*iz), x fastest; N = nx*ny*nz.
 *   - b = unknowns (= equations) per cell: 2 (oil-water) or 3 (black oil).
 *     Unknown order (p, Sw, x3) with x3 = Sg (saturated cell) or pb
 *     (undersaturated cell); equation order (water, oil, gas).
 *   - vectors on the device are component-major: v[c*N + i] (FP64).
 *   - Jacobian blocks: J[((d*b + r)*b + c)*N + i] = dR_r(i)/dx_c(nbr_d(i)),
 *     d = 0 centre, 1 -x, 2 +x, 3 -y, 4 +y, 5 -z, 6 +z; blocks that point
 *     outside the grid are zero.
 *   - units: bar, m, day, mD, cP, kg/m3; residuals in kg/day.
 *
 * Ownership and errors
 *   - the library owns every device buffer it allocates; callers own their
 *     host arrays (copied on entry) and any device pointers they pass.
 *   - every call returns sim_status; nothing aborts or throws across the ABI
 *     and no kernel traps.  The first error is kept (sticky) together with a
 *     message, readable with sim_last_error(), until sim_clear_error().
 *   - all work is ordered on the CUDA stream given to sim_create (NULL: the
 *     library creates its own).  Calls that return host data synchronise it.
 */
#ifndef GB300_SIM_H
#define GB300_SIM_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SIM_OK = 0,
    SIM_EINVAL = 1,            /* bad argument or inconsistent input */
    SIM_ENOMEM = 2,            /* device allocation failed */
    SIM_ECUDA = 3,             /* CUDA runtime error */
    SIM_ENAN = 4,              /* non-finite residual or update */
    SIM_ENOCONV_LINEAR = 5,    /* FGMRES hit its restart limit */
    SIM_ENOCONV_NEWTON = 6,    /* Newton failed and the time-step cuts ran out */
    SIM_ETIMEOUT = 7,          /* a bounded device wait gave up */
    SIM_ELIMIT = 8             /* a size limit of the implementation was exceeded */
} sim_status;

typedef struct sim sim_t;

/* structured grid (Sec. 2.4: structured grids, finite differences) */
typedef struct {
    int32_t nx, ny, nz;
    double dx, dy, dz;          /* cell size, m */
    double top_depth;           /* depth of the top face, m (depth positive down) */
} sim_grid;

/* rock: host arrays of N doubles, copied at sim_create */
typedef struct {
    const double *kx, *ky, *kz; /* absolute permeability, mD */
    const double *poro;         /* porosity at p_ref */
    double c_rock, p_ref;       /* phi = poro (1 + c_rock (p - p_ref)) */
} sim_rock;

/* fluid (Sec. 2.1-2.2).  model 2: rho = rho_ref exp(c (p - p_ref)), constant
   viscosities.  model 3: tabulated Bo, Rs, mu_o, Bg, mu_g (piecewise linear,
   linear extrapolation), undersaturated Bo = Bo(pb)(1 - bo_c_us (p - pb)),
   mu_o = mu_o(pb)(1 + muo_c_us (p - pb)), 1/Bw = 1 + bw_c (p - bw_pref).
   Relative permeability: Corey curves, Stone II for k_ro (model 3). */
typedef struct {
    int32_t model;
    double rho_w_ref, rho_o_ref, c_w, c_o, mu_w, mu_o;
    double rho_ws, rho_os, rho_gs, bw_c, bw_pref, bo_c_us, muo_c_us;
    int32_t npvt;               /* table nodes (2..64) */
    const double *pvt_p, *pvt_bo, *pvt_rs, *pvt_muo, *pvt_bg, *pvt_mug;
    double swc, sor, sgc, sorg, nw, now, ng, nog;
    double cnv_rho[3];          /* per-component density scale of the CNV test */
} sim_fluid;

#define SIM_WELL_PRODUCER 0
#define SIM_WELL_WATER_INJECTOR 1
#define SIM_WELL_BHP 0          /* fixed bottom-hole pressure (Eq. 7) */
#define SIM_WELL_WATER_RATE 1   /* fixed water rate (Eq. 8); producers and injectors */
#define SIM_WELL_OIL_RATE 2     /* fixed oil rate (Eq. 9); producers only */
/* vertical well perforated in layers k_top..k_bot (Sec. 2.3).  Under a rate
   control the well's bottom-hole pressure is an unknown of the Newton system
   (Eq. 16) and bhp is its initial guess.  No two perforations (of any wells)
   may share a cell. */
typedef struct {
    int32_t i, j, k_top, k_bot, type;
    double bhp;                 /* bar, at the depth of the top perforation */
    double r_w, skin;           /* Peaceman well radius (m) and skin */
    int32_t control;            /* SIM_WELL_BHP, SIM_WELL_WATER_RATE or SIM_WELL_OIL_RATE */
    double rate;                /* target component mass rate summed over the perforations,
                                   kg/day, positive into the reservoir (rate controls) */
} sim_well;

#define SIM_PRECOND_NONE 0
#define SIM_PRECOND_BJACOBI 1
#define SIM_PRECOND_CPR 2
#define SIM_STAGE2_BJACOBI 0
#define SIM_STAGE2_ILU0_RB 1
#define SIM_PRECISION_FP64 0
#define SIM_PRECISION_MIXED 1   /* FP32 preconditioner + FP32 Krylov directions Z */
#define SIM_DECOUPLE_QI 0       /* quasi-IMPES: pressure row J_0 - d_ps D_ss^-1 J_s (Sec. 3.2) */
#define SIM_DECOUPLE_ABF 1      /* alternate block factorisation: D_ii^-1 J (Sec. 3.2) */
#define SIM_KRYLOV_FGMRES 0     /* right-preconditioned FGMRES(gmres_m), restarts */
#define SIM_KRYLOV_BICGSTAB 1   /* right-preconditioned BiCGSTAB (the paper's solver, Sec. 4) */
#define SIM_FORCING_FIXED 0     /* theta = lin_tol on every Newton iteration */
#define SIM_FORCING_EW1 1       /* Eq. (14) choice 1: ||b^l - r^{l-1}|| / ||b^{l-1}|| */
#define SIM_FORCING_EW2 2       /* Eq. (14) choice 2: | ||b^l|| - ||r^{l-1}|| | / ||b^{l-1}|| */
#define SIM_FORCING_EW3 3       /* Eq. (14) choice 3: gamma (||b^l|| / ||b^{l-1}||)^beta */

typedef struct {
    double newton_tol;          /* CNV tolerance */
    int32_t newton_max;         /* Newton iterations per time step */
    double lin_tol;             /* forcing term theta: ||b - J dx|| <= theta ||b|| */
    int32_t gmres_m, gmres_max_restarts;   /* 1 <= m <= 32 */
    int32_t precond, stage2;
    double amg_theta;           /* strength threshold */
    int32_t amg_rounds;         /* handshake rounds per matching pass */
    int32_t amg_coarse_max;     /* coarsest level size (<= 1024) */
    int32_t amg_max_levels;
    double chop_ds, chop_dp;    /* Appleyard chop limits */
    int32_t max_cuts;           /* time-step halvings per sim_step */
    int32_t precision;          /* SIM_PRECISION_* */
    int32_t amg_cycles;         /* V-cycles per stage-P application (>= 1) */
    int32_t graphs;             /* 1: replay each FGMRES restart cycle as a CUDA graph */
    int32_t decouple;           /* SIM_DECOUPLE_*: left scaling applied before the CPR stages */
    int32_t cpr_stages;         /* 2: stage P then stage F; 3: F, P, F (CPR-FPF) */
    int32_t krylov;             /* SIM_KRYLOV_*: outer Krylov method of every linear solve */
    int32_t lin_max_iter;       /* BiCGSTAB iteration limit per solve (>= 1) */
    int32_t forcing;            /* SIM_FORCING_*: forcing term theta_l of the Newton loop */
    double ew_gamma, ew_beta;   /* constants of forcing choice 3 (gamma in (0, 1], beta > 0) */
    double theta_max;           /* theta of a Newton solve's first iteration and upper bound (lin_tol..1) */
    int32_t fused_coarse;       /* 1: the coarse AMG levels of a V-cycle run in one cluster launch */
    int32_t orth;               /* FGMRES Gram-Schmidt: 0 CGS2 (always two passes), 1 the second pass only
                                   when the first removed more than half of ||w||^2 */
} sim_options;

typedef struct {
    int32_t iterations, restarts, converged;
    double b_norm, r_norm;      /* ||b||, true ||b - J x|| at exit */
} sim_linear_info;

/* Per-phase figures of a Newton call: device time between CUDA events
   recorded on the handle's stream (microseconds) and the algorithmic bytes of
   the phase, i.e. what its kernels must read and write at least once, from
   the sizes alone (not measured traffic):
     assembly  read x, the step's accumulation, T, porosity; write R, J:
               N (7 b^2 + 3 b + 4) 8
     setup     decoupling reads J, writes Ahat (t bytes per value: 8 FP64,
               4 mixed) and A_p; ILU(0) / block Jacobi reads Ahat, writes the
               inverted diagonal blocks; each coarsening reads its level's
               matrix four times and writes the next level and its map:
               N (7 b^2 (8 + 2 t) + 7 * 8 + b^2 t) + sum_l (4 w_l n_l 12 + w_{l+1} n_{l+1} 12 + 4 n_l)
     solve     per FGMRES iteration with basis vectors 0..j: the product
               (7 b^2 + b) 8 N + b N tz (tz: the direction's precision), one
               CPR application (restriction, V-cycle: three passes over each
               level's matrix, stage F: pressure columns of Ahat, the ILU
               blocks, vectors), the Gram-Schmidt passes (3 (j + 1) + 7) n 8
               (n = b N); per restart the solution update, one product and the
               residual; BiCGSTAB: two products, two applications and 12
               vector passes per iteration
     update    read dx, x; write x: 3 b N 8
   The newton_* counts of sim_step_info sum over substeps; the phase fields
   sum over every Newton iteration of the call (failed substeps included). */
typedef struct {
    double assemble_us, setup_us, solve_us, update_us;
    double assemble_bytes, setup_bytes, solve_bytes, update_bytes;
} sim_phase_info;

typedef struct {
    int32_t newton_iterations;  /* linear solves performed */
    int32_t linear_iterations;
    int32_t converged;
    int32_t linear_failures;
    double cnv;
    sim_phase_info phase;
    /* final true relative residual ||b - J dx|| / ||b|| of the linear solve
       (the largest over the solves of a sim_newton_solve call); 0 without a solve */
    double lin_residual;
} sim_newton_info;

typedef struct {
    int32_t cuts, newton_iterations, linear_iterations, substeps, ok;
    sim_phase_info phase;
    /* mass-balance error of the step (Eq. 3, conservation): the largest over its
       accepted substeps and the components c of |M_c(end) - M_c(start) - dt q_c|
       / sum_c M_c(end), with M the component masses in place and q the wells'
       net mass rate into the reservoir */
    double mb_error;
} sim_step_info;

typedef struct {
    int64_t kernel_launches;    /* kernels launched by this handle so far */
    int64_t newton_iterations, linear_iterations;
    int64_t device_bytes;       /* device memory held by the handle */
    int32_t spmv_block, amg_block;   /* launch shapes in use (see sim_autotune) */
    int32_t stage_block;             /* threads per block of the stage-F sweeps */
} sim_stats;

/* Create a simulator (copies every host array).  Validates sizes, table
   monotonicity, well positions (no two perforations in one cell).
   cuda_stream: a cudaStream_t or NULL.  *out receives the handle; on error
   *out is NULL and the message is printed by sim_last_error(NULL). */
sim_status sim_create(const sim_grid *g, const sim_rock *r, const sim_fluid *f,
                      const sim_well *w, int32_t nwells, const sim_options *o,
                      void *cuda_stream, sim_t **out);
void sim_destroy(sim_t *s);

/* Accepted state (host arrays of N): pressure, Sw, x3 (Sg or pb), phase
   (1 saturated, 0 undersaturated; ignored for oil-water).  set_state also
   zeroes the cumulative well masses and starts a new time step from it.
   A non-finite value in p, Sw or x3 returns SIM_ENAN (sticky) and leaves
   the handle's state as it was.  get_state followed by set_state on a handle
   of the same case resumes a run: the following steps reproduce an
   uninterrupted run bit for bit (BHP-controlled wells; the BHP unknowns of
   rate-controlled wells are restored with sim_set_well_bhp). */
sim_status sim_set_state(sim_t *s, const double *p, const double *sw, const double *x3, const int8_t *phase);
sim_status sim_get_state(sim_t *s, double *p, double *sw, double *x3, int8_t *phase);

/* Advance by dt days (Algorithm 1 per step; a failed Newton solve halves the
   step, at most max_cuts times). */
sim_status sim_step(sim_t *s, double dt, sim_step_info *info);
/* Newton loop of Algorithm 1 for one step of dt from the accepted state
   (no cuts; on failure the iterate is left where Newton stopped). */
sim_status sim_newton_solve(sim_t *s, double dt, sim_newton_info *info);
/* One Newton iteration at the current iterate: assemble, test CNV, solve
   J dx = -R, update.  info->converged = 1 means CNV already met (no solve). */
sim_status sim_newton_step(sim_t *s, double dt, sim_newton_info *info);
/* Accept the current iterate as the converged state of a time step of
   length dt: the well rates of the last assembly are added to the cumulative
   well masses (times dt) and the next step starts from it (its accumulation
   terms are formed).  For callers that drive Newton themselves with
   sim_newton_step (the converged x of Algorithm 1 is the step's solution);
   sim_step does this after every converged substep. */
sim_status sim_accept_step(sim_t *s, double dt);
/* Solve J x = b with the current Jacobian to ||b - J x|| <= lin_tol ||b||
   (FGMRES or BiCGSTAB per options.krylov, with the configured
   preconditioner).  b_dev, x_dev: device pointers, N*b doubles each,
   component-major; they may not alias.  Returns SIM_ENOCONV_LINEAR (not
   sticky) when the restart / iteration limit is hit; x_dev then holds the
   last iterate.  In the Newton loop (sim_step, sim_newton_solve) the
   tolerance is the forcing term of options.forcing instead. */
sim_status sim_linear_solve(sim_t *s, const double *b_dev, double *x_dev, sim_linear_info *info);

/* ---- inspection entry points (used by the parity tests) ---- */
/* current Newton iterate, host arrays: x[b*N] component-major, phase[N];
   a non-finite x returns SIM_ENAN (sticky) with the iterate unchanged */
sim_status sim_set_iterate(sim_t *s, const double *x, const int8_t *phase);
sim_status sim_get_iterate(sim_t *s, double *x, int8_t *phase);
/* residual and Jacobian at the current iterate for step length dt */
sim_status sim_assemble(sim_t *s, double dt);
sim_status sim_get_residual(sim_t *s, double *R);       /* host, b*N */
sim_status sim_get_jacobian(sim_t *s, double *J);       /* host, 7*b*b*N */
sim_status sim_set_jacobian(sim_t *s, const double *J); /* host, 7*b*b*N */
sim_status sim_cnv(sim_t *s, double dt, double *cnv);
/* y = J x, device pointers (component-major, FP64) */
sim_status sim_spmv(sim_t *s, const double *x_dev, double *y_dev);
sim_status sim_precond_setup(sim_t *s);
sim_status sim_precond_apply(sim_t *s, const double *r_dev, double *z_dev);
/* quasi-IMPES weights w[b*N] and pressure-block coefficients ap[7*N] */
sim_status sim_get_qi(sim_t *s, double *w, double *ap);
int32_t sim_amg_levels(sim_t *s);
/* level size and ELL width (level 0 is the 7-point stencil: width 7) */
sim_status sim_amg_level_info(sim_t *s, int32_t level, int32_t *n, int32_t *width);
/* fine -> coarse aggregate map of a level (n ints; not for the coarsest) */
sim_status sim_amg_level_agg(sim_t *s, int32_t level, int32_t *agg);
/* ELL matrix of a level >= 1: col[width*n] (-1 padding), val[width*n],
   entry k of row i at k*n + i, columns ascending */
sim_status sim_amg_level_ell(sim_t *s, int32_t level, int32_t *col, double *val);
sim_status sim_component_mass(sim_t *s, double *m3);
sim_status sim_cumulative_well_mass(sim_t *s, double *m3);
sim_status sim_well_rates(sim_t *s, double *q3);
/* Well unknowns (Eq. 16).  Every well has a bottom-hole pressure p_h; under
   BHP control its equation is p_h - c = 0, under a rate control the summed
   component rate minus the target.  The Newton system
       [A    A_pw] [dx ]     [R  ]
       [A_wp A_ww] [dph] = - [R_w]
   is solved through S = A - A_pw A_ww^-1 A_wp (A_ww diagonal): sim_spmv and
   sim_linear_solve act with S, and the CPR preconditioner is built from S
   restricted to the 7-point block pattern.  Host arrays: bhp, Rw, Aww
   [nwells]; Apw, Awp [nperf][b] (perforations top to bottom, wells in input
   order); q [nwells][3] component rates at the last assembly (kg/day). */
int32_t sim_perforations(sim_t *s);
sim_status sim_get_well_bhp(sim_t *s, double *bhp);
sim_status sim_set_well_bhp(sim_t *s, const double *bhp);
sim_status sim_well_component_rates(sim_t *s, double *q);
sim_status sim_get_well_system(sim_t *s, double *Rw, double *Apw, double *Awp, double *Aww);
/* replaces the border blocks of the last assembly (tests feed identical
   systems to two implementations, as with sim_set_jacobian) */
sim_status sim_set_well_system(sim_t *s, const double *Rw, const double *Apw, const double *Awp, const double *Aww);
sim_status sim_get_stats(sim_t *s, sim_stats *st);
int32_t sim_block_size(sim_t *s);

/* CNV convergence measure for callers that cannot allocate device memory.
   The paper has no counterpart: this is a deployment aid, not part of the
   method.  Some callers cannot call cudaMalloc -- their device memory belongs
   to another allocator (a framework's caching allocator or a fixed, pre-sized
   arena), or they run a time-critical Newton loop where an allocation's
   latency and the device synchronisation it may imply are not acceptable.
   This entry point needs no handle and allocates nothing: it computes the
   same quantity as sim_cnv, max_i,c |R_c(i)| dt / (poro_i dx dy dz cnv_rho_c),
   from buffers the caller owns.
     R_dev     device, b*N doubles, component-major residual (kg/day)
     poro_dev  device, N doubles, porosity at the reference pressure
     cnv_rho   host, b doubles (> 0), per-component density scale
     cnv_dev   device, 1 double: receives the result (NaN if any R is NaN)
     cuda_stream  cudaStream_t or NULL; the call is asynchronous on it.
   Scratch: a library-owned static device array of 457 doubles (3,656
   bytes: 456 per-block partial maxima plus a ticket word), held by every GPU
   that loads the library until the process exits; no cudaMalloc / cudaFree
   is ever made.  Every call looks up that array's device address
   (cudaGetSymbolAddress, no allocation) on the caller's current device, so
   a device reset between calls leaves no stale address behind; the first
   call on a device may also load the library's device code, so make that
   first call before any stream capture.  All calls share the array and it keeps the
   last call's contents (the ticket is cleared by each call): calls that
   overlap on the GPU (other streams, other threads) race and must not
   overlap.  Limits: b in {2, 3}; N*b < 2^31 (32-bit indexing), larger
   grids fail with SIM_ELIMIT.  Errors are reported through the return code
   and sim_last_error(NULL). */
sim_status sim_cnv_noalloc(int32_t nx, int32_t ny, int32_t nz, double dx, double dy, double dz, int32_t b,
                           const double *R_dev, const double *poro_dev, const double *cnv_rho, double dt,
                           double *cnv_dev, void *cuda_stream);

/* Autotuner: assembles at the current iterate for step dt, then times the
   block SpMV with blocks of 64..512 threads and one CPR application with
   AMG level kernels of 64..256 threads and stage-F sweeps of 32..256
   threads, and keeps the fastest shapes for this handle.  Results do not
   depend on the shapes (each row's arithmetic is the same); only speed does. */
sim_status sim_autotune(sim_t *s, double dt);
/* The same with the shapes cached in a JSON file (created if absent), one
   entry per (block size, precision, grid dimensions):
     {"b3_fp64_100x100x20": {"spmv": 256, "amg": 128, "stage": 64}, ...}
   An entry for this handle's key is applied without timing (*from_cache = 1);
   otherwise sim_autotune runs and its shapes are written into the file
   (*from_cache = 0; the file is replaced by rename, so readers never see a
   partial one).  from_cache may be NULL. */
sim_status sim_autotune_cached(sim_t *s, double dt, const char *json_path, int32_t *from_cache);
/* Device time of one hot operation (measurement only; no paper counterpart):
   `reps` launches on the handle's stream, each bracketed by CUDA events and
   preceded by a 256 MB write that evicts its operands from L2.  which = 0: the
   product y = S x of sim_spmv; 1: one CPR application as in sim_precond_apply
   (set up first if needed).  Operands are the handle's own work vectors
   (zeroed), so the caller's data are untouched; the eviction buffer is
   allocated and freed inside the call.  which = 2: one FGMRES Arnoldi
   orthogonalisation step (the Gram-Schmidt passes against min(16, m) basis
   vectors and the normalisation of the new one), as inside a restart cycle.
   *us = average microseconds per launch. */
sim_status sim_time_op(sim_t *s, int32_t which, int32_t reps, double *us);
/* Run report (no paper counterpart; the paper reports steps, Newton and
   linear iterations and times per run): a JSON object with the grid, model,
   options, the run's counters (time steps, failed steps, accepted substeps,
   cuts, simulated days, Newton and linear iterations, linear solves that hit
   their limit, kernel launches), each phase's device time summed over every
   Newton call of the handle (microseconds, CUDA events) with its algorithmic
   bytes and the GB/s they imply, the device memory held and the launch shapes.
   buf receives the text with its terminating NUL when cap >= *len + 1;
   otherwise the call returns SIM_EINVAL (not sticky) with *len set, so that
   buf = NULL, cap = 0 queries the size. */
sim_status sim_run_report(sim_t *s, char *buf, int64_t cap, int64_t *len);

/* ---- ensemble (no paper counterpart) ----
   Independent simulators (e.g. geological realisations on grids of different
   sizes) advanced together on one GPU.  The batch does not own the members;
   members must own distinct CUDA streams and live on the current device.

   SIM_BATCH_LOCKSTEP (the default where every member allows it: the same
   block size, precision and solver options, two-stage CPR with one V-cycle,
   FGMRES with a fixed forcing term, no learned stage, no rate-controlled
   wells, at most 16 AMG levels): the members' Newton loops advance in
   rounds.  Per round each member in its step assembles and tests CNV
   (accepting converged substeps and halving failed ones, as sim_step does)
   and sets up its preconditioner -- concurrently, one worker thread and
   stream per member -- and then one batched FGMRES solves every member's
   Newton system at once: each Krylov operation (the block SpMV, each CPR
   stage, each Gram-Schmidt pass) is a single launch over all members, a
   restart cycle is one CUDA graph on the batch's own stream, and a member
   whose solve has converged drops out of the remaining launches.  Each
   member computes what its own sim_step computes.
   SIM_BATCH_CONCURRENT: each member's sim_step runs on its own stream from
   a pool worker (the members' kernels overlap on the device). */
#define SIM_BATCH_LOCKSTEP 0
#define SIM_BATCH_CONCURRENT 1
typedef struct sim_batch sim_batch_t;
/* nthreads <= 0: min(n, 64) worker threads */
sim_status sim_batch_create(int32_t n, sim_t *const *members, int32_t nthreads, sim_batch_t **out);
void sim_batch_destroy(sim_batch_t *b);
/* SIM_EINVAL for an unknown mode, or LOCKSTEP when the members do not allow it */
sim_status sim_batch_set_mode(sim_batch_t *b, int32_t mode);
int32_t sim_batch_mode(sim_batch_t *b);
/* one time step dt[k] for every member k; infos / member_status (n
   entries, may be NULL) receive each member's result; returns the first
   non-OK member status.  In lockstep mode the solve time of a round is
   counted in the phase info of every member that solved in it. */
sim_status sim_batch_step(sim_batch_t *b, const double *dt, sim_step_info *infos, sim_status *member_status);
/* lockstep rounds and member solves so far, and kernels launched by the
   batched solves (graph nodes included) */
sim_status sim_batch_stats(sim_batch_t *b, int64_t *rounds, int64_t *solves, int64_t *launches);
const char *sim_batch_last_error(sim_batch_t *b);
/* host seconds spent so far in the lockstep phases: the members' Newton phases
   (assembly, CNV test, accepting or cutting, CPR set-up), the batched solves,
   and the updates */
sim_status sim_batch_phase_seconds(sim_batch_t *b, double *newton, double *solve, double *update);

/* ---- learned pressure stage (no paper counterpart) ----
   A 3-D convolutional network: 4 layers of 3x3x3 kernels (zero padding),
   channels 4 -> 16 -> 16 -> 16 -> 1, ReLU between layers; BF16 weights and
   activations, FP32 accumulation on the tensor cores (forward and data
   gradient on tcgen05 with tensor-memory accumulators and TMA-staged inputs,
   weight gradient on mma.sync), FP32 master weights updated by Adam on the
   device.  Inputs per cell (x [N][4] FP32,
   cell-major): the normalised pressure residual and three standardised log
   face-transmissibility sums; output y [N] FP32: a normalised pressure
   correction.  Parameters as one flat FP32 array: for each layer, W[27][cin][cout]
   (tap t = (dz+1)*9 + (dy+1)*3 + (dx+1)) then b[cout]. */
typedef struct sim_net sim_net_t;
sim_status sim_net_create(int32_t nx, int32_t ny, int32_t nz, uint64_t seed, void *cuda_stream, sim_net_t **out);
void sim_net_destroy(sim_net_t *n);
int64_t sim_net_param_count(sim_net_t *n);
sim_status sim_net_set_params(sim_net_t *n, const float *params);   /* host array */
sim_status sim_net_get_params(sim_net_t *n, float *params);         /* host array */
/* y = net(x); device pointers, asynchronous on the net's stream */
sim_status sim_net_forward(sim_net_t *n, const float *x_dev, float *y_dev);
/* mean-squared-error loss against target [N] and its gradient (host, flat like the parameters; may be NULL) */
sim_status sim_net_loss_grad(sim_net_t *n, const float *x_dev, const float *target_dev, double *loss, float *grads);
/* one Adam step (beta 0.9 / 0.999) on the loss; loss may be NULL (then no synchronisation) */
sim_status sim_net_train_step(sim_net_t *n, const float *x_dev, const float *target_dev, float lr, double *loss);
const char *sim_net_last_error(sim_net_t *n);
/* Device time of one convolution kernel on the net's grid (measurement only):
   `reps` launches on the net's stream, each bracketed by CUDA events and
   preceded by a 256 MB write that evicts L2.  which = 0: the forward
   convolution of hidden layer 2 (16 -> 16 channels, bias and ReLU fused);
   1: the weight gradient of that layer (the kernel and its fold of the
   per-CTA partials); 2: its data gradient.  The operands are the net's own
   buffers: activations of the last forward pass (zero before any) and
   gradient buffers, which the call overwrites.  *us = average microseconds per
   launch; SIM_EINVAL for a bad which or reps < 1. */
sim_status sim_net_time_conv(sim_net_t *n, int32_t which, int32_t reps, double *us);
/* Testing hook for the convolutions' bounded waits (no paper counterpart): in
   the next forward pass, CTA 0 of the first convolution does not copy staged
   slab `slab` of its sequence (0 = the first) and does not arm its barrier, so
   the MMA thread's wait for it gives up after about 2 s; the CTA then stops
   its roles, lets its copies land, frees its tensor memory and sets the
   status word, and that call returns SIM_ETIMEOUT (sticky for this net).  No
   fault and no hang: every wait is bounded.  SIM_EINVAL for slab < 0. */
sim_status sim_net_inject_stall(sim_net_t *n, int32_t slab);
/* Use net (same grid; not owned, must outlive its use) as an extra CPR stage
   after the AMG V-cycles: the pressure residual left by stage P is normalised,
   the network's correction c, scaled by the minimal-residual step
   alpha = (A_p c . r') / (A_p c . A_p c) so that it never increases the 2-norm
   of that residual, is added to the pressure update.  enable = 0
   turns it off.  A solve whose first restart cycle reduces the residual by
   less than 10x (or turns non-finite) is redone with plain CPR. */
sim_status sim_set_learned_stage(sim_t *s, sim_net_t *net, int32_t enable);
/* Training pairs from the last linear solve: for the first k Krylov vectors
   v_j of its last restart cycle (k <= its iterations + 1), with f = the
   decoupled pressure residual (L v_j)_p and e_p one stage-P V-cycle on it,
   x_j = features of r' = f - A_p e_p (the residual the learned stage sees,
   normalised by its RMS) and y_j = A_p^-1 r' approximated by eight V-cycles
   of iterative refinement (normalised by its own RMS).  x_dev [k][N][4],
   y_dev [k][N] (device, FP32).  k outside 1..sim_learned_available(s)
   returns SIM_EINVAL without making the handle's error sticky. */
sim_status sim_learned_pairs(sim_t *s, int32_t k, float *x_dev, float *y_dev);
/* Krylov vectors available to sim_learned_pairs after the last solve */
int32_t sim_learned_available(sim_t *s);
/* number of solves that fell back to plain CPR */
int64_t sim_learned_fallbacks(sim_t *s);

/* Diagnostics (no paper counterpart): FP64 and FP32 fused-multiply-add rates
   of the current device, measured with independent FMA chains (8 or 16 per
   thread, 4 or 8 blocks of 256 threads per SM; the best shape is reported)
   and CUDA events; the roofline of the FP64-bound kernels is taken against
   the FP64 rate.  Allocates a small scratch buffer; synchronises the device. */
sim_status sim_probe_fma_rates(double *fp64_fma_per_s, double *fp32_fma_per_s);
/* The FP64 pipe's rate per clock: the best FP64 shape of the probe above,
   with the SM clock it ran at (clock64 cycles against %globaltimer
   nanoseconds over each block's loop, median over blocks).  *fma_per_s: FMAs
   per second; *sm_mhz: that clock; *fma_per_clk_per_sm = fma_per_s / (SMs x
   clock), the measured FMAs per clock per SM, which times the SMs and the
   clock of a run gives that run's FP64 peak. */
sim_status sim_probe_fp64_pipe(double *fma_per_s, double *sm_mhz, double *fma_per_clk_per_sm);

const char *sim_last_error(sim_t *s);   /* s may be NULL: last create error */
void sim_clear_error(sim_t *s);

#ifdef __cplusplus
}
#endif
#endif
