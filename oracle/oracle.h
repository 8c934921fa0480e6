/*
 * CPU oracle for the fully implicit oil-water / black-oil Newton step.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow, FP64 statement
 * of what the GPU path computes.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code, header or table
 * with the CUDA library; the two meet only through the seeded input arrays.
 *
 * Followed passages (paper sections / equations):
 *   Eq. (1)-(3)  black-oil mass conservation with Darcy flux
 *   Eq. (4)      closure relations (capillary pressure taken as zero, Sec. 4.1)
 *   Eq. (5)      two-phase oil-water model
 *   Eq. (6)      well rate per perforation, Peaceman well index (Sec. 2.3)
 *   Eq. (7)      fixed bottom-hole pressure control
 *   Eq. (10)     backward Euler in time
 *   Eq. (11)     cell-centred transmissibility on a structured grid
 *   Algorithm 1  inexact Newton with forcing term theta
 *   Eq. (16)     pressure / saturation block ordering of the Jacobian
 *   Sec. 2.4.2   CPR-type two-stage preconditioning with quasi-IMPES
 *                decoupling and AMG on the pressure block
 * Readings of passages the paper leaves open are stated where they are used.
 *
 * Layouts (oracle-private): vectors interleaved per cell, v[i*b + c];
 * Jacobian blocks J[((i*7 + d)*b + r)*b + c], d = 0 centre, 1 -x, 2 +x,
 * 3 -y, 4 +y, 5 -z, 6 +z.  Cell index i = ix + nx*(iy + ny*iz).
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

typedef struct {
    int32_t nx, ny, nz;
    double dx, dy, dz, top_depth;
    int32_t model;                 /* 2 oil-water, 3 black oil */
    const double *kx, *ky, *kz, *poro;
    double c_rock, p_ref;
    /* oil-water fluid: rho = rho_ref * exp(c (p - p_ref)) */
    double rho_w_ref, rho_o_ref, c_w, c_o, mu_w, mu_o;
    /* black-oil fluid */
    double rho_ws, rho_os, rho_gs, bw_c, bw_pref, bo_c_us, muo_c_us;
    int32_t npvt;
    const double *pvt_p, *pvt_bo, *pvt_rs, *pvt_muo, *pvt_bg, *pvt_mug;
    /* relative permeability (Corey two-phase curves, Stone II for three phases) */
    double swc, sor, sgc, sorg, nw, now, ng, nog;
    /* wells: type 0 producer, 1 water injector; BHP control */
    int32_t nwells;
    const int32_t *w_i, *w_j, *w_k0, *w_k1, *w_type;
    const double *w_bhp, *w_rw, *w_skin;
    /* scaling densities of the CNV convergence test, per component */
    double cnv_rho[3];
    /* nonlinear / linear solver options */
    double newton_tol; int32_t newton_max;
    double lin_tol; int32_t gmres_m, gmres_max_restarts;
    int32_t precond;               /* 0 none, 1 block-Jacobi, 2 CPR */
    int32_t stage2;                /* CPR second stage: 0 block-Jacobi, 1 red-black block ILU(0),
                                      2 natural-order block ILU(0) (a study of the ordering; the CUDA
                                      path has 0 and 1) */
    double amg_theta; int32_t amg_rounds, amg_coarse_max, amg_max_levels;
    double chop_ds, chop_dp; int32_t max_cuts;
    int32_t amg_cycles;            /* V-cycles per stage-P application (>= 1) */
    int32_t decouple;              /* 0 quasi-IMPES, 1 ABF (alternate block factorisation) */
    int32_t cpr_stages;            /* 2: P then F; 3: F, P, F (CPR-FPF) */
    int32_t krylov;                /* 0 FGMRES(m), 1 BiCGSTAB (the paper's solver, Sec. 4) */
    int32_t lin_max_iter;          /* BiCGSTAB iteration limit per solve */
    int32_t forcing;               /* 0: theta = lin_tol; 1, 2, 3: the choices of Eq. (14) */
    double ew_gamma, ew_beta;      /* constants of choice 3 */
    double theta_max;              /* theta of the first Newton iteration and upper safeguard */
    /* well controls (NULL: every well under BHP control).  Control 0: fixed
       BHP (Eq. 7); 1: fixed water rate, 2: fixed oil rate (Eq. 8-9), the
       target being the component's mass rate summed over the perforations,
       kg/day, positive into the reservoir; the BHP is then an unknown whose
       initial guess is w_bhp.  Injectors take water-rate control only. */
    const int32_t *w_ctrl;
    const double *w_rate;
    int32_t orth;                  /* FGMRES: 0 CGS2; 1 second Gram-Schmidt pass only when the first
                                      removed more than half of ||w||^2 (Daniel et al. 1976) */
} ora_input;

typedef struct {
    int32_t iterations;            /* FGMRES inner iterations or BiCGSTAB iterations */
    int32_t restarts;
    int32_t converged;
    double b_norm, r_norm;         /* ||b||, true ||b - A x|| at exit */
} ora_lin_info;

typedef struct {
    int32_t newton_iterations;     /* linear solves performed */
    int32_t linear_iterations;
    int32_t converged;
    int32_t linear_failures;
    double cnv;                    /* CNV at exit */
} ora_newton_info;

typedef struct {
    int32_t cuts, newton_iterations, linear_iterations, substeps, ok;
} ora_step_info;

typedef struct ora_sim ora_sim;

ora_sim *ora_create(const ora_input *in);
void ora_destroy(ora_sim *s);
int ora_block_size(const ora_sim *s);
void ora_set_state(ora_sim *s, const double *p, const double *sw, const double *x3, const int8_t *ph);
void ora_get_state(const ora_sim *s, double *p, double *sw, double *x3, int8_t *ph);
void ora_set_iterate(ora_sim *s, const double *x, const int8_t *ph);
void ora_get_iterate(const ora_sim *s, double *x, int8_t *ph);
void ora_assemble(ora_sim *s, double dt);
void ora_get_residual(const ora_sim *s, double *R);
void ora_get_jacobian(const ora_sim *s, double *J);
void ora_set_jacobian(ora_sim *s, const double *J);
double ora_cnv(const ora_sim *s, double dt);
void ora_spmv(const ora_sim *s, const double *x, double *y);
void ora_precond_setup(ora_sim *s);
void ora_precond_apply(ora_sim *s, const double *r, double *z);
int ora_linear_solve(ora_sim *s, const double *b, double *x, ora_lin_info *info);
int ora_newton_step(ora_sim *s, double dt, ora_newton_info *info);
int ora_newton_solve(ora_sim *s, double dt, ora_newton_info *info);
int ora_step(ora_sim *s, double dt, ora_step_info *info);
/* Well unknowns (Eq. 16): every well has a bottom-hole pressure p_h; a
   BHP-controlled well has the equation p_h - c = 0, a rate-controlled one
   sum_m q_{c,m} - target = 0.  The Newton system
       [A    A_pw] [dx ]     [R  ]
       [A_wp A_ww] [dph] = - [R_w]
   is solved through the Schur complement S = A - A_pw A_ww^-1 A_wp (A_ww is
   diagonal, one entry per well): ora_spmv and ora_linear_solve act with S.
   Layouts: bhp, R_w, A_ww [nwells]; A_pw, A_wp [nperf][b] in the order of the
   wells' perforations (top to bottom, wells in input order). */
void ora_get_well_bhp(const ora_sim *s, double *bhp);
void ora_set_well_bhp(ora_sim *s, const double *bhp);
int ora_perforations(const ora_sim *s);
void ora_get_well_system(const ora_sim *s, double *Rw, double *Apw, double *Awp, double *Aww);
/* component mass rates of each well at the last assembly, [nwells][3] (kg/day, + into the reservoir) */
void ora_well_component_rates(const ora_sim *s, double *q);

/* forcing terms of the last ora_newton_solve: per linear solve theta_l, ||b^l||
   and the true ||b^l - A dx|| at its exit; returns the number of solves (<= max) */
int ora_forcing_history(const ora_sim *s, double *theta, double *b_norm, double *r_norm, int max);
void ora_component_mass(const ora_sim *s, double *m);
void ora_cumulative_well_mass(const ora_sim *s, double *m);
void ora_well_rates(const ora_sim *s, double *q);
void ora_get_qi(const ora_sim *s, double *w, double *ap);
int ora_amg_levels(const ora_sim *s);
int ora_amg_level_n(const ora_sim *s, int level);
int ora_amg_level_nnz(const ora_sim *s, int level);
void ora_amg_level_csr(const ora_sim *s, int level, int32_t *rowptr, int32_t *col, double *val);
void ora_amg_level_agg(const ora_sim *s, int level, int32_t *agg);
void ora_ilu_dinv(const ora_sim *s, double *dinv);

/* standalone pieces used by the pins */
int ora_dense_lu_solve(int n, double *A, double *b);
int ora_match_pass(int n, const int32_t *rowptr, const int32_t *col, const double *val,
                   double theta, int rounds, int32_t *partner);
double ora_props_probe(const ora_input *in, int what, double p, double sw, double x3, int ph, double *grad);
#endif
