/*
 * CPU oracle: plain, sequential, FP64 statement of the fully implicit Newton
 * step of the paper (TEST INFRASTRUCTURE ONLY -- see oracle.h).
 *
 * Everything here is written for a reader checking it against the paper by
 * eye: one loop per mathematical step, no blocking, no fusion, no threads.
 * Derivatives are carried by small forward-mode dual numbers, so the
 * Jacobian is the exact derivative of the residual that the same code
 * evaluates (and the tests pin it against central finite differences).
 *
 * Readings of points the paper leaves open (all shared with the GPU path by
 * definition, not by code):
 *  - z is depth, positive downwards.  The well rate Eq. (6) is used as
 *    printed; the potential of Eq. (4) is taken as Phi = p - rho g z / 1e5
 *    (bar), i.e. the printed "+" is read as the elevation convention, so that
 *    a fluid column at rest has no flow.
 *  - capillary pressure is zero (Sec. 4.1 neglects it).
 *  - two-point flux with harmonic transmissibility, single-point upstream
 *    weighting per phase (upstream = the cell of higher potential; a tie goes
 *    to the lower-index cell), arithmetic mean phase density in the gravity
 *    term.
 *  - Peaceman well index for a vertical well in an anisotropic cell; water
 *    injectors inject water at the cell's total mobility; backflow allowed.
 *  - primary unknowns (p, Sw) for oil-water and (p, Sw, Sg | pb) for black
 *    oil with per-cell variable switching (Sec. 2.4.1 lists the unknowns).
 *  - equations ordered (water, oil, gas) per cell; unknowns (p, Sw, x3).
 *  - CPR: quasi-IMPES weights w = (1, -d_ps D_ss^-1) from the diagonal block;
 *    stage P = one aggregation-AMG V(1,1) cycle on the decoupled pressure
 *    block; stage F = block ILU(0) in red-black order (or block-Jacobi) of
 *    the decoupled matrix applied to the stage-P residual.
 */
#include "oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define GRAV 9.80665
/* Darcy unit factor: q [m3/day] = C k[mD] A[m2] dp[bar] / (mu[cP] L[m]) */
#define DARCY_C (86400.0 * 9.869233e-16 * 1e5 / 1e-3)

/* ------------------------------------------------------------------------ */
/* dual numbers: value + gradient with respect to the cell's own unknowns    */
/* ------------------------------------------------------------------------ */
typedef struct { double v, d[3]; } dual;

static dual dc(double v) { dual r; r.v = v; r.d[0] = r.d[1] = r.d[2] = 0.0; return r; }
static dual dv(double v, int k) { dual r = dc(v); r.d[k] = 1.0; return r; }
static dual dadd(dual a, dual b) { dual r; r.v = a.v + b.v; for (int k = 0; k < 3; k++) r.d[k] = a.d[k] + b.d[k]; return r; }
static dual dsub(dual a, dual b) { dual r; r.v = a.v - b.v; for (int k = 0; k < 3; k++) r.d[k] = a.d[k] - b.d[k]; return r; }
static dual dmul(dual a, dual b) { dual r; r.v = a.v * b.v; for (int k = 0; k < 3; k++) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
static dual ddiv(dual a, dual b) {
    dual r; r.v = a.v / b.v;
    for (int k = 0; k < 3; k++) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v);
    return r;
}
static dual dscale(dual a, double s) { dual r; r.v = a.v * s; for (int k = 0; k < 3; k++) r.d[k] = a.d[k] * s; return r; }
static dual dshift(dual a, double s) { a.v += s; return a; }
static dual dexp(dual a) { dual r; r.v = exp(a.v); for (int k = 0; k < 3; k++) r.d[k] = r.v * a.d[k]; return r; }

/* normalised saturation clipped to [0, 1], raised to the Corey exponent */
static dual corey(dual s, double n) {
    if (s.v <= 0.0) return dc(0.0);
    if (s.v >= 1.0) return dc(1.0);
    dual r; r.v = pow(s.v, n);
    double dr = n * pow(s.v, n - 1.0);
    for (int k = 0; k < 3; k++) r.d[k] = dr * s.d[k];
    return r;
}

/* piecewise-linear table, linear extrapolation beyond the end nodes */
static dual table(const double *xp, const double *yp, int n, dual x) {
    int k = 0;
    while (k + 1 <= n - 2 && x.v >= xp[k + 1]) k++;
    double slope = (yp[k + 1] - yp[k]) / (xp[k + 1] - xp[k]);
    return dshift(dscale(dshift(x, -xp[k]), slope), yp[k]);
}

/* ------------------------------------------------------------------------ */
/* per-cell properties (Eq. 3-5 ingredients)                                 */
/* ------------------------------------------------------------------------ */
enum { PW = 0, PO = 1, PG = 2 };           /* phases */
enum { CW = 0, CO = 1, CG = 2 };           /* components = equation rows */

typedef struct {
    dual acc[3];        /* component mass in the cell, kg */
    dual rho[3];        /* phase mass density, kg/m3 */
    dual mob[3][3];     /* mob[phase][component] = component density in phase * kr / mu */
    dual lamt;          /* total mobility sum kr/mu, 1/cP */
    dual rhow;          /* water mass per water volume */
    dual kr[3];
    dual bo, rs, muo;
    double pv0;
} cellprops;

/* which components each phase carries */
static int carries(int model, int a, int c) {
    if (a == PW) return c == CW;
    if (a == PO) return c == CO || (model == 3 && c == CG);
    if (a == PG) return model == 3 && c == CG;
    return 0;
}

static void eval_props(const ora_input *in, double poro, double vol, const double *x, int ph, cellprops *o) {
    memset(o, 0, sizeof(*o));
    dual P = dv(x[0], 0), SW = dv(x[1], 1);
    dual phi = dscale(dshift(dscale(dshift(P, -in->p_ref), in->c_rock), 1.0), poro);
    dual pv = dscale(phi, vol);
    o->pv0 = poro * vol;
    if (in->model == 2) {
        dual rw = dscale(dexp(dscale(dshift(P, -in->p_ref), in->c_w)), in->rho_w_ref);
        dual ro = dscale(dexp(dscale(dshift(P, -in->p_ref), in->c_o)), in->rho_o_ref);
        dual se = dscale(dshift(SW, -in->swc), 1.0 / (1.0 - in->swc - in->sor));
        dual krw = corey(se, in->nw);
        dual kro = corey(dsub(dc(1.0), se), in->now);
        dual so = dsub(dc(1.0), SW);
        o->acc[CW] = dmul(pv, dmul(rw, SW));
        o->acc[CO] = dmul(pv, dmul(ro, so));
        o->rho[PW] = rw; o->rho[PO] = ro; o->rho[PG] = dc(0.0);
        o->mob[PW][CW] = dscale(dmul(rw, krw), 1.0 / in->mu_w);
        o->mob[PO][CO] = dscale(dmul(ro, kro), 1.0 / in->mu_o);
        o->lamt = dadd(dscale(krw, 1.0 / in->mu_w), dscale(kro, 1.0 / in->mu_o));
        o->rhow = rw;
        o->kr[PW] = krw; o->kr[PO] = kro; o->kr[PG] = dc(0.0);
        return;
    }
    /* black oil */
    dual SG, BO, RS, MUO;
    if (ph) {               /* saturated: x3 = Sg, oil at its bubble point */
        SG = dv(x[2], 2);
        BO = table(in->pvt_p, in->pvt_bo, in->npvt, P);
        RS = table(in->pvt_p, in->pvt_rs, in->npvt, P);
        MUO = table(in->pvt_p, in->pvt_muo, in->npvt, P);
    } else {                /* undersaturated: x3 = pb, no free gas */
        dual PB = dv(x[2], 2);
        SG = dc(0.0);
        dual dpu = dsub(P, PB);
        BO = dmul(table(in->pvt_p, in->pvt_bo, in->npvt, PB), dsub(dc(1.0), dscale(dpu, in->bo_c_us)));
        RS = table(in->pvt_p, in->pvt_rs, in->npvt, PB);
        MUO = dmul(table(in->pvt_p, in->pvt_muo, in->npvt, PB), dadd(dc(1.0), dscale(dpu, in->muo_c_us)));
    }
    dual bwi = dshift(dscale(dshift(P, -in->bw_pref), in->bw_c), 1.0);          /* 1/Bw */
    dual boi = ddiv(dc(1.0), BO);                                              /* 1/Bo */
    dual bgi = ddiv(dc(1.0), table(in->pvt_p, in->pvt_bg, in->npvt, P));      /* 1/Bg */
    dual MUG = table(in->pvt_p, in->pvt_mug, in->npvt, P);
    dual SO = dsub(dsub(dc(1.0), SW), SG);

    /* Corey two-phase curves and Stone II (normalised so that krow(Swc) = 1) */
    dual krw = corey(dscale(dshift(SW, -in->swc), 1.0 / (1.0 - in->swc - in->sor)), in->nw);
    dual krow = corey(dscale(dsub(dc(1.0 - in->sor), SW), 1.0 / (1.0 - in->swc - in->sor)), in->now);
    dual krg = corey(dscale(dshift(SG, -in->sgc), 1.0 / (1.0 - in->swc - in->sorg - in->sgc)), in->ng);
    dual krog = corey(dscale(dsub(dc(1.0 - in->swc - in->sorg), SG), 1.0 / (1.0 - in->swc - in->sorg)), in->nog);
    dual kro = dsub(dmul(dadd(krow, krw), dadd(krog, krg)), dadd(krw, krg));
    if (kro.v < 0.0) kro = dc(0.0);

    o->acc[CW] = dmul(pv, dscale(dmul(bwi, SW), in->rho_ws));
    o->acc[CO] = dmul(pv, dscale(dmul(boi, SO), in->rho_os));
    o->acc[CG] = dmul(pv, dscale(dadd(dmul(RS, dmul(boi, SO)), dmul(bgi, SG)), in->rho_gs));
    o->rho[PW] = dscale(bwi, in->rho_ws);
    o->rho[PO] = dmul(dshift(dscale(RS, in->rho_gs), in->rho_os), boi);
    o->rho[PG] = dscale(bgi, in->rho_gs);
    dual lw = dscale(krw, 1.0 / in->mu_w);
    dual lo = ddiv(kro, MUO);
    dual lg = ddiv(krg, MUG);
    o->mob[PW][CW] = dmul(o->rho[PW], lw);
    o->mob[PO][CO] = dmul(dscale(boi, in->rho_os), lo);
    o->mob[PO][CG] = dmul(dscale(dmul(RS, boi), in->rho_gs), lo);
    o->mob[PG][CG] = dmul(o->rho[PG], lg);
    o->lamt = dadd(dadd(lw, lo), lg);
    o->rhow = o->rho[PW];
    o->kr[PW] = krw; o->kr[PO] = kro; o->kr[PG] = krg;
    o->bo = BO; o->rs = RS; o->muo = MUO;
}

/* ------------------------------------------------------------------------ */
/* simulator state                                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n, nnz;
    int32_t *rowptr, *col;
    double *val, *dl1;
    int32_t *agg;       /* fine -> next level (absent on the coarsest) */
    int32_t *moff, *mem;/* members of each next-level aggregate, ascending (CSR) */
    double *lu;         /* coarsest: dense LU factors */
    int32_t *piv;
    double *t1, *t2, *t3;
} level_t;

struct ora_sim {
    ora_input in;
    double *kx, *ky, *kz, *poro, *pvt[6];
    int32_t *wi_, *wj_, *wk0, *wk1, *wt;
    double *wbhp, *wrw, *wskin;
    int N, b;
    double vol;
    double *T[3];       /* transmissibility to the + neighbour in x, y, z */
    double *depth;
    int nperf;
    int32_t *perf_cell, *perf_type;
    double *perf_wi, *perf_zh;
    int32_t *perf_well;                /* perforation -> well */
    int32_t *cell_perf;                /* cell -> perforation of a rate-controlled well, or -1 */
    int32_t *wctrl; double *wrate;     /* per well control and target */
    double *wp, *wp_old;               /* per well bottom-hole pressure (an unknown under rate control) */
    double *apw, *awp;                 /* [nperf][b]: dR_cell/dp_h and dR_w/dx_cell */
    double *aww, *rw;                  /* [nw]: dR_w/dp_h and the well equation's residual */
    double *qwell;                     /* [nw][3] component rates per well */
    double *Jp;                        /* preconditioner matrix: J plus the wells' Schur complement on the stencil */
    int nrate;                         /* rate-controlled wells */
    double *x, *x_old; int8_t *ph, *ph_old;
    double *mold;
    double *R, *J;
    double qtot[3], cum_well[3];
    cellprops *props;
    /* CPR */
    double *qiw, *lsc, *ahat, *dinv;   /* qiw: first row of the per-cell left scaling lsc */
    int nlev;
    level_t lev[32];
    int precond_ready;
    /* Krylov workspace */
    double *V, *Z, *w, *r, *tmp, *tmp2, *tmp3;
    double *H, *g, *cs, *sn, *y;
    double theta;                  /* forcing term of the next linear solve */
    int nhist;                     /* forcing history of the last Newton solve */
    double hist_theta[64], hist_b[64], hist_r[64];
    double *rlin;                  /* linear residual b - A dx left by the last Newton solve */
};

static void *xmalloc(size_t n) { void *p = calloc(n ? n : 1, 1); if (!p) { fprintf(stderr, "oracle: out of memory\n"); abort(); } return p; }
static double *dup_d(const double *a, int n) { double *r = xmalloc(sizeof(double) * n); memcpy(r, a, sizeof(double) * n); return r; }
static int32_t *dup_i(const int32_t *a, int n) { int32_t *r = xmalloc(sizeof(int32_t) * (n ? n : 1)); if (n) memcpy(r, a, sizeof(int32_t) * n); return r; }

static void cell_ijk(const ora_sim *s, int i, int *ix, int *iy, int *iz) {
    *ix = i % s->in.nx; *iy = (i / s->in.nx) % s->in.ny; *iz = i / (s->in.nx * s->in.ny);
}

/* neighbour of cell i in direction d (1..6), or -1 outside the grid */
static int nbr(const ora_sim *s, int i, int d) {
    int ix, iy, iz; cell_ijk(s, i, &ix, &iy, &iz);
    int nx = s->in.nx, ny = s->in.ny, nz = s->in.nz;
    switch (d) {
    case 0: return i;
    case 1: return ix > 0 ? i - 1 : -1;
    case 2: return ix < nx - 1 ? i + 1 : -1;
    case 3: return iy > 0 ? i - nx : -1;
    case 4: return iy < ny - 1 ? i + nx : -1;
    case 5: return iz > 0 ? i - nx * ny : -1;
    case 6: return iz < nz - 1 ? i + nx * ny : -1;
    }
    return -1;
}
static int opp(int d) { return d == 0 ? 0 : (d % 2 ? d + 1 : d - 1); }

#define JB(s, i, d) (&(s)->J[(((size_t)(i) * 7 + (d)) * (s)->b) * (s)->b])
#define JP(s, i, d) (&(s)->Jp[(((size_t)(i) * 7 + (d)) * (s)->b) * (s)->b])
#define AH(s, i, d) (&(s)->ahat[(((size_t)(i) * 7 + (d)) * (s)->b) * (s)->b])

ora_sim *ora_create(const ora_input *in) {
    ora_sim *s = xmalloc(sizeof(ora_sim));
    s->in = *in;
    int N = in->nx * in->ny * in->nz;
    s->N = N; s->b = in->model == 3 ? 3 : 2;
    s->kx = dup_d(in->kx, N); s->ky = dup_d(in->ky, N); s->kz = dup_d(in->kz, N); s->poro = dup_d(in->poro, N);
    s->in.kx = s->kx; s->in.ky = s->ky; s->in.kz = s->kz; s->in.poro = s->poro;
    if (in->model == 3) {
        const double *src[6] = {in->pvt_p, in->pvt_bo, in->pvt_rs, in->pvt_muo, in->pvt_bg, in->pvt_mug};
        for (int t = 0; t < 6; t++) s->pvt[t] = dup_d(src[t], in->npvt);
        s->in.pvt_p = s->pvt[0]; s->in.pvt_bo = s->pvt[1]; s->in.pvt_rs = s->pvt[2];
        s->in.pvt_muo = s->pvt[3]; s->in.pvt_bg = s->pvt[4]; s->in.pvt_mug = s->pvt[5];
    }
    int nw = in->nwells;
    s->wi_ = dup_i(in->w_i, nw); s->wj_ = dup_i(in->w_j, nw); s->wk0 = dup_i(in->w_k0, nw);
    s->wk1 = dup_i(in->w_k1, nw); s->wt = dup_i(in->w_type, nw);
    s->wbhp = dup_d(in->w_bhp, nw ? nw : 1); s->wrw = dup_d(in->w_rw, nw ? nw : 1); s->wskin = dup_d(in->w_skin, nw ? nw : 1);
    s->in.w_i = s->wi_; s->in.w_j = s->wj_; s->in.w_k0 = s->wk0; s->in.w_k1 = s->wk1; s->in.w_type = s->wt;
    s->in.w_bhp = s->wbhp; s->in.w_rw = s->wrw; s->in.w_skin = s->wskin;

    int nx = in->nx, ny = in->ny, nz = in->nz;
    double dx = in->dx, dy = in->dy, dz = in->dz;
    s->vol = dx * dy * dz;
    /* Eq. (11): geometric part of the transmissibility, harmonic average of
       the two half-cell conductances */
    for (int a = 0; a < 3; a++) s->T[a] = xmalloc(sizeof(double) * N);
    s->depth = xmalloc(sizeof(double) * N);
    for (int i = 0; i < N; i++) {
        int ix, iy, iz; cell_ijk(s, i, &ix, &iy, &iz);
        s->depth[i] = in->top_depth + (iz + 0.5) * dz;
        if (ix < nx - 1) s->T[0][i] = DARCY_C * 2.0 * dy * dz / (dx / s->kx[i] + dx / s->kx[i + 1]);
        if (iy < ny - 1) s->T[1][i] = DARCY_C * 2.0 * dx * dz / (dy / s->ky[i] + dy / s->ky[i + nx]);
        if (iz < nz - 1) s->T[2][i] = DARCY_C * 2.0 * dx * dy / (dz / s->kz[i] + dz / s->kz[i + nx * ny]);
    }
    /* perforations with the Peaceman well index (vertical well) */
    int np = 0;
    for (int w = 0; w < nw; w++) np += s->wk1[w] - s->wk0[w] + 1;
    s->nperf = np;
    s->perf_cell = xmalloc(sizeof(int32_t) * (np + 1)); s->perf_type = xmalloc(sizeof(int32_t) * (np + 1));
    s->perf_wi = xmalloc(sizeof(double) * (np + 1)); s->perf_zh = xmalloc(sizeof(double) * (np + 1));
    s->perf_well = xmalloc(sizeof(int32_t) * (np + 1));
    s->wctrl = xmalloc(sizeof(int32_t) * (nw + 1)); s->wrate = xmalloc(sizeof(double) * (nw + 1));
    s->wp = xmalloc(sizeof(double) * (nw + 1)); s->wp_old = xmalloc(sizeof(double) * (nw + 1));
    s->aww = xmalloc(sizeof(double) * (nw + 1)); s->rw = xmalloc(sizeof(double) * (nw + 1));
    s->qwell = xmalloc(sizeof(double) * 3 * (nw + 1));
    s->apw = xmalloc(sizeof(double) * (np + 1) * 3); s->awp = xmalloc(sizeof(double) * (np + 1) * 3);
    s->cell_perf = xmalloc(sizeof(int32_t) * N);
    for (int i = 0; i < N; i++) s->cell_perf[i] = -1;
    s->nrate = 0;
    for (int w = 0; w < nw; w++) {
        s->wctrl[w] = in->w_ctrl ? in->w_ctrl[w] : 0;
        s->wrate[w] = in->w_rate ? in->w_rate[w] : 0.0;
        s->wp[w] = s->wbhp[w];
        if (s->wctrl[w]) s->nrate++;
    }
    s->in.w_ctrl = s->wctrl; s->in.w_rate = s->wrate;
    np = 0;
    for (int w = 0; w < nw; w++) {
        double zh = in->top_depth + (s->wk0[w] + 0.5) * dz;
        for (int k = s->wk0[w]; k <= s->wk1[w]; k++) {
            int c = s->wi_[w] + nx * (s->wj_[w] + ny * k);
            double kxx = s->kx[c], kyy = s->ky[c];
            double ro = 0.28 * sqrt(sqrt(kyy / kxx) * dx * dx + sqrt(kxx / kyy) * dy * dy)
                        / (pow(kyy / kxx, 0.25) + pow(kxx / kyy, 0.25));
            s->perf_cell[np] = c;
            s->perf_type[np] = s->wt[w];
            s->perf_wi[np] = 2.0 * M_PI * DARCY_C * sqrt(kxx * kyy) * dz / (log(ro / s->wrw[w]) + s->wskin[w]);
            s->perf_zh[np] = zh;
            s->perf_well[np] = w;
            if (s->wctrl[w]) {
                if (s->cell_perf[c] >= 0) {
                    fprintf(stderr, "oracle: two rate-controlled perforations in cell %d\n", c);
                    return NULL;     /* the caller treats NULL as an input error */
                }
                s->cell_perf[c] = np;
            }
            np++;
        }
    }
    int b = s->b;
    s->x = xmalloc(sizeof(double) * N * b); s->x_old = xmalloc(sizeof(double) * N * b);
    s->ph = xmalloc(N); s->ph_old = xmalloc(N);
    s->mold = xmalloc(sizeof(double) * N * b);
    s->R = xmalloc(sizeof(double) * N * b);
    s->J = xmalloc(sizeof(double) * (size_t)N * 7 * b * b);
    s->Jp = xmalloc(sizeof(double) * (size_t)N * 7 * b * b);
    s->props = xmalloc(sizeof(cellprops) * N);
    s->qiw = xmalloc(sizeof(double) * N * b);
    s->lsc = xmalloc(sizeof(double) * (size_t)N * b * b);
    s->ahat = xmalloc(sizeof(double) * (size_t)N * 7 * b * b);
    s->dinv = xmalloc(sizeof(double) * (size_t)N * b * b);
    int m = in->gmres_m, n = N * b;
    s->V = xmalloc(sizeof(double) * (size_t)(m + 1 > 5 ? m + 1 : 5) * n);    /* BiCGSTAB uses 5 */
    s->Z = xmalloc(sizeof(double) * (size_t)(m > 2 ? m : 2) * n);
    s->w = xmalloc(sizeof(double) * n); s->r = xmalloc(sizeof(double) * n);
    s->rlin = xmalloc(sizeof(double) * n);
    s->theta = in->lin_tol;
    s->tmp = xmalloc(sizeof(double) * n); s->tmp2 = xmalloc(sizeof(double) * n); s->tmp3 = xmalloc(sizeof(double) * n);
    s->H = xmalloc(sizeof(double) * (m + 1) * (m + 1));
    s->g = xmalloc(sizeof(double) * (m + 1)); s->cs = xmalloc(sizeof(double) * (m + 1));
    s->sn = xmalloc(sizeof(double) * (m + 1)); s->y = xmalloc(sizeof(double) * (m + 1));
    return s;
}

static void free_levels(ora_sim *s) {
    for (int l = 0; l < s->nlev; l++) {
        level_t *L = &s->lev[l];
        free(L->rowptr); free(L->col); free(L->val); free(L->dl1); free(L->agg); free(L->moff); free(L->mem);
        free(L->lu); free(L->piv); free(L->t1); free(L->t2); free(L->t3);
        memset(L, 0, sizeof(*L));
    }
    s->nlev = 0;
}

void ora_destroy(ora_sim *s) {
    if (!s) return;
    free_levels(s);
    free(s->kx); free(s->ky); free(s->kz); free(s->poro);
    for (int t = 0; t < 6; t++) free(s->pvt[t]);
    free(s->wi_); free(s->wj_); free(s->wk0); free(s->wk1); free(s->wt); free(s->wbhp); free(s->wrw); free(s->wskin);
    for (int a = 0; a < 3; a++) free(s->T[a]);
    free(s->depth); free(s->perf_cell); free(s->perf_type); free(s->perf_wi); free(s->perf_zh); free(s->perf_well);
    free(s->cell_perf); free(s->wctrl); free(s->wrate); free(s->wp); free(s->wp_old); free(s->aww); free(s->rw); free(s->qwell);
    free(s->apw); free(s->awp); free(s->Jp);
    free(s->x); free(s->x_old); free(s->ph); free(s->ph_old); free(s->mold); free(s->R); free(s->J); free(s->props);
    free(s->qiw); free(s->lsc); free(s->ahat); free(s->dinv);
    free(s->V); free(s->Z); free(s->w); free(s->r); free(s->rlin); free(s->tmp); free(s->tmp2); free(s->tmp3);
    free(s->H); free(s->g); free(s->cs); free(s->sn); free(s->y);
    free(s);
}

int ora_block_size(const ora_sim *s) { return s->b; }

/* accumulation of the last accepted state (the f^n of Eq. 10) */
static void begin_step(ora_sim *s) {
    int b = s->b;
    memcpy(s->x_old, s->x, sizeof(double) * s->N * b);
    memcpy(s->ph_old, s->ph, s->N);
    memcpy(s->wp_old, s->wp, sizeof(double) * s->in.nwells);
    for (int i = 0; i < s->N; i++) {
        cellprops cp;
        eval_props(&s->in, s->poro[i], s->vol, &s->x[i * b], s->ph[i], &cp);
        for (int c = 0; c < b; c++) s->mold[i * b + c] = cp.acc[c].v;
    }
}

void ora_set_state(ora_sim *s, const double *p, const double *sw, const double *x3, const int8_t *ph) {
    int b = s->b;
    for (int i = 0; i < s->N; i++) {
        s->x[i * b] = p[i]; s->x[i * b + 1] = sw[i];
        if (b == 3) s->x[i * b + 2] = x3[i];
        s->ph[i] = b == 3 ? ph[i] : 1;
    }
    begin_step(s);
    s->cum_well[0] = s->cum_well[1] = s->cum_well[2] = 0.0;
}

void ora_get_state(const ora_sim *s, double *p, double *sw, double *x3, int8_t *ph) {
    int b = s->b;
    for (int i = 0; i < s->N; i++) {
        p[i] = s->x[i * b]; sw[i] = s->x[i * b + 1];
        x3[i] = b == 3 ? s->x[i * b + 2] : 0.0;
        ph[i] = s->ph[i];
    }
}

void ora_set_iterate(ora_sim *s, const double *x, const int8_t *ph) {
    memcpy(s->x, x, sizeof(double) * s->N * s->b);
    memcpy(s->ph, ph, s->N);
}
void ora_get_iterate(const ora_sim *s, double *x, int8_t *ph) {
    memcpy(x, s->x, sizeof(double) * s->N * s->b);
    memcpy(ph, s->ph, s->N);
}

/* ------------------------------------------------------------------------ */
/* residual and Jacobian (Eq. 3/5 discretised by Eq. 10-11, wells Eq. 6-7)   */
/* ------------------------------------------------------------------------ */
void ora_assemble(ora_sim *s, double dt) {
    const ora_input *in = &s->in;
    int N = s->N, b = s->b, np = in->model == 3 ? 3 : 2;
    memset(s->R, 0, sizeof(double) * N * b);
    memset(s->J, 0, sizeof(double) * (size_t)N * 7 * b * b);
    for (int i = 0; i < N; i++) eval_props(in, s->poro[i], s->vol, &s->x[i * b], s->ph[i], &s->props[i]);

    /* accumulation (f^{n+1} - f^n) / dt */
    for (int i = 0; i < N; i++) {
        double *D = JB(s, i, 0);
        for (int c = 0; c < b; c++) {
            s->R[i * b + c] += (s->props[i].acc[c].v - s->mold[i * b + c]) / dt;
            for (int k = 0; k < b; k++) D[c * b + k] += s->props[i].acc[c].d[k] / dt;
        }
    }
    /* inter-cell fluxes, each face once in the orientation (L, R = L + stride) */
    int strides[3] = {1, in->nx, in->nx * in->ny};
    for (int L = 0; L < N; L++) {
        for (int a = 0; a < 3; a++) {
            int Rr = nbr(s, L, 2 * a + 2);
            if (Rr < 0) continue;
            (void)strides;
            double T = s->T[a][L];
            const cellprops *PL = &s->props[L], *PR = &s->props[Rr];
            double gdz = GRAV * (s->depth[Rr] - s->depth[L]) / 1e5;
            for (int ph = 0; ph < np; ph++) {
                double rbar = 0.5 * (PL->rho[ph].v + PR->rho[ph].v);
                double dphi = (s->x[Rr * b] - s->x[L * b]) - rbar * gdz;
                double dphiL[3], dphiR[3];
                for (int k = 0; k < 3; k++) {
                    dphiL[k] = -gdz * 0.5 * PL->rho[ph].d[k];
                    dphiR[k] = -gdz * 0.5 * PR->rho[ph].d[k];
                }
                dphiL[0] -= 1.0; dphiR[0] += 1.0;
                int upR = dphi > 0.0;
                const cellprops *PU = upR ? PR : PL;
                for (int c = 0; c < b; c++) {
                    if (!carries(in->model, ph, c)) continue;
                    const dual *m = &PU->mob[ph][c];
                    double F = T * m->v * dphi;
                    double dFL[3], dFR[3];
                    for (int k = 0; k < b; k++) {
                        dFL[k] = T * ((upR ? 0.0 : m->d[k] * dphi) + m->v * dphiL[k]);
                        dFR[k] = T * ((upR ? m->d[k] * dphi : 0.0) + m->v * dphiR[k]);
                    }
                    /* F flows from R into L */
                    s->R[L * b + c] -= F;
                    s->R[Rr * b + c] += F;
                    double *JLL = JB(s, L, 0), *JLR = JB(s, L, 2 * a + 2);
                    double *JRR = JB(s, Rr, 0), *JRL = JB(s, Rr, 2 * a + 1);
                    for (int k = 0; k < b; k++) {
                        JLL[c * b + k] -= dFL[k];
                        JLR[c * b + k] -= dFR[k];
                        JRR[c * b + k] += dFR[k];
                        JRL[c * b + k] += dFL[k];
                    }
                }
            }
        }
    }
    /* wells, Eq. (6); each well's bottom-hole pressure p_h is the current
       value of its unknown (fixed under BHP control).  The border blocks of
       Eq. (16): A_pw = dR_cell/dp_h per perforation; the well equation is
       p_h - c = 0 (BHP control, Eq. 7) or the perforations' summed rate of
       the controlled component minus its target (Eq. 8-9) */
    s->qtot[0] = s->qtot[1] = s->qtot[2] = 0.0;
    for (int w = 0; w < in->nwells; w++) {
        s->qwell[w * 3] = s->qwell[w * 3 + 1] = s->qwell[w * 3 + 2] = 0.0;
        if (s->wctrl[w]) { s->rw[w] = -s->wrate[w]; s->aww[w] = 0.0; }
        else { s->rw[w] = s->wp[w] - s->wbhp[w]; s->aww[w] = 1.0; }
    }
    for (int q = 0; q < s->nperf; q++) {
        int i = s->perf_cell[q], w = s->perf_well[q];
        const cellprops *P = &s->props[i];
        double WI = s->perf_wi[q];
        double dh = GRAV * (s->perf_zh[q] - s->depth[i]) / 1e5;
        double p = s->x[i * b];
        double *D = JB(s, i, 0);
        double *apw = &s->apw[q * 3], *awp = &s->awp[q * 3];
        for (int k = 0; k < 3; k++) { apw[k] = 0.0; awp[k] = 0.0; }
        const int cc = s->wctrl[w] == 1 ? CW : (s->wctrl[w] == 2 ? CO : -1);   /* controlled component */
        const double Dw = s->wp[w] - p - P->rho[PW].v * dh;   /* head of the water-filled injector */
        if (s->perf_type[q] == 1 && (Dw >= 0.0 || s->wctrl[w])) {
            /* water injector: water at the cell's total mobility.  A rate-
               controlled injector keeps this form for a negative head too: its
               solution injects, and the form keeps dR_w/dp_h from vanishing on
               the Newton path */
            dual lam = dmul(P->rhow, P->lamt);
            double qw = WI * lam.v * Dw;
            s->R[i * b + CW] -= qw;
            s->qtot[CW] += qw;
            s->qwell[w * 3 + CW] += qw;
            apw[CW] -= WI * lam.v;
            for (int k = 0; k < b; k++) {
                double dD = (k == 0 ? -1.0 : 0.0) - P->rho[PW].d[k] * dh;
                double dq = WI * (lam.d[k] * Dw + lam.v * dD);
                D[CW * b + k] -= dq;
                if (cc == CW) awp[k] += dq;
            }
            if (cc == CW) { s->rw[w] += qw; s->aww[w] += WI * lam.v; }
        } else {
            /* producer (Eq. 6 per phase), or a BHP-controlled injector whose
               water head is below the cell pressure: the cell's phases flow
               into the wellbore at their own mobilities, driven for the
               injector by its water head (continuous with injection at Dw = 0) */
            const int inj = s->perf_type[q] == 1;
            for (int ph = 0; ph < np; ph++) {
                double Dp = inj ? Dw : s->wp[w] - p - P->rho[ph].v * dh;
                const int hp = inj ? PW : ph;             /* phase whose density sets the head */
                for (int c = 0; c < b; c++) {
                    if (!carries(in->model, ph, c)) continue;
                    const dual *m = &P->mob[ph][c];
                    double qc = WI * m->v * Dp;
                    s->R[i * b + c] -= qc;
                    s->qtot[c] += qc;
                    s->qwell[w * 3 + c] += qc;
                    apw[c] -= WI * m->v;
                    for (int k = 0; k < b; k++) {
                        double dD = (k == 0 ? -1.0 : 0.0) - P->rho[hp].d[k] * dh;
                        double dq = WI * (m->d[k] * Dp + m->v * dD);
                        D[c * b + k] -= dq;
                        if (c == cc) awp[k] += dq;
                    }
                    if (c == cc) { s->rw[w] += qc; s->aww[w] += WI * m->v; }
                }
            }
        }
    }
    s->precond_ready = 0;
}

/* well measure of the Newton test: largest |R_w| / max(|target|, 1 kg/day)
   over the rate-controlled wells (BHP wells meet p_h = c exactly) */
static double well_cnv(const ora_sim *s) {
    double m = 0.0;
    for (int w = 0; w < s->in.nwells; w++) {
        if (!s->wctrl[w]) continue;
        double sc = fabs(s->wrate[w]) > 1.0 ? fabs(s->wrate[w]) : 1.0;
        double v = fabs(s->rw[w]) / sc;
        if (!(v <= m)) m = v;
    }
    return m;
}

void ora_get_well_bhp(const ora_sim *s, double *bhp) { memcpy(bhp, s->wp, sizeof(double) * s->in.nwells); }
void ora_set_well_bhp(ora_sim *s, const double *bhp) { memcpy(s->wp, bhp, sizeof(double) * s->in.nwells); }
int ora_perforations(const ora_sim *s) { return s->nperf; }
void ora_well_component_rates(const ora_sim *s, double *q) { memcpy(q, s->qwell, sizeof(double) * 3 * s->in.nwells); }
void ora_get_well_system(const ora_sim *s, double *Rw, double *Apw, double *Awp, double *Aww) {
    int b = s->b;
    memcpy(Rw, s->rw, sizeof(double) * s->in.nwells);
    memcpy(Aww, s->aww, sizeof(double) * s->in.nwells);
    for (int q = 0; q < s->nperf; q++)
        for (int c = 0; c < b; c++) { Apw[q * b + c] = s->apw[q * 3 + c]; Awp[q * b + c] = s->awp[q * 3 + c]; }
}

void ora_get_residual(const ora_sim *s, double *R) { memcpy(R, s->R, sizeof(double) * s->N * s->b); }
void ora_get_jacobian(const ora_sim *s, double *J) { memcpy(J, s->J, sizeof(double) * (size_t)s->N * 7 * s->b * s->b); }
void ora_set_jacobian(ora_sim *s, const double *J) {
    memcpy(s->J, J, sizeof(double) * (size_t)s->N * 7 * s->b * s->b);
    s->precond_ready = 0;
}

/* CNV: largest component residual in pore-volume-saturation units */
double ora_cnv(const ora_sim *s, double dt) {
    double m = 0.0;
    for (int i = 0; i < s->N; i++) {
        double pv0 = s->poro[i] * s->vol;
        for (int c = 0; c < s->b; c++) {
            double v = fabs(s->R[i * s->b + c]) * dt / (pv0 * s->in.cnv_rho[c]);
            if (!(v <= m)) m = v;       /* NaN propagates */
        }
    }
    return m;
}

void ora_component_mass(const ora_sim *s, double *m) {
    m[0] = m[1] = m[2] = 0.0;
    for (int i = 0; i < s->N; i++) {
        cellprops cp;
        eval_props(&s->in, s->poro[i], s->vol, &s->x[i * s->b], s->ph[i], &cp);
        for (int c = 0; c < s->b; c++) m[c] += cp.acc[c].v;
    }
}
void ora_cumulative_well_mass(const ora_sim *s, double *m) { for (int c = 0; c < 3; c++) m[c] = s->cum_well[c]; }
void ora_well_rates(const ora_sim *s, double *q) { for (int c = 0; c < 3; c++) q[c] = s->qtot[c]; }

/* ------------------------------------------------------------------------ */
/* small dense algebra                                                       */
/* ------------------------------------------------------------------------ */
static void inv_block(int b, const double *A, double *Ai) {
    if (b == 2) {
        double det = A[0] * A[3] - A[1] * A[2];
        Ai[0] = A[3] / det; Ai[1] = -A[1] / det; Ai[2] = -A[2] / det; Ai[3] = A[0] / det;
    } else {
        double c00 = A[4] * A[8] - A[5] * A[7];
        double c01 = A[5] * A[6] - A[3] * A[8];
        double c02 = A[3] * A[7] - A[4] * A[6];
        double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
        Ai[0] = c00 / det; Ai[1] = (A[2] * A[7] - A[1] * A[8]) / det; Ai[2] = (A[1] * A[5] - A[2] * A[4]) / det;
        Ai[3] = c01 / det; Ai[4] = (A[0] * A[8] - A[2] * A[6]) / det; Ai[5] = (A[2] * A[3] - A[0] * A[5]) / det;
        Ai[6] = c02 / det; Ai[7] = (A[1] * A[6] - A[0] * A[7]) / det; Ai[8] = (A[0] * A[4] - A[1] * A[3]) / det;
    }
}
static void matmul_block(int b, const double *A, const double *B, double *C) {
    for (int r = 0; r < b; r++)
        for (int c = 0; c < b; c++) {
            double t = 0.0;
            for (int k = 0; k < b; k++) t += A[r * b + k] * B[k * b + c];
            C[r * b + c] = t;
        }
}
static void matvec_block(int b, const double *A, const double *x, double *y) {
    for (int r = 0; r < b; r++) { double t = 0.0; for (int k = 0; k < b; k++) t += A[r * b + k] * x[k]; y[r] = t; }
}

/* dense LU with partial pivoting, row-major, in place; returns 0 on success */
static int lu_factor(int n, double *A, int32_t *piv) {
    for (int k = 0; k < n; k++) {
        int p = k; double best = fabs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; i++) if (fabs(A[(size_t)i * n + k]) > best) { best = fabs(A[(size_t)i * n + k]); p = i; }
        piv[k] = p;
        if (best == 0.0) return -1;
        if (p != k) for (int j = 0; j < n; j++) { double t = A[(size_t)k * n + j]; A[(size_t)k * n + j] = A[(size_t)p * n + j]; A[(size_t)p * n + j] = t; }
        for (int i = k + 1; i < n; i++) {
            double l = A[(size_t)i * n + k] / A[(size_t)k * n + k];
            A[(size_t)i * n + k] = l;
            for (int j = k + 1; j < n; j++) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
        }
    }
    return 0;
}
static void lu_solve(int n, const double *LU, const int32_t *piv, double *x) {
    for (int k = 0; k < n; k++) if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
    for (int i = 0; i < n; i++) { double t = x[i]; for (int j = 0; j < i; j++) t -= LU[(size_t)i * n + j] * x[j]; x[i] = t; }
    for (int i = n - 1; i >= 0; i--) { double t = x[i]; for (int j = i + 1; j < n; j++) t -= LU[(size_t)i * n + j] * x[j]; x[i] = t / LU[(size_t)i * n + i]; }
}
int ora_dense_lu_solve(int n, double *A, double *b) {
    int32_t *piv = xmalloc(sizeof(int32_t) * n);
    int rc = lu_factor(n, A, piv);
    if (rc == 0) lu_solve(n, A, piv, b);
    free(piv);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* sparse matrix-vector product with the 7-point block Jacobian              */
/* ------------------------------------------------------------------------ */
static void block_spmv(const ora_sim *s, const double *A, const double *x, double *y) {
    int b = s->b;
    for (int i = 0; i < s->N; i++) {
        double acc[3] = {0, 0, 0}, t[3];
        for (int d = 0; d < 7; d++) {
            int j = nbr(s, i, d);
            if (j < 0) continue;
            matvec_block(b, &A[(((size_t)i * 7 + d) * b) * b], &x[j * b], t);
            for (int r = 0; r < b; r++) acc[r] += t[r];
        }
        for (int r = 0; r < b; r++) y[i * b + r] = acc[r];
    }
}
/* y = S x, S = A - A_pw A_ww^-1 A_wp (the wells' unknowns eliminated): the
   stencil product, then per well u = (A_wp x) / A_ww subtracted through A_pw */
static void op_apply(const ora_sim *s, const double *x, double *y) {
    int b = s->b;
    block_spmv(s, s->J, x, y);
    if (!s->nrate) return;
    for (int w = 0; w < s->in.nwells; w++) {
        if (!s->wctrl[w]) continue;
        double u = 0.0;
        for (int q = 0; q < s->nperf; q++) {
            if (s->perf_well[q] != w) continue;
            for (int k = 0; k < b; k++) u += s->awp[q * 3 + k] * x[s->perf_cell[q] * b + k];
        }
        u /= s->aww[w];
        for (int q = 0; q < s->nperf; q++) {
            if (s->perf_well[q] != w) continue;
            for (int c = 0; c < b; c++) y[s->perf_cell[q] * b + c] -= s->apw[q * 3 + c] * u;
        }
    }
}
void ora_spmv(const ora_sim *s, const double *x, double *y) { op_apply(s, x, y); }

/* ------------------------------------------------------------------------ */
/* aggregation AMG on the pressure block                                     */
/* ------------------------------------------------------------------------ */
/* splitmix64 finaliser, used only to break exact ties between equal edge
   strengths deterministically (a symmetric key of the unordered pair) */
static uint64_t edge_hash(int a, int b) {
    uint64_t lo = (uint64_t)(a < b ? a : b), hi = (uint64_t)(a < b ? b : a);
    uint64_t z = ((hi << 32) | lo) + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* strength band of a positive coupling: its binary exponent (one band per
   factor of two), read from the IEEE-754 bit pattern */
static int strength_band(double a) {
    uint64_t u; memcpy(&u, &a, sizeof(u));
    return (int)((u >> 52) & 0x7FF);
}

/* one matching pass: rounds of handshakes among unmatched nodes.  In each
   round every unmatched node picks, among its unmatched strong neighbours
   (strong: -a_ij >= theta * max_k -a_ik), the one in the highest strength
   band, ties broken by the larger pair hash, then by the smaller index;
   mutual picks become pairs.  partner[i] = -1 for nodes left single. */
int ora_match_pass(int n, const int32_t *rowptr, const int32_t *col, const double *val,
                   double theta, int rounds, int32_t *partner) {
    int32_t *pick = xmalloc(sizeof(int32_t) * (n ? n : 1));
    for (int i = 0; i < n; i++) partner[i] = -1;
    int done_rounds = 0;
    for (int r = 0; r < rounds; r++) {
        for (int i = 0; i < n; i++) {
            pick[i] = -1;
            if (partner[i] >= 0) continue;
            double mx = 0.0;
            for (int k = rowptr[i]; k < rowptr[i + 1]; k++)
                if (col[k] != i && -val[k] > mx) mx = -val[k];
            if (mx <= 0.0) continue;
            int best = -1, bs = 0; uint64_t bh = 0;
            for (int k = rowptr[i]; k < rowptr[i + 1]; k++) {
                int j = col[k];
                if (j == i || partner[j] >= 0) continue;
                double a = -val[k];
                if (!(a > 0.0) || a < theta * mx) continue;
                int band = strength_band(a);
                uint64_t h = edge_hash(i, j);
                if (best < 0 || band > bs || (band == bs && (h > bh || (h == bh && j < best)))) { best = j; bs = band; bh = h; }
            }
            pick[i] = best;
        }
        int any = 0;
        for (int i = 0; i < n; i++)
            if (partner[i] < 0 && pick[i] >= 0 && pick[pick[i]] == i) { partner[i] = pick[i]; any = 1; }
        done_rounds++;
        if (!any) break;
    }
    free(pick);
    return done_rounds;
}

/* aggregates of one pass: matched pairs, plus every single node that has a
   strong matched neighbour joining the aggregate of the strongest such
   neighbour (same key as the matching); other single nodes stay alone.
   Aggregates are numbered in the order of their lowest-index founder
   (pair leader or lone node).  Returns the number of aggregates. */
static int form_aggregates(int n, const int32_t *rowptr, const int32_t *col, const double *val, double theta,
                           const int32_t *partner, int32_t *agg) {
    int32_t *host = xmalloc(sizeof(int32_t) * (n ? n : 1));
    for (int i = 0; i < n; i++) {
        host[i] = -1;
        if (partner[i] >= 0) continue;
        double mx = 0.0;
        for (int k = rowptr[i]; k < rowptr[i + 1]; k++)
            if (col[k] != i && -val[k] > mx) mx = -val[k];
        if (mx <= 0.0) continue;
        int best = -1, bs = 0; uint64_t bh = 0;
        for (int k = rowptr[i]; k < rowptr[i + 1]; k++) {
            int j = col[k];
            if (j == i || partner[j] < 0) continue;
            double a = -val[k];
            if (!(a > 0.0) || a < theta * mx) continue;
            int band = strength_band(a);
            uint64_t h = edge_hash(i, j);
            if (best < 0 || band > bs || (band == bs && (h > bh || (h == bh && j < best)))) { best = j; bs = band; bh = h; }
        }
        host[i] = best;
    }
    int nc = 0;
    for (int i = 0; i < n; i++) {
        int p = partner[i];
        if ((p >= 0 && i < p) || (p < 0 && host[i] < 0)) agg[i] = nc++;
        else agg[i] = -1;
    }
    for (int i = 0; i < n; i++) {
        int p = partner[i];
        if (p >= 0 && i > p) agg[i] = agg[p];
    }
    for (int i = 0; i < n; i++) {
        if (partner[i] < 0 && host[i] >= 0) {
            int h = host[i], hp = partner[h];
            agg[i] = agg[h < hp ? h : hp];
        }
    }
    free(host);
    return nc;
}

/* members of each aggregate in ascending order (CSR) */
static void members_of(int n, const int32_t *agg, int nc, int32_t **moff_out, int32_t **mem_out) {
    int32_t *moff = xmalloc(sizeof(int32_t) * (nc + 1)), *mem = xmalloc(sizeof(int32_t) * (n ? n : 1));
    int32_t *pos = xmalloc(sizeof(int32_t) * (nc + 1));
    for (int i = 0; i < n; i++) moff[agg[i] + 1]++;
    for (int I = 0; I < nc; I++) moff[I + 1] += moff[I];
    for (int I = 0; I < nc; I++) pos[I] = moff[I];
    for (int i = 0; i < n; i++) mem[pos[agg[i]]++] = i;
    free(pos);
    *moff_out = moff; *mem_out = mem;
}

/* Galerkin product P^T A P for piecewise-constant P: coarse row I sums the
   rows of its members (ascending member order, then column order) into
   columns agg[j]; coarse columns sorted ascending */
static void galerkin(int n, const int32_t *rowptr, const int32_t *col, const double *val,
                     const int32_t *agg, const int32_t *moff, const int32_t *mem, int nc,
                     int32_t **rp_out, int32_t **col_out, double **val_out) {
    int cap = 64;
    int32_t *cols = xmalloc(sizeof(int32_t) * cap); double *vals = xmalloc(sizeof(double) * cap);
    int32_t *rp = xmalloc(sizeof(int32_t) * (nc + 1));
    size_t nnzcap = (size_t)rowptr[n] + 16, nnz = 0;
    int32_t *oc = xmalloc(sizeof(int32_t) * nnzcap); double *ov = xmalloc(sizeof(double) * nnzcap);
    for (int I = 0; I < nc; I++) {
        int cnt = 0;
        for (int t = moff[I]; t < moff[I + 1]; t++) {
            int m = mem[t];
            for (int k = rowptr[m]; k < rowptr[m + 1]; k++) {
                int Jc = agg[col[k]], f = -1;
                for (int q = 0; q < cnt; q++) if (cols[q] == Jc) { f = q; break; }
                if (f < 0) {
                    if (cnt == cap) { cap *= 2; cols = realloc(cols, sizeof(int32_t) * cap); vals = realloc(vals, sizeof(double) * cap); }
                    cols[cnt] = Jc; vals[cnt] = 0.0; f = cnt++;
                }
                vals[f] += val[k];
            }
        }
        /* insertion sort by column */
        for (int a = 1; a < cnt; a++) {
            int cj = cols[a]; double cv = vals[a]; int q = a - 1;
            while (q >= 0 && cols[q] > cj) { cols[q + 1] = cols[q]; vals[q + 1] = vals[q]; q--; }
            cols[q + 1] = cj; vals[q + 1] = cv;
        }
        rp[I] = (int32_t)nnz;
        if (nnz + cnt > nnzcap) { nnzcap = 2 * (nnz + cnt); oc = realloc(oc, sizeof(int32_t) * nnzcap); ov = realloc(ov, sizeof(double) * nnzcap); }
        for (int q = 0; q < cnt; q++) { oc[nnz] = cols[q]; ov[nnz] = vals[q]; nnz++; }
    }
    rp[nc] = (int32_t)nnz;
    free(cols); free(vals);
    *rp_out = rp; *col_out = oc; *val_out = ov;
}

/* a Galerkin row wider than this stops the coarsening (shared with the device) */
#define AMG_MAX_ROW 512
static int max_row(const int32_t *rp, int n) {
    int m = 0;
    for (int i = 0; i < n; i++) if (rp[i + 1] - rp[i] > m) m = rp[i + 1] - rp[i];
    return m;
}

static void level_finish(level_t *L) {
    L->dl1 = xmalloc(sizeof(double) * L->n);
    for (int i = 0; i < L->n; i++) {
        double t = 0.0;
        for (int k = L->rowptr[i]; k < L->rowptr[i + 1]; k++) t += fabs(L->val[k]);
        L->dl1[i] = t;
    }
    L->nnz = L->rowptr[L->n];
    L->t1 = xmalloc(sizeof(double) * L->n); L->t2 = xmalloc(sizeof(double) * L->n); L->t3 = xmalloc(sizeof(double) * L->n);
}

static void amg_setup(ora_sim *s, int32_t *rp0, int32_t *col0, double *val0, int n0) {
    free_levels(s);
    const ora_input *in = &s->in;
    level_t *L = &s->lev[0];
    L->n = n0; L->rowptr = rp0; L->col = col0; L->val = val0;
    level_finish(L);
    s->nlev = 1;
    while (1) {
        L = &s->lev[s->nlev - 1];
        if (L->n <= in->amg_coarse_max || s->nlev >= in->amg_max_levels || s->nlev >= 32) break;
        int n = L->n;
        int32_t *p1 = xmalloc(sizeof(int32_t) * n), *agg1 = xmalloc(sizeof(int32_t) * n);
        ora_match_pass(n, L->rowptr, L->col, L->val, in->amg_theta, in->amg_rounds, p1);
        int n1 = form_aggregates(n, L->rowptr, L->col, L->val, in->amg_theta, p1, agg1);
        int32_t *o1, *m1;
        members_of(n, agg1, n1, &o1, &m1);
        int32_t *rp1, *c1; double *v1;
        galerkin(n, L->rowptr, L->col, L->val, agg1, o1, m1, n1, &rp1, &c1, &v1);
        if (max_row(rp1, n1) > AMG_MAX_ROW) {   /* too wide: this level is the coarsest */
            free(p1); free(agg1); free(o1); free(m1); free(rp1); free(c1); free(v1);
            break;
        }
        int32_t *p2 = xmalloc(sizeof(int32_t) * n1), *agg2 = xmalloc(sizeof(int32_t) * n1);
        ora_match_pass(n1, rp1, c1, v1, in->amg_theta, in->amg_rounds, p2);
        int n2 = form_aggregates(n1, rp1, c1, v1, in->amg_theta, p2, agg2);
        int32_t *o2, *m2;
        members_of(n1, agg2, n2, &o2, &m2);
        int stalled = 4 * (long)n2 > 3 * (long)n;   /* coarsening stalled (> 3/4 kept) */
        if (!stalled) {
            level_t *C = &s->lev[s->nlev];
            galerkin(n1, rp1, c1, v1, agg2, o2, m2, n2, &C->rowptr, &C->col, &C->val);
            if (max_row(C->rowptr, n2) > AMG_MAX_ROW) {
                free(C->rowptr); free(C->col); free(C->val);
                C->rowptr = NULL; C->col = NULL; C->val = NULL;
                stalled = 1;
            }
        }
        if (!stalled) {
            level_t *C = &s->lev[s->nlev];
            C->n = n2;
            L->agg = xmalloc(sizeof(int32_t) * n);
            for (int i = 0; i < n; i++) L->agg[i] = agg2[agg1[i]];
            members_of(n, L->agg, n2, &L->moff, &L->mem);
            level_finish(C);
            s->nlev++;
        }
        free(p1); free(agg1); free(o1); free(m1); free(rp1); free(c1); free(v1);
        free(p2); free(agg2); free(o2); free(m2);
        if (stalled) break;
    }
    /* coarsest level: dense LU */
    L = &s->lev[s->nlev - 1];
    int n = L->n;
    L->lu = xmalloc(sizeof(double) * (size_t)n * n);
    L->piv = xmalloc(sizeof(int32_t) * n);
    for (int i = 0; i < n; i++)
        for (int k = L->rowptr[i]; k < L->rowptr[i + 1]; k++) L->lu[(size_t)i * n + L->col[k]] += L->val[k];
    lu_factor(n, L->lu, L->piv);
}

static void csr_residual(const level_t *L, const double *f, const double *e, double *r) {
    for (int i = 0; i < L->n; i++) {
        double t = 0.0;
        for (int k = L->rowptr[i]; k < L->rowptr[i + 1]; k++) t += L->val[k] * e[L->col[k]];
        r[i] = f[i] - t;
    }
}

/* V(1,1) cycle with l1-Jacobi smoothing, zero initial guess */
static void vcycle(ora_sim *s, int l, const double *f, double *e) {
    level_t *L = &s->lev[l];
    int n = L->n;
    if (l == s->nlev - 1) {
        memcpy(e, f, sizeof(double) * n);
        lu_solve(n, L->lu, L->piv, e);
        return;
    }
    level_t *C = &s->lev[l + 1];
    for (int i = 0; i < n; i++) e[i] = f[i] / L->dl1[i];
    csr_residual(L, f, e, L->t1);
    double *fc = C->t2, *ec = C->t3;
    for (int I = 0; I < C->n; I++) {
        double t = 0.0;
        for (int q = L->moff[I]; q < L->moff[I + 1]; q++) t += L->t1[L->mem[q]];
        fc[I] = t;
    }
    vcycle(s, l + 1, fc, ec);
    for (int i = 0; i < n; i++) e[i] += ec[L->agg[i]];
    csr_residual(L, f, e, L->t1);
    for (int i = 0; i < n; i++) e[i] += L->t1[i] / L->dl1[i];
}

/* ------------------------------------------------------------------------ */
/* CPR preconditioner (Sec. 2.4.2)                                           */
/* ------------------------------------------------------------------------ */
void ora_precond_setup(ora_sim *s) {
    int N = s->N, b = s->b;
    const ora_input *in = &s->in;
    /* the preconditioner is built from Jp: the Schur complement S of the well
       unknowns restricted to the 7-point block pattern, i.e. J minus
       A_pw[q] A_ww^-1 A_wp[q'] for perforations q, q' of one rate-controlled
       well whose cells coincide or are stencil neighbours */
    memcpy(s->Jp, s->J, sizeof(double) * (size_t)N * 7 * b * b);
    for (int q = 0; q < s->nperf; q++) {
        int w = s->perf_well[q];
        if (!s->wctrl[w]) continue;
        int i = s->perf_cell[q];
        for (int q2 = 0; q2 < s->nperf; q2++) {
            if (s->perf_well[q2] != w) continue;
            for (int d = 0; d < 7; d++) {
                if (nbr(s, i, d) != s->perf_cell[q2]) continue;
                double *B = JP(s, i, d);
                for (int r = 0; r < b; r++)
                    for (int c = 0; c < b; c++) B[r * b + c] -= s->apw[q * 3 + r] * s->awp[q2 * 3 + c] / s->aww[w];
            }
        }
    }
    if (in->precond == 1) {
        for (int i = 0; i < N; i++) inv_block(b, JP(s, i, 0), &s->dinv[(size_t)i * b * b]);
        s->precond_ready = 1;
        return;
    }
    if (in->precond != 2) { s->precond_ready = 1; return; }
    /* decoupling: a per-cell left scaling L_i of the cell's equations.
       quasi-IMPES: the pressure (first) row becomes w^T times the rows with
       w = (1, -d_ps D_ss^-1) from the diagonal block D = J_ii, the other rows
       stay; ABF: L_i = D^-1 (alternate block factorisation). */
    for (int i = 0; i < N; i++) {
        const double *D = JP(s, i, 0);
        double *L = &s->lsc[(size_t)i * b * b];
        if (in->decouple == 1) {
            inv_block(b, D, L);
        } else {
            double w1, w2 = 0.0;
            if (b == 2) {
                w1 = -(D[1] / D[3]);
            } else {
                double det = D[4] * D[8] - D[5] * D[7];
                w1 = (D[2] * D[7] - D[1] * D[8]) / det;
                w2 = (D[1] * D[5] - D[2] * D[4]) / det;
            }
            for (int t = 0; t < b * b; t++) L[t] = (t / b == t % b) ? 1.0 : 0.0;
            L[1] = w1;
            if (b == 3) L[2] = w2;
        }
        for (int c = 0; c < b; c++) s->qiw[i * b + c] = L[c];
    }
    /* decoupled matrix Ahat_ij = L_i J_ij (products summed in row order) */
    for (int i = 0; i < N; i++) {
        const double *L = &s->lsc[(size_t)i * b * b];
        for (int d = 0; d < 7; d++) {
            const double *A = JP(s, i, d);
            double *Ah = AH(s, i, d);
            for (int r = 0; r < b; r++)
                for (int c = 0; c < b; c++) {
                    double t = L[r * b] * A[c];
                    t = t + L[r * b + 1] * A[b + c];
                    if (b == 3) t = t + L[r * b + 2] * A[2 * b + c];
                    Ah[r * b + c] = t;
                }
        }
    }
    /* pressure block as CSR with ascending columns: -z, -y, -x, centre, +x, +y, +z */
    static const int dorder[7] = {5, 3, 1, 0, 2, 4, 6};
    int32_t *rp = xmalloc(sizeof(int32_t) * (N + 1));
    int32_t *col = xmalloc(sizeof(int32_t) * (size_t)N * 7);
    double *val = xmalloc(sizeof(double) * (size_t)N * 7);
    int nnz = 0;
    for (int i = 0; i < N; i++) {
        rp[i] = nnz;
        for (int t = 0; t < 7; t++) {
            int d = dorder[t], j = nbr(s, i, d);
            if (j < 0) continue;
            col[nnz] = j; val[nnz] = AH(s, i, d)[0]; nnz++;
        }
    }
    rp[N] = nnz;
    amg_setup(s, rp, col, val, N);
    /* second stage on the decoupled matrix */
    for (int i = 0; i < N; i++) {
        int ix, iy, iz; cell_ijk(s, i, &ix, &iy, &iz);
        double *Di = &s->dinv[(size_t)i * b * b];
        if (in->stage2 == 1 && ((ix + iy + iz) & 1)) continue;   /* black cells after all red ones */
        if (in->stage2 == 2) continue;                              /* natural order: below */
        inv_block(b, AH(s, i, 0), Di);
    }
    if (in->stage2 == 2) {
        /* natural (lexicographic) order: on the 7-point pattern ILU(0) only
           modifies the diagonal blocks, D_i = Ahat_ii - sum over the lower
           neighbours j (-x, -y, -z) of Ahat_ij D_j^-1 Ahat_ji */
        for (int i = 0; i < N; i++) {
            double D[9], T1[9], T2[9];
            memcpy(D, AH(s, i, 0), sizeof(double) * b * b);
            for (int d = 1; d < 7; d += 2) {
                int k = nbr(s, i, d);
                if (k < 0) continue;
                matmul_block(b, &s->dinv[(size_t)k * b * b], AH(s, k, opp(d)), T1);
                matmul_block(b, AH(s, i, d), T1, T2);
                for (int t = 0; t < b * b; t++) D[t] -= T2[t];
            }
            inv_block(b, D, &s->dinv[(size_t)i * b * b]);
        }
    }
    if (in->stage2 == 1) {
        for (int i = 0; i < N; i++) {
            int ix, iy, iz; cell_ijk(s, i, &ix, &iy, &iz);
            if (!((ix + iy + iz) & 1)) continue;
            double D[9], T1[9], T2[9];
            memcpy(D, AH(s, i, 0), sizeof(double) * b * b);
            for (int d = 1; d < 7; d++) {
                int k = nbr(s, i, d);
                if (k < 0) continue;
                matmul_block(b, &s->dinv[(size_t)k * b * b], AH(s, k, opp(d)), T1);
                matmul_block(b, AH(s, i, d), T1, T2);
                for (int t = 0; t < b * b; t++) D[t] -= T2[t];
            }
            inv_block(b, D, &s->dinv[(size_t)i * b * b]);
        }
    }
    s->precond_ready = 1;
}

/* stage F: one application of red-black block ILU(0) (or block-Jacobi) of
   the decoupled matrix: out = M_F^-1 rhs */
static void stage_f(ora_sim *s, const double *rhs, double *out) {
    int N = s->N, b = s->b;
    double t[3], u[3];
    if (s->in.stage2 == 2) {
        /* natural order: (D + L) D^-1 (D + U) x = rhs with L, U the lower (-x, -y,
           -z) and upper (+x, +y, +z) neighbour blocks of Ahat */
        for (int i = 0; i < N; i++) {          /* forward: y = (D + L)^-1 rhs, D y_i = rhs_i - L y */
            for (int c = 0; c < b; c++) t[c] = rhs[i * b + c];
            for (int d = 1; d < 7; d += 2) {
                int k = nbr(s, i, d);
                if (k < 0) continue;
                matvec_block(b, AH(s, i, d), &out[k * b], u);
                for (int c = 0; c < b; c++) t[c] -= u[c];
            }
            matvec_block(b, &s->dinv[(size_t)i * b * b], t, &out[i * b]);
        }
        for (int i = N - 1; i >= 0; i--) {     /* backward: x_i = y_i - D_i^-1 U x */
            for (int c = 0; c < b; c++) t[c] = 0.0;
            for (int d = 2; d < 7; d += 2) {
                int k = nbr(s, i, d);
                if (k < 0) continue;
                matvec_block(b, AH(s, i, d), &out[k * b], u);
                for (int c = 0; c < b; c++) t[c] += u[c];
            }
            matvec_block(b, &s->dinv[(size_t)i * b * b], t, u);
            for (int c = 0; c < b; c++) out[i * b + c] -= u[c];
        }
        return;
    }
    if (s->in.stage2 != 1) {
        for (int i = 0; i < N; i++) matvec_block(b, &s->dinv[(size_t)i * b * b], &rhs[i * b], &out[i * b]);
        return;
    }
    for (int i = 0; i < N; i++) {           /* forward, red */
        int ix, iy, iz; cell_ijk(s, i, &ix, &iy, &iz);
        if ((ix + iy + iz) & 1) continue;
        matvec_block(b, &s->dinv[(size_t)i * b * b], &rhs[i * b], &out[i * b]);
    }
    for (int i = 0; i < N; i++) {           /* forward, black */
        int ix, iy, iz; cell_ijk(s, i, &ix, &iy, &iz);
        if (!((ix + iy + iz) & 1)) continue;
        for (int c = 0; c < b; c++) t[c] = rhs[i * b + c];
        for (int d = 1; d < 7; d++) {
            int k = nbr(s, i, d);
            if (k < 0) continue;
            matvec_block(b, AH(s, i, d), &out[k * b], u);
            for (int c = 0; c < b; c++) t[c] -= u[c];
        }
        matvec_block(b, &s->dinv[(size_t)i * b * b], t, &out[i * b]);
    }
    for (int i = 0; i < N; i++) {           /* backward, red (black unchanged) */
        int ix, iy, iz; cell_ijk(s, i, &ix, &iy, &iz);
        if ((ix + iy + iz) & 1) continue;
        for (int c = 0; c < b; c++) t[c] = 0.0;
        for (int d = 1; d < 7; d++) {
            int k = nbr(s, i, d);
            if (k < 0) continue;
            matvec_block(b, AH(s, i, d), &out[k * b], u);
            for (int c = 0; c < b; c++) t[c] += u[c];
        }
        matvec_block(b, &s->dinv[(size_t)i * b * b], t, u);
        for (int c = 0; c < b; c++) out[i * b + c] -= u[c];
    }
}

/* stage P: AMG V-cycles on fp, each on the residual left by the previous ones */
static void stage_p(ora_sim *s, const double *fp, double *ep) {
    vcycle(s, 0, fp, ep);
    for (int c = 1; c < s->in.amg_cycles; c++) {
        level_t *L0 = &s->lev[0];
        double *rp = L0->t2, *dp = L0->t3;
        csr_residual(L0, fp, ep, rp);
        vcycle(s, 0, rp, dp);
        for (int i = 0; i < s->N; i++) ep[i] += dp[i];
    }
}

void ora_precond_apply(ora_sim *s, const double *r, double *z) {
    int N = s->N, b = s->b;
    const ora_input *in = &s->in;
    if (!s->precond_ready) ora_precond_setup(s);
    if (in->precond == 0) { memcpy(z, r, sizeof(double) * N * b); return; }
    if (in->precond == 1) {
        for (int i = 0; i < N; i++) matvec_block(b, &s->dinv[(size_t)i * b * b], &r[i * b], &z[i * b]);
        return;
    }
    double *rh = s->tmp, *ep = s->tmp2, *fp = s->tmp3;
    /* decoupled residual rh = L r */
    for (int i = 0; i < N; i++) {
        const double *L = &s->lsc[(size_t)i * b * b];
        for (int rr = 0; rr < b; rr++) {
            double t = L[rr * b] * r[i * b];
            t = t + L[rr * b + 1] * r[i * b + 1];
            if (b == 3) t = t + L[rr * b + 2] * r[i * b + 2];
            rh[i * b + rr] = t;
        }
    }
    double *x0 = NULL;
    if (in->cpr_stages == 3) {
        /* CPR-FPF: a stage F first; stage P then works on what it leaves */
        x0 = xmalloc(sizeof(double) * N * b);
        stage_f(s, rh, x0);
        block_spmv(s, s->ahat, x0, z);                       /* z = Ahat x0 */
        for (int t = 0; t < N * b; t++) rh[t] -= z[t];        /* rh = residual after the first F */
    }
    for (int i = 0; i < N; i++) fp[i] = rh[i * b];
    stage_p(s, fp, ep);
    /* residual of the decoupled system after stage P (pressure columns only) */
    for (int i = 0; i < N; i++) {
        for (int c = 0; c < b; c++) {
            double t = rh[i * b + c];
            for (int d = 0; d < 7; d++) {
                int j = nbr(s, i, d);
                if (j < 0) continue;
                t -= AH(s, i, d)[c * b] * ep[j];
            }
            z[i * b + c] = t;      /* z holds r2 for now */
        }
    }
    memcpy(rh, z, sizeof(double) * N * b);
    stage_f(s, rh, z);
    for (int i = 0; i < N; i++) z[i * b] += ep[i];
    if (x0) {
        for (int t = 0; t < N * b; t++) z[t] += x0[t];
        free(x0);
    }
}

void ora_get_qi(const ora_sim *s, double *w, double *ap) {
    memcpy(w, s->qiw, sizeof(double) * s->N * s->b);
    for (int i = 0; i < s->N; i++)
        for (int d = 0; d < 7; d++) ap[i * 7 + d] = s->ahat[(((size_t)i * 7 + d) * s->b) * s->b];
}
int ora_amg_levels(const ora_sim *s) { return s->nlev; }
int ora_amg_level_n(const ora_sim *s, int l) { return s->lev[l].n; }
int ora_amg_level_nnz(const ora_sim *s, int l) { return s->lev[l].nnz; }
void ora_amg_level_csr(const ora_sim *s, int l, int32_t *rp, int32_t *col, double *val) {
    const level_t *L = &s->lev[l];
    memcpy(rp, L->rowptr, sizeof(int32_t) * (L->n + 1));
    memcpy(col, L->col, sizeof(int32_t) * L->nnz);
    memcpy(val, L->val, sizeof(double) * L->nnz);
}
void ora_amg_level_agg(const ora_sim *s, int l, int32_t *agg) {
    const level_t *L = &s->lev[l];
    if (L->agg) memcpy(agg, L->agg, sizeof(int32_t) * L->n);
}
void ora_ilu_dinv(const ora_sim *s, double *dinv) { memcpy(dinv, s->dinv, sizeof(double) * (size_t)s->N * s->b * s->b); }

/* ------------------------------------------------------------------------ */
/* right-preconditioned FGMRES(m) with classical Gram-Schmidt + one full     */
/* reorthogonalisation, Givens rotations, zero initial guess (the inexact solve of Algorithm 1, Eq. 13) */
/* ------------------------------------------------------------------------ */
static double dot(const double *a, const double *b, int n) { double t = 0.0; for (int i = 0; i < n; i++) t += a[i] * b[i]; return t; }

static int bicgstab(ora_sim *s, const double *bvec, double *x, ora_lin_info *info);

int ora_linear_solve(ora_sim *s, const double *bvec, double *x, ora_lin_info *info) {
    const ora_input *in = &s->in;
    if (in->krylov == 1) return bicgstab(s, bvec, x, info);
    int n = s->N * s->b, m = in->gmres_m;
    ora_lin_info li; memset(&li, 0, sizeof(li));
    if (!s->precond_ready) ora_precond_setup(s);
    double bn = sqrt(dot(bvec, bvec, n));
    li.b_norm = bn;
    for (int i = 0; i < n; i++) x[i] = 0.0;
    if (bn == 0.0) { li.converged = 1; memcpy(s->r, bvec, sizeof(double) * n); if (info) *info = li; return 0; }
    double tol = s->theta * bn;
    memcpy(s->r, bvec, sizeof(double) * n);
    double beta = bn;
    double *H = s->H, *g = s->g, *cs = s->cs, *sn = s->sn, *y = s->y, *h2 = s->tmp3;
    (void)h2;
    double hcol[64], hre[64];
    for (int cyc = 0; cyc <= in->gmres_max_restarts; cyc++) {
        double *V0 = s->V;
        for (int i = 0; i < n; i++) V0[i] = s->r[i] / beta;
        for (int j = 0; j <= m; j++) g[j] = 0.0;
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m; j++) {
            double *vj = s->V + (size_t)j * n, *zj = s->Z + (size_t)j * n, *w = s->w;
            ora_precond_apply(s, vj, zj);
            op_apply(s, zj, w);
            /* CGS pass 1 */
            const double wn2 = dot(w, w, n);
            for (int i = 0; i <= j; i++) hcol[i] = dot(s->V + (size_t)i * n, w, n);
            for (int i = 0; i <= j; i++) { const double *vi = s->V + (size_t)i * n; for (int t = 0; t < n; t++) w[t] -= hcol[i] * vi[t]; }
            /* CGS pass 2: always (CGS2), or when pass 1 removed more than half of
               ||w||^2, i.e. ||w||^2 - sum h^2 < ||w||^2 / 2 (selective form) */
            double hh = 0.0;
            for (int i = 0; i <= j; i++) hh += hcol[i] * hcol[i];
            if (!in->orth || hh > 0.5 * wn2) {
                for (int i = 0; i <= j; i++) hre[i] = dot(s->V + (size_t)i * n, w, n);
                for (int i = 0; i <= j; i++) { const double *vi = s->V + (size_t)i * n; for (int t = 0; t < n; t++) w[t] -= hre[i] * vi[t]; }
                for (int i = 0; i <= j; i++) hcol[i] += hre[i];
            }
            double hn = sqrt(dot(w, w, n));
            double *vn = s->V + (size_t)(j + 1) * n;
            if (hn > 0.0) for (int t = 0; t < n; t++) vn[t] = w[t] / hn;
            else for (int t = 0; t < n; t++) vn[t] = 0.0;
            /* previous rotations on column j */
            for (int i = 0; i < j; i++) {
                double a = hcol[i], c2 = hcol[i + 1];
                hcol[i] = cs[i] * a + sn[i] * c2;
                hcol[i + 1] = -sn[i] * a + cs[i] * c2;
            }
            double a = hcol[j], bb = hn;
            double rr = sqrt(a * a + bb * bb);
            if (rr == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
            else { cs[j] = a / rr; sn[j] = bb / rr; }
            hcol[j] = rr;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            for (int i = 0; i <= j; i++) H[i * (m + 1) + j] = hcol[i];
            li.iterations++;
            k = j + 1;
            if (fabs(g[j + 1]) <= tol) break;
        }
        /* back substitution H y = g */
        for (int i = k - 1; i >= 0; i--) {
            double t = g[i];
            for (int c = i + 1; c < k; c++) t -= H[i * (m + 1) + c] * y[c];
            y[i] = t / H[i * (m + 1) + i];
        }
        for (int i = 0; i < k; i++) { const double *zi = s->Z + (size_t)i * n; for (int t = 0; t < n; t++) x[t] += y[i] * zi[t]; }
        op_apply(s, x, s->w);
        for (int t = 0; t < n; t++) s->r[t] = bvec[t] - s->w[t];
        beta = sqrt(dot(s->r, s->r, n));
        li.r_norm = beta;
        if (beta <= tol) { li.converged = 1; break; }
        if (!(beta == beta)) break;
        li.restarts++;
    }
    if (info) *info = li;
    return li.converged ? 0 : 1;
}

/* right-preconditioned BiCGSTAB (van der Vorst), the Krylov solver of the
   paper's experiments (Sec. 4), zero initial guess.  When the recursive
   residual meets the tolerance, the true residual b - A x decides; if it does
   not, or on a breakdown (rho, (rhat, v) or omega zero), the method restarts
   from the current x with rhat = r.  One iteration = two preconditioner
   applications and two products with A (half an iteration counts as one). */
static int bicgstab(ora_sim *s, const double *bvec, double *x, ora_lin_info *info) {
    const ora_input *in = &s->in;
    const int n = s->N * s->b;
    ora_lin_info li; memset(&li, 0, sizeof(li));
    if (!s->precond_ready) ora_precond_setup(s);
    const double bn = sqrt(dot(bvec, bvec, n));
    li.b_norm = bn;
    for (int i = 0; i < n; i++) x[i] = 0.0;
    double *r = s->r;
    memcpy(r, bvec, sizeof(double) * n);
    if (bn == 0.0) { li.converged = 1; if (info) *info = li; return 0; }
    const double tol = s->theta * bn;
    double *rh = s->V, *p = s->V + n, *v = s->V + 2 * (size_t)n, *sv = s->V + 3 * (size_t)n,
           *t = s->V + 4 * (size_t)n, *ph = s->Z, *sh = s->Z + n;
    memcpy(rh, r, sizeof(double) * n);
    double rho_old = 1.0, alpha = 1.0, omega = 1.0;
    int fresh = 1;                       /* first iteration of a (re)start */
    li.r_norm = bn;
    while (li.iterations < in->lin_max_iter) {
        const double rho = dot(rh, r, n);
        int check = 0, breakdown = 0;
        if (rho == 0.0 || !(rho == rho)) breakdown = 1;     /* r orthogonal to rh (r = 0 after a restart) */
        else {
            if (fresh) memcpy(p, r, sizeof(double) * n);
            else {
                const double beta = (rho / rho_old) * (alpha / omega);
                for (int i = 0; i < n; i++) p[i] = r[i] + beta * (p[i] - omega * v[i]);
            }
            ora_precond_apply(s, p, ph);
            op_apply(s, ph, v);
            const double rv = dot(rh, v, n);
            li.iterations++;
            if (rv == 0.0 || !(rv == rv)) breakdown = 1;
            else {
                alpha = rho / rv;
                for (int i = 0; i < n; i++) sv[i] = r[i] - alpha * v[i];
                if (sqrt(dot(sv, sv, n)) <= tol) {
                    for (int i = 0; i < n; i++) x[i] += alpha * ph[i];
                    check = 1;
                } else {
                    ora_precond_apply(s, sv, sh);
                    op_apply(s, sh, t);
                    const double tt = dot(t, t, n);
                    omega = tt > 0.0 ? dot(t, sv, n) / tt : 0.0;
                    for (int i = 0; i < n; i++) x[i] += alpha * ph[i] + omega * sh[i];
                    for (int i = 0; i < n; i++) r[i] = sv[i] - omega * t[i];
                    if (sqrt(dot(r, r, n)) <= tol) check = 1;
                    else if (omega == 0.0 || !(omega == omega)) breakdown = 1;
                }
            }
        }
        rho_old = rho;
        fresh = 0;
        if (check || breakdown) {
            op_apply(s, x, s->w);
            for (int i = 0; i < n; i++) r[i] = bvec[i] - s->w[i];
            li.r_norm = sqrt(dot(r, r, n));
            if (li.r_norm <= tol) { li.converged = 1; break; }
            if (!(li.r_norm == li.r_norm) || li.iterations >= in->lin_max_iter) break;
            memcpy(rh, r, sizeof(double) * n);
            fresh = 1;
            li.restarts++;
        }
    }
    if (!li.converged) {
        op_apply(s, x, s->w);
        for (int i = 0; i < n; i++) r[i] = bvec[i] - s->w[i];
        li.r_norm = sqrt(dot(r, r, n));
    }
    if (info) *info = li;
    return li.converged ? 0 : 1;
}

/* ------------------------------------------------------------------------ */
/* inexact Newton (Algorithm 1) and time stepping                            */
/* ------------------------------------------------------------------------ */
/* x += dx with the per-cell Appleyard chop, saturations clamped to their
   physical range, then the black-oil variable switch: free gas vanishing
   (Sg < 0) makes the cell undersaturated at pb = p; pb rising above p, or
   the oil leaving the cell (no oil, no bubble point), makes it saturated at
   Sg = 0 */
static void newton_update(ora_sim *s, const double *dx) {
    int b = s->b;
    const ora_input *in = &s->in;
    for (int i = 0; i < s->N; i++) {
        double *xi = &s->x[i * b];
        const double *d = &dx[i * b];
        double ds = fabs(d[1]), dp = fabs(d[0]);
        if (b == 3) { if (s->ph[i]) { if (fabs(d[2]) > ds) ds = fabs(d[2]); } else { if (fabs(d[2]) > dp) dp = fabs(d[2]); } }
        double f = 1.0;
        if (ds > in->chop_ds) f = in->chop_ds / ds;
        if (dp > in->chop_dp && in->chop_dp / dp < f) f = in->chop_dp / dp;
        for (int c = 0; c < b; c++) xi[c] += f * d[c];
        /* saturations stay physical: 0 <= Sw <= 1, Sg <= 1 - Sw */
        if (xi[1] < 0.0) xi[1] = 0.0;
        if (xi[1] > 1.0) xi[1] = 1.0;
        if (b == 3) {
            if (s->ph[i] && xi[2] < 0.0) { s->ph[i] = 0; xi[2] = xi[0]; }
            else if (!s->ph[i] && xi[2] > xi[0]) { s->ph[i] = 1; xi[2] = 0.0; }
            if (!s->ph[i] && xi[1] > 1.0 - 1e-6) { s->ph[i] = 1; xi[2] = 0.0; }
            if (s->ph[i] && xi[2] > 1.0 - xi[1]) xi[2] = 1.0 - xi[1];
        }
    }
}

static int finite_vec(const double *a, int n) { for (int i = 0; i < n; i++) if (!(a[i] - a[i] == 0.0)) return 0; return 1; }

/* right-hand side of the reduced system: -R + A_pw A_ww^-1 R_w */
static void reduced_rhs(const ora_sim *s, double *rhs) {
    int b = s->b, n = s->N * b;
    for (int t = 0; t < n; t++) rhs[t] = -s->R[t];
    if (!s->nrate) return;
    for (int q = 0; q < s->nperf; q++) {
        int w = s->perf_well[q];
        if (!s->wctrl[w]) continue;
        double u = s->rw[w] / s->aww[w];
        for (int c = 0; c < b; c++) rhs[s->perf_cell[q] * b + c] += s->apw[q * 3 + c] * u;
    }
}

/* well update from the cell update: dp_h = (-R_w - A_wp dx) / A_ww, limited
   to chop_dp like a cell pressure (zero for BHP-controlled wells) */
static int well_update(ora_sim *s, const double *dx) {
    int b = s->b;
    for (int w = 0; w < s->in.nwells; w++) {
        if (!s->wctrl[w]) continue;
        double t = -s->rw[w];
        for (int q = 0; q < s->nperf; q++) {
            if (s->perf_well[q] != w) continue;
            for (int k = 0; k < b; k++) t -= s->awp[q * 3 + k] * dx[s->perf_cell[q] * b + k];
        }
        double d = t / s->aww[w];
        if (d != d) return 0;                                    /* NaN: the solve failed */
        if (fabs(d) > s->in.chop_dp) d = d > 0 ? s->in.chop_dp : -s->in.chop_dp;   /* also +-inf */
        s->wp[w] += d;
    }
    return 1;
}

/* one Newton iteration: assemble, solve J dx = -R, update */
int ora_newton_step(ora_sim *s, double dt, ora_newton_info *info) {
    int n = s->N * s->b;
    ora_assemble(s, dt);
    double cnv = ora_cnv(s, dt);
    ora_newton_info ni; memset(&ni, 0, sizeof(ni));
    ni.cnv = cnv;
    if (cnv <= s->in.newton_tol && well_cnv(s) <= s->in.newton_tol) { ni.converged = 1; if (info) *info = ni; return 0; }
    double *rhs = xmalloc(sizeof(double) * n), *dx = xmalloc(sizeof(double) * n);
    reduced_rhs(s, rhs);
    ora_lin_info li;
    ora_linear_solve(s, rhs, dx, &li);
    ni.newton_iterations = 1; ni.linear_iterations = li.iterations; ni.linear_failures = !li.converged;
    int ok = finite_vec(dx, n);
    if (ok) ok = well_update(s, dx);
    if (ok) newton_update(s, dx);
    free(rhs); free(dx);
    if (info) *info = ni;
    return ok ? 0 : 2;
}

/* forcing term theta_l of Algorithm 1 (Eq. 14).  Reading: norms are 2-norms of
   the raw residual; r^{l-1} is the linear residual b^{l-1} - A dx left by the
   previous solve; choice 2 takes the absolute value of its numerator; choice 3
   uses gamma, beta as given.  The first iteration of a Newton solve uses
   theta_max.  Safeguards of Eisenstat and Walker (1996): theta does not fall
   below theta_{l-1}^((1+sqrt 5)/2) (choices 1, 2) or gamma theta_{l-1}^beta
   (choice 3) while that bound exceeds 0.1; then lin_tol <= theta <= theta_max. */
static double forcing_term(const ora_sim *s, int l, const double *bl, double bnorm, double bprev, double rprev,
                           double theta_prev) {
    const ora_input *in = &s->in;
    if (in->forcing == 0) return in->lin_tol;
    if (l == 0) return in->theta_max;
    const int n = s->N * s->b;
    double th, guard;
    if (in->forcing == 1) {
        double t2 = 0.0;
        for (int i = 0; i < n; i++) { const double d = bl[i] - s->rlin[i]; t2 += d * d; }
        th = sqrt(t2) / bprev;
        guard = pow(theta_prev, 0.5 * (1.0 + sqrt(5.0)));
    } else if (in->forcing == 2) {
        th = fabs(bnorm - rprev) / bprev;
        guard = pow(theta_prev, 0.5 * (1.0 + sqrt(5.0)));
    } else {
        th = in->ew_gamma * pow(bnorm / bprev, in->ew_beta);
        guard = in->ew_gamma * pow(theta_prev, in->ew_beta);
    }
    if (guard > 0.1 && guard > th) th = guard;
    if (th > in->theta_max) th = in->theta_max;
    if (th < in->lin_tol) th = in->lin_tol;
    return th;
}

/* Newton loop of Algorithm 1 until CNV <= tol; 0 = converged */
int ora_newton_solve(ora_sim *s, double dt, ora_newton_info *info) {
    int n = s->N * s->b;
    ora_newton_info ni; memset(&ni, 0, sizeof(ni));
    double *rhs = xmalloc(sizeof(double) * n), *dx = xmalloc(sizeof(double) * n);
    int rc = 1;
    double bprev = 0.0, rprev = 0.0, theta = s->in.lin_tol;
    s->nhist = 0;
    for (int l = 0;; l++) {
        ora_assemble(s, dt);
        double cnv = ora_cnv(s, dt);
        ni.cnv = cnv;
        if (!(cnv == cnv)) { rc = 2; break; }
        if (cnv <= s->in.newton_tol && well_cnv(s) <= s->in.newton_tol) { rc = 0; ni.converged = 1; break; }
        if (l >= s->in.newton_max) { rc = 1; break; }
        reduced_rhs(s, rhs);
        const double bnorm = sqrt(dot(rhs, rhs, n));
        theta = forcing_term(s, l, rhs, bnorm, bprev, rprev, theta);
        s->theta = theta;
        ora_lin_info li;
        ora_linear_solve(s, rhs, dx, &li);
        s->theta = s->in.lin_tol;
        bprev = bnorm; rprev = li.r_norm;
        memcpy(s->rlin, s->r, sizeof(double) * n);
        if (s->nhist < 64) {
            s->hist_theta[s->nhist] = theta; s->hist_b[s->nhist] = bnorm; s->hist_r[s->nhist] = li.r_norm;
            s->nhist++;
        }
        ni.newton_iterations++; ni.linear_iterations += li.iterations; ni.linear_failures += !li.converged;
        if (!finite_vec(dx, n) || !well_update(s, dx)) { rc = 2; break; }
        newton_update(s, dx);
    }
    free(rhs); free(dx);
    if (info) *info = ni;
    return rc;
}

int ora_forcing_history(const ora_sim *s, double *theta, double *b_norm, double *r_norm, int max) {
    int k = s->nhist < max ? s->nhist : max;
    for (int i = 0; i < k; i++) { theta[i] = s->hist_theta[i]; b_norm[i] = s->hist_b[i]; r_norm[i] = s->hist_r[i]; }
    return k;
}

/* advance by dt; a failed Newton solve restores the last state and halves the step */
int ora_step(ora_sim *s, double dt, ora_step_info *info) {
    ora_step_info si; memset(&si, 0, sizeof(si));
    double remaining = dt, h = dt;
    int rc = 0;
    while (remaining > 1e-12 * dt) {
        if (h > remaining) h = remaining;
        ora_newton_info ni;
        int r = ora_newton_solve(s, h, &ni);
        si.newton_iterations += ni.newton_iterations;
        si.linear_iterations += ni.linear_iterations;
        if (r == 0) {
            for (int c = 0; c < 3; c++) s->cum_well[c] += h * s->qtot[c];
            remaining -= h;
            si.substeps++;
            begin_step(s);
        } else {
            memcpy(s->x, s->x_old, sizeof(double) * s->N * s->b);
            memcpy(s->wp, s->wp_old, sizeof(double) * s->in.nwells);
            memcpy(s->ph, s->ph_old, s->N);
            si.cuts++;
            if (si.cuts > s->in.max_cuts) { rc = 1; break; }
            h *= 0.5;
        }
    }
    si.ok = rc == 0;
    if (info) *info = si;
    return rc;
}

/* property probe for the closed-form pins */
double ora_props_probe(const ora_input *in, int what, double p, double sw, double x3, int ph, double *grad) {
    cellprops cp;
    double x[3] = {p, sw, x3};
    eval_props(in, 1.0, 1.0, x, ph, &cp);
    dual r;
    switch (what) {
    case 0: r = cp.kr[PW]; break;
    case 1: r = cp.kr[PO]; break;
    case 2: r = cp.kr[PG]; break;
    case 3: r = cp.rho[PW]; break;
    case 4: r = cp.rho[PO]; break;
    case 5: r = cp.rho[PG]; break;
    case 6: r = cp.mob[PW][CW]; break;
    case 7: r = cp.mob[PO][CO]; break;
    case 8: r = cp.mob[PO][CG]; break;
    case 9: r = cp.mob[PG][CG]; break;
    case 10: r = cp.bo; break;
    case 11: r = cp.rs; break;
    case 12: r = cp.muo; break;
    case 13: r = cp.acc[CW]; break;
    case 14: r = cp.acc[CO]; break;
    case 15: r = cp.acc[CG]; break;
    case 16: r = cp.lamt; break;
    default: r = dc(NAN);
    }
    if (grad) for (int k = 0; k < 3; k++) grad[k] = r.d[k];
    return r.v;
}
