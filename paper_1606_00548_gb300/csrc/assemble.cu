// Residual and Jacobian assembly on the device (FP64), Newton update, norms.
//
// Discretisation (paper Sec. 2.4): backward Euler (Eq. 10), two-point
// cell-centred fluxes with transmissibility K kr rho A / (mu dd) (Eq. 11),
// phase potentials from Eq. (4) with zero capillary pressure, wells by the
// sink/source rate of Eq. (6) under BHP control (Eq. 7) with the Peaceman
// index.  Readings of the open points: depth z positive down with
// Phi = p - rho g z; harmonic face transmissibility; single-point upstream
// weighting per phase (tie -> lower-index cell); arithmetic-mean face density;
// water injectors inject at the cell's total mobility.
//
// Layout: x, R [c][N]; J [d][r][c][N]; per-cell flux properties
// [q][1+b][N] with q = phase densities then (phase, component) mobilities.
// One thread per cell writes only its own rows, so no atomics are needed;
// each face flux is evaluated by both of its cells in the same canonical
// (L, R) orientation, so the two contributions cancel exactly.

#include "sim_internal.cuh"

namespace {

template <int B>
struct Dl {
    double v, d[B];
};

template <int B> __device__ __forceinline__ Dl<B> cst(double v) {
    Dl<B> r; r.v = v;
#pragma unroll
    for (int k = 0; k < B; k++) r.d[k] = 0.0;
    return r;
}
template <int B> __device__ __forceinline__ Dl<B> var(double v, int which) {
    Dl<B> r = cst<B>(v);
#pragma unroll
    for (int k = 0; k < B; k++) r.d[k] = (k == which) ? 1.0 : 0.0;
    return r;
}
template <int B> __device__ __forceinline__ Dl<B> operator+(Dl<B> a, Dl<B> b) {
    Dl<B> r; r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < B; k++) r.d[k] = a.d[k] + b.d[k];
    return r;
}
template <int B> __device__ __forceinline__ Dl<B> operator-(Dl<B> a, Dl<B> b) {
    Dl<B> r; r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < B; k++) r.d[k] = a.d[k] - b.d[k];
    return r;
}
template <int B> __device__ __forceinline__ Dl<B> operator*(Dl<B> a, Dl<B> b) {
    Dl<B> r; r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < B; k++) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
template <int B> __device__ __forceinline__ Dl<B> operator/(Dl<B> a, Dl<B> b) {
    Dl<B> r; r.v = a.v / b.v;
    double ib2 = 1.0 / (b.v * b.v);
#pragma unroll
    for (int k = 0; k < B; k++) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) * ib2;
    return r;
}
template <int B> __device__ __forceinline__ Dl<B> operator*(Dl<B> a, double s) {
    Dl<B> r; r.v = a.v * s;
#pragma unroll
    for (int k = 0; k < B; k++) r.d[k] = a.d[k] * s;
    return r;
}
template <int B> __device__ __forceinline__ Dl<B> operator+(Dl<B> a, double s) { a.v += s; return a; }
template <int B> __device__ __forceinline__ Dl<B> operator-(double s, Dl<B> a) {
    Dl<B> r; r.v = s - a.v;
#pragma unroll
    for (int k = 0; k < B; k++) r.d[k] = -a.d[k];
    return r;
}
template <int B> __device__ __forceinline__ Dl<B> dexp(Dl<B> a) {
    Dl<B> r; r.v = exp(a.v);
#pragma unroll
    for (int k = 0; k < B; k++) r.d[k] = r.v * a.d[k];
    return r;
}
// Corey curve of a normalised saturation, clipped to [0, 1]
template <int B> __device__ __forceinline__ Dl<B> corey(Dl<B> s, double n) {
    if (s.v <= 0.0) return cst<B>(0.0);
    if (s.v >= 1.0) return cst<B>(1.0);
    Dl<B> r;
    double dr;
    if (n == 2.0) { r.v = s.v * s.v; dr = 2.0 * s.v; }
    else { r.v = pow(s.v, n); dr = n * pow(s.v, n - 1.0); }
#pragma unroll
    for (int k = 0; k < B; k++) r.d[k] = dr * s.d[k];
    return r;
}
// piecewise-linear table with linear extrapolation
template <int B> __device__ __forceinline__ Dl<B> lut(const double *xp, const double *yp, int n, Dl<B> x) {
    int k = 0;
    while (k + 1 <= n - 2 && x.v >= xp[k + 1]) k++;
    double slope = (yp[k + 1] - yp[k]) / (xp[k + 1] - xp[k]);
    Dl<B> r; r.v = (x.v - xp[k]) * slope + yp[k];
#pragma unroll
    for (int k2 = 0; k2 < B; k2++) r.d[k2] = x.d[k2] * slope;
    return r;
}

// phase / pair bookkeeping: pairs (phase, component) carried by the flux
// b = 2: (w,w) (o,o);  b = 3: (w,w) (o,o) (o,g) (g,g)
template <int B> struct Layout {
    static constexpr int NPH = B;
    static constexpr int NPAIR = (B == 2) ? 2 : 4;
    static constexpr int NQ = NPH + NPAIR;
    __device__ static int pair_phase(int q) { return B == 2 ? q : (q == 0 ? 0 : (q <= 2 ? 1 : 2)); }
    __device__ static int pair_comp(int q) { return B == 2 ? q : (q == 0 ? 0 : (q == 1 ? 1 : 2)); }
};

template <int B>
struct Props {
    Dl<B> acc[B];
    Dl<B> rho[B];
    Dl<B> mob[Layout<B>::NPAIR];
    Dl<B> lamt;
};

// per-cell properties, Eq. (3)-(5) ingredients
template <int B>
__device__ void cell_props(const FluidConst &f, double poro, double vol, double p, double sw, double x3, int ph,
                           Props<B> &o) {
    Dl<B> P = var<B>(p, 0), SW = var<B>(sw, 1);
    Dl<B> pv = ((P + (-f.p_ref)) * f.c_rock + 1.0) * poro * vol;
    if constexpr (B == 2) {
        Dl<B> rw = dexp((P + (-f.p_ref)) * f.c_w) * f.rho_w_ref;
        Dl<B> ro = dexp((P + (-f.p_ref)) * f.c_o) * f.rho_o_ref;
        Dl<B> se = (SW + (-f.swc)) * (1.0 / (1.0 - f.swc - f.sor));
        Dl<B> krw = corey(se, f.nw);
        Dl<B> kro = corey(1.0 - se, f.now);
        o.acc[0] = pv * (rw * SW);
        o.acc[1] = pv * (ro * (1.0 - SW));
        o.rho[0] = rw; o.rho[1] = ro;
        o.mob[0] = (rw * krw) * (1.0 / f.mu_w);
        o.mob[1] = (ro * kro) * (1.0 / f.mu_o);
        o.lamt = krw * (1.0 / f.mu_w) + kro * (1.0 / f.mu_o);
        return;
    } else {
        Dl<B> SG, BO, RS, MUO;
        if (ph) {
            SG = var<B>(x3, 2);
            BO = lut(f.pvt_p, f.pvt_bo, f.npvt, P);
            RS = lut(f.pvt_p, f.pvt_rs, f.npvt, P);
            MUO = lut(f.pvt_p, f.pvt_muo, f.npvt, P);
        } else {
            Dl<B> PB = var<B>(x3, 2);
            SG = cst<B>(0.0);
            Dl<B> dpu = P - PB;
            BO = lut(f.pvt_p, f.pvt_bo, f.npvt, PB) * (1.0 - dpu * f.bo_c_us);
            RS = lut(f.pvt_p, f.pvt_rs, f.npvt, PB);
            MUO = lut(f.pvt_p, f.pvt_muo, f.npvt, PB) * (dpu * f.muo_c_us + 1.0);
        }
        Dl<B> bwi = (P + (-f.bw_pref)) * f.bw_c + 1.0;
        Dl<B> one = cst<B>(1.0);
        Dl<B> boi = one / BO;
        Dl<B> bgi = one / lut(f.pvt_p, f.pvt_bg, f.npvt, P);
        Dl<B> MUG = lut(f.pvt_p, f.pvt_mug, f.npvt, P);
        Dl<B> SO = (1.0 - SW) - SG;
        Dl<B> krw = corey((SW + (-f.swc)) * (1.0 / (1.0 - f.swc - f.sor)), f.nw);
        Dl<B> krow = corey(((1.0 - f.sor) - SW) * (1.0 / (1.0 - f.swc - f.sor)), f.now);
        Dl<B> krg = corey((SG + (-f.sgc)) * (1.0 / (1.0 - f.swc - f.sorg - f.sgc)), f.ng);
        Dl<B> krog = corey(((1.0 - f.swc - f.sorg) - SG) * (1.0 / (1.0 - f.swc - f.sorg)), f.nog);
        // Stone II with krow(Swc) = 1
        Dl<B> kro = (krow + krw) * (krog + krg) - (krw + krg);
        if (kro.v < 0.0) kro = cst<B>(0.0);
        o.acc[0] = pv * ((bwi * SW) * f.rho_ws);
        o.acc[1] = pv * ((boi * SO) * f.rho_os);
        o.acc[2] = pv * ((RS * (boi * SO) + bgi * SG) * f.rho_gs);
        o.rho[0] = bwi * f.rho_ws;
        o.rho[1] = (RS * f.rho_gs + f.rho_os) * boi;
        o.rho[2] = bgi * f.rho_gs;
        Dl<B> lw = krw * (1.0 / f.mu_w);
        Dl<B> lo = kro / MUO;
        Dl<B> lg = krg / MUG;
        o.mob[0] = o.rho[0] * lw;
        o.mob[1] = (boi * f.rho_os) * lo;
        o.mob[2] = ((RS * boi) * f.rho_gs) * lo;
        o.mob[3] = o.rho[2] * lg;
        o.lamt = (lw + lo) + lg;
    }
}

__device__ __forceinline__ void cell_xyz(const GridDesc &g, int i, int &ix, int &iy, int &iz) {
    ix = i % g.nx;
    int t = i / g.nx;
    iy = t % g.ny;
    iz = t / g.ny;
}
__device__ __forceinline__ int nbr_of(const GridDesc &g, int i, int ix, int iy, int iz, int d) {
    switch (d) {
    case 1: return ix > 0 ? i - 1 : -1;
    case 2: return ix < g.nx - 1 ? i + 1 : -1;
    case 3: return iy > 0 ? i - g.nx : -1;
    case 4: return iy < g.ny - 1 ? i + g.nx : -1;
    case 5: return iz > 0 ? i - g.nx * g.ny : -1;
    case 6: return iz < g.nz - 1 ? i + g.nx * g.ny : -1;
    }
    return i;
}

// ---------------------------------------------------------------------------
// geometry: transmissibilities (Eq. 11, harmonic) and Peaceman well indices
// ---------------------------------------------------------------------------
__global__ void geometry_kernel(GridDesc g, const double *__restrict__ kx, const double *__restrict__ ky,
                                const double *__restrict__ kz, double *__restrict__ T) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int ix, iy, iz;
    cell_xyz(g, i, ix, iy, iz);
    double tx = 0.0, ty = 0.0, tz = 0.0;
    if (ix < g.nx - 1) tx = SIM_DARCY * 2.0 * g.dy * g.dz / (g.dx / kx[i] + g.dx / kx[i + 1]);
    if (iy < g.ny - 1) ty = SIM_DARCY * 2.0 * g.dx * g.dz / (g.dy / ky[i] + g.dy / ky[i + g.nx]);
    if (iz < g.nz - 1) tz = SIM_DARCY * 2.0 * g.dx * g.dy / (g.dz / kz[i] + g.dz / kz[i + g.nx * g.ny]);
    T[i] = tx;
    T[g.N + i] = ty;
    T[2 * g.N + i] = tz;
}

__global__ void peaceman_kernel(GridDesc g, int nperf, const int *__restrict__ cell, const double *__restrict__ kx,
                                const double *__restrict__ ky, const double *__restrict__ rw,
                                const double *__restrict__ skin, double *__restrict__ wi) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nperf) return;
    int c = cell[q];
    double a = kx[c], b = ky[c];
    double ro = 0.28 * sqrt(sqrt(b / a) * g.dx * g.dx + sqrt(a / b) * g.dy * g.dy) / (pow(b / a, 0.25) + pow(a / b, 0.25));
    wi[q] = 2.0 * M_PI * SIM_DARCY * sqrt(a * b) * g.dz / (log(ro / rw[q]) + skin[q]);
}

// ---------------------------------------------------------------------------
// accumulation only (mass at the start of a step, component totals)
// ---------------------------------------------------------------------------
template <int B>
__global__ void accumulation_kernel(FluidConst f, GridDesc g, const double *__restrict__ x, const int8_t *__restrict__ ph,
                                    const double *__restrict__ poro, double *__restrict__ acc) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    Props<B> P;
    cell_props<B>(f, poro[i], g.dx * g.dy * g.dz, x[i], x[g.N + i], B == 3 ? x[2 * g.N + i] : 0.0, B == 3 ? ph[i] : 1, P);
#pragma unroll
    for (int c = 0; c < B; c++) acc[c * g.N + i] = P.acc[c].v;
}

// ---------------------------------------------------------------------------
// assembly pass 1: properties, accumulation rows of R and of the centre block
// ---------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(SIM_THREADS) props_kernel(FluidConst f, GridDesc g, const double *__restrict__ x,
                                                            const int8_t *__restrict__ ph, const double *__restrict__ poro,
                                                            const double *__restrict__ mold, double inv_dt,
                                                            double *__restrict__ props, double *__restrict__ R,
                                                            double *__restrict__ J) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    const long N = g.N;
    Props<B> P;
    cell_props<B>(f, poro[i], g.dx * g.dy * g.dz, x[i], x[N + i], B == 3 ? x[2 * N + i] : 0.0, B == 3 ? ph[i] : 1, P);
    constexpr int W = B + 1;
#pragma unroll
    for (int a = 0; a < B; a++) {
        props[(a * W) * N + i] = P.rho[a].v;
#pragma unroll
        for (int k = 0; k < B; k++) props[(a * W + 1 + k) * N + i] = P.rho[a].d[k];
    }
#pragma unroll
    for (int q = 0; q < Layout<B>::NPAIR; q++) {
        int base = (B + q) * W;
        props[base * N + i] = P.mob[q].v;
#pragma unroll
        for (int k = 0; k < B; k++) props[(base + 1 + k) * N + i] = P.mob[q].d[k];
    }
#pragma unroll
    for (int c = 0; c < B; c++) {
        R[c * N + i] = (P.acc[c].v - mold[c * N + i]) * inv_dt;
#pragma unroll
        for (int k = 0; k < B; k++) J[(c * B + k) * N + i] = P.acc[c].d[k] * inv_dt;
    }
}

// ---------------------------------------------------------------------------
// assembly pass 2: upwinded Darcy fluxes through the six faces of each cell
// ---------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(SIM_THREADS) flux_kernel(GridDesc g, const double *__restrict__ x,
                                                           const double *__restrict__ props,
                                                           const double *__restrict__ T, double *__restrict__ R,
                                                           double *__restrict__ J) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    const long N = g.N;
    constexpr int W = B + 1;
    constexpr int NQ = Layout<B>::NQ;
    int ix, iy, iz;
    cell_xyz(g, i, ix, iy, iz);
    double Ri[B], Jc[B * B];
#pragma unroll
    for (int c = 0; c < B; c++) Ri[c] = R[c * N + i];
#pragma unroll
    for (int t = 0; t < B * B; t++) Jc[t] = J[t * N + i];
    double own[NQ * W];
#pragma unroll
    for (int t = 0; t < NQ * W; t++) own[t] = props[t * N + i];
    const double p_i = x[i];
    const double depth_i = g.top + (iz + 0.5) * g.dz;
    const int order[6] = {5, 3, 1, 2, 4, 6};
#pragma unroll 1
    for (int oi = 0; oi < 6; oi++) {
        const int d = order[oi];
        const int j = nbr_of(g, i, ix, iy, iz, d);
        double Jd[B * B];
#pragma unroll
        for (int t = 0; t < B * B; t++) Jd[t] = 0.0;
        if (j >= 0) {
            const bool iL = (d % 2) == 0;         // + direction: this cell is L
            const int axis = (d - 1) / 2;
            const int L = iL ? i : j;
            const double Tf = T[axis * N + L];
            double nb[NQ * W];
#pragma unroll
            for (int t = 0; t < NQ * W; t++) nb[t] = props[t * N + j];
            // L / R views of the two cells' properties without taking addresses
#define PLV(t) (iL ? own[(t)] : nb[(t)])
#define PRV(t) (iL ? nb[(t)] : own[(t)])
            const int jz = (d == 5) ? iz - 1 : ((d == 6) ? iz + 1 : iz);
            const double depth_j = g.top + (jz + 0.5) * g.dz;
            const double gdz = SIM_GRAV * ((iL ? depth_j : depth_i) - (iL ? depth_i : depth_j)) / 1e5;
            const double pL = iL ? p_i : x[j], pR = iL ? x[j] : p_i;
#pragma unroll
            for (int a = 0; a < B; a++) {
                const double rbar = 0.5 * (PLV(a * W) + PRV(a * W));
                const double dphi = (pR - pL) - rbar * gdz;
                double dphiL[B], dphiR[B];
#pragma unroll
                for (int k = 0; k < B; k++) {
                    dphiL[k] = -gdz * 0.5 * PLV(a * W + 1 + k);
                    dphiR[k] = -gdz * 0.5 * PRV(a * W + 1 + k);
                }
                dphiL[0] -= 1.0;
                dphiR[0] += 1.0;
                const bool upR = dphi > 0.0;
#pragma unroll
                for (int q = 0; q < Layout<B>::NPAIR; q++) {
                    if (Layout<B>::pair_phase(q) != a) continue;
                    const int c = Layout<B>::pair_comp(q);
                    // upstream cell is the neighbour exactly when (upR == iL)
                    const bool useNb = (upR == iL);
#define MV(t) (useNb ? nb[(B + q) * W + (t)] : own[(B + q) * W + (t)])
                    const double m0 = MV(0);
                    const double F = Tf * m0 * dphi;
#pragma unroll
                    for (int k = 0; k < B; k++) {
                        const double dFL = Tf * ((upR ? 0.0 : MV(1 + k) * dphi) + m0 * dphiL[k]);
                        const double dFR = Tf * ((upR ? MV(1 + k) * dphi : 0.0) + m0 * dphiR[k]);
                        if (iL) { Jc[c * B + k] -= dFL; Jd[c * B + k] -= dFR; }
                        else { Jc[c * B + k] += dFR; Jd[c * B + k] += dFL; }
                    }
                    if (iL) Ri[c] -= F; else Ri[c] += F;
                }
            }
        }
#pragma unroll
        for (int t = 0; t < B * B; t++) J[(d * B * B + t) * N + i] = Jd[t];
    }
#undef PLV
#undef PRV
#undef MV
#pragma unroll
    for (int c = 0; c < B; c++) R[c * N + i] = Ri[c];
#pragma unroll
    for (int t = 0; t < B * B; t++) J[t * N + i] = Jc[t];
}

// ---------------------------------------------------------------------------
// assembly pass 3: well terms (Eq. 6) at the perforated cells; one block.
// Perforations occupy distinct cells (checked at creation).
// ---------------------------------------------------------------------------
// Border blocks of Eq. (16) per perforation q: apw[c][q] = dR_c/dp_h and,
// for the well's controlled component cc, awp[k][q] = dq_cc/dx_k; the
// controlled rate of the perforation goes to qcc[q].  One block; afterwards
// one thread per well sums its perforations in order: R_w, A_ww, the rates.
template <int B>
__global__ void well_kernel(FluidConst f, GridDesc g, const double *__restrict__ x, const int8_t *__restrict__ ph,
                            const double *__restrict__ poro, int nperf, const int *__restrict__ cell,
                            const int *__restrict__ type, const double *__restrict__ wi, const double *__restrict__ zh,
                            const int *__restrict__ pwell, const int *__restrict__ woff, int nwells,
                            const int *__restrict__ wctrl, const double *__restrict__ wrate,
                            const double *__restrict__ wbhp_c, const double *__restrict__ wp, double *__restrict__ R,
                            double *__restrict__ J, double *__restrict__ apw, double *__restrict__ awp,
                            double *__restrict__ qperf, double *__restrict__ rw, double *__restrict__ aww,
                            double *__restrict__ qwell, double *__restrict__ wcnv, double *__restrict__ qtot) {
    __shared__ double part[SIM_THREADS][3];
    __shared__ double wmax[SIM_THREADS];
    const long N = g.N;
    double qs[3] = {0.0, 0.0, 0.0};
    for (int q = threadIdx.x; q < nperf; q += blockDim.x) {
        const int i = cell[q];
        const int iz = i / (g.nx * g.ny);
        const int w = pwell[q];
        const int ctrl = wctrl[w];
        const int cc = ctrl == 1 ? 0 : (ctrl == 2 ? 1 : -1);    // controlled component (water 0, oil 1)
        Props<B> P;
        const double p = x[i];
        cell_props<B>(f, poro[i], g.dx * g.dy * g.dz, p, x[N + i], B == 3 ? x[2 * N + i] : 0.0, B == 3 ? ph[i] : 1, P);
        const double dh = SIM_GRAV * (zh[q] - (g.top + (iz + 0.5) * g.dz)) / 1e5;
        const double W = wi[q];
        const double bhp = wp[w];
        double a_pw[3] = {0.0, 0.0, 0.0}, a_wp[3] = {0.0, 0.0, 0.0}, qc4[4] = {0.0, 0.0, 0.0, 0.0};
        const double Dw = bhp - p - P.rho[0].v * dh;     // head of a water-filled injector
        const bool inj = type[q] == SIM_WELL_WATER_INJECTOR;
        if (inj && (Dw >= 0.0 || ctrl)) {
            // water at the cell's total mobility; a rate-controlled injector keeps
            // this form for a negative head too (its solution injects, and the
            // form keeps dR_w/dp_h from vanishing on the Newton path)
            const Dl<B> lam = P.rho[0] * P.lamt;
            const double qw = W * lam.v * Dw;
            R[i] -= qw;
            qs[0] += qw;
            qc4[0] = qw;
            a_pw[0] -= W * lam.v;
#pragma unroll
            for (int k = 0; k < B; k++) {
                const double dD = (k == 0 ? -1.0 : 0.0) - P.rho[0].d[k] * dh;
                const double dq = W * (lam.d[k] * Dw + lam.v * dD);
                J[k * N + i] -= dq;
                if (cc == 0) a_wp[k] += dq;
            }
            if (cc == 0) { qc4[3] = qw; }
        } else {
            // producer (Eq. 6 per phase), or a BHP-controlled injector in
            // backflow: the cell's phases leave at their own mobilities, driven
            // for the injector by its water head (continuous at Dw = 0)
#pragma unroll
            for (int a = 0; a < B; a++) {
                const double Dp = inj ? Dw : bhp - p - P.rho[a].v * dh;
                const int hp = inj ? 0 : a;
#pragma unroll
                for (int pq = 0; pq < Layout<B>::NPAIR; pq++) {
                    if (Layout<B>::pair_phase(pq) != a) continue;
                    const int c = Layout<B>::pair_comp(pq);
                    const Dl<B> &m = P.mob[pq];
                    const double qc = W * m.v * Dp;
                    R[c * N + i] -= qc;
                    qs[c] += qc;
                    qc4[c] += qc;
                    a_pw[c] -= W * m.v;
#pragma unroll
                    for (int k = 0; k < B; k++) {
                        const double dD = (k == 0 ? -1.0 : 0.0) - P.rho[hp].d[k] * dh;
                        const double dq = W * (m.d[k] * Dp + m.v * dD);
                        J[(c * B + k) * N + i] -= dq;
                        if (c == cc) a_wp[k] += dq;
                    }
                    if (c == cc) qc4[3] = qc;
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 3; c++) {
            apw[(long)c * nperf + q] = a_pw[c];
            awp[(long)c * nperf + q] = a_wp[c];
        }
#pragma unroll
        for (int c = 0; c < 4; c++) qperf[(long)c * nperf + q] = qc4[c];
    }
    for (int c = 0; c < 3; c++) part[threadIdx.x][c] = qs[c];
    __syncthreads();    // qperf and apw of every perforation are visible to the block
    double mx = 0.0;
    for (int w = threadIdx.x; w < nwells; w += blockDim.x) {
        const int ctrl = wctrl[w];
        double r = ctrl ? -wrate[w] : wp[w] - wbhp_c[w], a = ctrl ? 0.0 : 1.0;
        double qw[3] = {0.0, 0.0, 0.0};
        const int cc = ctrl == 1 ? 0 : 1;
        for (int q = woff[w]; q < woff[w + 1]; q++) {
            for (int c = 0; c < 3; c++) qw[c] += qperf[(long)c * nperf + q];
            if (ctrl) {
                r += qperf[3L * nperf + q];
                a -= apw[(long)cc * nperf + q];
            }
        }
        rw[w] = r;
        aww[w] = a;
        for (int c = 0; c < 3; c++) qwell[(long)c * nwells + w] = qw[c];
        if (ctrl) {
            const double sc = fabs(wrate[w]) > 1.0 ? fabs(wrate[w]) : 1.0;
            const double v = fabs(r) / sc;
            if (!(v <= mx)) mx = v;        // NaN propagates
        }
    }
    wmax[threadIdx.x] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[3] = {0.0, 0.0, 0.0}, m = 0.0;
        for (int k = 0; k < (int)blockDim.x; k++) {
            for (int c = 0; c < 3; c++) t[c] += part[k][c];
            if (!(wmax[k] <= m)) m = wmax[k];
        }
        for (int c = 0; c < 3; c++) qtot[c] = t[c];
        *wcnv = m;
    }
}

// b += A_pw A_ww^-1 R_w at the perforations of rate-controlled wells
// (the right-hand side of the system with the well unknowns eliminated)
__global__ void well_rhs_kernel(long N, int b, int nperf, const int *__restrict__ cell, const int *__restrict__ pwell,
                                const int *__restrict__ wctrl, const double *__restrict__ apw,
                                const double *__restrict__ rw, const double *__restrict__ aww, double *__restrict__ rhs) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nperf) return;
    const int w = pwell[q];
    if (!wctrl[w]) return;
    const double u = rw[w] / aww[w];
    const int i = cell[q];
    for (int c = 0; c < b; c++) rhs[c * N + i] += apw[(long)c * nperf + q] * u;
}

// dp_h = (-R_w - A_wp dx) / A_ww, limited to chop_dp; one warp per well
__global__ void well_update_kernel(long N, int b, int nperf, int nwells, const int *__restrict__ cell,
                                   const int *__restrict__ woff, const int *__restrict__ wctrl,
                                   const double *__restrict__ awp, const double *__restrict__ rw,
                                   const double *__restrict__ aww, const double *__restrict__ dx, double chop_dp,
                                   double *__restrict__ wp) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= nwells || !wctrl[w]) return;
    double t = 0.0;
    for (int q = woff[w] + lane; q < woff[w + 1]; q += 32) {
        const int i = cell[q];
        for (int k = 0; k < b; k++) t += awp[(long)k * nperf + q] * dx[k * N + i];
    }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) {
        double d = (-rw[w] - t) / aww[w];
        if (fabs(d) > chop_dp) d = d > 0 ? chop_dp : -chop_dp;
        wp[w] += d;
    }
}

// y -= A_pw A_ww^-1 A_wp x at the rate-controlled wells' perforations; one warp per well
template <typename X>
__global__ void well_op_kernel(long N, int b, int nperf, int nwells, const int *__restrict__ cell,
                               const int *__restrict__ woff, const int *__restrict__ wctrl,
                               const double *__restrict__ apw, const double *__restrict__ awp,
                               const double *__restrict__ aww, const X *__restrict__ x, double *__restrict__ y,
                               const int *done) {
    if (done && *(volatile const int *)done) return;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= nwells || !wctrl[w]) return;
    double t = 0.0;
    for (int q = woff[w] + lane; q < woff[w + 1]; q += 32) {
        const int i = cell[q];
        for (int k = 0; k < b; k++) t += awp[(long)k * nperf + q] * (double)x[k * N + i];
    }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    const double u = __shfl_sync(0xffffffffu, t, 0) / aww[w];
    for (int q = woff[w] + lane; q < woff[w + 1]; q += 32) {
        const int i = cell[q];
        for (int c = 0; c < b; c++) y[c * N + i] -= apw[(long)c * nperf + q] * u;
    }
}

// ---------------------------------------------------------------------------
// reductions: CNV max, component mass, non-finite count (deterministic:
// fixed grid, per-block partials reduced in block order by the last block)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double nanmax(double a, double b) { return (b > a || b != b) ? b : a; }

template <int OP>   // 0 sum, 1 max (NaN-propagating)
__device__ __forceinline__ double block_reduce(double v) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) {
        double t = __shfl_down_sync(0xffffffffu, v, o);
        v = OP == 0 ? v + t : nanmax(v, t);
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : (OP == 0 ? 0.0 : 0.0);
        for (int o = 16; o > 0; o >>= 1) {
            double t = __shfl_down_sync(0xffffffffu, v, o);
            v = OP == 0 ? v + t : nanmax(v, t);
        }
    }
    return v;   // valid in thread 0
}

// last block of the grid folds the per-block partials [nv][gridDim] into out[nv]
template <int OP>
__device__ void finish_grid(double *partials, int nv, unsigned int *ticket, double *out) {
    __shared__ bool last;
    __threadfence();
    if (threadIdx.x == 0) {
        unsigned int t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // one warp per value, lanes stride over the partials, fixed shuffle tree
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int v = wid; v < nv; v += nw) {
        double acc = 0.0;
        for (int k = lane; k < (int)gridDim.x; k += 32) {
            const double p = __ldcg(partials + (long)v * gridDim.x + k);
            acc = OP == 0 ? acc + p : nanmax(acc, p);
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double t = __shfl_down_sync(0xffffffffu, acc, o);
            acc = OP == 0 ? acc + t : nanmax(acc, t);
        }
        if (lane == 0) out[v] = acc;
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

template <int B>
__global__ void cnv_kernel(GridDesc g, const double *__restrict__ R, const double *__restrict__ poro, double dt,
                           FluidConst f, double *partials, unsigned int *ticket, double *out) {
    const long N = g.N;
    const double vol = g.dx * g.dy * g.dz;
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double pv0 = poro[i] * vol;
#pragma unroll
        for (int c = 0; c < B; c++) m = nanmax(m, fabs(R[c * N + i]) * dt / (pv0 * f.cnv_rho[c]));
    }
    m = block_reduce<1>(m);
    if (threadIdx.x == 0) partials[blockIdx.x] = m;
    finish_grid<1>(partials, 1, ticket, out);
}

template <int B>
__global__ void mass_kernel(FluidConst f, GridDesc g, const double *__restrict__ x, const int8_t *__restrict__ ph,
                            const double *__restrict__ poro, double *partials, unsigned int *ticket, double *out) {
    const long N = g.N;
    double m[B];
#pragma unroll
    for (int c = 0; c < B; c++) m[c] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        Props<B> P;
        cell_props<B>(f, poro[i], g.dx * g.dy * g.dz, x[i], x[N + i], B == 3 ? x[2 * N + i] : 0.0, B == 3 ? ph[i] : 1, P);
#pragma unroll
        for (int c = 0; c < B; c++) m[c] += P.acc[c].v;
    }
#pragma unroll
    for (int c = 0; c < B; c++) {
        double t = block_reduce<0>(m[c]);
        if (threadIdx.x == 0) partials[c * gridDim.x + blockIdx.x] = t;
    }
    finish_grid<0>(partials, B, ticket, out);
}

__global__ void nonfinite_kernel(const double *__restrict__ v, long n, double *partials, unsigned int *ticket, double *out) {
    double c = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) c += 1.0;
    c = block_reduce<0>(c);
    if (threadIdx.x == 0) partials[blockIdx.x] = c;
    finish_grid<0>(partials, 1, ticket, out);
}

// ---------------------------------------------------------------------------
// Newton update: Appleyard chop, saturation clamp, black-oil variable switch
// ---------------------------------------------------------------------------
template <int B>
__global__ void update_kernel(int N, double chop_ds, double chop_dp, const double *__restrict__ dx, double *__restrict__ x,
                              int8_t *__restrict__ ph) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double d[B], xi[B];
#pragma unroll
    for (int c = 0; c < B; c++) { d[c] = dx[c * N + i]; xi[c] = x[c * N + i]; }
    int sat = B == 3 ? ph[i] : 1;
    double ds = fabs(d[1]), dp = fabs(d[0]);
    if (B == 3) {
        if (sat) { if (fabs(d[2]) > ds) ds = fabs(d[2]); }
        else { if (fabs(d[2]) > dp) dp = fabs(d[2]); }
    }
    double fct = 1.0;
    if (ds > chop_ds) fct = chop_ds / ds;
    if (dp > chop_dp && chop_dp / dp < fct) fct = chop_dp / dp;
#pragma unroll
    for (int c = 0; c < B; c++) xi[c] += fct * d[c];
    if (xi[1] < 0.0) xi[1] = 0.0;
    if (xi[1] > 1.0) xi[1] = 1.0;
    if (B == 3) {
        if (sat && xi[2] < 0.0) { sat = 0; xi[2] = xi[0]; }
        else if (!sat && xi[2] > xi[0]) { sat = 1; xi[2] = 0.0; }
        if (!sat && xi[1] > 1.0 - 1e-6) { sat = 1; xi[2] = 0.0; }
        if (sat && xi[2] > 1.0 - xi[1]) xi[2] = 1.0 - xi[1];
        ph[i] = (int8_t)sat;
    }
#pragma unroll
    for (int c = 0; c < B; c++) x[c * N + i] = xi[c];
}

}  // namespace

// ===========================================================================
// host launchers
// ===========================================================================
static double *poro_of(sim_t *s) { return s->poro; }

sim_status k_geometry(sim_t *s, const double *kx, const double *ky, const double *kz, const double *poro,
                      const int *wcell, const int *wtype, const int *pwell, const double *wzh, const double *wrw,
                      const double *wskin) {
    const int N = s->N;
    double *dk = (double *)sim_alloc(s, sizeof(double) * 3 * (size_t)N);
    if (!dk) return s->err;
    SIM_CK(s, cudaMemcpyAsync(dk, kx, sizeof(double) * N, cudaMemcpyHostToDevice, s->stream));
    SIM_CK(s, cudaMemcpyAsync(dk + N, ky, sizeof(double) * N, cudaMemcpyHostToDevice, s->stream));
    SIM_CK(s, cudaMemcpyAsync(dk + 2 * (size_t)N, kz, sizeof(double) * N, cudaMemcpyHostToDevice, s->stream));
    SIM_CK(s, cudaMemcpyAsync(s->poro, poro, sizeof(double) * N, cudaMemcpyHostToDevice, s->stream));
    geometry_kernel<<<sim_blocks(N), SIM_THREADS, 0, s->stream>>>(s->gd, dk, dk + N, dk + 2 * (size_t)N, s->T);
    SIM_LAUNCHED(s);
    const int np = s->nperf;
    if (np > 0) {
        double *tmp = (double *)sim_alloc(s, sizeof(double) * 2 * (size_t)np);
        if (!tmp) return s->err;
        SIM_CK(s, cudaMemcpyAsync(s->perf_cell, wcell, sizeof(int) * np, cudaMemcpyHostToDevice, s->stream));
        SIM_CK(s, cudaMemcpyAsync(s->perf_type, wtype, sizeof(int) * np, cudaMemcpyHostToDevice, s->stream));
        SIM_CK(s, cudaMemcpyAsync(s->perf_well, pwell, sizeof(int) * np, cudaMemcpyHostToDevice, s->stream));
        SIM_CK(s, cudaMemcpyAsync(s->perf_zh, wzh, sizeof(double) * np, cudaMemcpyHostToDevice, s->stream));
        SIM_CK(s, cudaMemcpyAsync(tmp, wrw, sizeof(double) * np, cudaMemcpyHostToDevice, s->stream));
        SIM_CK(s, cudaMemcpyAsync(tmp + np, wskin, sizeof(double) * np, cudaMemcpyHostToDevice, s->stream));
        peaceman_kernel<<<sim_blocks(np), SIM_THREADS, 0, s->stream>>>(s->gd, np, s->perf_cell, dk, dk + N, tmp, tmp + np,
                                                                       s->perf_wi);
        SIM_LAUNCHED(s);
        SIM_CK(s, cudaStreamSynchronize(s->stream));
        sim_free(s, tmp);
    }
    SIM_CK(s, cudaStreamSynchronize(s->stream));
    sim_free(s, dk);
    return SIM_OK;
}

sim_status k_accumulation(sim_t *s, const double *x, const int8_t *ph, double *acc) {
    if (s->b == 2)
        accumulation_kernel<2><<<sim_blocks(s->N), SIM_THREADS, 0, s->stream>>>(s->fc, s->gd, x, ph, poro_of(s), acc);
    else
        accumulation_kernel<3><<<sim_blocks(s->N), SIM_THREADS, 0, s->stream>>>(s->fc, s->gd, x, ph, poro_of(s), acc);
    SIM_LAUNCHED(s);
    return SIM_OK;
}

template <int B>
static sim_status assemble_b(sim_t *s, double dt) {
    const int N = s->N;
    props_kernel<B><<<sim_blocks(N), SIM_THREADS, 0, s->stream>>>(s->fc, s->gd, s->x, s->ph, poro_of(s), s->mold,
                                                                  1.0 / dt, s->props, s->R, s->J);
    SIM_LAUNCHED(s);
    flux_kernel<B><<<sim_blocks(N), SIM_THREADS, 0, s->stream>>>(s->gd, s->x, s->props, s->T, s->R, s->J);
    SIM_LAUNCHED(s);
    if (s->nwells > 0) {
        well_kernel<B><<<1, SIM_THREADS, 0, s->stream>>>(s->fc, s->gd, s->x, s->ph, poro_of(s), s->nperf, s->perf_cell,
                                                         s->perf_type, s->perf_wi, s->perf_zh, s->perf_well, s->woff,
                                                         s->nwells, s->wctrl, s->wrate, s->wbhp_c, s->wp, s->R, s->J,
                                                         s->apw, s->awp, s->qperf, s->rw, s->aww, s->qwell, s->wcnv,
                                                         s->qtot);
        SIM_LAUNCHED(s);
    } else {
        SIM_CK(s, cudaMemsetAsync(s->qtot, 0, sizeof(double) * 3, s->stream));
        SIM_CK(s, cudaMemsetAsync(s->wcnv, 0, sizeof(double), s->stream));
    }
    return SIM_OK;
}

sim_status k_assemble(sim_t *s, double dt) {
    s->precond_ready = false;
    return s->b == 2 ? assemble_b<2>(s, dt) : assemble_b<3>(s, dt);
}

sim_status k_well_rhs(sim_t *s, double *rhs) {
    if (s->nrate == 0) return SIM_OK;
    well_rhs_kernel<<<sim_blocks(s->nperf), SIM_THREADS, 0, s->stream>>>(s->N, s->b, s->nperf, s->perf_cell, s->perf_well,
                                                                         s->wctrl, s->apw, s->rw, s->aww, rhs);
    SIM_LAUNCHED(s);
    return SIM_OK;
}

sim_status k_well_update(sim_t *s, const double *dx) {
    if (s->nrate == 0) return SIM_OK;
    well_update_kernel<<<sim_blocks((long)s->nwells * 32), SIM_THREADS, 0, s->stream>>>(
        s->N, s->b, s->nperf, s->nwells, s->perf_cell, s->woff, s->wctrl, s->awp, s->rw, s->aww, dx, s->opt.chop_dp, s->wp);
    SIM_LAUNCHED(s);
    return SIM_OK;
}

template <typename X>
sim_status k_well_op(sim_t *s, const X *x, double *y, const int *done) {
    if (s->nrate == 0) return SIM_OK;
    well_op_kernel<X><<<sim_blocks((long)s->nwells * 32), SIM_THREADS, 0, s->stream>>>(
        s->N, s->b, s->nperf, s->nwells, s->perf_cell, s->woff, s->wctrl, s->apw, s->awp, s->aww, x, y, done);
    SIM_LAUNCHED(s);
    return SIM_OK;
}
template sim_status k_well_op<double>(sim_t *, const double *, double *, const int *);
template sim_status k_well_op<float>(sim_t *, const float *, double *, const int *);

sim_status k_cnv(sim_t *s, double dt, double *cnv_host, double *well_cnv_host) {
    if (s->b == 2)
        cnv_kernel<2><<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(s->gd, s->R, poro_of(s), dt, s->fc, s->red, s->ticket, s->scal);
    else
        cnv_kernel<3><<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(s->gd, s->R, poro_of(s), dt, s->fc, s->red, s->ticket, s->scal);
    SIM_LAUNCHED(s);
    SIM_CK(s, cudaMemcpyAsync(s->h_pinned, s->scal, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    if (well_cnv_host) SIM_CK(s, cudaMemcpyAsync(s->h_pinned + 1, s->wcnv, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    SIM_CK(s, cudaStreamSynchronize(s->stream));
    *cnv_host = s->h_pinned[0];
    if (well_cnv_host) *well_cnv_host = s->h_pinned[1];
    return SIM_OK;
}

sim_status k_component_mass(sim_t *s, double *m3) {
    if (s->b == 2)
        mass_kernel<2><<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(s->fc, s->gd, s->x, s->ph, poro_of(s), s->red, s->ticket, s->scal);
    else
        mass_kernel<3><<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(s->fc, s->gd, s->x, s->ph, poro_of(s), s->red, s->ticket, s->scal);
    SIM_LAUNCHED(s);
    SIM_CK(s, cudaMemcpyAsync(s->h_pinned, s->scal, sizeof(double) * 3, cudaMemcpyDeviceToHost, s->stream));
    SIM_CK(s, cudaStreamSynchronize(s->stream));
    for (int c = 0; c < 3; c++) m3[c] = c < s->b ? s->h_pinned[c] : 0.0;
    return SIM_OK;
}

sim_status k_newton_update(sim_t *s, const double *dx) {
    if (s->b == 2)
        update_kernel<2><<<sim_blocks(s->N), SIM_THREADS, 0, s->stream>>>(s->N, s->opt.chop_ds, s->opt.chop_dp, dx, s->x, s->ph);
    else
        update_kernel<3><<<sim_blocks(s->N), SIM_THREADS, 0, s->stream>>>(s->N, s->opt.chop_ds, s->opt.chop_dp, dx, s->x, s->ph);
    SIM_LAUNCHED(s);
    return SIM_OK;
}

sim_status k_finite(sim_t *s, const double *v, long n, int *ok) {
    nonfinite_kernel<<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(v, n, s->red, s->ticket, s->scal);
    SIM_LAUNCHED(s);
    SIM_CK(s, cudaMemcpyAsync(s->h_pinned, s->scal, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    SIM_CK(s, cudaStreamSynchronize(s->stream));
    *ok = s->h_pinned[0] == 0.0;
    return SIM_OK;
}

// ===========================================================================
// CNV without device allocation (sim_cnv_noalloc)
//
// Scratch: the per-block partial maxima and the last-block ticket live in a
// file-scope device array of NOALLOC_SCRATCH = SIM_RED_BLOCKS + 1 doubles
// (456 partials and one ticket word: 457 doubles, 3,656 bytes), held by every
// GPU that loads the library until the process exits.  Host code never uses
// the array's name as a pointer (on the host it is only a stand-in): every
// call looks the device address up with cudaGetSymbolAddress, with the
// caller's device current, so no address outlives a device reset.
// ===========================================================================
namespace {
constexpr int NOALLOC_SCRATCH = SIM_RED_BLOCKS + 1;   // partials + ticket word
static __device__ __align__(256) double g_cnv_scratch[NOALLOC_SCRATCH];

template <int B>
__global__ void cnv_noalloc_kernel(GridDesc g, const double *__restrict__ R, const double *__restrict__ poro, double dt,
                                   double r0, double r1, double r2, double *scratch, double *out) {
    const long N = g.N;
    const double vol = g.dx * g.dy * g.dz;
    const double rho[3] = {r0, r1, r2};
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double pv0 = poro[i] * vol;
#pragma unroll
        for (int c = 0; c < B; c++) m = nanmax(m, fabs(R[c * N + i]) * dt / (pv0 * rho[c]));
    }
    m = block_reduce<1>(m);
    if (threadIdx.x == 0) scratch[blockIdx.x] = m;
    finish_grid<1>(scratch, 1, (unsigned int *)(scratch + SIM_RED_BLOCKS), out);
}
}  // namespace

extern "C" sim_status sim_cnv_noalloc(int32_t nx, int32_t ny, int32_t nz, double dx, double dy, double dz, int32_t b,
                                      const double *R_dev, const double *poro_dev, const double *cnv_rho, double dt,
                                      double *cnv_dev, void *cuda_stream) {
    if (!R_dev || !poro_dev || !cnv_rho || !cnv_dev) return sim_fail(nullptr, SIM_EINVAL, "sim_cnv_noalloc: NULL pointer");
    if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0 && dy > 0 && dz > 0) || !(dt > 0) || (b != 2 && b != 3))
        return sim_fail(nullptr, SIM_EINVAL, "sim_cnv_noalloc: bad grid, block size or dt");
    for (int c = 0; c < b; c++)
        if (!(cnv_rho[c] > 0)) return sim_fail(nullptr, SIM_EINVAL, "sim_cnv_noalloc: cnv_rho must be positive");
    const long long N = (long long)nx * ny * nz;
    if (N * b > 0x7fffffffLL)
        return sim_fail(nullptr, SIM_ELIMIT, "sim_cnv_noalloc: N*b must stay below 2^31 (32-bit indexing)");
    int dev = 0;   // the caller's current device: the one whose copy of the array is used
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return sim_fail(nullptr, SIM_ECUDA, std::string("sim_cnv_noalloc: ") + cudaGetErrorString(e));
    // the array's device address on that device (a lookup, no allocation)
    double *scratch = nullptr;
    e = cudaGetSymbolAddress((void **)&scratch, g_cnv_scratch);
    if (e != cudaSuccess || !scratch)
        return sim_fail(nullptr, SIM_ECUDA, std::string("sim_cnv_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the ticket must start at zero; the partials are overwritten before use
    e = cudaMemsetAsync(scratch + SIM_RED_BLOCKS, 0, sizeof(double), st);
    if (e != cudaSuccess) return sim_fail(nullptr, SIM_ECUDA, std::string("sim_cnv_noalloc: ") + cudaGetErrorString(e));
    GridDesc g;
    g.nx = nx; g.ny = ny; g.nz = nz; g.N = (int)N; g.dx = dx; g.dy = dy; g.dz = dz; g.top = 0.0; g.H = 0;
    const double r2 = b == 3 ? cnv_rho[2] : 1.0;
    if (b == 2)
        cnv_noalloc_kernel<2><<<SIM_RED_BLOCKS, SIM_THREADS, 0, st>>>(g, R_dev, poro_dev, dt, cnv_rho[0], cnv_rho[1], r2,
                                                                     scratch, cnv_dev);
    else
        cnv_noalloc_kernel<3><<<SIM_RED_BLOCKS, SIM_THREADS, 0, st>>>(g, R_dev, poro_dev, dt, cnv_rho[0], cnv_rho[1], r2,
                                                                     scratch, cnv_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return sim_fail(nullptr, SIM_ECUDA, std::string("sim_cnv_noalloc: ") + cudaGetErrorString(e));
    return SIM_OK;
}
