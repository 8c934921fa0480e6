// Internal declarations of the GB300 reservoir library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/sim.h"

#include <nvtx3/nvToolsExt.h>

// NVTX range over a host scope (a phase of a step); no cost unless a tool such
// as a profiler attaches to NVTX
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

#define SIM_GRAV 9.80665
#define SIM_DARCY (86400.0 * 9.869233e-16 * 1e5 / 1e-3)
#define SIM_MAX_PVT 64
#define SIM_MAX_M 32
#define SIM_MAX_ELL 512      // widest coarse AMG row: a wider Galerkin row stops coarsening
#define SIM_RED_BLOCKS 456   // 3 x 152 SMs: grid of the reduction kernels (one wave at <= 85 registers)
#define SIM_THREADS 256

// fluid and rock constants, passed by value as a kernel parameter (about
// 3.3 KB, under the 4 KB parameter limit), so handles never share state
struct FluidConst {
    int model, b, npvt;
    double rho_w_ref, rho_o_ref, c_w, c_o, mu_w, mu_o;
    double rho_ws, rho_os, rho_gs, bw_c, bw_pref, bo_c_us, muo_c_us;
    double swc, sor, sgc, sorg, nw, now, ng, nog;
    double c_rock, p_ref;
    double pvt_p[SIM_MAX_PVT], pvt_bo[SIM_MAX_PVT], pvt_rs[SIM_MAX_PVT], pvt_muo[SIM_MAX_PVT],
        pvt_bg[SIM_MAX_PVT], pvt_mug[SIM_MAX_PVT];
    double cnv_rho[3];
};

struct GridDesc {
    int nx, ny, nz, N;
    double dx, dy, dz, top;
    int H;              // cells of one colour in the colour-split arrays: ceil(nx / 2) ny nz
};

// device control block of one FGMRES solve (Givens, Hessenberg, flags)
struct KrylovCtl {
    int done;           // 1 once the Arnoldi residual estimate met the tolerance
    int k;              // inner iterations completed in the current cycle
    int active;         // batched solves: 1 while this member's solve goes on
    int iters;          // batched solves: inner iterations of this member's solve
    double tol, beta, rnorm2;
    double h[SIM_MAX_M + 1], h2[SIM_MAX_M + 1];
    double g[SIM_MAX_M + 1], cs[SIM_MAX_M + 1], sn[SIM_MAX_M + 1], y[SIM_MAX_M + 1];
    double H[(SIM_MAX_M + 1) * (SIM_MAX_M + 1)];
    unsigned int counter;   // last-block reduction ticket
    unsigned int pad2;
};

// One member of a batched FGMRES solve (an ensemble of independent systems):
// its operands, read by the batched kernels from a device table
struct KMember {
    GridDesc g;
    long n;                  // b N
    double theta;            // relative tolerance of this member's solve
    const double *J;
    double *V, *w, *r, *x;   // Krylov basis, work vector, residual, solution
    const double *rhs;       // right-hand side; null: the member does not solve in this round
    void *Z;                 // preconditioned directions (FP64 or FP32)
    KrylovCtl *ctl;
    double *red;             // the member's reduction partials and ticket
    unsigned int *ticket;
};

// BiCGSTAB scalars (device); flag: 1 recursive residual met the tolerance,
// 2 breakdown, 3 iteration limit (each also sets done)
struct BicgCtl {
    int done, flag, it, half_j;
    int fresh, max_it;
    double tol, rho, rho_old, alpha, omega, rnorm;
};

struct AmgLevel {
    int n = 0, width = 0;        // level 0: width 7, structured
    int *col = nullptr;          // ELL columns [width][n] (levels >= 1), -1 padding
    int *colA = nullptr;         // the same with padding on the row's own column (apply)
    double *val = nullptr;       // ELL values, FP64 (setup precision)
    void *valT = nullptr;        // ELL values in apply precision (float copy for mixed)
    void *dinvT = nullptr;       // 1 / l1 row sums, apply precision
    int *agg = nullptr;          // fine -> next level
    int *moff = nullptr, *mem = nullptr;   // members of each next-level aggregate, ascending (CSR)
    void *f = nullptr, *e = nullptr, *e2 = nullptr;   // V-cycle vectors (apply precision)
    void *coarse_inv = nullptr;  // coarsest: dense inverse, row-major n*n (FP64 in both forms)
};

struct sim {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    sim_status err = SIM_OK;
    std::string msg;
    FluidConst fc;
    GridDesc gd;
    sim_options opt;
    int N = 0, b = 0;
    int64_t launches = 0, newton_total = 0, linear_total = 0;
    size_t bytes = 0;
    // run totals for the run report: time steps (completed / failed), accepted
    // substeps, cuts, linear solves that hit their limit, simulated days, and the
    // per-phase device time and algorithmic bytes summed over every Newton call
    int64_t run_steps = 0, run_failed_steps = 0, run_substeps = 0, run_cuts = 0, run_lin_failures = 0;
    double run_days = 0.0, run_max_mb = 0.0;
    sim_phase_info run_phase = {};
    double m_start[3] = {0.0, 0.0, 0.0};   // component masses of the current step's start
    double last_mb = 0.0;                   // mass-balance error of the last accepted substep
    std::vector<void *> allocs;

    // geometry
    double *T = nullptr;         // [3][N] transmissibility to the + neighbour
    double *poro = nullptr;      // [N] porosity at p_ref
    int nperf = 0;
    int *perf_cell = nullptr, *perf_type = nullptr;
    double *perf_wi = nullptr, *perf_zh = nullptr;
    // wells (Eq. 16): perforations are grouped by well, woff[w]..woff[w+1]
    int nwells = 0, nrate = 0;
    int *perf_well = nullptr, *woff = nullptr, *wctrl = nullptr;
    double *wrate = nullptr;                 // [nwells] target of rate controls
    double *wbhp_c = nullptr;                // [nwells] BHP of BHP controls
    double *wp = nullptr, *wp_old = nullptr; // [nwells] bottom-hole pressures (unknowns under rate control)
    double *apw = nullptr, *awp = nullptr;   // [3][nperf] border blocks dR_cell/dp_h, dR_w/dx_cell
    double *aww = nullptr, *rw = nullptr;    // [nwells] dR_w/dp_h, well equation residual
    double *qwell = nullptr;                 // [3][nwells] component rates per well
    double *qperf = nullptr;                 // [4][nperf] component rates and the controlled rate per perforation
    double *wcnv = nullptr;                  // device scalar: largest |R_w| / max(|target|, 1)
    int *cell_perf = nullptr;                // [N] perforation of a rate-controlled well, or -1 (rate wells only)
    std::vector<int> h_wctrl;

    // state
    double *x = nullptr, *x_old = nullptr;   // [b][N]
    int8_t *ph = nullptr, *ph_old = nullptr;
    double *mold = nullptr;                  // [b][N]
    double *R = nullptr, *J = nullptr;       // [b][N], [7][b][b][N]
    double *props = nullptr;                 // [nq*4][N]
    double *qtot = nullptr;                  // [3] well rates of the last assembly
    double cum_well[3] = {0, 0, 0};

    // reductions
    double *red = nullptr;       // partial sums [SIM_MAX_M+2][SIM_RED_BLOCKS]
    double *scal = nullptr;      // small device scalars
    unsigned int *ticket = nullptr;
    double *h_pinned = nullptr;  // pinned host mirror for small reads
    cudaEvent_t pev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // phase marks of a Newton iteration

    // Krylov
    int m = 0;
    double *V = nullptr;         // [(m+1)][n]
    void *Z = nullptr;           // [m][n], FP64 or FP32
    double *w = nullptr, *r = nullptr, *xl = nullptr, *bl = nullptr, *dx = nullptr;
    KrylovCtl *ctl = nullptr;
    KrylovCtl *ctl_host = nullptr;
    cudaGraphExec_t cycle_exec = nullptr;   // captured restart cycle
    int64_t setup_gen = 0, cycle_gen = -1, graph_nodes = 0;
    int cycle_learned = -1;                  // learned-stage state the graph was captured with
    int tune_spmv = SIM_THREADS, tune_amg = 128, tune_stage = 64;   // block sizes picked by sim_autotune
    int last_cycle_k = 0;                    // inner iterations of the last restart cycle
    // BiCGSTAB: control block and the graph of one chunk of iterations
    BicgCtl *bctl = nullptr, *bctl_host = nullptr;
    cudaGraphExec_t bicg_exec = nullptr;
    int64_t bicg_gen = -1, bicg_nodes = 0;
    const double *bicg_x = nullptr;          // solution vector the chunk graph was captured with
    // inexact Newton: forcing term of the next solve, last linear residual b - J dx
    double theta = 0.0;
    double *rlin = nullptr;

    // CPR
    bool precond_ready = false;
    double *qiw = nullptr;       // [b][N]
    void *qiwT = nullptr;        // [b][N] apply precision (aliases qiw in FP64 mode)
    double *ap = nullptr;        // [7][N] pressure block, FP64
    void *apT = nullptr;         // [7][N] apply precision (aliases ap in FP64 mode)
    void *ahat = nullptr;        // [7][b][b][N] decoupled matrix, apply precision
    void *dinv = nullptr;        // [b][b][N] ILU / block-Jacobi inverse diagonal blocks
    double *dinv_d = nullptr;    // FP64 scratch of the same
    void *r2 = nullptr;          // [b][N] stage-2 work vector (apply precision)
    void *rpT = nullptr, *epacc = nullptr;   // [N] stage-P residual and accumulated correction
    // learned pressure stage (extra CPR stage after the V-cycles)
    sim_net_t *net = nullptr;
    int learned_on = 0;          // requested
    int learned_active = 0;      // used by the current solve (falls back to 0)
    int64_t learned_fallbacks = 0;
    float *lfeat = nullptr;      // [N][3] standardised log transmissibility features
    float *lx = nullptr, *ly = nullptr;   // [N][4] network input, [N] output
    void *lres = nullptr;        // [N] pressure residual after stage P (apply precision)
    void *lep = nullptr;         // [N] pressure correction after the learned stage
    double *lrms = nullptr;      // device scalar
    void *zr = nullptr;          // [b][N]
    double *lsc = nullptr;       // [b][b][N] per-cell left scaling L (quasi-IMPES or ABF)
    void *lscT = nullptr;        // [b][b][N] apply precision (aliases lsc in FP64 mode)
    void *rhT = nullptr, *x0 = nullptr;   // [b][N] CPR-FPF: L r - Ahat x0 and the first stage-F result
    std::vector<AmgLevel> lev;
    // AMG setup scratch
    int *partner = nullptr, *pick = nullptr, *host = nullptr, *flag = nullptr, *cnt = nullptr;
    int *aggA = nullptr, *moffA = nullptr, *memA = nullptr, *aggB = nullptr, *moffB = nullptr, *memB = nullptr;
    int *scan = nullptr, *iscal = nullptr;
    int *tcol = nullptr; double *tval = nullptr;   // intermediate (pass-1) matrix
    int tcap = 0;
};

// ---- error helpers --------------------------------------------------------
sim_status sim_fail(sim_t *s, sim_status st, const std::string &m);
bool sim_cuda_ok(sim_t *s, cudaError_t e, const char *what);
#define SIM_CK(s, call) do { if (!sim_cuda_ok((s), (call), #call)) return (s)->err; } while (0)
#define SIM_LAUNCHED(s) do { (s)->launches++; if (!sim_cuda_ok((s), cudaGetLastError(), "kernel launch")) return (s)->err; } while (0)
void *sim_alloc(sim_t *s, size_t bytes);
void sim_free(sim_t *s, void *p);
inline int sim_blocks(long n, int t = SIM_THREADS) { long b = (n + t - 1) / t; return (int)(b < 1 ? 1 : b); }
bool sim_mixed(const sim_t *s);

// ---- assemble.cu ----------------------------------------------------------
sim_status k_geometry(sim_t *s, const double *kx, const double *ky, const double *kz, const double *poro,
                      const int *wcell_host, const int *wtype_host, const int *pwell_host,
                      const double *wzh_host, const double *wrw_host, const double *wskin_host);
sim_status k_well_rhs(sim_t *s, double *b);                          // b += A_pw A_ww^-1 R_w
sim_status k_well_update(sim_t *s, const double *dx);                // p_h += dp_h (rate wells)
template <typename X> sim_status k_well_op(sim_t *s, const X *x, double *y, const int *done);   // y -= A_pw A_ww^-1 A_wp x
sim_status k_accumulation(sim_t *s, const double *x, const int8_t *ph, double *acc);   // acc [b][N]
sim_status k_assemble(sim_t *s, double dt);
sim_status k_cnv(sim_t *s, double dt, double *cnv_host, double *well_cnv_host = nullptr);
sim_status k_component_mass(sim_t *s, double *m3_host);
sim_status k_newton_update(sim_t *s, const double *dx);
sim_status k_finite(sim_t *s, const double *v, long n, int *ok_host);

// ---- sim_api.cu: the pieces of a Newton iteration (ensemble runtime) --------
sim_status nl_assemble_test(sim_t *s, double dt, int *state, sim_phase_info *ph);   // 0 solve, 1 converged, 2 non-finite
sim_status nl_prepare_solve(sim_t *s, sim_phase_info *ph);
sim_status nl_finish_solve(sim_t *s, const sim_linear_info &li, bool *finite_ok, sim_phase_info *ph);
sim_status nl_restore(sim_t *s);
sim_status accept_step(sim_t *s, double dt);
// a finished time step (sim_step or one member of a batch step) into the run totals
void run_record_step(sim_t *s, const sim_step_info &si, sim_status st);

// ---- krylov.cu ------------------------------------------------------------
sim_status k_spmv(sim_t *s, const double *x, double *y);                 // y = J x
sim_status k_spmv_f(sim_t *s, const float *x, double *y);
sim_status k_fgmres(sim_t *s, const double *b, double *x, sim_linear_info *info);
sim_status k_bicgstab(sim_t *s, const double *b, double *x, sim_linear_info *info);
sim_status k_linear_solve(sim_t *s, const double *b, double *x, sim_linear_info *info);
sim_status k_diff_norm2(sim_t *s, const double *a, const double *b, long n, double *out);
sim_status k_norm2(sim_t *s, const double *v, long n, double *out_host);
sim_status k_spmv_block(sim_t *s, const double *x, double *y, int block);
// FGMRES batched over ensemble members: every Krylov operation one launch for all
struct KrylovBatch;
KrylovBatch *k_batch_new();
void k_batch_free(KrylovBatch *kb);
int64_t k_batch_launches(const KrylovBatch *kb);
sim_status k_fgmres_batch(KrylovBatch *kb, sim_t *const *ms, int nm, cudaStream_t st, sim_linear_info *infos,
                          std::string *err);
sim_status k_orth_step(sim_t *s, int nv);              // measurement: one Arnoldi orthogonalisation step
double k_orth_step_bytes(const sim_t *s, int nv);      // its algorithmic bytes

// ---- cpr.cu ---------------------------------------------------------------
sim_status cpr_setup(sim_t *s);
sim_status cpr_apply(sim_t *s, const double *r, void *z, const int *done);   // z FP64 or FP32 (Z type)
void cpr_free(sim_t *s);
// batched CPR application over ensemble members (tables and work lists)
struct CprBatch;
bool cpr_batchable(sim_t *const *ms, int nm);
CprBatch *cpr_batch_new();
void cpr_batch_free(CprBatch *cb);
cudaError_t cpr_batch_build(CprBatch *cb, sim_t *const *ms, int nm, cudaStream_t st);   // after every member's setup
int cpr_batch_apply(const CprBatch *cb, cudaStream_t st, int j);                         // launches, or -1
sim_status cpr_copy_level_ell(sim_t *s, int level, int *col, double *val);
sim_status cpr_learned_pairs(sim_t *s, int k, float *x_dev, float *y_dev);
sim_status cpr_learned_features(sim_t *s);

// ---- learned.cu -----------------------------------------------------------
sim_status net_infer(sim_net_t *n, const float *x_dev, float *y_dev, cudaStream_t st, const int *done);
int64_t net_launches(sim_net_t *n);
// the convolutions' status word after the stream has drained: 0 fine, > 0 a
// bounded wait gave up, < 0 the read itself failed
int net_status_word(sim_net_t *n, cudaStream_t st);
int net_cells(sim_net_t *n);
