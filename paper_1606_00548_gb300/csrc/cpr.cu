// CPR two-stage preconditioner on the device (paper Sec. 2.4.2).
//
//   setup (FP64):  quasi-IMPES weights w_i = (1, -d_ps D_ss^-1) from the
//                  diagonal block; decoupled matrix Ahat (pressure row
//                  replaced by w^T rows); pressure block A_p; aggregation AMG
//                  hierarchy of A_p; red-black block ILU(0) (or block-Jacobi)
//                  of Ahat.
//   apply (T):     rp = w^T r; e_p = V(1,1)-cycle(A_p, rp);
//                  r2 = rhat - Ahat[:, p] e_p;  z = ILU0(Ahat)^-1 r2 + e_p.
// T = double for the plain form, float for the mixed form (FP32 hierarchy,
// factors and smoothers; the FGMRES outer loop stays FP64).
//
// AMG: two pairwise matching passes per level (handshakes among unmatched
// nodes; candidate = strongest unmatched strong neighbour compared by
// strength band (binary exponent), then a symmetric splitmix64 pair hash,
// then the smaller index); piecewise-constant prolongation; Galerkin coarse
// operators summed in member order then column order; l1-Jacobi V(1,1);
// dense inverse on the coarsest level.  The setup is deterministic and its
// integer results do not depend on thread scheduling.
//
// Layouts: level 0 is the 7-point stencil A_p [7][N]; coarser levels are ELL,
// entry k of row i at k*n + i, columns ascending, -1 padding.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>

#include "sim_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int MAXE = SIM_MAX_ELL;

__device__ __forceinline__ bool skip(const int *done) { return done != nullptr && *(volatile const int *)done; }

struct Cell { int i, ix, iy, iz; };
__device__ __forceinline__ Cell cell_of(const GridDesc &g, int i) {
    Cell c; c.i = i; c.ix = i % g.nx; const int t = i / g.nx; c.iy = t % g.ny; c.iz = t / g.ny; return c;
}
__device__ __forceinline__ int nbrc(const GridDesc &g, const Cell &c, int d) {
    switch (d) {
    case 0: return c.i;
    case 1: return c.ix > 0 ? c.i - 1 : -1;
    case 2: return c.ix < g.nx - 1 ? c.i + 1 : -1;
    case 3: return c.iy > 0 ? c.i - g.nx : -1;
    case 4: return c.iy < g.ny - 1 ? c.i + g.nx : -1;
    case 5: return c.iz > 0 ? c.i - g.nx * g.ny : -1;
    default: return c.iz < g.nz - 1 ? c.i + g.nx * g.ny : -1;
    }
}
__device__ __forceinline__ int nbr7(const GridDesc &g, int i, int d) {
    const int ix = i % g.nx, t = i / g.nx, iy = t % g.ny, iz = t / g.ny;
    switch (d) {
    case 0: return i;
    case 1: return ix > 0 ? i - 1 : -1;
    case 2: return ix < g.nx - 1 ? i + 1 : -1;
    case 3: return iy > 0 ? i - g.nx : -1;
    case 4: return iy < g.ny - 1 ? i + g.nx : -1;
    case 5: return iz > 0 ? i - g.nx * g.ny : -1;
    default: return iz < g.nz - 1 ? i + g.nx * g.ny : -1;
    }
}
// thread t of a launch over one colour (0: ix+iy+iz even, 1: odd): slot k of
// x-row r holds the cell ix = 2k or 2k+1 of that colour, so a warp's threads
// all work (a launch over every cell would leave half of each warp idle)
__device__ __forceinline__ int colour_cell(const GridDesc &g, long t, int colour) {
    const int hx = (g.nx + 1) >> 1;
    const long r = t / hx;
    const int k = (int)(t - r * hx);
    if (r >= (long)g.ny * g.nz) return -1;
    const int iy = (int)(r % g.ny), iz = (int)(r / g.ny);
    const int ix = 2 * k + (((iy + iz) & 1) != colour ? 1 : 0);
    if (ix >= g.nx) return -1;
    return (int)(ix + (long)g.nx * r);
}

// Colour-split storage of the blocks the red-black sweeps read (Ahat and the
// inverted diagonal blocks): colour (ix + iy + iz) & 1 first, then the cell's
// slot in colour_cell's order, so the threads of a one-colour sweep read
// consecutive positions (component-major storage by cell would hand each warp
// sectors half filled with the other colour's blocks).  2 H positions.
__device__ __forceinline__ long cslot(const GridDesc &g, int ix, int iy, int iz) {
    return (long)((ix + iy + iz) & 1) * g.H + (long)(iy + g.ny * iz) * ((g.nx + 1) >> 1) + (ix >> 1);
}
__device__ __forceinline__ long cslot_of(const GridDesc &g, int i) {
    const int ix = i % g.nx, t = i / g.nx, iy = t % g.ny, iz = t / g.ny;
    return cslot(g, ix, iy, iz);
}

__device__ __forceinline__ int opp(int d) { return d == 0 ? 0 : ((d & 1) ? d + 1 : d - 1); }
__device__ __forceinline__ bool is_black(const GridDesc &g, int i) {
    const int ix = i % g.nx, t = i / g.nx, iy = t % g.ny, iz = t / g.ny;
    return ((ix + iy + iz) & 1) != 0;
}

// A row of a level matrix: structured (level 0) or ELL
template <typename V>
struct Mat {
    bool st;
    bool selfpad;    // ELL padded with (self column, 0) instead of -1: no early exit
    bool diff;       // difference form: the diagonal slot holds the row sum (see row_dot)
    GridDesc g;      // structured
    const V *val;    // structured: [7][n]; ELL: [width][n]
    const int *col;  // ELL
    int n, width;
};

// visit the entries of row i in ascending column order: f(col, val)
// (self-padded ELL rows end with zero entries on the diagonal column)
template <typename V, typename F>
__device__ __forceinline__ void for_row(const Mat<V> &A, int i, F f) {
    if (A.st) {
        const int nx = A.g.nx, ny = A.g.ny, nxy = nx * ny;
        const int ix = i % nx, t = i / nx, iy = t % ny, iz = t / ny;
        const long n = A.n;
        if (iz > 0) f(i - nxy, A.val[5 * n + i]);
        if (iy > 0) f(i - nx, A.val[3 * n + i]);
        if (ix > 0) f(i - 1, A.val[1 * n + i]);
        f(i, A.val[i]);
        if (ix < nx - 1) f(i + 1, A.val[2 * n + i]);
        if (iy < ny - 1) f(i + nx, A.val[4 * n + i]);
        if (iz < A.g.nz - 1) f(i + nxy, A.val[6 * n + i]);
    } else if (A.selfpad) {
        // batches of 8 entries: the batch's loads are issued together, then f
        // runs on them in column-slot order
        for (int k0 = 0; k0 < A.width; k0 += 8) {
            int jj[8];
            V vv[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const long q = (long)(k0 + u) * A.n + i;
                const bool ok = k0 + u < A.width;
                jj[u] = ok ? A.col[q] : i;
                vv[u] = ok ? A.val[q] : V(0);
            }
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (k0 + u < A.width) f(jj[u], vv[u]);
        }
    } else {
        // -1 padding sits only at the end of a row: skipping it instead of
        // stopping there visits the same entries in the same order, and the
        // column loads no longer wait on one another
#pragma unroll 4
        for (int k = 0; k < A.width; k++) {
            const int j = A.col[(long)k * A.n + i];
            if (j >= 0) f(j, A.val[(long)k * A.n + i]);
        }
    }
}

// A_i . e.  In the difference form (the FP32 copies of the pressure matrices)
// the diagonal slot holds the row sum d_i = sum_j a_ij, computed in FP64, and
// A_i . e = d_i e_i + sum_{j != i} a_ij (e_j - e_i): the small row sum (the
// accumulation term, 1e-4 to 1e-7 of the off-diagonals where permeability is
// high) survives rounding to FP32, where a_ii + sum_{j != i} a_ij would lose it.
template <typename T>
__device__ __forceinline__ T row_dot(const Mat<T> &A, int i, const T *__restrict__ e) {
    T t = (T)0;
    if (A.diff) {
        const T ei = e[i];
        for_row(A, i, [&](int j, T v) { t += (j == i) ? v * ei : v * (e[j] - ei); });
    } else {
        for_row(A, i, [&](int j, T v) { t += v * e[j]; });
    }
    return t;
}

__global__ void selfpad_kernel(int n, int W, const int *__restrict__ col, int *__restrict__ colA) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)n * W) return;
    const int i = (int)(t % n);
    const int c = col[t];
    colA[t] = c < 0 ? i : c;
}

// ---------------------------------------------------------------------------
// quasi-IMPES decoupling (FP64, rounding-exact: no contraction)
// ---------------------------------------------------------------------------
// rate-controlled wells' Schur term in the preconditioner matrix: block (i, d)
// of J loses A_pw[q] A_ww^-1 A_wp[q'] when cell i holds perforation q and its
// neighbour j holds perforation q' of the same rate-controlled well
struct WellCorr {
    const int *cell_perf = nullptr;   // null: no rate-controlled wells
    const int *pwell = nullptr;
    const double *apw = nullptr, *awp = nullptr, *aww = nullptr;   // [3][nperf], [nwells]
    int nperf = 0;
};

// block (row cell i, direction d, neighbour j) of the preconditioner matrix,
// the correction rounded as written (the AMG hierarchy is built bit-exactly)
template <int B>
__device__ __forceinline__ void load_jblock(const double *__restrict__ J, long N, int i, int d, int j, const WellCorr &wc,
                                            double *Jb) {
#pragma unroll
    for (int t = 0; t < B * B; t++) Jb[t] = J[(long)(d * B * B + t) * N + i];
    if (!wc.cell_perf || j < 0) return;
    const int q = wc.cell_perf[i];
    if (q < 0) return;
    const int q2 = wc.cell_perf[j];
    if (q2 < 0 || wc.pwell[q2] != wc.pwell[q]) return;
    const double a = wc.aww[wc.pwell[q]];
#pragma unroll
    for (int r = 0; r < B; r++)
#pragma unroll
        for (int c = 0; c < B; c++)
            Jb[r * B + c] = __dsub_rn(Jb[r * B + c],
                                      __ddiv_rn(__dmul_rn(wc.apw[(long)r * wc.nperf + q], wc.awp[(long)c * wc.nperf + q2]), a));
}

template <int B>
__device__ __forceinline__ void qi_weights(const double *D, double *w) {
    const double D01 = D[0 * B + 1], D11 = D[1 * B + 1];
    w[0] = 1.0;
    if constexpr (B == 2) {
        w[1] = -(D01 / D11);
    } else {
        const double D02 = D[0 * B + 2];
        const double D12 = D[1 * B + 2], D21 = D[2 * B + 1], D22 = D[2 * B + 2];
        const double det = __dsub_rn(__dmul_rn(D11, D22), __dmul_rn(D12, D21));
        w[1] = __ddiv_rn(__dsub_rn(__dmul_rn(D02, D21), __dmul_rn(D01, D22)), det);
        w[2] = __ddiv_rn(__dsub_rn(__dmul_rn(D01, D12), __dmul_rn(D02, D11)), det);
    }
}

// decoupled block (row cell i, direction d): Ahat = L_i J_id, products summed in
// row order without contraction (quasi-IMPES: L = [w^T; 0 I], so the pressure
// row is J_0c + w1 J_1c + w2 J_2c exactly as the oracle forms it)
template <int B>
__device__ __forceinline__ void ahat_block(const double *__restrict__ J, long N, int i, int d, int j, const WellCorr &wc,
                                           const double *L, double *A) {
    double Jb[B * B];
    load_jblock<B>(J, N, i, d, j, wc, Jb);
#pragma unroll
    for (int r = 0; r < B; r++)
#pragma unroll
        for (int c = 0; c < B; c++) {
            double t = __dmul_rn(L[r * B], Jb[c]);
            t = __dadd_rn(t, __dmul_rn(L[r * B + 1], Jb[B + c]));
            if (B == 3) t = __dadd_rn(t, __dmul_rn(L[r * B + 2], Jb[2 * B + c]));
            A[r * B + c] = t;
        }
}

template <int B>
__device__ __forceinline__ void load_lsc(const double *__restrict__ lsc, long N, int i, double *L) {
#pragma unroll
    for (int t = 0; t < B * B; t++) L[t] = lsc[(long)t * N + i];
}

// inverse of a diagonal block by cofactors, every operation rounded as written
// (the ABF scaling feeds the AMG hierarchy, which is built bit-exactly)
template <int B>
__device__ __forceinline__ void inv_block_rn(const double *A, double *Ai) {
#define M_(a, b) __dmul_rn(A[a], A[b])
    if constexpr (B == 2) {
        const double det = __dsub_rn(M_(0, 3), M_(1, 2));
        Ai[0] = __ddiv_rn(A[3], det); Ai[1] = __ddiv_rn(-A[1], det);
        Ai[2] = __ddiv_rn(-A[2], det); Ai[3] = __ddiv_rn(A[0], det);
    } else {
        const double c00 = __dsub_rn(M_(4, 8), M_(5, 7));
        const double c01 = __dsub_rn(M_(5, 6), M_(3, 8));
        const double c02 = __dsub_rn(M_(3, 7), M_(4, 6));
        const double det = __dadd_rn(__dadd_rn(__dmul_rn(A[0], c00), __dmul_rn(A[1], c01)), __dmul_rn(A[2], c02));
        Ai[0] = __ddiv_rn(c00, det);
        Ai[1] = __ddiv_rn(__dsub_rn(M_(2, 7), M_(1, 8)), det);
        Ai[2] = __ddiv_rn(__dsub_rn(M_(1, 5), M_(2, 4)), det);
        Ai[3] = __ddiv_rn(c01, det);
        Ai[4] = __ddiv_rn(__dsub_rn(M_(0, 8), M_(2, 6)), det);
        Ai[5] = __ddiv_rn(__dsub_rn(M_(2, 3), M_(0, 5)), det);
        Ai[6] = __ddiv_rn(c02, det);
        Ai[7] = __ddiv_rn(__dsub_rn(M_(1, 6), M_(0, 7)), det);
        Ai[8] = __ddiv_rn(__dsub_rn(M_(0, 4), M_(1, 3)), det);
    }
#undef M_
}

// left scaling per cell (quasi-IMPES or ABF), its first row, the pressure
// block A_p and the decoupled matrix in the apply precision
template <int B, typename T>
__global__ void qi_kernel(GridDesc g, const double *__restrict__ J, WellCorr wc, int abf, double *__restrict__ lsc,
                          T *__restrict__ lscT, double *__restrict__ qiw, T *__restrict__ qiwT, double *__restrict__ ap,
                          T *__restrict__ apT, T *__restrict__ ahat) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const long N = g.N;
    if (i >= N) return;
    double L[B * B], D[B * B];
    load_jblock<B>(J, N, i, 0, i, wc, D);
    if (abf) {
        inv_block_rn<B>(D, L);
    } else {
        double w[3] = {1.0, 0.0, 0.0};
        qi_weights<B>(D, w);
#pragma unroll
        for (int t = 0; t < B * B; t++) L[t] = (t / B == t % B) ? 1.0 : 0.0;
        L[1] = w[1];
        if (B == 3) L[2] = w[2];
    }
#pragma unroll
    for (int t = 0; t < B * B; t++) { lsc[(long)t * N + i] = L[t]; lscT[(long)t * N + i] = (T)L[t]; }
#pragma unroll
    for (int c = 0; c < B; c++) { qiw[(long)c * N + i] = L[c]; qiwT[(long)c * N + i] = (T)L[c]; }
    const Cell cc = cell_of(g, i);
    const long NS = 2L * g.H, si = cslot(g, cc.ix, cc.iy, cc.iz);
    double rsum = 0.0;                   // FP32 copy: row sum of A_p on the diagonal slot (difference form)
    for (int d = 0; d < 7; d++) {
        double A[B * B];
        const int j = nbrc(g, cc, d);
        ahat_block<B>(J, N, i, d, j, wc, L, A);
        const bool has = j >= 0;
        ap[(long)d * N + i] = has ? A[0] : 0.0;
        apT[(long)d * N + i] = has ? (T)A[0] : (T)0;
        if (sizeof(T) == sizeof(float) && has) rsum += A[0];
#pragma unroll
        for (int t = 0; t < B * B; t++) ahat[(long)(d * B * B + t) * NS + si] = (T)A[t];
    }
    if (sizeof(T) == sizeof(float)) apT[i] = (T)rsum;
}

// ---------------------------------------------------------------------------
// block inverses and red-black ILU(0) setup (FP64)
// ---------------------------------------------------------------------------
template <int B>
__device__ __forceinline__ void inv_block(const double *A, double *Ai) {
    if constexpr (B == 2) {
        const double det = A[0] * A[3] - A[1] * A[2];
        Ai[0] = A[3] / det; Ai[1] = -A[1] / det; Ai[2] = -A[2] / det; Ai[3] = A[0] / det;
    } else {
        const double c00 = A[4] * A[8] - A[5] * A[7];
        const double c01 = A[5] * A[6] - A[3] * A[8];
        const double c02 = A[3] * A[7] - A[4] * A[6];
        const double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
        const double id = 1.0 / det;
        Ai[0] = c00 * id; Ai[1] = (A[2] * A[7] - A[1] * A[8]) * id; Ai[2] = (A[1] * A[5] - A[2] * A[4]) * id;
        Ai[3] = c01 * id; Ai[4] = (A[0] * A[8] - A[2] * A[6]) * id; Ai[5] = (A[2] * A[3] - A[0] * A[5]) * id;
        Ai[6] = c02 * id; Ai[7] = (A[1] * A[6] - A[0] * A[7]) * id; Ai[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    }
}

// mode 0: inverse of Ahat_ii for every cell (block-Jacobi) or red cells only (mode 1);
// mode 2: inverse of J_ii (plain block-Jacobi, no decoupling)
template <int B>
__global__ void diag_inv_kernel(GridDesc g, const double *__restrict__ J, WellCorr wc, const double *__restrict__ lsc,
                                int mode, double *__restrict__ dinv) {
    const long N = g.N;
    const int i = mode == 1 ? colour_cell(g, blockIdx.x * (long)blockDim.x + threadIdx.x, 0)
                            : (blockIdx.x * blockDim.x + threadIdx.x < N ? (int)(blockIdx.x * blockDim.x + threadIdx.x) : -1);
    if (i < 0) return;
    double L[B * B], A[B * B], Ai[B * B];
    if (mode == 2) {
        load_jblock<B>(J, N, i, 0, i, wc, A);
    } else {
        load_lsc<B>(lsc, N, i, L);
        ahat_block<B>(J, N, i, 0, i, wc, L, A);
    }
    inv_block<B>(A, Ai);
    const long NS = 2L * g.H, si = cslot_of(g, i);
#pragma unroll
    for (int t = 0; t < B * B; t++) dinv[(long)t * NS + si] = Ai[t];
}

// black cells: D = Ahat_ii - sum_d Ahat_{i,d} Dinv_k Ahat_{k,opp(d)}
template <int B>
__global__ void __launch_bounds__(SIM_THREADS, 2) ilu_black_kernel(GridDesc g, const double *__restrict__ J, WellCorr wc,
                                                                   const double *__restrict__ lsc,
                                                                   double *__restrict__ dinv) {
    const int i = colour_cell(g, blockIdx.x * (long)blockDim.x + threadIdx.x, 1);
    const long N = g.N;
    if (i < 0) return;
    double Li[B * B];
    load_lsc<B>(lsc, N, i, Li);
    double D[B * B];
    ahat_block<B>(J, N, i, 0, i, wc, Li, D);
    for (int d = 1; d < 7; d++) {
        const int k = nbr7(g, i, d);
        if (k < 0) continue;
        double Lk[B * B], Aik[B * B], Aki[B * B], Dk[B * B], T1[B * B];
        load_lsc<B>(lsc, N, k, Lk);
        ahat_block<B>(J, N, i, d, k, wc, Li, Aik);
        ahat_block<B>(J, N, k, opp(d), i, wc, Lk, Aki);
        const long sk = cslot_of(g, k);
#pragma unroll
        for (int t = 0; t < B * B; t++) Dk[t] = dinv[(long)t * 2L * g.H + sk];
#pragma unroll
        for (int r = 0; r < B; r++)
#pragma unroll
            for (int c = 0; c < B; c++) {
                double s = 0.0;
#pragma unroll
                for (int q = 0; q < B; q++) s += Dk[r * B + q] * Aki[q * B + c];
                T1[r * B + c] = s;
            }
#pragma unroll
        for (int r = 0; r < B; r++)
#pragma unroll
            for (int c = 0; c < B; c++) {
                double s = 0.0;
#pragma unroll
                for (int q = 0; q < B; q++) s += Aik[r * B + q] * T1[q * B + c];
                D[r * B + c] -= s;
            }
    }
    double Di[B * B];
    inv_block<B>(D, Di);
    const long NS = 2L * g.H, si = cslot_of(g, i);
#pragma unroll
    for (int t = 0; t < B * B; t++) dinv[(long)t * NS + si] = Di[t];
}

// FP32 copy of an ELL level in the difference form: the diagonal entry is
// replaced by the row sum (computed in FP64), the others rounded as they are
__global__ void cast_diff_kernel(int n, int W, const int *__restrict__ col, const double *__restrict__ val,
                                 float *__restrict__ valT) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double rs = 0.0;
    for (int k = 0; k < W; k++) {
        const int j = col[(long)k * n + i];
        if (j < 0) break;
        rs += val[(long)k * n + i];
    }
    for (int k = 0; k < W; k++) {
        const long t = (long)k * n + i;
        const int j = col[t];
        valT[t] = j == i ? (float)rs : (float)val[t];
    }
}

template <typename T>
__global__ void cast_kernel(const double *__restrict__ a, T *__restrict__ b, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) b[i] = (T)a[i];
}

// ---------------------------------------------------------------------------
// AMG setup kernels (FP64 values, integer results)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long edge_hash(int a, int b) {
    const unsigned long long lo = (unsigned long long)(a < b ? a : b), hi = (unsigned long long)(a < b ? b : a);
    unsigned long long z = ((hi << 32) | lo) + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__device__ __forceinline__ int strength_band(double a) {
    return (int)((__double_as_longlong(a) >> 52) & 0x7FF);
}

__global__ void match_pick_kernel(Mat<double> A, const int *__restrict__ partner, int *__restrict__ pick, double theta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    pick[i] = -1;
    if (partner[i] >= 0) return;
    double mx = 0.0;
    for_row(A, i, [&](int j, double a) { if (j != i && -a > mx) mx = -a; });
    if (mx <= 0.0) return;
    int best = -1, bs = 0;
    unsigned long long bh = 0ULL;
    const double lim = theta * mx;
    for_row(A, i, [&](int j, double v) {
        if (j == i || partner[j] >= 0) return;
        const double a = -v;
        if (!(a > 0.0) || a < lim) return;
        const int band = strength_band(a);
        const unsigned long long h = edge_hash(i, j);
        if (best < 0 || band > bs || (band == bs && (h > bh || (h == bh && j < best)))) { best = j; bs = band; bh = h; }
    });
    pick[i] = best;
}

__global__ void match_confirm_kernel(int n, const int *__restrict__ pick, int *__restrict__ partner) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = pick[i];
    if (partner[i] < 0 && p >= 0 && pick[p] == i) partner[i] = p;
}

// single nodes join the aggregate of their strongest strong matched
// neighbour (same key as the matching): host[i], or -1
__global__ void host_kernel(Mat<double> A, const int *__restrict__ partner, int *__restrict__ host, double theta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    host[i] = -1;
    if (partner[i] >= 0) return;
    double mx = 0.0;
    for_row(A, i, [&](int j, double a) { if (j != i && -a > mx) mx = -a; });
    if (mx <= 0.0) return;
    int best = -1, bs = 0;
    unsigned long long bh = 0ULL;
    const double lim = theta * mx;
    for_row(A, i, [&](int j, double v) {
        if (j == i || partner[j] < 0) return;
        const double a = -v;
        if (!(a > 0.0) || a < lim) return;
        const int band = strength_band(a);
        const unsigned long long h = edge_hash(i, j);
        if (best < 0 || band > bs || (band == bs && (h > bh || (h == bh && j < best)))) { best = j; bs = band; bh = h; }
    });
    host[i] = best;
}

// founders: pair leaders (lower index of a pair) and lone nodes without a host
__global__ void founder_kernel(int n, const int *__restrict__ partner, const int *__restrict__ host, int *__restrict__ flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = partner[i];
    flag[i] = ((p >= 0 && i < p) || (p < 0 && host[i] < 0)) ? 1 : 0;
}

// generic exclusive scan of n ints in chunks of SCAN_CHUNK per block
constexpr int SCAN_CHUNK = 4096;
__global__ void scan_sum_kernel(int n, const int *__restrict__ in, int *__restrict__ bsum) {
    __shared__ int sh[SIM_THREADS];
    const int base = blockIdx.x * SCAN_CHUNK;
    int c = 0;
    for (int t = threadIdx.x; t < SCAN_CHUNK; t += blockDim.x) {
        const int i = base + t;
        if (i < n) c += in[i];
    }
    sh[threadIdx.x] = c;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = sh[0];
}

// single block: exclusive scan of nb block sums in place, total into *total
__global__ void scan_blocks_kernel(int nb, int *__restrict__ bsum, int *__restrict__ total) {
    __shared__ int carry;
    __shared__ int sh[1024];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? bsum[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            const int t = (int)threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) bsum[i] = carry + sh[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += sh[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// out[i] = sum_{k<i} in[k]; out[n] = total
__global__ void scan_write_kernel(int n, const int *__restrict__ in, const int *__restrict__ bsum, const int *__restrict__ total,
                                  int *__restrict__ out) {
    __shared__ int sh[SIM_THREADS];
    const int base = blockIdx.x * SCAN_CHUNK;
    constexpr int PER = SCAN_CHUNK / SIM_THREADS;
    const int t0 = base + threadIdx.x * PER;
    int local = 0;
    for (int k = 0; k < PER; k++) { const int i = t0 + k; if (i < n) local += in[i]; }
    sh[threadIdx.x] = local;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        const int t = (int)threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    int run = bsum[blockIdx.x] + sh[threadIdx.x] - local;
    for (int k = 0; k < PER; k++) {
        const int i = t0 + k;
        if (i >= n) break;
        out[i] = run;
        run += in[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = *total;
}

// aggregate of every node: founders own ids; pair followers take the
// leader's; absorbed nodes take their host pair's
__global__ void agg_kernel(int n, const int *__restrict__ partner, const int *__restrict__ host, const int *__restrict__ id,
                           int *__restrict__ agg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = partner[i];
    int a;
    if (p >= 0) a = id[i < p ? i : p];
    else if (host[i] < 0) a = id[i];
    else { const int h = host[i], hp = partner[h]; a = id[h < hp ? h : hp]; }
    agg[i] = a;
}

__global__ void count_kernel(int n, const int *__restrict__ agg, int *__restrict__ cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[agg[i]], 1);
}
__global__ void fill_kernel(int n, const int *__restrict__ agg, const int *__restrict__ moff, int *__restrict__ pos,
                            int *__restrict__ mem) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int a = agg[i];
    mem[moff[a] + atomicAdd(&pos[a], 1)] = i;
}
// members of each aggregate in ascending order (the fill order is arbitrary)
__global__ void sort_members_kernel(int nc, const int *__restrict__ moff, int *__restrict__ mem) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    const int a0 = moff[I], a1 = moff[I + 1];
    for (int a = a0 + 1; a < a1; a++) {
        const int v = mem[a];
        int t = a - 1;
        while (t >= a0 && mem[t] > v) { mem[t + 1] = mem[t]; t--; }
        mem[t + 1] = v;
    }
}

// Galerkin row I of P^T A P, one warp per row.  The members' row entries,
// mapped to aggregate columns, are staged in member-then-column order (the
// order of the sequential definition); each distinct column sums its entries
// in that order, and the distinct columns are ranked ascending.  Rows whose
// list exceeds kGalCap entries are left to galerkin_kernel.
constexpr int kGalWarps = 8, kGalCap = 256;

__global__ void __launch_bounds__(kGalWarps * 32) galerkin_warp_kernel(
    Mat<double> A, const int *__restrict__ agg, const int *__restrict__ moff, const int *__restrict__ mem, int nc,
    int mode, int *__restrict__ len, int W, int *__restrict__ ccol, double *__restrict__ cval, int *err) {
    __shared__ int scol[kGalWarps][kGalCap];
    __shared__ double sval[kGalWarps][kGalCap];
    __shared__ unsigned char sfirst[kGalWarps][kGalCap];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int I = blockIdx.x * kGalWarps + w;
    if (I >= nc) return;                          // whole warp
    int *cl = scol[w];
    double *vl = sval[w];
    unsigned char *fl = sfirst[w];
    // 1. the ordered list
    int L = 0;
    bool over = false;
    for (int q = moff[I]; q < moff[I + 1] && !over; q++) {
        const int m = mem[q];
        if (A.st) {
            // structured row: the 7-point entries in ascending column order
            const int nx = A.g.nx, ny = A.g.ny, nxy = nx * ny;
            const int ix = m % nx, t = m / nx, iy = t % ny, iz = t / ny;
            const long n = A.n;
            const int dirs[7] = {5, 3, 1, 0, 2, 4, 6};
            const int offs[7] = {-nxy, -nx, -1, 0, 1, nx, nxy};
            bool ok = false;
            int col = 0, d = 0;
            if (lane < 7) {
                d = dirs[lane];
                ok = (d == 0) || (d == 1 && ix > 0) || (d == 2 && ix < nx - 1) || (d == 3 && iy > 0) ||
                     (d == 4 && iy < ny - 1) || (d == 5 && iz > 0) || (d == 6 && iz < A.g.nz - 1);
                col = m + offs[lane];
            }
            const unsigned bal = __ballot_sync(0xffffffffu, ok);
            const int cnt = __popc(bal);
            if (L + cnt > kGalCap) { over = true; break; }
            if (ok) {
                const int pos = L + __popc(bal & ((1u << lane) - 1u));
                cl[pos] = agg[col];
                vl[pos] = A.val[d * n + m];
            }
            L += cnt;
        } else {
            for (int k0 = 0; k0 < A.width; k0 += 32) {
                const int k = k0 + lane;
                int col = -1;
                double v = 0.0;
                if (k < A.width) { col = A.col[(long)k * A.n + m]; if (col >= 0) v = A.val[(long)k * A.n + m]; }
                const bool ok = col >= 0;
                const unsigned bal = __ballot_sync(0xffffffffu, ok);
                const int cnt = __popc(bal);
                if (L + cnt > kGalCap) { over = true; break; }
                if (ok) {
                    const int pos = L + __popc(bal & ((1u << lane) - 1u));
                    cl[pos] = agg[col];
                    vl[pos] = v;
                }
                L += cnt;
                if (cnt < 32) break;              // -1 padding: the row has ended
            }
        }
    }
    if (over) {                                   // galerkin_kernel takes this row
        if (mode == 0 && lane == 0) len[I] = -1;
        return;
    }
    __syncwarp();
    // 2. first occurrences, their count, their ordered sums and ranks
    int D = 0;
    for (int p0 = 0; p0 < L; p0 += 32) {
        const int p = p0 + lane;
        bool first = false;
        if (p < L) {
            first = true;
            const int c = cl[p];
            for (int q = 0; q < p; q++) if (cl[q] == c) { first = false; break; }
            fl[p] = first;
        }
        D += __popc(__ballot_sync(0xffffffffu, first));
    }
    if (D > MAXE) { if (lane == 0) atomicExch(err, 1); return; }
    if (mode == 0) {
        if (lane == 0) { len[I] = D; atomicMax(len + nc, D); }
        return;
    }
    __syncwarp();
    for (int p0 = 0; p0 < L; p0 += 32) {
        const int p = p0 + lane;
        if (p >= L || !fl[p]) continue;
        const int c = cl[p];
        double sum = 0.0;
        for (int q = p; q < L; q++) if (cl[q] == c) sum = __dadd_rn(sum, vl[q]);
        int rank = 0;                             // distinct columns below c
        for (int q = 0; q < L; q++) rank += (fl[q] && cl[q] < c);
        ccol[(long)rank * nc + I] = c;
        cval[(long)rank * nc + I] = sum;
    }
    for (int t = D + lane; t < W; t += 32) {
        ccol[(long)t * nc + I] = -1;
        cval[(long)t * nc + I] = 0.0;
    }
}

// Galerkin row I of P^T A P, one thread per row (rows with long lists):
// members moff/mem (ascending), entries summed in member order then column
// order, columns sorted ascending.
// mode 0: row length into len[I]; mode 1: write the ELL row of width W
__global__ void galerkin_kernel(Mat<double> A, const int *__restrict__ agg, const int *__restrict__ moff,
                                const int *__restrict__ mem, int nc, int mode, int *__restrict__ len, int W,
                                int *__restrict__ ccol, double *__restrict__ cval, int *err) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    // rows the warp kernel left: len = -1 after its counting pass; this kernel
    // then stores -(count) - 2, so the filling pass finds the same rows
    if (mode == 0 ? len[I] != -1 : len[I] >= 0) return;
    int cols[MAXE];
    double vals[MAXE];
    int cnt = 0;
    bool over = false;
    for (int q = moff[I]; q < moff[I + 1]; q++) {
        const int m = mem[q];
        for_row(A, m, [&](int j, double a) {
            const int Jc = agg[j];
            int f = -1;
            for (int t = 0; t < cnt; t++) if (cols[t] == Jc) { f = t; break; }
            if (f < 0) {
                if (cnt == MAXE) { over = true; return; }
                cols[cnt] = Jc; vals[cnt] = 0.0; f = cnt++;
            }
            vals[f] = __dadd_rn(vals[f], a);
        });
    }
    if (over) { atomicExch(err, 1); return; }
    for (int a = 1; a < cnt; a++) {
        const int cj = cols[a];
        const double cv = vals[a];
        int t = a - 1;
        while (t >= 0 && cols[t] > cj) { cols[t + 1] = cols[t]; vals[t + 1] = vals[t]; t--; }
        cols[t + 1] = cj; vals[t + 1] = cv;
    }
    if (mode == 0) { len[I] = -cnt - 2; atomicMax(len + nc, cnt); return; }
    for (int t = 0; t < W; t++) {
        ccol[(long)t * nc + I] = t < cnt ? cols[t] : -1;
        cval[(long)t * nc + I] = t < cnt ? vals[t] : 0.0;
    }
}

__global__ void compose_kernel(int n, const int *__restrict__ aggA, const int *__restrict__ aggB, int *__restrict__ agg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) agg[i] = aggB[aggA[i]];
}
template <typename T>
__global__ void l1_kernel(Mat<double> A, T *__restrict__ dinv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    double s = 0.0;
    for_row(A, i, [&](int, double a) { s += fabs(a); });
    dinv[i] = (T)(1.0 / s);
}

// Gauss-Jordan step k without pivoting on the augmented [A | Inv] (n x 2n),
// read from src and written to dst: the coarse pressure block is
// diagonally dominant with a positive diagonal, so the pivots stay positive.
// Gauss-Jordan elimination without pivoting of [A | I] on the coarsest level,
// in one launch of an 8-CTA cluster: step k writes, from the matrix left by
// step k-1 (ping-pong buffers), pivot row k divided by its pivot and every
// other row minus its column-k entry times that row; a cluster barrier
// separates the steps; the result ends in A1 for odd n, else A0
constexpr int kGjMax = 1024;   // largest coarsest level (rows)

// A pivot whose magnitude is not above kGjPivotTol times the l1 norm of its
// row of A (rn) -- zero, denormal, NaN, or pure rounding noise -- sets *bad;
// the elimination still runs to its end (the cluster barriers need every CTA)
// and the host turns the flag into an error instead of using the inverse.
constexpr double kGjPivotTol = 1e-14;

__device__ __forceinline__ void gj_check_pivot(double piv, double rnorm, int *bad) {
    if (!(fabs(piv) > kGjPivotTol * rnorm)) *(volatile int *)bad = 1;
}

__global__ void __cluster_dims__(8, 1, 1) __launch_bounds__(1024, 1)
gj_cluster_kernel(int n, double *__restrict__ A0, double *__restrict__ A1, const double *__restrict__ rn, int *bad) {
    __shared__ double pk[2 * kGjMax];   // the pivot row over its pivot, per CTA (one division per entry)
    const int w = 2 * n;
    // CTA c owns rows c, c + 8, ...; its threads stride over the columns (no index division)
    const int tpr = blockDim.x < (unsigned)w ? blockDim.x : w;    // threads per row
    const int rows_at_once = blockDim.x / tpr;
    const int r0 = threadIdx.x / tpr, j0 = threadIdx.x % tpr;
    for (int k = 0; k < n; k++) {
        const double *src = (k & 1) ? A1 : A0;
        double *dst = (k & 1) ? A0 : A1;
        const double piv = src[(long)k * w + k];
        if (blockIdx.x == 0 && threadIdx.x == 0) gj_check_pivot(piv, rn[k], bad);
        for (int j = threadIdx.x; j < w; j += blockDim.x) pk[j] = src[(long)k * w + j] / piv;
        __syncthreads();
        if (r0 < rows_at_once) {
            for (int i = blockIdx.x + r0 * gridDim.x; i < n; i += rows_at_once * gridDim.x) {
                const double f = src[(long)i * w + k];
                const double *si = src + (long)i * w;
                double *di = dst + (long)i * w;
                for (int j = j0; j < w; j += tpr) di[j] = (i == k) ? pk[j] : si[j] - f * pk[j];
            }
        }
        __threadfence();
        cg::this_cluster().sync();   // also keeps pk from being overwritten early
    }
}

// The same elimination with the augmented matrix held in the shared memory of
// the CTAs of one cluster (8, or 16 where the part schedules a cluster that
// large; n <= kGjSmem), kGjPanel pivots at a time: CTA c
// owns a block of rows; for each panel of up to kGjPanel consecutive pivot
// rows (all in one CTA) the owner reduces the panel to the identity on its
// pivot columns (Gauss-Jordan within the panel), one cluster barrier
// publishes it (double-buffered by panel parity), and every CTA reads it
// through distributed shared memory and subtracts, from each of its other
// rows, the panel rows times that row's entries in the pivot columns.  In
// exact arithmetic this is the pivot-by-pivot elimination; it needs one
// cluster barrier per panel instead of one per pivot.  The right half of the
// result is written to inv.
constexpr int kGjSmem = 256, kGjPanel = 4;

__global__ void __launch_bounds__(1024, 1)
gj_dsmem_kernel(int n, const double *__restrict__ aug, double *__restrict__ inv, const double *__restrict__ rn,
                int *bad) {
    extern __shared__ double gsm[];
    cg::cluster_group cl = cg::this_cluster();
    const int nc = (int)cl.num_blocks(), w = 2 * n, rpc = (n + nc - 1) / nc;   // rows per CTA
    const int me = (int)cl.block_rank(), tid = threadIdx.x, bd = blockDim.x;
    double *R = gsm;                                      // [rpc][w] own rows
    double *P = R + (long)rpc * w;                        // [2][kGjPanel][w] panels (by panel parity)
    double *PL = P + 2L * kGjPanel * w;                   // [kGjPanel][w] local copy of the current panel
    double *F = PL + (long)kGjPanel * w;                  // [rpc][kGjPanel] own rows' pivot-column entries
    const int base = me * rpc, nrows = max(0, min(rpc, n - base));
    for (int t = tid; t < nrows * w; t += bd) R[t] = aug[(long)base * w + t];
    __syncthreads();
    int panel = 0;
    for (int c = 0; c < nc; c++) {
        const int cb = c * rpc, cn = max(0, min(rpc, n - cb));
        for (int k0 = cb; k0 < cb + cn; k0 += kGjPanel, panel++) {
            const int ps = min(kGjPanel, cb + cn - k0);
            double *Pb = P + (long)(panel & 1) * kGjPanel * w;
            // the panel rows are zero outside columns [k0, n + k0 + ps) (left of k0
            // eliminated, right of n + k0 + ps still the untouched identity), so only
            // that window of width n + ps changes: half the FP64 work of the full 2n
            const int j0 = k0, wa = n + ps;
            if (me == c) {
                for (int t = tid; t < ps * w; t += bd) Pb[t] = R[(long)(k0 - base) * w + t];
                __syncthreads();
                for (int q = 0; q < ps; q++) {
                    const double piv = Pb[(long)q * w + k0 + q];
                    if (tid == 0) gj_check_pivot(piv, rn[k0 + q], bad);
                    __syncthreads();
                    for (int j = j0 + tid; j < j0 + wa; j += bd) Pb[(long)q * w + j] = Pb[(long)q * w + j] / piv;
                    __syncthreads();
                    double fu[kGjPanel];
#pragma unroll
                    for (int u = 0; u < kGjPanel; u++) fu[u] = u < ps ? Pb[(long)u * w + k0 + q] : 0.0;
                    __syncthreads();
                    for (int t = tid; t < ps * wa; t += bd) {
                        const int u = t / wa, j = j0 + (t - u * wa);
                        if (u != q) Pb[(long)u * w + j] = Pb[(long)u * w + j] - fu[u] * Pb[(long)q * w + j];
                    }
                    __syncthreads();
                }
            }
            cl.sync();
            const double *rP = cl.map_shared_rank(Pb, c);
            for (int t = tid; t < ps * wa; t += bd) {
                const int u = t / wa, j = j0 + (t - u * wa);
                PL[(long)u * w + j] = rP[(long)u * w + j];
            }
            for (int t = tid; t < nrows * ps; t += bd) {
                const int r = t / ps, u = t - r * ps;
                F[r * kGjPanel + u] = R[(long)r * w + k0 + u];
            }
            __syncthreads();
            for (int t = tid; t < nrows * wa; t += bd) {
                const int r = t / wa, j = j0 + (t - r * wa), gi = base + r;
                double *Rr = R + (long)r * w + j;
                if (gi >= k0 && gi < k0 + ps) {
                    *Rr = PL[(long)(gi - k0) * w + j];
                } else {
                    double v = *Rr;
                    for (int u = 0; u < ps; u++) v -= F[r * kGjPanel + u] * PL[(long)u * w + j];
                    *Rr = v;
                }
            }
            __syncthreads();
        }
    }
    cl.sync();                                            // no CTA leaves while another may read its panels
    for (int t = tid; t < nrows * n; t += bd) {
        const int r = t / n, j = t - r * n;
        inv[(long)(base + r) * n + j] = R[(long)r * w + n + j];
    }
}

static size_t gj_dsmem_bytes(int n, int nc) {
    const int w = 2 * n, rpc = (n + nc - 1) / nc;
    return sizeof(double) * ((size_t)rpc * w + 3 * (size_t)kGjPanel * w + (size_t)rpc * kGjPanel);
}

// [A | I], one thread per entry (row i, column j of the n x 2n array)
// CTAs of the Gauss-Jordan cluster: 16 (a non-portable size) when the
// occupancy query finds room for one such cluster at the largest shared-memory
// size, else the portable 8; the query launches nothing
static int gj_cluster_ctas() {
    if (cudaFuncSetAttribute(gj_dsmem_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        (void)cudaGetLastError();
        return 8;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(16); cfg.blockDim = dim3(1024); cfg.dynamicSmemBytes = gj_dsmem_bytes(kGjSmem, 16);
    cfg.attrs = at; cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, gj_dsmem_kernel, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        return 8;
    }
    return clusters > 0 ? 16 : 8;
}

__global__ void gj_init_kernel(Mat<double> A, double *__restrict__ aug) {
    const long w = 2L * A.n;
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)A.n * w) return;
    const int i = (int)(t / w), j = (int)(t - (long)i * w);
    double v = (j - A.n == i) ? 1.0 : 0.0;
    if (j < A.n) for_row(A, i, [&](int c, double a) { if (c == j) v += a; });
    aug[t] = v;
}

// l1 norm of each row of the coarsest matrix (the scale of the pivot test)
__global__ void gj_rownorm_kernel(Mat<double> A, double *__restrict__ rn) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    double t = 0.0;
    for_row(A, i, [&](int, double a) { t += fabs(a); });
    rn[i] = t;
}

template <typename T>
__global__ void gj_extract_kernel(int n, const double *__restrict__ aug, T *__restrict__ inv) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)n * n) return;
    const int i = (int)(t / n), j = (int)(t % n);
    inv[t] = (T)aug[(long)i * 2 * n + n + j];
}

// ---------------------------------------------------------------------------
// apply kernels (precision T)
// ---------------------------------------------------------------------------
// L2 prefetch of part `part` of `parts` of [p, p + bytes), its ends rounded
// inwards to 16 bytes (a bulk prefetch is a hint; it never leaves the range)
__device__ __forceinline__ void l2_prefetch_part(const void *p, size_t bytes, int part, int parts) {
    if (p == nullptr || bytes < 16) return;
    const size_t a = (size_t)p, e = a + bytes;
    const size_t chunk = (bytes / parts + 15) & ~(size_t)15;
    size_t lo = (a + (size_t)part * chunk + 15) & ~(size_t)15;
    size_t hi = (a + (size_t)(part + 1) * chunk) & ~(size_t)15;
    if (hi > (e & ~(size_t)15)) hi = e & ~(size_t)15;
    if (hi <= lo) return;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((unsigned)(hi - lo)) : "memory");
}

// arrays to bring into L2 ahead of their use (the coarse levels of a V-cycle):
// the first kernel of stage P issues the prefetches, the cluster launch of the
// coarse levels starts tens of microseconds later with its data in L2
constexpr int kPrefetchMax = 16;
struct L2Prefetch {
    int count;
    const void *p[kPrefetchMax];
    unsigned long long bytes[kPrefetchMax];
};
constexpr int kPrefetchParts = 8;
__device__ __forceinline__ void issue_prefetch(const L2Prefetch &pf) {
    if (blockIdx.x < kPrefetchParts && (int)threadIdx.x < pf.count)
        l2_prefetch_part(pf.p[threadIdx.x], pf.bytes[threadIdx.x], blockIdx.x, kPrefetchParts);
}

// f0 = first row of L times r (quasi-IMPES: L_00 = 1); e0 = f0 / l1
template <int B, typename T>
__device__ __forceinline__ void restrict_p_row(int N, const double *__restrict__ r, const T *__restrict__ wT, int full,
                                               const T *__restrict__ dinv0, T *__restrict__ f0, T *__restrict__ e0,
                                               int i) {
    // explicit FMAs: the same rounding in every kernel that inlines the row
    const T r0 = full ? wT[i] * (T)r[i] : (T)r[i];
    T t = fma(wT[(long)N + i], (T)r[(long)N + i], r0);
    if (B == 3) t = fma(wT[2L * N + i], (T)r[2L * N + i], t);
    f0[i] = t;
    e0[i] = t * dinv0[i];
}

template <int B, typename T>
__global__ void restrict_p_kernel(int N, const double *__restrict__ r, const T *__restrict__ wT, int full,
                                  const T *__restrict__ dinv0, T *__restrict__ f0, T *__restrict__ e0, const L2Prefetch pf,
                                  const int *done) {
    if (skip(done)) return;
    issue_prefetch(pf);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    restrict_p_row<B, T>(N, r, wT, full, dinv0, f0, e0, i);
}

// r = f - A e (one thread per fine row: coalesced stencil / ELL reads)
template <typename T>
__global__ void amg_resid_kernel(Mat<T> A, const T *__restrict__ f, const T *__restrict__ e, T *__restrict__ r,
                                 const int *done) {
    if (skip(done)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    r[i] = f[i] - row_dot(A, i, e);
}

// f_c = P^T r of coarse row I
template <typename T>
__device__ __forceinline__ void amg_restrict_row(const T *__restrict__ r, const int *__restrict__ moff,
                                                 const int *__restrict__ mem, T *__restrict__ fc, T *__restrict__ ec,
                                                 const T *__restrict__ dinvc, int I) {
    // members in batches of 8: the batch's indices, then its gathers, then the
    // sum in member order (a plain loop would wait on each load in turn)
    const int q0 = moff[I], q1 = moff[I + 1];
    T s = (T)0;
    for (int qb = q0; qb < q1; qb += 8) {
        int m[8];
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; u++) m[u] = qb + u < q1 ? mem[qb + u] : -1;
#pragma unroll
        for (int u = 0; u < 8; u++) v[u] = m[u] >= 0 ? r[m[u]] : (T)0;
#pragma unroll
        for (int u = 0; u < 8; u++)
            if (qb + u < q1) s += v[u];
    }
    fc[I] = s;
    if (ec) ec[I] = s * dinvc[I];
}

// f_c = P^T r (members in ascending order); e_c = f_c / l1 (coarse pre-smoothing)
template <typename T>
__global__ void amg_restrict_kernel(const T *__restrict__ r, const int *__restrict__ moff, const int *__restrict__ mem,
                                    int nc, T *__restrict__ fc, T *__restrict__ ec, const T *__restrict__ dinvc,
                                    const int *done) {
    if (skip(done)) return;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    amg_restrict_row<T>(r, moff, mem, fc, ec, dinvc, I);
}


// e += P e_c
template <typename T>
__global__ void amg_prolong_kernel(int n, const int *__restrict__ agg, const T *__restrict__ ec, T *__restrict__ e,
                                   const int *done) {
    if (skip(done)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) e[i] += ec[agg[i]];
}

// e2 = e + (f - A e) / l1 (post-smoothing)
template <typename T>
__global__ void amg_smooth_kernel(Mat<T> A, const T *__restrict__ f, const T *__restrict__ e, const T *__restrict__ dinv,
                                  T *__restrict__ e2, const int *done) {
    if (skip(done)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    e2[i] = e[i] + (f[i] - row_dot(A, i, e)) * dinv[i];
}

// next stage-P cycle: f0 = rp - A_p ep; e0 = f0 / l1
template <typename T>
__global__ void cycle_next_kernel(Mat<T> A, const T *__restrict__ rp, const T *__restrict__ ep, const T *__restrict__ dinv,
                                  T *__restrict__ f0, T *__restrict__ e0, const int *done) {
    if (skip(done)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const T f = rp[i] - row_dot(A, i, ep);
    f0[i] = f;
    e0[i] = f * dinv[i];
}

// y = x (mode 0) or y += x (mode 1)
template <typename T>
__global__ void copy_add_kernel(int n, const T *__restrict__ x, T *__restrict__ y, int mode, const int *done) {
    if (skip(done)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = mode ? y[i] + x[i] : x[i];
}

// e = Inv f on the coarsest level (FP64 inverse and sum): one warp per row
template <typename T>
__global__ void coarse_solve_kernel(int n, const double *__restrict__ Inv, const T *__restrict__ f, T *__restrict__ e,
                                    const int *done) {
    if (skip(done)) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s += Inv[(long)warp * n + j] * (double)f[j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) e[warp] = (T)s;
}

// ---- the coarse end of the V-cycle in one launch --------------------------
// Levels l0..nl-1 (each at most kCoarseRows rows) run inside one thread-block
// cluster: the same row operations as the per-level kernels, with a cluster
// barrier between dependent sweeps instead of a kernel boundary.  On entry
// level l0 holds f and its pre-smoothed e; on exit its corrected vector is e2.
constexpr int kCoarseCtas = 8, kCoarseThreads = 1024, kCoarseRows = 2 * kCoarseCtas * kCoarseThreads;
constexpr int kCoarseMaxLevels = 24;

template <typename T>
struct CoarseLevel {
    int n, width, diff;
    const int *colA;     // self-padded ELL columns [width][n]
    const T *val;        // [width][n]
    const T *dinv;       // 1 / l1 row sums
    const int *agg;      // row -> next-level aggregate
    const int *moff, *mem;
    T *f, *e, *e2;
};

template <typename T>
struct CoarseCycle {
    int nlev;                          // levels in lv (the last one is the coarsest)
    const double *inv;                 // coarsest: dense inverse, row-major (FP64)
    CoarseLevel<T> lv[kCoarseMaxLevels];
};

template <typename T>
__device__ __forceinline__ T ell_dot(const CoarseLevel<T> &L, int i, const T *__restrict__ e) {
    T t = (T)0;
    if (L.diff) {                                  // difference form (see row_dot)
        const T ei = e[i];
#pragma unroll 4
        for (int k = 0; k < L.width; k++) {
            const int j = L.colA[(long)k * L.n + i];
            const T v = L.val[(long)k * L.n + i];
            t += (j == i) ? v * ei : v * (e[j] - ei);
        }
        return t;
    }
#pragma unroll 4
    for (int k = 0; k < L.width; k++) t += L.val[(long)k * L.n + i] * e[L.colA[(long)k * L.n + i]];
    return t;
}

__device__ __forceinline__ void cluster_barrier() {
    __threadfence();                   // global writes of this thread before the barrier
    cg::this_cluster().sync();
}

// the cycle run by CTA `rank` of the nb CTAs of one cluster
template <typename T>
__device__ __forceinline__ void coarse_cycle_body(const CoarseCycle<T> &cc, int rank, int nb) {
    // each sweep splits a level's rows into one contiguous block per CTA, so every
    // SM of the cluster carries an equal share of a small level's L2 traffic
    // (a grid-wide thread index would leave a 1,000-row level to one or two SMs)
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    auto lo_of = [&](int n) { const int per = (n + nb - 1) / nb; return min(n, rank * per); };
    auto hi_of = [&](int n) { const int per = (n + nb - 1) / nb; return min(n, (rank + 1) * per); };
    const int last = cc.nlev - 1;
    // the matrices of the levels below the first and the dense inverse come into
    // L2 while the first level is swept: one bulk prefetch per (array, CTA)
    if (threadIdx.x < 32) {
        const int t = threadIdx.x;
        const int lv = 1 + t / 4, a = t % 4;
        if (lv <= last) {
            const CoarseLevel<T> &Q = cc.lv[lv];
            const size_t ell = (size_t)Q.width * Q.n;
            if (a == 0) l2_prefetch_part(Q.colA, sizeof(int) * ell, rank, nb);
            else if (a == 1) l2_prefetch_part(Q.val, sizeof(T) * ell, rank, nb);
            else if (a == 2) l2_prefetch_part(Q.dinv, sizeof(T) * Q.n, rank, nb);
            else if (lv < last) l2_prefetch_part(Q.mem, sizeof(int) * Q.n, rank, nb);
            else l2_prefetch_part(cc.inv, sizeof(double) * (size_t)Q.n * Q.n, rank, nb);
        }
    }
    for (int l = 0; l < last; l++) {
        const CoarseLevel<T> &L = cc.lv[l], &C = cc.lv[l + 1];
        for (int i = lo_of(L.n) + threadIdx.x; i < hi_of(L.n); i += blockDim.x) L.e2[i] = L.f[i] - ell_dot(L, i, L.e);
        cluster_barrier();
        for (int I = lo_of(C.n) + threadIdx.x; I < hi_of(C.n); I += blockDim.x) {
            T s = (T)0;
            for (int q = L.moff[I]; q < L.moff[I + 1]; q++) s += L.e2[L.mem[q]];
            C.f[I] = s;
            if (l + 1 < last) C.e[I] = s * C.dinv[I];
        }
        cluster_barrier();
    }
    {
        const CoarseLevel<T> &C = cc.lv[last];
        for (int r = lo_of(C.n) + wib; r < hi_of(C.n); r += wpb) {
            double s = 0.0;
#pragma unroll 4
            for (int j = lane; j < C.n; j += 32) s += cc.inv[(long)r * C.n + j] * (double)C.f[j];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) C.e[r] = (T)s;
        }
    }
    cluster_barrier();
    for (int l = last - 1; l >= 0; l--) {
        const CoarseLevel<T> &L = cc.lv[l], &C = cc.lv[l + 1];
        const T *ec = (l + 1 == last) ? C.e : C.e2;
        for (int i = lo_of(L.n) + threadIdx.x; i < hi_of(L.n); i += blockDim.x) L.e[i] += ec[L.agg[i]];
        cluster_barrier();
        for (int i = lo_of(L.n) + threadIdx.x; i < hi_of(L.n); i += blockDim.x)
            L.e2[i] = L.e[i] + (L.f[i] - ell_dot(L, i, L.e)) * L.dinv[i];
        if (l > 0) cluster_barrier();
    }
}

template <typename T>
__global__ void __cluster_dims__(kCoarseCtas, 1, 1) __launch_bounds__(kCoarseThreads, 1)
coarse_cycle_kernel(const __grid_constant__ CoarseCycle<T> cc, const int *done) {
    if (skip(done)) return;            // uniform over the cluster: no thread reaches a barrier alone
    // (a grid constant: the body reads the description in parameter space, no copy)
    coarse_cycle_body<T>(cc, (int)blockIdx.x, (int)gridDim.x);
}

// stage F, pass 1: r2 = rhat - Ahat[:,p] e_p; red cells z = Dinv r2, black keep r2.
// rhat = L r from the FP64 residual (lscT = null: quasi-IMPES, only the first row
// differs from the identity) or, when r is null, the given vector rh; ep may be null.
template <int B, typename T>
__device__ __forceinline__ void stage2_a_row(const GridDesc &g, const double *__restrict__ r, const T *__restrict__ wT,
                                             const T *__restrict__ lscT, const T *__restrict__ rh,
                                             const T *__restrict__ ahat, const T *__restrict__ dinv,
                                             const T *__restrict__ ep, T *__restrict__ r2, T *__restrict__ z, int rb,
                                             int i) {
    const long N = g.N;
    T v[B];
    if (!r) {
#pragma unroll
        for (int c = 0; c < B; c++) v[c] = rh[(long)c * N + i];
    } else if (lscT) {
        T u[B];
#pragma unroll
        for (int c = 0; c < B; c++) u[c] = (T)r[(long)c * N + i];
#pragma unroll
        for (int rr = 0; rr < B; rr++) {
            T t = fma(lscT[(long)(rr * B + 1) * N + i], u[1], lscT[(long)(rr * B) * N + i] * u[0]);
            if (B == 3) t = fma(lscT[(long)(rr * B + 2) * N + i], u[2], t);
            v[rr] = t;
        }
    } else {
#pragma unroll
        for (int c = 0; c < B; c++) v[c] = (T)r[(long)c * N + i];
        T rp = fma(wT[(long)N + i], v[1], v[0]);
        if (B == 3) rp = fma(wT[2L * N + i], v[2], rp);
        v[0] = rp;
    }
    const Cell cc = cell_of(g, i);
    const long NS = 2L * g.H, si = cslot(g, cc.ix, cc.iy, cc.iz);
    if (ep) {
#pragma unroll
        for (int d = 0; d < 7; d++) {
            const int j = nbrc(g, cc, d);
            if (j < 0) continue;
            const T e = ep[j];
#pragma unroll
            for (int c = 0; c < B; c++) v[c] -= ahat[(long)(d * B * B + c * B) * NS + si] * e;
        }
    }
    if (rb && is_black(g, i)) {
#pragma unroll
        for (int c = 0; c < B; c++) r2[(long)c * N + i] = v[c];
        return;
    }
#pragma unroll
    for (int c = 0; c < B; c++) {
        T s = (T)0;
#pragma unroll
        for (int q = 0; q < B; q++) s += dinv[(long)(c * B + q) * NS + si] * v[q];
        z[(long)c * N + i] = s;
    }
}

template <int B, typename T>
__global__ void stage2_a_kernel(GridDesc g, const double *__restrict__ r, const T *__restrict__ wT,
                                const T *__restrict__ lscT, const T *__restrict__ rh, const T *__restrict__ ahat,
                                const T *__restrict__ dinv, const T *__restrict__ ep, T *__restrict__ r2,
                                T *__restrict__ z, int rb, const int *done) {
    if (skip(done)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    stage2_a_row<B, T>(g, r, wT, lscT, rh, ahat, dinv, ep, r2, z, rb, i);
}

// CPR-FPF, after the first stage F (x0): rh = L r - Ahat x0 over the full 7-point
// block stencil; f0 = rh_p, e0 = f0 / l1 start stage P
template <int B, typename T>
__global__ void fpf_resid_kernel(GridDesc g, const double *__restrict__ r, const T *__restrict__ wT,
                                 const T *__restrict__ lscT, const T *__restrict__ ahat, const T *__restrict__ x0,
                                 const T *__restrict__ dinv0, T *__restrict__ rh, T *__restrict__ f0, T *__restrict__ e0,
                                 const L2Prefetch pf, const int *done) {
    if (skip(done)) return;
    issue_prefetch(pf);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const long N = g.N;
    if (i >= N) return;
    T v[B], u[B];
#pragma unroll
    for (int c = 0; c < B; c++) u[c] = (T)r[(long)c * N + i];
    if (lscT) {
#pragma unroll
        for (int rr = 0; rr < B; rr++) {
            T t = lscT[(long)(rr * B) * N + i] * u[0] + lscT[(long)(rr * B + 1) * N + i] * u[1];
            if (B == 3) t += lscT[(long)(rr * B + 2) * N + i] * u[2];
            v[rr] = t;
        }
    } else {
#pragma unroll
        for (int c = 0; c < B; c++) v[c] = u[c];
        T rp = v[0] + wT[(long)N + i] * v[1];
        if (B == 3) rp += wT[2L * N + i] * v[2];
        v[0] = rp;
    }
    const Cell cc = cell_of(g, i);
    const long NS = 2L * g.H, si = cslot(g, cc.ix, cc.iy, cc.iz);
#pragma unroll
    for (int d = 0; d < 7; d++) {
        const int j = nbrc(g, cc, d);
        if (j < 0) continue;
        T xj[B];
#pragma unroll
        for (int c = 0; c < B; c++) xj[c] = x0[(long)c * N + j];
#pragma unroll
        for (int rr = 0; rr < B; rr++)
#pragma unroll
            for (int c = 0; c < B; c++) v[rr] -= ahat[(long)(d * B * B + rr * B + c) * NS + si] * xj[c];
    }
#pragma unroll
    for (int c = 0; c < B; c++) rh[(long)c * N + i] = v[c];
    f0[i] = v[0];
    e0[i] = v[0] * dinv0[i];
}

// stage-F output of component r: x (+ e_p on the pressure row) (+ addv, the first
// stage F of CPR-FPF), added in the order the stages ran
template <typename T>
__device__ __forceinline__ T fin(T x, int r, int i, long N, const T *__restrict__ ep, const T *__restrict__ addv) {
    if (r == 0 && ep) x += ep[i];
    if (addv) x += addv[(long)r * N + i];
    return x;
}

// stage F, pass 2 (black cells): z = Dinv (r2 - sum_d Ahat_{i,d} z_red(nbr)); out = z + e_p
template <int B, typename T, typename TZ>
__device__ __forceinline__ void stage2_b_row(const GridDesc &g, const T *__restrict__ ahat, const T *__restrict__ dinv,
                                             const T *__restrict__ r2, T *__restrict__ z, const T *__restrict__ ep,
                                             const T *__restrict__ addv, TZ *__restrict__ out, int i) {
    const long N = g.N;
    const Cell cc = cell_of(g, i);
    const long NS = 2L * g.H, si = cslot(g, cc.ix, cc.iy, cc.iz);
    T t[B];
#pragma unroll
    for (int c = 0; c < B; c++) t[c] = r2[(long)c * N + i];
#pragma unroll
    for (int d = 1; d < 7; d++) {
        const int k = nbrc(g, cc, d);
        if (k < 0) continue;
        T zk[B];
#pragma unroll
        for (int c = 0; c < B; c++) zk[c] = z[(long)c * N + k];
#pragma unroll
        for (int r = 0; r < B; r++)
#pragma unroll
            for (int c = 0; c < B; c++) t[r] -= ahat[(long)(d * B * B + r * B + c) * NS + si] * zk[c];
    }
#pragma unroll
    for (int r = 0; r < B; r++) {
        T s = (T)0;
#pragma unroll
        for (int q = 0; q < B; q++) s += dinv[(long)(r * B + q) * NS + si] * t[q];
        z[(long)r * N + i] = s;
        out[(long)r * N + i] = (TZ)fin<T>(s, r, i, N, ep, addv);
    }
}

template <int B, typename T, typename TZ>
__global__ void stage2_b_kernel(GridDesc g, const T *__restrict__ ahat, const T *__restrict__ dinv,
                                const T *__restrict__ r2, T *__restrict__ z, const T *__restrict__ ep,
                                const T *__restrict__ addv, TZ *__restrict__ out, const int *done) {
    if (skip(done)) return;
    const int i = colour_cell(g, blockIdx.x * (long)blockDim.x + threadIdx.x, 1);
    if (i < 0) return;
    stage2_b_row<B, T, TZ>(g, ahat, dinv, r2, z, ep, addv, out, i);
}

// stage F, pass 3 (red cells): x = z - Dinv sum_d Ahat_{i,d} z_black(nbr); out = x + e_p
// (rb = 0: block-Jacobi, out = z + e_p for every cell)
template <int B, typename T, typename TZ>
__device__ __forceinline__ void stage2_c_row(const GridDesc &g, const T *__restrict__ ahat, const T *__restrict__ dinv,
                                             const T *__restrict__ z, const T *__restrict__ ep,
                                             const T *__restrict__ addv, TZ *__restrict__ out, int rb, int i) {
    const long N = g.N;
    if (!rb) {
#pragma unroll
        for (int r = 0; r < B; r++) {
            out[(long)r * N + i] = (TZ)fin<T>(z[(long)r * N + i], r, i, N, ep, addv);
        }
        return;
    }
    const Cell cc = cell_of(g, i);
    const long NS = 2L * g.H, si = cslot(g, cc.ix, cc.iy, cc.iz);
    T t[B];
#pragma unroll
    for (int c = 0; c < B; c++) t[c] = (T)0;
#pragma unroll
    for (int d = 1; d < 7; d++) {
        const int k = nbrc(g, cc, d);
        if (k < 0) continue;
        T zk[B];
#pragma unroll
        for (int c = 0; c < B; c++) zk[c] = z[(long)c * N + k];
#pragma unroll
        for (int r = 0; r < B; r++)
#pragma unroll
            for (int c = 0; c < B; c++) t[r] += ahat[(long)(d * B * B + r * B + c) * NS + si] * zk[c];
    }
#pragma unroll
    for (int r = 0; r < B; r++) {
        T s = (T)0;
#pragma unroll
        for (int q = 0; q < B; q++) s += dinv[(long)(r * B + q) * NS + si] * t[q];
        out[(long)r * N + i] = (TZ)fin<T>(z[(long)r * N + i] - s, r, i, N, ep, addv);
    }
}

template <int B, typename T, typename TZ>
__global__ void stage2_c_kernel(GridDesc g, const T *__restrict__ ahat, const T *__restrict__ dinv, const T *__restrict__ z,
                                const T *__restrict__ ep, const T *__restrict__ addv, TZ *__restrict__ out, int rb,
                                const int *done) {
    if (skip(done)) return;
    const int i = rb ? colour_cell(g, blockIdx.x * (long)blockDim.x + threadIdx.x, 0)   // red cells
                     : (blockIdx.x * blockDim.x + threadIdx.x < (unsigned)g.N ? (int)(blockIdx.x * blockDim.x + threadIdx.x) : -1);
    if (i < 0) return;
    stage2_c_row<B, T, TZ>(g, ahat, dinv, z, ep, addv, out, rb, i);
}

// no preconditioner / plain block-Jacobi on J (no decoupling)
template <int B, typename TZ>
__global__ void simple_prec_kernel(GridDesc g, const double *__restrict__ r, const double *__restrict__ dinv, TZ *__restrict__ z,
                                   int use_dinv, const int *done) {
    if (skip(done)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const long N = g.N;
    if (i >= N) return;
    const long NS = 2L * g.H, si = cslot_of(g, i);
    double v[B];
#pragma unroll
    for (int c = 0; c < B; c++) v[c] = r[(long)c * N + i];
#pragma unroll
    for (int rr = 0; rr < B; rr++) {
        double s = v[rr];
        if (use_dinv) {
            s = 0.0;
#pragma unroll
            for (int q = 0; q < B; q++) s += dinv[(long)(rr * B + q) * NS + si] * v[q];
        }
        z[(long)rr * N + i] = (TZ)s;
    }
}

// ---- learned stage helpers ------------------------------------------------
// RMS of a vector into *out (per-block partials folded in block order by the last block)
template <typename T>
__global__ void rms_kernel(int n, const T *__restrict__ v, double *partials, unsigned int *ticket, double *out,
                           const int *done) {
    if (skip(done)) return;
    __shared__ double sh[SIM_THREADS];
    __shared__ bool last;
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += (double)v[i] * (double)v[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < (int)gridDim.x; b++) t += __ldcg(partials + b);
        *out = sqrt(t / n);
        *ticket = 0u;
    }
}

// network input: [r / rms, three standardised log-transmissibility features]
template <typename T>
__global__ void learned_in_kernel(int n, const T *__restrict__ r, const double *__restrict__ rms,
                                  const float *__restrict__ feat, float *__restrict__ x, const int *done) {
    if (skip(done)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double sc = *rms > 0.0 ? 1.0 / *rms : 0.0;
    x[(long)i * 4] = (float)((double)r[i] * sc);
    x[(long)i * 4 + 1] = feat[(long)i * 3];
    x[(long)i * 4 + 2] = feat[(long)i * 3 + 1];
    x[(long)i * 4 + 3] = feat[(long)i * 3 + 2];
}

// q = A_p c with c = y * rms (the network's correction in pressure units)
template <typename T>
__global__ void learned_apply_kernel(Mat<T> A, const float *__restrict__ y, const double *__restrict__ rms,
                                     T *__restrict__ q, const int *done) {
    if (skip(done)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const double sc = *rms;
    T t = (T)0;
    const T yi = (T)((double)y[i] * sc);
    for_row(A, i, [&](int j, T v) {
        const T yj = (T)((double)y[j] * sc);
        t += A.diff ? ((j == i) ? v * yi : v * (yj - yi)) : v * yj;
    });
    q[i] = t;
}

// minimal-residual step alpha = (q . r) / (q . q) into out[1] (0 if q = 0)
template <typename T>
__global__ void mr_step_kernel(int n, const T *__restrict__ q, const T *__restrict__ r, double *partials,
                               unsigned int *ticket, double *out, const int *done) {
    if (skip(done)) return;
    __shared__ double s1[SIM_THREADS], s2[SIM_THREADS];
    __shared__ bool last;
    double a = 0.0, c = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        a += (double)q[i] * (double)r[i];
        c += (double)q[i] * (double)q[i];
    }
    s1[threadIdx.x] = a; s2[threadIdx.x] = c;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) { s1[threadIdx.x] += s1[threadIdx.x + o]; s2[threadIdx.x] += s2[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { partials[2 * blockIdx.x] = s1[0]; partials[2 * blockIdx.x + 1] = s2[0]; }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        double ta = 0.0, tc = 0.0;
        for (int b = 0; b < (int)gridDim.x; b++) { ta += __ldcg(partials + 2 * b); tc += __ldcg(partials + 2 * b + 1); }
        out[1] = tc > 0.0 ? ta / tc : 0.0;
        *ticket = 0u;
    }
}

// ep_out = ep + alpha * y * rms
template <typename T>
__global__ void learned_out_kernel(int n, const T *__restrict__ ep, const float *__restrict__ y,
                                   const double *__restrict__ rms, T *__restrict__ out, const int *done) {
    if (skip(done)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = ep[i] + (T)(rms[1] * (double)y[i] * rms[0]);
}

// training pair j: x_j = [f / rms(f), features], y_j = e / rms(e) (the stage's
// minimal-residual step restores the scale at inference)
template <typename T>
__global__ void pair_kernel(int n, const T *__restrict__ f, const T *__restrict__ e, const double *__restrict__ rms,
                            const float *__restrict__ feat, float *__restrict__ x, float *__restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double sc = rms[0] > 0.0 ? 1.0 / rms[0] : 0.0;
    const double se = rms[1] > 0.0 ? 1.0 / rms[1] : 0.0;
    x[(long)i * 4] = (float)((double)f[i] * sc);
    x[(long)i * 4 + 1] = feat[(long)i * 3];
    x[(long)i * 4 + 2] = feat[(long)i * 3 + 1];
    x[(long)i * 4 + 3] = feat[(long)i * 3 + 2];
    y[i] = (float)((double)e[i] * se);
}

// log of the summed face transmissibilities per direction
__global__ void logt_kernel(GridDesc g, const double *__restrict__ T, float *__restrict__ feat) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    const Cell c = cell_of(g, i);
    const long N = g.N;
    const double sx = T[i] + (c.ix > 0 ? T[i - 1] : 0.0);
    const double sy = T[N + i] + (c.iy > 0 ? T[N + i - g.nx] : 0.0);
    const double sz = T[2L * N + i] + (c.iz > 0 ? T[2L * N + i - g.nx * g.ny] : 0.0);
    feat[(long)i * 3] = (float)log(sx + 1e-30);
    feat[(long)i * 3 + 1] = (float)log(sy + 1e-30);
    feat[(long)i * 3 + 2] = (float)log(sz + 1e-30);
}

__global__ void standardize_kernel(int n, float *__restrict__ feat, float m0, float m1, float m2, float s0, float s1,
                                   float s2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    feat[(long)i * 3] = s0 > 0.f ? (feat[(long)i * 3] - m0) / s0 : 0.f;
    feat[(long)i * 3 + 1] = s1 > 0.f ? (feat[(long)i * 3 + 1] - m1) / s1 : 0.f;
    feat[(long)i * 3 + 2] = s2 > 0.f ? (feat[(long)i * 3 + 2] - m2) / s2 : 0.f;
}

}  // namespace

// ===========================================================================
// host side
// ===========================================================================
bool sim_mixed(const sim_t *s) { return s->opt.precision == SIM_PRECISION_MIXED; }

static void *dev_alloc_async(sim_t *s, size_t bytes) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(&p, bytes, s->stream);
    if (e != cudaSuccess) { sim_cuda_ok(s, e, "cudaMallocAsync (AMG hierarchy)"); return nullptr; }
    return p;
}
static void dev_free_async(sim_t *s, void *p) { if (p) cudaFreeAsync(p, s->stream); }

static void free_level(sim_t *s, AmgLevel &L) {
    // valT may alias the FP64 values or the level-0 stencil owned by the handle
    if (L.valT != (void *)L.val && L.valT != s->apT) dev_free_async(s, L.valT);
    dev_free_async(s, L.col); dev_free_async(s, L.colA); dev_free_async(s, L.val); dev_free_async(s, L.dinvT);
    dev_free_async(s, L.agg); dev_free_async(s, L.moff); dev_free_async(s, L.mem); dev_free_async(s, L.f); dev_free_async(s, L.e);
    dev_free_async(s, L.e2); dev_free_async(s, L.coarse_inv);
    L = AmgLevel();
}

void cpr_free(sim_t *s) {
    for (auto &L : s->lev) free_level(s, L);
    s->lev.clear();
}

static Mat<double> level_mat(sim_t *s, const AmgLevel &L, int l) {
    Mat<double> A;
    A.st = (l == 0); A.selfpad = false; A.diff = false; A.g = s->gd; A.n = L.n; A.width = L.width;
    A.val = l == 0 ? s->ap : L.val;
    A.col = L.col;
    return A;
}
template <typename T>
static Mat<T> level_matT(sim_t *s, const AmgLevel &L, int l) {
    Mat<T> A;
    A.st = (l == 0); A.selfpad = true; A.diff = sizeof(T) == sizeof(float); A.g = s->gd; A.n = L.n; A.width = L.width;
    A.val = (const T *)L.valT;
    A.col = L.colA;
    return A;
}

// exclusive scan of n ints: out[0..n] (out[n] = total); returns total or -1
static int scan_ints(sim_t *s, const int *in, int n, int *out) {
    const int nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    scan_sum_kernel<<<nb, SIM_THREADS, 0, s->stream>>>(n, in, s->scan);
    scan_blocks_kernel<<<1, 1024, 0, s->stream>>>(nb, s->scan, s->iscal);
    scan_write_kernel<<<nb, SIM_THREADS, 0, s->stream>>>(n, in, s->scan, s->iscal, out);
    s->launches += 3;
    if (!sim_cuda_ok(s, cudaGetLastError(), "scan")) return -1;
    if (!sim_cuda_ok(s, cudaMemcpyAsync(&s->h_pinned[0], s->iscal, sizeof(int), cudaMemcpyDeviceToHost, s->stream), "copy")) return -1;
    if (!sim_cuda_ok(s, cudaStreamSynchronize(s->stream), "sync")) return -1;
    int total = 0;
    memcpy(&total, &s->h_pinned[0], sizeof(int));
    return total;
}

// members of each of nc aggregates in ascending order: moff[nc+1], mem[n]
static bool build_members(sim_t *s, const int *agg, int n, int nc, int *moff, int *mem) {
    if (!sim_cuda_ok(s, cudaMemsetAsync(s->cnt, 0, sizeof(int) * (nc + 1), s->stream), "memset")) return false;
    count_kernel<<<sim_blocks(n), SIM_THREADS, 0, s->stream>>>(n, agg, s->cnt);
    s->launches++;
    if (scan_ints(s, s->cnt, nc, moff) < 0) return false;
    if (!sim_cuda_ok(s, cudaMemsetAsync(s->cnt, 0, sizeof(int) * (nc + 1), s->stream), "memset")) return false;
    fill_kernel<<<sim_blocks(n), SIM_THREADS, 0, s->stream>>>(n, agg, moff, s->cnt, mem);
    sort_members_kernel<<<sim_blocks(nc), SIM_THREADS, 0, s->stream>>>(nc, moff, mem);
    s->launches += 2;
    return sim_cuda_ok(s, cudaGetLastError(), "members");
}

// one aggregation pass on A (n rows): matching rounds, absorption of single
// nodes, numbering by founders; agg[n], members moff/mem; returns nc or -1
static int aggregate_pass(sim_t *s, const Mat<double> &A, int *agg, int *moff, int *mem) {
    const int n = A.n;
    if (!sim_cuda_ok(s, cudaMemsetAsync(s->partner, 0xff, sizeof(int) * n, s->stream), "memset")) return -1;
    for (int r = 0; r < s->opt.amg_rounds; r++) {
        match_pick_kernel<<<sim_blocks(n), SIM_THREADS, 0, s->stream>>>(A, s->partner, s->pick, s->opt.amg_theta);
        match_confirm_kernel<<<sim_blocks(n), SIM_THREADS, 0, s->stream>>>(n, s->pick, s->partner);
        s->launches += 2;
    }
    host_kernel<<<sim_blocks(n), SIM_THREADS, 0, s->stream>>>(A, s->partner, s->host, s->opt.amg_theta);
    founder_kernel<<<sim_blocks(n), SIM_THREADS, 0, s->stream>>>(n, s->partner, s->host, s->flag);
    s->launches += 2;
    const int nc = scan_ints(s, s->flag, n, s->pick);   // pick reused as founder ids
    if (nc < 0) return -1;
    agg_kernel<<<sim_blocks(n), SIM_THREADS, 0, s->stream>>>(n, s->partner, s->host, s->pick, agg);
    s->launches++;
    if (!build_members(s, agg, n, nc, moff, mem)) return -1;
    return nc;
}

// Galerkin product into a freshly allocated ELL matrix; returns width or -1.
static int galerkin(sim_t *s, const Mat<double> &A, const int *agg, const int *moff, const int *mem, int nc, int **col,
                    double **val) {
    int *len = (int *)dev_alloc_async(s, sizeof(int) * (nc + 1));
    if (!len) return -1;
    if (!sim_cuda_ok(s, cudaMemsetAsync(len + nc, 0, sizeof(int), s->stream), "memset")) return -1;
    if (!sim_cuda_ok(s, cudaMemsetAsync(s->iscal + 1, 0, sizeof(int), s->stream), "memset")) return -1;
    const int gw = (nc + kGalWarps - 1) / kGalWarps;
    galerkin_warp_kernel<<<gw, kGalWarps * 32, 0, s->stream>>>(A, agg, moff, mem, nc, 0, len, 0, nullptr, nullptr,
                                                              s->iscal + 1);
    galerkin_kernel<<<sim_blocks(nc), SIM_THREADS, 0, s->stream>>>(A, agg, moff, mem, nc, 0, len, 0, nullptr, nullptr,
                                                                   s->iscal + 1);
    s->launches += 2;
    int hv[2];
    if (!sim_cuda_ok(s, cudaMemcpyAsync(&s->h_pinned[0], len + nc, sizeof(int), cudaMemcpyDeviceToHost, s->stream), "copy") ||
        !sim_cuda_ok(s, cudaMemcpyAsync((char *)&s->h_pinned[0] + 4, s->iscal + 1, sizeof(int), cudaMemcpyDeviceToHost, s->stream), "copy") ||
        !sim_cuda_ok(s, cudaStreamSynchronize(s->stream), "sync"))
        return -1;
    memcpy(hv, &s->h_pinned[0], 8);
    if (hv[1]) { dev_free_async(s, len); return 0; }   // wider than SIM_MAX_ELL: caller stops coarsening
    const int W = hv[0] < 1 ? 1 : hv[0];
    *col = (int *)dev_alloc_async(s, sizeof(int) * (size_t)W * nc);
    *val = (double *)dev_alloc_async(s, sizeof(double) * (size_t)W * nc);
    if (!*col || !*val) return -1;
    galerkin_warp_kernel<<<gw, kGalWarps * 32, 0, s->stream>>>(A, agg, moff, mem, nc, 1, len, W, *col, *val,
                                                              s->iscal + 1);
    galerkin_kernel<<<sim_blocks(nc), SIM_THREADS, 0, s->stream>>>(A, agg, moff, mem, nc, 1, len, W, *col, *val,
                                                                   s->iscal + 1);
    s->launches += 2;
    dev_free_async(s, len);
    if (!sim_cuda_ok(s, cudaGetLastError(), "Galerkin")) return -1;
    return W;
}

template <typename T>
static sim_status finish_levels(sim_t *s) {
    // l1 inverse diagonals, apply-precision values, work vectors; coarsest dense inverse
    const int nl = (int)s->lev.size();
    for (int l = 0; l < nl; l++) {
        AmgLevel &L = s->lev[l];
        Mat<double> A = level_mat(s, L, l);
        L.dinvT = dev_alloc_async(s, sizeof(T) * L.n);
        L.f = dev_alloc_async(s, sizeof(T) * L.n);
        L.e = dev_alloc_async(s, sizeof(T) * L.n);
        L.e2 = dev_alloc_async(s, sizeof(T) * L.n);
        if (!L.dinvT || !L.f || !L.e || !L.e2) return s->err;
        l1_kernel<T><<<sim_blocks(L.n), SIM_THREADS, 0, s->stream>>>(A, (T *)L.dinvT);
        s->launches++;
        if (l > 0) {
            L.colA = (int *)dev_alloc_async(s, sizeof(int) * (size_t)L.width * L.n);
            if (!L.colA) return s->err;
            selfpad_kernel<<<sim_blocks((long)L.width * L.n), SIM_THREADS, 0, s->stream>>>(L.n, L.width, L.col, L.colA);
            s->launches++;
            if (sizeof(T) == sizeof(double)) {
                L.valT = L.val;              // FP64 apply reads the setup values
            } else {
                L.valT = dev_alloc_async(s, sizeof(T) * (size_t)L.width * L.n);
                if (!L.valT) return s->err;
                cast_diff_kernel<<<sim_blocks(L.n), SIM_THREADS, 0, s->stream>>>(L.n, L.width, L.col, L.val,
                                                                                (float *)L.valT);
                s->launches++;
            }
        }
    }
    // coarsest: dense Gauss-Jordan inverse in FP64
    AmgLevel &C = s->lev[nl - 1];
    const int n = C.n;
    const size_t aug = (size_t)n * 2 * n;
    double *A0 = (double *)dev_alloc_async(s, sizeof(double) * aug);
    double *A1 = (double *)dev_alloc_async(s, sizeof(double) * aug);
    double *rn = (double *)dev_alloc_async(s, sizeof(double) * n);
    if (!A0 || !A1 || !rn) return s->err;
    int *bad = s->iscal + 4;
    SIM_CK(s, cudaMemsetAsync(bad, 0, sizeof(int), s->stream));
    gj_init_kernel<<<sim_blocks(2L * n * n), SIM_THREADS, 0, s->stream>>>(level_mat(s, C, nl - 1), A0);
    s->launches++;
    gj_rownorm_kernel<<<sim_blocks(n), SIM_THREADS, 0, s->stream>>>(level_mat(s, C, nl - 1), rn);
    s->launches++;
    static bool dsmem_ok = cudaFuncSetAttribute(gj_dsmem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)gj_dsmem_bytes(kGjSmem, 8)) == cudaSuccess;
    static int gj_ctas = gj_cluster_ctas();
    const bool in_smem = dsmem_ok && n <= kGjSmem;
    if (!in_smem) {
        gj_cluster_kernel<<<8, 1024, 0, s->stream>>>(n, A0, A1, rn, bad);
        s->launches++;
    }
    // the coarsest inverse stays FP64 in both forms: the coarse matrices of
    // strongly heterogeneous fields are ill-conditioned, and the product is tiny
    C.coarse_inv = dev_alloc_async(s, sizeof(double) * (size_t)n * n);
    if (!C.coarse_inv) return s->err;
    if (in_smem) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = gj_ctas; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(gj_ctas); cfg.blockDim = dim3(1024); cfg.dynamicSmemBytes = gj_dsmem_bytes(n, gj_ctas);
        cfg.stream = s->stream; cfg.attrs = at; cfg.numAttrs = 1;
        if (!sim_cuda_ok(s, cudaLaunchKernelEx(&cfg, gj_dsmem_kernel, n, (const double *)A0, (double *)C.coarse_inv,
                                               (const double *)rn, bad),
                         "coarsest inverse"))
            return s->err;
    } else {
        gj_extract_kernel<double><<<sim_blocks((long)n * n), SIM_THREADS, 0, s->stream>>>(n, (n & 1) ? A1 : A0,
                                                                                        (double *)C.coarse_inv);
    }
    s->launches++;
    dev_free_async(s, A0); dev_free_async(s, A1); dev_free_async(s, rn);
    SIM_CK(s, cudaGetLastError());
    // the pivot test of the elimination (no pivoting: a vanishing pivot would
    // leave inf / NaN in the coarsest inverse)
    SIM_CK(s, cudaMemcpyAsync(&s->h_pinned[0], bad, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    SIM_CK(s, cudaStreamSynchronize(s->stream));
    int hb = 0;
    memcpy(&hb, &s->h_pinned[0], sizeof(int));
    if (hb) return sim_fail(s, SIM_ENAN, "coarsest AMG level: a Gauss-Jordan pivot is not above 1e-14 of its row's l1 norm");
    return SIM_OK;
}

static sim_status amg_setup(sim_t *s) {
    cpr_free(s);
    AmgLevel L0;
    L0.n = s->N; L0.width = 7;
    s->lev.push_back(L0);
    const int cmax = s->opt.amg_coarse_max;
    while (true) {
        const int l = (int)s->lev.size() - 1;
        AmgLevel &L = s->lev[l];
        if (L.n <= cmax || (int)s->lev.size() >= s->opt.amg_max_levels) break;
        const int n = L.n;
        Mat<double> A = level_mat(s, L, l);
        const int n1 = aggregate_pass(s, A, s->aggA, s->moffA, s->memA);
        if (n1 < 0) return s->err;
        int *c1 = nullptr; double *v1 = nullptr;
        const int W1 = galerkin(s, A, s->aggA, s->moffA, s->memA, n1, &c1, &v1);
        if (W1 < 0) return s->err;
        if (W1 == 0) break;   // a coarse row wider than SIM_MAX_ELL: this level is the coarsest
        Mat<double> A1; A1.st = false; A1.selfpad = false; A1.diff = false; A1.g = s->gd; A1.n = n1; A1.width = W1; A1.col = c1; A1.val = v1;
        const int n2 = aggregate_pass(s, A1, s->aggB, s->moffB, s->memB);
        if (n2 < 0) return s->err;
        if (4L * n2 > 3L * n) {   // coarsening stalled: this level is the coarsest
            dev_free_async(s, c1); dev_free_async(s, v1);
            break;
        }
        AmgLevel C;
        C.n = n2;
        const int W2 = galerkin(s, A1, s->aggB, s->moffB, s->memB, n2, &C.col, &C.val);
        if (W2 < 0) return s->err;
        if (W2 == 0) { dev_free_async(s, c1); dev_free_async(s, v1); break; }
        C.width = W2;
        AmgLevel &Lr = s->lev[l];    // (reference still valid: no push yet)
        Lr.agg = (int *)dev_alloc_async(s, sizeof(int) * n);
        Lr.moff = (int *)dev_alloc_async(s, sizeof(int) * (size_t)(n2 + 1));
        Lr.mem = (int *)dev_alloc_async(s, sizeof(int) * (size_t)n);
        if (!Lr.agg || !Lr.moff || !Lr.mem) return s->err;
        compose_kernel<<<sim_blocks(n), SIM_THREADS, 0, s->stream>>>(n, s->aggA, s->aggB, Lr.agg);
        s->launches++;
        if (!build_members(s, Lr.agg, n, n2, Lr.moff, Lr.mem)) return s->err;
        dev_free_async(s, c1); dev_free_async(s, v1);
        s->lev.push_back(C);
    }
    if (s->lev.back().n > 1024) return sim_fail(s, SIM_ELIMIT, "AMG coarsest level larger than 1024 rows");
    return sim_mixed(s) ? finish_levels<float>(s) : finish_levels<double>(s);
}

// blocks of a launch over one colour (colour_cell)
static int colour_blocks(const sim_t *s, int threads = SIM_THREADS) {
    return sim_blocks((long)((s->gd.nx + 1) / 2) * s->gd.ny * s->gd.nz, threads);
}

// stage-F sweeps of a batched application in blocks of 64 threads (the default of
// sim_autotune's stage-F shape: at 0.3-0.6 waves the finer blocks spread a
// launch's FP64 work more evenly over the SMs than blocks of 256)
constexpr int kStageThreads = 64;

template <int B, typename T>
static sim_status setup_bt(sim_t *s) {
    const int N = s->N;
    const int nb = sim_blocks(N), nbc = colour_blocks(s);
    WellCorr wc;
    if (s->nrate > 0) {
        wc.cell_perf = s->cell_perf; wc.pwell = s->perf_well;
        wc.apw = s->apw; wc.awp = s->awp; wc.aww = s->aww; wc.nperf = s->nperf;
    }
    if (s->opt.precond == SIM_PRECOND_BJACOBI) {
        diag_inv_kernel<B><<<nb, SIM_THREADS, 0, s->stream>>>(s->gd, s->J, wc, s->lsc, 2, s->dinv_d);
        SIM_LAUNCHED(s);
        return SIM_OK;
    }
    if (s->opt.precond != SIM_PRECOND_CPR) return SIM_OK;
    qi_kernel<B, T><<<nb, SIM_THREADS, 0, s->stream>>>(s->gd, s->J, wc, s->opt.decouple == SIM_DECOUPLE_ABF, s->lsc,
                                                       (T *)s->lscT, s->qiw, (T *)s->qiwT, s->ap, (T *)s->apT,
                                                       (T *)s->ahat);
    SIM_LAUNCHED(s);
    if (amg_setup(s) != SIM_OK) return s->err;
    s->lev[0].valT = s->apT;
    const int rb = s->opt.stage2 == SIM_STAGE2_ILU0_RB;
    diag_inv_kernel<B><<<rb ? nbc : nb, SIM_THREADS, 0, s->stream>>>(s->gd, s->J, wc, s->lsc, rb ? 1 : 0, s->dinv_d);
    SIM_LAUNCHED(s);
    if (rb) {
        ilu_black_kernel<B><<<nbc, SIM_THREADS, 0, s->stream>>>(s->gd, s->J, wc, s->lsc, s->dinv_d);
        SIM_LAUNCHED(s);
    }
    if (sizeof(T) != sizeof(double)) {
        cast_kernel<T><<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(s->dinv_d, (T *)s->dinv, (long)B * B * 2 * s->gd.H);
        SIM_LAUNCHED(s);
    }
    return SIM_OK;
}

sim_status cpr_setup(sim_t *s) {
    sim_status st;
    if (s->b == 2) st = sim_mixed(s) ? setup_bt<2, float>(s) : setup_bt<2, double>(s);
    else st = sim_mixed(s) ? setup_bt<3, float>(s) : setup_bt<3, double>(s);
    if (st != SIM_OK) return st;
    s->precond_ready = true;
    s->setup_gen++;
    return SIM_OK;
}

// first level handled by the one-launch coarse cycle (nl: no fusion)
static int coarse_start(const sim_t *s) {
    const int nl = (int)s->lev.size();
    if (nl < 3) return nl;
    int l0 = nl - 1;
    while (l0 - 1 >= 1 && s->lev[l0 - 1].n <= kCoarseRows && nl - (l0 - 1) <= kCoarseMaxLevels) l0--;
    return (nl - l0 >= 3) ? l0 : nl;   // worth a launch only when it replaces several
}

// the arrays the cluster launch of the coarse levels reads (none without it)
template <typename T>
static L2Prefetch coarse_prefetch(const sim_t *s) {
    L2Prefetch pf{};
    const int nl = (int)s->lev.size();
    const int lf = s->opt.fused_coarse ? coarse_start(s) : nl;
    auto add = [&](const void *p, size_t bytes) {
        if (p && bytes >= 16 && pf.count < kPrefetchMax) { pf.p[pf.count] = p; pf.bytes[pf.count] = bytes; pf.count++; }
    };
    for (int l = lf; l < nl; l++) {
        const AmgLevel &L = s->lev[l];
        const size_t ell = (size_t)L.width * L.n;
        if (l + 1 == nl) { add(L.coarse_inv, sizeof(double) * (size_t)L.n * L.n); break; }
        add(L.colA, sizeof(int) * ell);
        add(L.valT, sizeof(T) * ell);
        add(L.dinvT, sizeof(T) * L.n);
        add(L.mem, sizeof(int) * L.n);
    }
    return pf;
}

template <typename T>
static sim_status coarse_cycle(sim_t *s, int l0, const int *done) {
    const int nl = (int)s->lev.size();
    CoarseCycle<T> cc;
    cc.nlev = nl - l0;
    cc.inv = (const double *)s->lev[nl - 1].coarse_inv;
    for (int l = l0; l < nl; l++) {
        const AmgLevel &L = s->lev[l];
        CoarseLevel<T> &d = cc.lv[l - l0];
        d.n = L.n; d.width = L.width; d.diff = sizeof(T) == sizeof(float); d.colA = L.colA; d.val = (const T *)L.valT;
        d.dinv = (const T *)L.dinvT;
        d.agg = L.agg; d.moff = L.moff; d.mem = L.mem;
        d.f = (T *)L.f; d.e = (T *)L.e; d.e2 = (T *)L.e2;
    }
    coarse_cycle_kernel<T><<<kCoarseCtas, kCoarseThreads, 0, s->stream>>>(cc, done);
    SIM_LAUNCHED(s);
    return SIM_OK;
}

template <typename T>
static sim_status vcycle(sim_t *s, const int *done) {
    const int nl = (int)s->lev.size();
    const int lf = s->opt.fused_coarse ? coarse_start(s) : nl;
    // down: r = f - A e; f_{l+1} = P^T r; e_{l+1} = f_{l+1} / l1 (not on the coarsest)
    for (int l = 0; l + 1 < nl && l < lf; l++) {
        AmgLevel &L = s->lev[l], &C = s->lev[l + 1];
        const bool coarsest = (l + 1 == nl - 1);
        amg_resid_kernel<T><<<sim_blocks(L.n, s->tune_amg), s->tune_amg, 0, s->stream>>>(level_matT<T>(s, L, l), (const T *)L.f,
                                                                        (const T *)L.e, (T *)L.e2, done);
        SIM_LAUNCHED(s);
        amg_restrict_kernel<T><<<sim_blocks(C.n, s->tune_amg), s->tune_amg, 0, s->stream>>>((const T *)L.e2, L.moff, L.mem, C.n, (T *)C.f,
                                                                           coarsest ? nullptr : (T *)C.e,
                                                                           (const T *)C.dinvT, done);
        SIM_LAUNCHED(s);
    }
    if (lf < nl) {
        if (coarse_cycle<T>(s, lf, done) != SIM_OK) return s->err;
    } else {
        AmgLevel &Cn = s->lev[nl - 1];
        coarse_solve_kernel<T><<<sim_blocks((long)Cn.n * 32), SIM_THREADS, 0, s->stream>>>(Cn.n, (const double *)Cn.coarse_inv,
                                                                                        (const T *)Cn.f, (T *)Cn.e, done);
        SIM_LAUNCHED(s);
    }
    // up: e_l += P e_{l+1}; e2_l = smooth(e_l); the corrected vector of level l is e2_l
    for (int l = (lf < nl ? lf : nl - 1) - 1; l >= 0; l--) {
        AmgLevel &L = s->lev[l], &C = s->lev[l + 1];
        const T *ec = (l + 1 == nl - 1) ? (const T *)C.e : (const T *)C.e2;
        amg_prolong_kernel<T><<<sim_blocks(L.n, s->tune_amg), s->tune_amg, 0, s->stream>>>(L.n, L.agg, ec, (T *)L.e, done);
        SIM_LAUNCHED(s);
        amg_smooth_kernel<T><<<sim_blocks(L.n, s->tune_amg), s->tune_amg, 0, s->stream>>>(level_matT<T>(s, L, l), (const T *)L.f,
                                                                         (const T *)L.e, (const T *)L.dinvT, (T *)L.e2,
                                                                         done);
        SIM_LAUNCHED(s);
    }
    return SIM_OK;
}

template <int B, typename T, typename TZ>
static sim_status apply_btz(sim_t *s, const double *r, TZ *z, const int *done) {
    const int N = s->N;
    const int nb = sim_blocks(N);
    if (s->opt.precond != SIM_PRECOND_CPR) {
        simple_prec_kernel<B, TZ><<<nb, SIM_THREADS, 0, s->stream>>>(s->gd, r, s->dinv_d, z,
                                                                   s->opt.precond == SIM_PRECOND_BJACOBI, done);
        SIM_LAUNCHED(s);
        return SIM_OK;
    }
    AmgLevel &L0 = s->lev[0];
    const int rb = s->opt.stage2 == SIM_STAGE2_ILU0_RB;
    const T *dinv = sizeof(T) == sizeof(double) ? (const T *)s->dinv_d : (const T *)s->dinv;
    const int full = s->opt.decouple == SIM_DECOUPLE_ABF;
    const T *lscT = full ? (const T *)s->lscT : nullptr;
    const bool fpf = s->opt.cpr_stages == 3;
    if (fpf) {
        // CPR-FPF: stage F on L r first (x0), then stage P on the residual it leaves
        stage2_a_kernel<B, T><<<sim_blocks(N, s->tune_stage), s->tune_stage, 0, s->stream>>>(s->gd, r, (const T *)s->qiwT, lscT, nullptr,
                                                                (const T *)s->ahat, dinv, nullptr, (T *)s->r2,
                                                                (T *)s->zr, rb, done);
        SIM_LAUNCHED(s);
        if (rb) {
            stage2_b_kernel<B, T, T><<<colour_blocks(s, s->tune_stage), s->tune_stage, 0, s->stream>>>(s->gd, (const T *)s->ahat, dinv, (const T *)s->r2,
                                                                       (T *)s->zr, nullptr, nullptr, (T *)s->x0, done);
            SIM_LAUNCHED(s);
        }
        stage2_c_kernel<B, T, T><<<rb ? colour_blocks(s, s->tune_stage) : sim_blocks(N, s->tune_stage), s->tune_stage, 0, s->stream>>>(s->gd, (const T *)s->ahat, dinv, (const T *)s->zr,
                                                                   nullptr, nullptr, (T *)s->x0, rb, done);
        SIM_LAUNCHED(s);
        fpf_resid_kernel<B, T><<<nb, SIM_THREADS, 0, s->stream>>>(s->gd, r, (const T *)s->qiwT, lscT, (const T *)s->ahat,
                                                                 (const T *)s->x0, (const T *)L0.dinvT, (T *)s->rhT,
                                                                 (T *)L0.f, (T *)L0.e, coarse_prefetch<T>(s), done);
        SIM_LAUNCHED(s);
    } else {
        restrict_p_kernel<B, T><<<nb, SIM_THREADS, 0, s->stream>>>(N, r, (const T *)s->qiwT, full, (const T *)L0.dinvT,
                                                                  (T *)L0.f, (T *)L0.e, coarse_prefetch<T>(s), done);
        SIM_LAUNCHED(s);
    }
    const T *ep;
    if (s->lev.size() == 1) {
        coarse_solve_kernel<T><<<sim_blocks((long)L0.n * 32), SIM_THREADS, 0, s->stream>>>(L0.n, (const double *)L0.coarse_inv,
                                                                                        (const T *)L0.f, (T *)L0.e2, done);
        SIM_LAUNCHED(s);
    } else if (vcycle<T>(s, done) != SIM_OK) {
        return s->err;
    }
    ep = (const T *)L0.e2;
    if (s->opt.amg_cycles > 1 && s->lev.size() > 1) {
        // further cycles on the pressure residual left by the previous ones
        copy_add_kernel<T><<<sim_blocks(N), SIM_THREADS, 0, s->stream>>>(N, (const T *)L0.f, (T *)s->rpT, 0, done);
        copy_add_kernel<T><<<sim_blocks(N), SIM_THREADS, 0, s->stream>>>(N, (const T *)L0.e2, (T *)s->epacc, 0, done);
        SIM_LAUNCHED(s);
        for (int c = 1; c < s->opt.amg_cycles; c++) {
            cycle_next_kernel<T><<<sim_blocks(N, 128), 128, 0, s->stream>>>(level_matT<T>(s, L0, 0), (const T *)s->rpT,
                                                                           (const T *)s->epacc, (const T *)L0.dinvT,
                                                                           (T *)L0.f, (T *)L0.e, done);
            SIM_LAUNCHED(s);
            if (vcycle<T>(s, done) != SIM_OK) return s->err;
            copy_add_kernel<T><<<sim_blocks(N), SIM_THREADS, 0, s->stream>>>(N, (const T *)L0.e2, (T *)s->epacc, 1, done);
            SIM_LAUNCHED(s);
        }
        ep = (const T *)s->epacc;
    }
    if (s->learned_active && s->net) {
        // extra stage: the network's correction of the pressure residual left by stage P
        const T *rp = (s->opt.amg_cycles > 1 && s->lev.size() > 1) ? (const T *)s->rpT : (const T *)L0.f;
        amg_resid_kernel<T><<<sim_blocks(N, 128), 128, 0, s->stream>>>(level_matT<T>(s, L0, 0), rp, ep, (T *)s->lres, done);
        SIM_LAUNCHED(s);
        rms_kernel<T><<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(N, (const T *)s->lres, s->red, s->ticket, s->lrms, done);
        SIM_LAUNCHED(s);
        learned_in_kernel<T><<<sim_blocks(N), SIM_THREADS, 0, s->stream>>>(N, (const T *)s->lres, s->lrms, s->lfeat, s->lx, done);
        SIM_LAUNCHED(s);
        const int64_t l0 = net_launches(s->net);
        if (net_infer(s->net, s->lx, s->ly, s->stream, done) != SIM_OK) return sim_fail(s, SIM_ECUDA, "learned stage inference");
        s->launches += net_launches(s->net) - l0;
        // minimal-residual scaling of the correction: never increases ||r'||_2
        learned_apply_kernel<T><<<sim_blocks(N, 128), 128, 0, s->stream>>>(level_matT<T>(s, L0, 0), s->ly, s->lrms,
                                                                          (T *)s->lep, done);
        SIM_LAUNCHED(s);
        mr_step_kernel<T><<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(N, (const T *)s->lep, (const T *)s->lres, s->red,
                                                                        s->ticket, s->lrms, done);
        SIM_LAUNCHED(s);
        learned_out_kernel<T><<<sim_blocks(N), SIM_THREADS, 0, s->stream>>>(N, ep, s->ly, s->lrms, (T *)s->lep, done);
        SIM_LAUNCHED(s);
        ep = (const T *)s->lep;
    }
    const T *addv = fpf ? (const T *)s->x0 : nullptr;
    stage2_a_kernel<B, T><<<sim_blocks(N, s->tune_stage), s->tune_stage, 0, s->stream>>>(s->gd, fpf ? nullptr : r, (const T *)s->qiwT, lscT,
                                                            (const T *)s->rhT, (const T *)s->ahat, dinv, ep, (T *)s->r2,
                                                            (T *)s->zr, rb, done);
    SIM_LAUNCHED(s);
    if (rb) {
        stage2_b_kernel<B, T, TZ><<<colour_blocks(s, s->tune_stage), s->tune_stage, 0, s->stream>>>(s->gd, (const T *)s->ahat, dinv, (const T *)s->r2,
                                                                    (T *)s->zr, ep, addv, z, done);
        SIM_LAUNCHED(s);
    }
    stage2_c_kernel<B, T, TZ><<<rb ? colour_blocks(s, s->tune_stage) : sim_blocks(N, s->tune_stage), s->tune_stage, 0, s->stream>>>(s->gd, (const T *)s->ahat, dinv, (const T *)s->zr, ep, addv,
                                                                z, rb, done);
    SIM_LAUNCHED(s);
    return SIM_OK;
}

sim_status cpr_apply(sim_t *s, const double *r, void *z, const int *done) {
    if (!s->precond_ready) { if (cpr_setup(s) != SIM_OK) return s->err; }
    if (s->b == 2)
        return sim_mixed(s) ? apply_btz<2, float, float>(s, r, (float *)z, done) : apply_btz<2, double, double>(s, r, (double *)z, done);
    return sim_mixed(s) ? apply_btz<3, float, float>(s, r, (float *)z, done) : apply_btz<3, double, double>(s, r, (double *)z, done);
}

// ===========================================================================
// CPR application batched over the members of an ensemble
//
// One launch per stage covers every member: the restriction, each V-cycle
// level's residual / restriction / prolongation / smoothing (a member takes
// part in the launches of the levels it has), the coarse end (one 8-CTA
// cluster per member for its fused coarse levels, or the dense product of its
// coarsest level) and the three stage-F sweeps.  Block b of a launch takes
// work[b] = (member, block of the member's rows), reads the member's operands
// from a device table and runs the single-system row arithmetic, so every
// member's result equals that of its own application.  A member whose restart
// cycle is done (its FGMRES control word) returns at once.
// ===========================================================================
namespace {
constexpr int kBatchLevels = 16;
constexpr int kBatchAmgThreads = 128;

template <typename T>
struct BLevel {
    Mat<T> A;                   // the level's matrix (apply precision)
    const T *dinv;              // 1 / l1 row sums
    const int *agg, *moff, *mem;
    T *f, *e, *e2;
    int n;
};

template <typename T>
struct CMember {
    GridDesc g;
    long n;                     // b N
    const double *V;            // input of application j: V + j n (FP64)
    T *Z;                       // output: Z + j n
    const T *wT, *lscT, *ahat, *dinv;
    T *r2, *zr;
    int full, rb, nl, lf;
    const double *inv;          // dense inverse of the coarsest level
    const CoarseCycle<T> *cc;   // the fused coarse levels (device copy) or null
    const int *done;
    BLevel<T> lv[kBatchLevels];
};

template <typename T>
__device__ __forceinline__ const CMember<T> &cmember(const CMember<T> *M, const int2 *work, int *vb) {
    const int2 wk = work[blockIdx.x];
    *vb = wk.y;
    return M[wk.x];
}

template <int B, typename T>
__global__ void b_restrict_p_kernel(const CMember<T> *M, const int2 *work, int j) {
    int vb;
    const CMember<T> &m = cmember(M, work, &vb);
    if (skip(m.done)) return;
    const int i = vb * blockDim.x + threadIdx.x;
    if (i >= m.g.N) return;
    const BLevel<T> &L0 = m.lv[0];
    restrict_p_row<B, T>(m.g.N, m.V + (size_t)j * m.n, m.wT, m.full, L0.dinv, L0.f, L0.e, i);
}

// down the V-cycle at level l: e2 = f - A e (mode 0, rows of l) or the
// restriction of e2 to level l + 1 (mode 1, rows of l + 1)
template <typename T>
__global__ void b_amg_down_kernel(const CMember<T> *M, const int2 *work, int l, int mode) {
    int vb;
    const CMember<T> &m = cmember(M, work, &vb);
    if (skip(m.done)) return;
    const int i = vb * blockDim.x + threadIdx.x;
    const BLevel<T> &L = m.lv[l];
    if (mode == 0) {
        if (i < L.n) L.e2[i] = L.f[i] - row_dot(L.A, i, L.e);
    } else {
        const BLevel<T> &C = m.lv[l + 1];
        if (i < C.n) amg_restrict_row<T>(L.e2, L.moff, L.mem, C.f, l + 1 == m.nl - 1 ? nullptr : C.e, C.dinv, i);
    }
}

// up the V-cycle at level l: e += P e_c (mode 0), then e2 = e + (f - A e) / l1 (mode 1)
template <typename T>
__global__ void b_amg_up_kernel(const CMember<T> *M, const int2 *work, int l, int mode) {
    int vb;
    const CMember<T> &m = cmember(M, work, &vb);
    if (skip(m.done)) return;
    const int i = vb * blockDim.x + threadIdx.x;
    const BLevel<T> &L = m.lv[l];
    if (i >= L.n) return;
    if (mode == 0) {
        const BLevel<T> &C = m.lv[l + 1];
        const T *ec = (l + 1 == m.nl - 1) ? C.e : C.e2;
        L.e[i] += ec[L.agg[i]];
    } else {
        L.e2[i] = L.e[i] + (L.f[i] - row_dot(L.A, i, L.e)) * L.dinv[i];
    }
}

// coarsest level without the fused cycle: e = Inv f, one warp per row (a
// one-level hierarchy writes e2 of level 0, the stage-P correction)
template <typename T>
__global__ void b_coarse_solve_kernel(const CMember<T> *M, const int2 *work) {
    int vb;
    const CMember<T> &m = cmember(M, work, &vb);
    if (skip(m.done)) return;
    const BLevel<T> &C = m.lv[m.nl - 1];
    const int warp = (vb * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= C.n) return;
    double s = 0.0;
    for (int q = lane; q < C.n; q += 32) s += m.inv[(long)warp * C.n + q] * (double)C.f[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) (m.nl == 1 ? C.e2 : C.e)[warp] = (T)s;
}

// the fused coarse levels: cluster c runs member members[c]
template <typename T>
__global__ void __cluster_dims__(kCoarseCtas, 1, 1) __launch_bounds__(kCoarseThreads, 1)
b_coarse_cycle_kernel(const CMember<T> *M, const int *members) {
    const CMember<T> &m = M[members[blockIdx.x / kCoarseCtas]];
    if (skip(m.done)) return;          // uniform over the cluster (one member)
    coarse_cycle_body<T>(*m.cc, (int)(blockIdx.x % kCoarseCtas), kCoarseCtas);
}

// stage F on the residual of stage P: sweep 0 (all cells), 1 (black), 2 (red,
// or all cells for block Jacobi)
template <int B, typename T>
__global__ void b_stage2_kernel(const CMember<T> *M, const int2 *work, int j, int sweep) {
    int vb;
    const CMember<T> &m = cmember(M, work, &vb);
    if (skip(m.done)) return;
    const long t = vb * (long)blockDim.x + threadIdx.x;
    const T *ep = m.lv[0].e2;
    T *out = m.Z + (size_t)j * m.n;
    if (sweep == 0) {
        if (t >= m.g.N) return;
        stage2_a_row<B, T>(m.g, m.V + (size_t)j * m.n, m.wT, m.lscT, nullptr, m.ahat, m.dinv, ep, m.r2, m.zr, m.rb, (int)t);
    } else if (sweep == 1) {
        const int i = colour_cell(m.g, t, 1);
        if (i >= 0) stage2_b_row<B, T, T>(m.g, m.ahat, m.dinv, m.r2, m.zr, ep, nullptr, out, i);
    } else {
        const int i = m.rb ? colour_cell(m.g, t, 0) : (t < m.g.N ? (int)t : -1);
        if (i >= 0) stage2_c_row<B, T, T>(m.g, m.ahat, m.dinv, m.zr, ep, nullptr, out, m.rb, i);
    }
}
}  // namespace

struct CprBatch {
    int nm = 0, b = 0, mixed = 0, rb = 0;
    void *dmem = nullptr;  size_t mem_cap = 0;    // CMember<T>[nm]
    void *dcc = nullptr;   size_t cc_cap = 0;     // CoarseCycle<T>[ncl]
    int2 *dwork = nullptr; size_t work_cap = 0;
    int *dcl = nullptr;    size_t cl_cap = 0;     // members with fused coarse levels
    int ncl = 0;
    struct List { long off = 0; int count = 0; };
    List cell256, cell64, stage1, stage2, cs;
    std::vector<List> down_r, down_c, up;
};

static cudaError_t grow(void **p, size_t *cap, size_t bytes) {
    if (bytes <= *cap) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr; *cap = 0;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) *cap = bytes;
    return e;
}

// the members' current hierarchies are batchable: the same options, block
// size and precision, two-stage CPR with one V-cycle, no learned stage, no
// rate-controlled wells, at most kBatchLevels levels
bool cpr_batchable(sim_t *const *ms, int nm) {
    if (nm < 1) return false;
    const sim_options &o = ms[0]->opt;
    for (int k = 0; k < nm; k++) {
        const sim_t *s = ms[k];
        const sim_options &p = s->opt;
        if (s->b != ms[0]->b || sim_mixed(s) != sim_mixed(ms[0]) || p.precond != SIM_PRECOND_CPR ||
            p.stage2 != o.stage2 || p.decouple != o.decouple || p.cpr_stages != 2 || p.amg_cycles != 1 ||
            p.krylov != SIM_KRYLOV_FGMRES || p.gmres_m != o.gmres_m || p.orth != o.orth || s->learned_on || s->nrate)
            return false;
    }
    return true;
}

template <typename T>
static cudaError_t batch_build_t(CprBatch *cb, sim_t *const *ms, int nm, cudaStream_t st) {
    std::vector<CMember<T>> hm(nm);
    std::vector<CoarseCycle<T>> hcc;
    std::vector<int> hcl;
    std::vector<int2> work;
    cb->down_r.clear(); cb->down_c.clear(); cb->up.clear();
    auto add_list = [&](CprBatch::List &L, auto blocks_of) {
        L.off = (long)work.size();
        for (int k = 0; k < nm; k++) {
            const int nb = blocks_of(k);
            for (int q = 0; q < nb; q++) work.push_back(make_int2(k, q));
        }
        L.count = (int)((long)work.size() - L.off);
    };
    int maxdown = 0, maxup = 0;
    for (int k = 0; k < nm; k++) {
        sim_t *s = ms[k];
        CMember<T> &m = hm[k];
        memset(&m, 0, sizeof(m));
        const int nl = (int)s->lev.size();
        if (nl < 1 || nl > kBatchLevels || !s->precond_ready) return cudaErrorInvalidValue;
        m.g = s->gd; m.n = (long)s->N * s->b;
        m.V = s->V; m.Z = (T *)s->Z;
        m.wT = (const T *)s->qiwT;
        m.full = s->opt.decouple == SIM_DECOUPLE_ABF;
        m.lscT = m.full ? (const T *)s->lscT : nullptr;
        m.ahat = (const T *)s->ahat;
        m.dinv = sizeof(T) == sizeof(double) ? (const T *)s->dinv_d : (const T *)s->dinv;
        m.r2 = (T *)s->r2; m.zr = (T *)s->zr;
        m.rb = s->opt.stage2 == SIM_STAGE2_ILU0_RB;
        m.nl = nl;
        m.lf = (s->opt.fused_coarse && nl > 1) ? coarse_start(s) : nl;
        m.inv = (const double *)s->lev[nl - 1].coarse_inv;
        m.done = &s->ctl->done;
        for (int l = 0; l < nl; l++) {
            AmgLevel &L = s->lev[l];
            BLevel<T> &d = m.lv[l];
            d.A = level_matT<T>(s, L, l);
            d.dinv = (const T *)L.dinvT; d.agg = L.agg; d.moff = L.moff; d.mem = L.mem;
            d.f = (T *)L.f; d.e = (T *)L.e; d.e2 = (T *)L.e2; d.n = L.n;
        }
        if (m.lf < nl) {
            CoarseCycle<T> cc;
            cc.nlev = nl - m.lf;
            cc.inv = m.inv;
            for (int l = m.lf; l < nl; l++) {
                const AmgLevel &L = s->lev[l];
                CoarseLevel<T> &d = cc.lv[l - m.lf];
                d.n = L.n; d.width = L.width; d.diff = sizeof(T) == sizeof(float); d.colA = L.colA;
                d.val = (const T *)L.valT; d.dinv = (const T *)L.dinvT;
                d.agg = L.agg; d.moff = L.moff; d.mem = L.mem;
                d.f = (T *)L.f; d.e = (T *)L.e; d.e2 = (T *)L.e2;
            }
            hcc.push_back(cc);
            hcl.push_back(k);
        }
        const int down = nl > 1 ? std::min(nl - 1, m.lf) : 0;
        const int top = nl > 1 ? (m.lf < nl ? m.lf : nl - 1) : 0;
        maxdown = std::max(maxdown, down);
        maxup = std::max(maxup, top);
    }
    auto down_of = [&](int k) { const CMember<T> &m = hm[k]; return m.nl > 1 ? std::min(m.nl - 1, m.lf) : 0; };
    auto top_of = [&](int k) { const CMember<T> &m = hm[k]; return m.nl > 1 ? (m.lf < m.nl ? m.lf : m.nl - 1) : 0; };
    add_list(cb->cell256, [&](int k) { return sim_blocks(hm[k].g.N, SIM_THREADS); });
    add_list(cb->cell64, [&](int k) { return sim_blocks(hm[k].g.N, kStageThreads); });
    add_list(cb->stage1, [&](int k) { return hm[k].rb ? colour_blocks(ms[k], kStageThreads) : 0; });
    add_list(cb->stage2, [&](int k) { return hm[k].rb ? colour_blocks(ms[k], kStageThreads) : sim_blocks(hm[k].g.N, kStageThreads); });
    add_list(cb->cs, [&](int k) { const CMember<T> &m = hm[k];
                                  return (m.nl == 1 || m.lf == m.nl) ? sim_blocks((long)m.lv[m.nl - 1].n * 32, SIM_THREADS) : 0; });
    cb->down_r.resize(maxdown); cb->down_c.resize(maxdown); cb->up.resize(maxup);
    for (int l = 0; l < maxdown; l++) {
        add_list(cb->down_r[l], [&](int k) { return l < down_of(k) ? sim_blocks(hm[k].lv[l].n, kBatchAmgThreads) : 0; });
        add_list(cb->down_c[l], [&](int k) { return l < down_of(k) ? sim_blocks(hm[k].lv[l + 1].n, kBatchAmgThreads) : 0; });
    }
    for (int l = 0; l < maxup; l++)
        add_list(cb->up[l], [&](int k) { return l < top_of(k) ? sim_blocks(hm[k].lv[l].n, kBatchAmgThreads) : 0; });
    cudaError_t e;
    if ((e = grow(&cb->dmem, &cb->mem_cap, sizeof(CMember<T>) * nm)) != cudaSuccess) return e;
    if ((e = grow((void **)&cb->dwork, &cb->work_cap, sizeof(int2) * std::max<size_t>(1, work.size()))) != cudaSuccess) return e;
    if (!hcc.empty()) {
        if ((e = grow(&cb->dcc, &cb->cc_cap, sizeof(CoarseCycle<T>) * hcc.size())) != cudaSuccess) return e;
        if ((e = grow((void **)&cb->dcl, &cb->cl_cap, sizeof(int) * hcl.size())) != cudaSuccess) return e;
        for (size_t c = 0; c < hcc.size(); c++) hm[hcl[c]].cc = (const CoarseCycle<T> *)cb->dcc + c;
        if ((e = cudaMemcpyAsync(cb->dcc, hcc.data(), sizeof(CoarseCycle<T>) * hcc.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(cb->dcl, hcl.data(), sizeof(int) * hcl.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    }
    cb->ncl = (int)hcl.size();
    if ((e = cudaMemcpyAsync(cb->dmem, hm.data(), sizeof(CMember<T>) * nm, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if (!work.empty() && (e = cudaMemcpyAsync(cb->dwork, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    // the host tables must outlive the asynchronous copies
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    cb->nm = nm; cb->b = ms[0]->b; cb->mixed = sim_mixed(ms[0]); cb->rb = hm[0].rb;
    return cudaSuccess;
}

CprBatch *cpr_batch_new() { return new CprBatch(); }

void cpr_batch_free(CprBatch *cb) {
    if (!cb) return;
    if (cb->dmem) cudaFree(cb->dmem);
    if (cb->dcc) cudaFree(cb->dcc);
    if (cb->dwork) cudaFree(cb->dwork);
    if (cb->dcl) cudaFree(cb->dcl);
    delete cb;
}

cudaError_t cpr_batch_build(CprBatch *cb, sim_t *const *ms, int nm, cudaStream_t st) {
    return sim_mixed(ms[0]) ? batch_build_t<float>(cb, ms, nm, st) : batch_build_t<double>(cb, ms, nm, st);
}

template <int B, typename T>
static int batch_apply_t(const CprBatch *cb, cudaStream_t st, int j) {
    const CMember<T> *M = (const CMember<T> *)cb->dmem;
    const int2 *W = cb->dwork;
    int launches = 0;
    auto go = [&](const CprBatch::List &L, int threads, auto launch) {
        if (L.count > 0) { launch(L.count, threads, W + L.off); launches++; }
    };
    go(cb->cell256, SIM_THREADS, [&](int n, int t, const int2 *w) { b_restrict_p_kernel<B, T><<<n, t, 0, st>>>(M, w, j); });
    for (size_t l = 0; l < cb->down_r.size(); l++) {
        go(cb->down_r[l], kBatchAmgThreads, [&](int n, int t, const int2 *w) { b_amg_down_kernel<T><<<n, t, 0, st>>>(M, w, (int)l, 0); });
        go(cb->down_c[l], kBatchAmgThreads, [&](int n, int t, const int2 *w) { b_amg_down_kernel<T><<<n, t, 0, st>>>(M, w, (int)l, 1); });
    }
    if (cb->ncl > 0) {
        b_coarse_cycle_kernel<T><<<cb->ncl * kCoarseCtas, kCoarseThreads, 0, st>>>(M, cb->dcl);
        launches++;
    }
    go(cb->cs, SIM_THREADS, [&](int n, int t, const int2 *w) { b_coarse_solve_kernel<T><<<n, t, 0, st>>>(M, w); });
    for (int l = (int)cb->up.size() - 1; l >= 0; l--) {
        go(cb->up[l], kBatchAmgThreads, [&](int n, int t, const int2 *w) { b_amg_up_kernel<T><<<n, t, 0, st>>>(M, w, l, 0); });
        go(cb->up[l], kBatchAmgThreads, [&](int n, int t, const int2 *w) { b_amg_up_kernel<T><<<n, t, 0, st>>>(M, w, l, 1); });
    }
    go(cb->cell64, kStageThreads, [&](int n, int t, const int2 *w) { b_stage2_kernel<B, T><<<n, t, 0, st>>>(M, w, j, 0); });
    go(cb->stage1, kStageThreads, [&](int n, int t, const int2 *w) { b_stage2_kernel<B, T><<<n, t, 0, st>>>(M, w, j, 1); });
    go(cb->stage2, kStageThreads, [&](int n, int t, const int2 *w) { b_stage2_kernel<B, T><<<n, t, 0, st>>>(M, w, j, 2); });
    return launches;
}

// one batched CPR application (input V_j, output Z_j of every member);
// returns the number of kernels launched, or -1 on a launch error
int cpr_batch_apply(const CprBatch *cb, cudaStream_t st, int j) {
    int n;
    if (cb->b == 2) n = cb->mixed ? batch_apply_t<2, float>(cb, st, j) : batch_apply_t<2, double>(cb, st, j);
    else n = cb->mixed ? batch_apply_t<3, float>(cb, st, j) : batch_apply_t<3, double>(cb, st, j);
    return cudaGetLastError() == cudaSuccess ? n : -1;
}

sim_status cpr_copy_level_ell(sim_t *s, int level, int *col, double *val) {
    if (level < 1 || level >= (int)s->lev.size()) return sim_fail(s, SIM_EINVAL, "level out of range");
    const AmgLevel &L = s->lev[level];
    SIM_CK(s, cudaMemcpyAsync(col, L.col, sizeof(int) * (size_t)L.width * L.n, cudaMemcpyDeviceToHost, s->stream));
    SIM_CK(s, cudaMemcpyAsync(val, L.val, sizeof(double) * (size_t)L.width * L.n, cudaMemcpyDeviceToHost, s->stream));
    SIM_CK(s, cudaStreamSynchronize(s->stream));
    return SIM_OK;
}

// Training pairs for the learned stage.  For Krylov vector v_j: f = (L v_j)_p,
// one stage-P V-cycle e_p, the residual it leaves r' = f - A_p e_p (the input
// of the learned stage in apply_btz), and as target the error that residual
// corresponds to, A_p^-1 r', approximated by kRefine V-cycles of iterative
// refinement.  Input r' / rms(r') with the log-transmissibility features;
// target normalised by its own RMS (the stage is scaled by minimal residual).
constexpr int kRefine = 8;

template <typename T>
static sim_status learned_pairs_t(sim_t *s, int k, float *x, float *y) {
    const int N = s->N;
    AmgLevel &L0 = s->lev[0];
    const int full = s->opt.decouple == SIM_DECOUPLE_ABF;
    const Mat<T> A0 = level_matT<T>(s, L0, 0);
    auto cycle = [&](void) -> sim_status {
        if (s->lev.size() == 1) {
            coarse_solve_kernel<T><<<sim_blocks((long)L0.n * 32), SIM_THREADS, 0, s->stream>>>(
                L0.n, (const double *)L0.coarse_inv, (const T *)L0.f, (T *)L0.e2, nullptr);
            SIM_LAUNCHED(s);
            return SIM_OK;
        }
        return vcycle<T>(s, nullptr);
    };
    for (int j = 0; j < k; j++) {
        const double *v = s->V + (size_t)j * N * s->b;
        if (s->b == 2) restrict_p_kernel<2, T><<<sim_blocks(N), SIM_THREADS, 0, s->stream>>>(N, v, (const T *)s->qiwT, full, (const T *)L0.dinvT, (T *)L0.f, (T *)L0.e, L2Prefetch{}, nullptr);
        else restrict_p_kernel<3, T><<<sim_blocks(N), SIM_THREADS, 0, s->stream>>>(N, v, (const T *)s->qiwT, full, (const T *)L0.dinvT, (T *)L0.f, (T *)L0.e, L2Prefetch{}, nullptr);
        SIM_LAUNCHED(s);
        if (cycle() != SIM_OK) return s->err;
        // r' = f - A_p e_p into rpT; the first refinement cycle starts from it
        amg_resid_kernel<T><<<sim_blocks(N, 128), 128, 0, s->stream>>>(A0, (const T *)L0.f, (const T *)L0.e2, (T *)s->rpT,
                                                                     nullptr);
        SIM_LAUNCHED(s);
        copy_add_kernel<T><<<sim_blocks(N), SIM_THREADS, 0, s->stream>>>(N, (const T *)s->rpT, (T *)s->lres, 0, nullptr);
        SIM_LAUNCHED(s);
        SIM_CK(s, cudaMemsetAsync(s->epacc, 0, sizeof(T) * (size_t)N, s->stream));
        for (int c = 0; c < kRefine; c++) {
            cycle_next_kernel<T><<<sim_blocks(N, 128), 128, 0, s->stream>>>(A0, (const T *)s->rpT, (const T *)s->epacc,
                                                                           (const T *)L0.dinvT, (T *)L0.f, (T *)L0.e, nullptr);
            SIM_LAUNCHED(s);
            if (cycle() != SIM_OK) return s->err;
            copy_add_kernel<T><<<sim_blocks(N), SIM_THREADS, 0, s->stream>>>(N, (const T *)L0.e2, (T *)s->epacc, 1, nullptr);
            SIM_LAUNCHED(s);
        }
        rms_kernel<T><<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(N, (const T *)s->lres, s->red, s->ticket, s->lrms, nullptr);
        SIM_LAUNCHED(s);
        rms_kernel<T><<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(N, (const T *)s->epacc, s->red, s->ticket, s->lrms + 1,
                                                                    nullptr);
        SIM_LAUNCHED(s);
        pair_kernel<T><<<sim_blocks(N), SIM_THREADS, 0, s->stream>>>(N, (const T *)s->lres, (const T *)s->epacc, s->lrms,
                                                                    s->lfeat, x + (size_t)j * N * 4, y + (size_t)j * N);
        SIM_LAUNCHED(s);
    }
    return SIM_OK;
}

sim_status cpr_learned_pairs(sim_t *s, int k, float *x, float *y) {
    if (s->opt.precond != SIM_PRECOND_CPR || !s->precond_ready || s->lev.empty())
        return sim_fail(s, SIM_EINVAL, "training pairs need a CPR preconditioner set up by a solve");
    return sim_mixed(s) ? learned_pairs_t<float>(s, k, x, y) : learned_pairs_t<double>(s, k, x, y);
}

sim_status cpr_learned_features(sim_t *s) {
    const int N = s->N;
    logt_kernel<<<sim_blocks(N), SIM_THREADS, 0, s->stream>>>(s->gd, s->T, s->lfeat);
    SIM_LAUNCHED(s);
    std::vector<float> h((size_t)N * 3);
    SIM_CK(s, cudaMemcpyAsync(h.data(), s->lfeat, sizeof(float) * 3 * (size_t)N, cudaMemcpyDeviceToHost, s->stream));
    SIM_CK(s, cudaStreamSynchronize(s->stream));
    double m[3] = {0, 0, 0}, q[3] = {0, 0, 0};
    for (int i = 0; i < N; i++)
        for (int c = 0; c < 3; c++) { const double v = h[(size_t)i * 3 + c]; m[c] += v; q[c] += v * v; }
    float mf[3], sf[3];
    for (int c = 0; c < 3; c++) {
        const double mu = m[c] / N, var = q[c] / N - mu * mu;
        mf[c] = (float)mu; sf[c] = (float)(var > 1e-12 ? std::sqrt(var) : 0.0);
    }
    standardize_kernel<<<sim_blocks(N), SIM_THREADS, 0, s->stream>>>(N, s->lfeat, mf[0], mf[1], mf[2], sf[0], sf[1], sf[2]);
    SIM_LAUNCHED(s);
    return SIM_OK;
}
