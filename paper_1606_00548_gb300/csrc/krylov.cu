// Block-stencil SpMV and right-preconditioned FGMRES(m) (FP64 outer loop).
//
// FGMRES with classical Gram-Schmidt plus one full re-orthogonalisation
// (CGS2), Givens rotations and restarts; it solves the Newton correction of
// Algorithm 1 to ||b - J dx|| <= theta ||b||.  One inner iteration is a fixed
// sequence of kernels with no host synchronisation: every kernel first reads
// the device flag ctl->done and returns at once when the Arnoldi residual
// estimate has already met the tolerance, so a whole restart cycle is
// enqueued up front and the host reads the control block once per cycle.
//
// Reductions are deterministic: a fixed grid, per-block partials reduced in
// block order by the last block to finish (ticket counter).
#include "sim_internal.cuh"

namespace {

__device__ __forceinline__ bool skip(const int *done) { return done != nullptr && *(volatile const int *)done; }

template <typename X> __device__ __forceinline__ double ld(const X *p, long i) { return (double)p[i]; }

// y = J x on the 7-point block stencil; blocks of absent neighbours are skipped
template <int B, typename X>
__device__ __forceinline__ void spmv_row(const GridDesc &g, const double *__restrict__ J, const X *__restrict__ x,
                                         double *__restrict__ y, int i) {
    const long N = g.N;
    const int ix = i % g.nx, t = i / g.nx, iy = t % g.ny, iz = t / g.ny;
    const int nxy = g.nx * g.ny;
    double acc[B];
#pragma unroll
    for (int r = 0; r < B; r++) acc[r] = 0.0;
#pragma unroll
    for (int d = 0; d < 7; d++) {
        int j;
        if (d == 0) j = i;
        else if (d == 1) j = ix > 0 ? i - 1 : -1;
        else if (d == 2) j = ix < g.nx - 1 ? i + 1 : -1;
        else if (d == 3) j = iy > 0 ? i - g.nx : -1;
        else if (d == 4) j = iy < g.ny - 1 ? i + g.nx : -1;
        else if (d == 5) j = iz > 0 ? i - nxy : -1;
        else j = iz < g.nz - 1 ? i + nxy : -1;
        if (j < 0) continue;
        double xv[B];
#pragma unroll
        for (int c = 0; c < B; c++) xv[c] = ld(x, (long)c * N + j);
        // accumulate straight into acc: b^2 FMAs per block and no separate adds
        // (the SpMV is bound by the FP64 pipe, not by HBM, on this part)
#pragma unroll
        for (int r = 0; r < B; r++)
#pragma unroll
            for (int c = 0; c < B; c++) acc[r] = fma(J[(long)((d * B + r) * B + c) * N + i], xv[c], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < B; r++) y[(long)r * N + i] = acc[r];
}

template <int B, typename X>
__global__ void __launch_bounds__(512) spmv_kernel(GridDesc g, const double *__restrict__ J,
                                                           const X *__restrict__ x, double *__restrict__ y,
                                                           const int *done) {
    if (skip(done)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    spmv_row<B, X>(g, J, x, y, i);
}

// ---- block reduction of nv partial sums into partials[k][gridDim] ----------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// A block's place in the grid its reduction spans: the launch's own grid
// (one system), or the member's share of a batched launch (one system per
// member of an ensemble; partials and tickets are the member's own).
struct VBlk { int id, count; };
__device__ __forceinline__ VBlk grid_blk() { return VBlk{(int)blockIdx.x, (int)gridDim.x}; }

template <int NV>
__device__ void block_partials(const double (&acc)[NV], int nv, double *partials, VBlk vb = grid_blk()) {
    __shared__ double sh[SIM_THREADS / 32][NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        if (k < nv) {
            double v = warp_sum(acc[k]);
            if (lane == 0) sh[wid][k] = v;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[w][k];
        partials[k * vb.count + vb.id] = s;
    }
}

// returns true in the last block to arrive (all partials visible)
__device__ bool last_block(unsigned int *ticket, int count = (int)gridDim.x) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = atomicAdd(ticket, 1u);
        last = (t == (unsigned int)count - 1);
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// one warp per value: lanes stride over the block partials, then a fixed
// shuffle tree (the summation order does not depend on timing).  A lane loads
// 8 of its partials before adding them in stride order, so the loads overlap
// instead of each waiting for the previous add.
__device__ void fold(const double *partials, int nv, double *out, int G = (int)gridDim.x) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = wid; k < nv; k += nw) {
        const double *p = partials + (long)k * G;
        double s = 0.0;
        for (int b0 = lane; b0 < G; b0 += 32 * 8) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; u++) v[u] = b0 + 32 * u < G ? __ldcg(p + b0 + 32 * u) : 0.0;
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (b0 + 32 * u < G) s += v[u];
        }
        s = warp_sum(s);
        if (lane == 0) out[k] = s;
    }
}

constexpr int NVMAX = SIM_MAX_M + 1;

// h[k] = V_k . w, k < NV (NV exact: no predicated work for absent vectors),
// and h[NV] = w . w (the norm the selective reorthogonalisation test needs).
// Above 20 vectors two blocks per SM (128 registers a thread) keep more of an
// element's NV loads in flight than three blocks at 80 registers.
template <int NV>
__device__ __forceinline__ void dots_body(const double *__restrict__ V, const double *__restrict__ w, long n,
                                          double *partials, unsigned int *ticket, double *out, VBlk vb) {
    double acc[NV + 1];
#pragma unroll
    for (int k = 0; k <= NV; k++) acc[k] = 0.0;
    for (long i = vb.id * (long)blockDim.x + threadIdx.x; i < n; i += (long)vb.count * blockDim.x) {
        const double wi = w[i];
#pragma unroll
        for (int k = 0; k < NV; k++) acc[k] += V[k * n + i] * wi;
        acc[NV] += wi * wi;
    }
    block_partials<NV + 1>(acc, NV + 1, partials, vb);
    if (last_block(ticket, vb.count)) {
        fold(partials, NV + 1, out, vb.count);
        if (threadIdx.x == 0) *ticket = 0u;
    }
}

template <int NV>
__global__ void __launch_bounds__(SIM_THREADS, NV > 20 ? 2 : 3) dots_kernel(const double *__restrict__ V, const double *__restrict__ w,
                                                           long n, double *partials, unsigned int *ticket,
                                                           double *out, const int *done) {
    if (skip(done)) return;
    dots_body<NV>(V, w, n, partials, ticket, out, grid_blk());
}

// second Gram-Schmidt pass needed?  Always for CGS2; for the selective form
// (Daniel, Gragg, Kaufman, Stewart 1976) when the first pass removed more than
// half of ||w||^2: ||w - V h||^2 = ||w||^2 - sum h^2 < ||w||^2 / 2.  Every
// thread evaluates it the same way from the same h.
__device__ __forceinline__ bool need_reorth(const double *h, int nv, int selective) {
    if (!selective) return true;
    double s = 0.0;
    for (int k = 0; k < nv; k++) s += h[k] * h[k];
    return s > 0.5 * h[nv];
}

// w -= sum_k h[k] V_k ; out[k] = V_k . w (second Gram-Schmidt pass); nothing
// when the selective test finds no second pass is needed.  A block takes
// tiles of 128 elements: each thread updates one element, keeping the tile's
// basis entries in shared memory, then thread (k, sub) accumulates
// V_k . w over the tile's elements sub, sub + 4, ... (few registers, so
// several blocks share an SM; rows padded to 132 doubles: conflict-free).
constexpr int kOrthTile = 128, kOrthPad = 132;

template <int NV>
__device__ __forceinline__ void orth_dots_body(const double *__restrict__ V, double *__restrict__ w, long n,
                                               const double *h, double *partials, unsigned int *ticket, double *out,
                                               int selective, VBlk vb) {
    if (!need_reorth(h, NV, selective)) return;
    __shared__ double sv[NV][kOrthPad];
    __shared__ double sw[kOrthTile];
    __shared__ double hs[NV];
    for (int k = threadIdx.x; k < NV; k += blockDim.x) hs[k] = h[k];
    __syncthreads();
    const int kk = threadIdx.x >> 2, sub = threadIdx.x & 3;   // dot slot of this thread
    double acc = 0.0;
    for (long base = (long)vb.id * kOrthTile; base < n; base += (long)vb.count * kOrthTile) {
        const long i = base + threadIdx.x;
        if (i < n) {
            double wi = w[i];
#pragma unroll
            for (int k = 0; k < NV; k++) {
                const double v = V[k * n + i];
                sv[k][threadIdx.x] = v;
                wi -= hs[k] * v;
            }
            w[i] = wi;
            sw[threadIdx.x] = wi;
        } else {
#pragma unroll
            for (int k = 0; k < NV; k++) sv[k][threadIdx.x] = 0.0;
            sw[threadIdx.x] = 0.0;
        }
        __syncthreads();
        if (kk < NV) {
#pragma unroll 8
            for (int e = sub; e < kOrthTile; e += 4) acc += sv[kk][e] * sw[e];
        }
        __syncthreads();
    }
    // the 4 threads of a slot are adjacent lanes: fold them, then one per slot writes
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (sub == 0 && kk < NV) partials[kk * vb.count + vb.id] = acc;
    if (last_block(ticket, vb.count)) {
        fold(partials, NV, out, vb.count);
        if (threadIdx.x == 0) *ticket = 0u;
    }
}

template <int NV>
__global__ void __launch_bounds__(kOrthTile) orth_dots_kernel(const double *__restrict__ V, double *__restrict__ w,
                                                             long n, const double *h, double *partials,
                                                             unsigned int *ticket, double *out, const int *done,
                                                             int selective) {
    if (skip(done)) return;
    orth_dots_body<NV>(V, w, n, h, partials, ticket, out, selective, grid_blk());
}

// w -= sum_k h2[k] V_k ; ||w||; last block: Hessenberg column j, Givens, test
// (NV = j + 1 at compile time: the NV basis loads of an element are unrolled
// and in flight together)
template <int NV>
__device__ __forceinline__ void orth_norm_body(const double *__restrict__ V, double *__restrict__ w, long n, int j,
                                               int m, double *partials, unsigned int *ticket, KrylovCtl *ctl,
                                               int selective, VBlk vb) {
    const int nv = NV;
    const bool re = need_reorth(ctl->h, nv, selective);   // else the first pass is subtracted here
    __shared__ double hs[NVMAX];
    for (int k = threadIdx.x; k < nv; k += blockDim.x) hs[k] = re ? ctl->h2[k] : ctl->h[k];
    __syncthreads();
    double acc[1] = {0.0};
    for (long i = vb.id * (long)blockDim.x + threadIdx.x; i < n; i += (long)vb.count * blockDim.x) {
        double wi = w[i];
#pragma unroll
        for (int k = 0; k < NV; k++) wi -= hs[k] * V[k * n + i];
        w[i] = wi;
        acc[0] += wi * wi;
    }
    block_partials<1>(acc, 1, partials, vb);
    if (last_block(ticket, vb.count)) {
        __shared__ double nrm;
        // the column and the earlier rotations, staged by the whole block so
        // that thread 0's rotation chain reads shared memory only
        __shared__ double col[NVMAX + 1], rcs[NVMAX + 1], rsn[NVMAX + 1];
        for (int k = threadIdx.x; k <= j; k += blockDim.x) {
            col[k] = re ? ctl->h[k] + ctl->h2[k] : ctl->h[k];
            rcs[k] = ctl->cs[k];
            rsn[k] = ctl->sn[k];
        }
        fold(partials, 1, &nrm, vb.count);
        __syncthreads();
        if (threadIdx.x == 0) {
            *ticket = 0u;
            const double hn = sqrt(nrm);
            // two-product sums written as explicit FMAs: every kernel that
            // inlines this body (one system or a batch) rounds them alike
            for (int k = 0; k < j; k++) {
                const double a = col[k], c2 = col[k + 1];
                col[k] = fma(rcs[k], a, rsn[k] * c2);
                col[k + 1] = fma(-rsn[k], a, rcs[k] * c2);
            }
            const double a = col[j], bb = hn;
            const double rr = sqrt(fma(a, a, bb * bb));
            double c, s;
            if (rr == 0.0) { c = 1.0; s = 0.0; }
            else { c = a / rr; s = bb / rr; }
            ctl->cs[j] = c; ctl->sn[j] = s;
            col[j] = rr;
            ctl->g[j + 1] = -s * ctl->g[j];
            ctl->g[j] = c * ctl->g[j];
            for (int k = 0; k <= j; k++) ctl->H[k * (SIM_MAX_M + 1) + j] = col[k];
            ctl->rnorm2 = hn;             // normaliser of v_{j+1}
            ctl->k = j + 1;
            if (fabs(ctl->g[j + 1]) <= ctl->tol || j + 1 >= m) ctl->done = 1;
        }
    }
}

template <int NV>
__global__ void __launch_bounds__(SIM_THREADS, NV > 20 ? 2 : 3) orth_norm_kernel(const double *__restrict__ V, double *__restrict__ w,
                                                                long n, int j, int m, double *partials,
                                                                unsigned int *ticket, KrylovCtl *ctl, int selective) {
    if (ctl->done) return;
    orth_norm_body<NV>(V, w, n, j, m, partials, ticket, ctl, selective, grid_blk());
}

// v = w / scale (scale = ctl->rnorm2 inside a cycle, ctl->beta at a restart)
__device__ __forceinline__ void scale_body(const double *__restrict__ w, double *__restrict__ v, long n,
                                           const KrylovCtl *ctl, int use_beta, VBlk vb) {
    const double sc = use_beta ? ctl->beta : ctl->rnorm2;
    const double inv = sc > 0.0 ? 1.0 / sc : 0.0;
    for (long i = vb.id * (long)blockDim.x + threadIdx.x; i < n; i += (long)vb.count * blockDim.x)
        v[i] = sc > 0.0 ? w[i] * inv : 0.0;
}

__global__ void scale_kernel(const double *__restrict__ w, double *__restrict__ v, long n, const KrylovCtl *ctl,
                             int use_beta) {
    if (!use_beta && ctl->done) return;
    scale_body(w, v, n, ctl, use_beta, grid_blk());
}

// y = H^{-1} g (k x k upper triangular), single thread
// (H and g staged in shared memory by the block, so the one thread that runs
// the dependent back substitution never waits on global memory)
__device__ __forceinline__ void backsolve_body(KrylovCtl *ctl) {
    constexpr int LD = SIM_MAX_M + 1;
    __shared__ double Hs[LD * LD], gs[LD], ys[LD];
    const int k = ctl->k;
    for (int t = threadIdx.x; t < k * LD; t += blockDim.x) Hs[t] = ctl->H[t];
    for (int t = threadIdx.x; t < k; t += blockDim.x) gs[t] = ctl->g[t];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = k - 1; i >= 0; i--) {
            double t = gs[i];
            for (int c = i + 1; c < k; c++) t -= Hs[i * LD + c] * ys[c];
            ys[i] = t / Hs[i * LD + i];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < k; t += blockDim.x) ctl->y[t] = ys[t];
}

__global__ void backsolve_kernel(KrylovCtl *ctl) { backsolve_body(ctl); }

// x += sum_k y_k Z_k
template <typename Z>
__device__ __forceinline__ void xupdate_body(double *__restrict__ x, const Z *__restrict__ Zb, long n,
                                             const KrylovCtl *ctl, VBlk vb) {
    __shared__ double ys[NVMAX];
    const int k = ctl->k;
    for (int t = threadIdx.x; t < k; t += blockDim.x) ys[t] = ctl->y[t];
    __syncthreads();
    for (long i = vb.id * (long)blockDim.x + threadIdx.x; i < n; i += (long)vb.count * blockDim.x) {
        double s = x[i];
        for (int t = 0; t < k; t++) s += ys[t] * (double)Zb[t * n + i];
        x[i] = s;
    }
}

template <typename Z>
__global__ void xupdate_kernel(double *__restrict__ x, const Z *__restrict__ Zb, long n, const KrylovCtl *ctl) {
    xupdate_body<Z>(x, Zb, n, ctl, grid_blk());
}

// r = b - y ; ||r|| into *out
__device__ __forceinline__ bool resid_body(const double *__restrict__ b, const double *__restrict__ y,
                                           double *__restrict__ r, long n, double *partials, unsigned int *ticket,
                                           double *out, VBlk vb) {
    double acc[1] = {0.0};
    for (long i = vb.id * (long)blockDim.x + threadIdx.x; i < n; i += (long)vb.count * blockDim.x) {
        const double v = b[i] - y[i];
        r[i] = v;
        acc[0] += v * v;
    }
    block_partials<1>(acc, 1, partials, vb);
    if (last_block(ticket, vb.count)) {
        __shared__ double nrm;
        fold(partials, 1, &nrm, vb.count);
        __syncthreads();
        if (threadIdx.x == 0) { *ticket = 0u; *out = sqrt(nrm); }
        return true;
    }
    return false;
}

__global__ void __launch_bounds__(SIM_THREADS) resid_kernel(const double *__restrict__ b, const double *__restrict__ y,
                                                            double *__restrict__ r, long n, double *partials,
                                                            unsigned int *ticket, double *out) {
    resid_body(b, y, r, n, partials, ticket, out, grid_blk());
}

__global__ void norm_kernel(const double *__restrict__ v, long n, double *partials, unsigned int *ticket, double *out) {
    double acc[1] = {0.0};
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) acc[0] += v[i] * v[i];
    block_partials<1>(acc, 1, partials);
    if (last_block(ticket)) {
        __shared__ double nrm;
        fold(partials, 1, &nrm);
        __syncthreads();
        if (threadIdx.x == 0) { *ticket = 0u; out[0] = sqrt(nrm); }
    }
}

// start of a restart cycle: clear flags and the Givens state, g = beta e1
// (ctl->tol is set once per solve)
__device__ __forceinline__ void cycle_init_body(KrylovCtl *ctl, int done) {
    const int t = threadIdx.x;
    if (t == 0) { ctl->done = done; ctl->k = 0; ctl->g[0] = ctl->beta; }
    for (int k = t + 1; k <= SIM_MAX_M; k += blockDim.x) ctl->g[k] = 0.0;
}

__global__ void cycle_init_kernel(KrylovCtl *ctl) { cycle_init_body(ctl, 0); }

// ---- the same operations batched over the members of an ensemble ----------
// One launch covers every member: block b of the launch takes the work item
// work[b] = (member, virtual block), finds the member's operands in the table
// M and runs the single-system body on its share (the member's reductions
// keep their own partials, ticket and virtual grid of SIM_RED_BLOCKS blocks,
// so each member's sums are the ones of a launch of its own).  A member whose
// solve has converged (ctl->active = 0) or whose cycle is done returns at once.
__device__ __forceinline__ const KMember &member_of(const KMember *M, const int2 *work, VBlk *vb, int count) {
    const int2 wk = work[blockIdx.x];
    vb->id = wk.y;
    vb->count = count;
    return M[wk.x];
}

__device__ __forceinline__ bool cycle_off(const KMember &m) { return *(volatile const int *)&m.ctl->done; }

// start of a solve: r = b, x = 0, beta = ||b||, tol = theta ||b||, active
// when beta is positive and finite
__global__ void __launch_bounds__(SIM_THREADS) b_start_kernel(const KMember *M, const int2 *work) {
    VBlk vb;
    const KMember &m = member_of(M, work, &vb, SIM_RED_BLOCKS);
    if (!m.rhs) return;                                  // not solving in this round
    double acc[1] = {0.0};
    for (long i = vb.id * (long)blockDim.x + threadIdx.x; i < m.n; i += (long)vb.count * blockDim.x) {
        const double v = m.rhs[i];
        m.r[i] = v;
        m.x[i] = 0.0;
        acc[0] += v * v;
    }
    block_partials<1>(acc, 1, m.red, vb);
    if (last_block(m.ticket, vb.count)) {
        __shared__ double nrm;
        fold(m.red, 1, &nrm, vb.count);
        __syncthreads();
        if (threadIdx.x == 0) {
            *m.ticket = 0u;
            const double bn = sqrt(nrm);
            m.ctl->beta = bn;
            m.ctl->tol = m.theta * bn;
            m.ctl->active = (bn > 0.0 && bn == bn) ? 1 : 0;
            m.ctl->k = 0;
            m.ctl->iters = 0;
        }
    }
}

__global__ void b_cycle_init_kernel(const KMember *M, const int2 *work) {
    VBlk vb;
    const KMember &m = member_of(M, work, &vb, 1);
    cycle_init_body(m.ctl, m.rhs && m.ctl->active ? 0 : 1);
}

// v_j = w / scale: j = 0 from the residual (use_beta), else from w
__global__ void b_scale_kernel(const KMember *M, const int2 *work, int j, int use_beta) {
    VBlk vb;
    const KMember &m = member_of(M, work, &vb, SIM_RED_BLOCKS);
    if (cycle_off(m)) return;
    scale_body(use_beta ? m.r : m.w, m.V + (size_t)j * m.n, m.n, m.ctl, use_beta, vb);
}

// w = J z_j (src 0, z_j in the direction precision) or w = J x (src 1)
template <int B, typename X>
__global__ void __launch_bounds__(512) b_spmv_kernel(const KMember *M, const int2 *work, int j, int src) {
    VBlk vb;
    const KMember &m = member_of(M, work, &vb, 0);
    if (src == 0 ? cycle_off(m) : !(m.rhs && m.ctl->active)) return;
    const int i = vb.id * blockDim.x + threadIdx.x;
    if (i >= m.g.N) return;
    const X *x = src == 0 ? (const X *)m.Z + (size_t)j * m.n : (const X *)m.x;
    spmv_row<B, X>(m.g, m.J, x, m.w, i);
}

template <int NV>
__global__ void __launch_bounds__(SIM_THREADS, NV > 20 ? 2 : 3) b_dots_kernel(const KMember *M, const int2 *work) {
    VBlk vb;
    const KMember &m = member_of(M, work, &vb, SIM_RED_BLOCKS);
    if (cycle_off(m)) return;
    dots_body<NV>(m.V, m.w, m.n, m.red, m.ticket, m.ctl->h, vb);
}

template <int NV>
__global__ void __launch_bounds__(kOrthTile) b_orth_dots_kernel(const KMember *M, const int2 *work, int selective) {
    VBlk vb;
    const KMember &m = member_of(M, work, &vb, 2 * SIM_RED_BLOCKS);
    if (cycle_off(m)) return;
    orth_dots_body<NV>(m.V, m.w, m.n, m.ctl->h, m.red, m.ticket, m.ctl->h2, selective, vb);
}

template <int NV>
__global__ void __launch_bounds__(SIM_THREADS, NV > 20 ? 2 : 3) b_orth_norm_kernel(const KMember *M, const int2 *work,
                                                                                  int mrestart, int selective) {
    VBlk vb;
    const KMember &m = member_of(M, work, &vb, SIM_RED_BLOCKS);
    if (cycle_off(m)) return;
    orth_norm_body<NV>(m.V, m.w, m.n, NV - 1, mrestart, m.red, m.ticket, m.ctl, selective, vb);
}

// after a cycle (members still solving): y = H^-1 g; x += Z y; w = J x; r = b - w
__global__ void b_backsolve_kernel(const KMember *M, const int2 *work) {
    VBlk vb;
    const KMember &m = member_of(M, work, &vb, 1);
    if (!(m.rhs && m.ctl->active)) return;
    backsolve_body(m.ctl);
}

template <typename Z>
__global__ void b_xupdate_kernel(const KMember *M, const int2 *work) {
    VBlk vb;
    const KMember &m = member_of(M, work, &vb, SIM_RED_BLOCKS);
    if (!(m.rhs && m.ctl->active)) return;
    xupdate_body<Z>(m.x, (const Z *)m.Z, m.n, m.ctl, vb);
}

// r = b - w, beta = ||r||; the member stays active while beta > tol (finite)
__global__ void __launch_bounds__(SIM_THREADS) b_resid_kernel(const KMember *M, const int2 *work) {
    VBlk vb;
    const KMember &m = member_of(M, work, &vb, SIM_RED_BLOCKS);
    if (!(m.rhs && m.ctl->active)) return;
    if (resid_body(m.rhs, m.w, m.r, m.n, m.red, m.ticket, &m.ctl->beta, vb) && threadIdx.x == 0) {
        const double beta = m.ctl->beta;
        m.ctl->iters += m.ctl->k;
        m.ctl->active = (beta > m.ctl->tol && beta == beta) ? 1 : 0;
    }
}

// launch the NV-specialised kernels for a runtime vector count nv <= SIM_MAX_M
template <int NV>
struct OrthDispatch {
    static void dots(int nv, cudaStream_t st, const double *V, const double *w, long n, double *part, unsigned int *tk,
                     double *out, const int *done) {
        if (nv == NV) dots_kernel<NV><<<SIM_RED_BLOCKS, SIM_THREADS, 0, st>>>(V, w, n, part, tk, out, done);
        else OrthDispatch<NV - 1>::dots(nv, st, V, w, n, part, tk, out, done);
    }
    static void norm(int nv, cudaStream_t st, const double *V, double *w, long n, int m, double *part, unsigned int *tk,
                     KrylovCtl *ctl, int sel) {
        if (nv == NV) orth_norm_kernel<NV><<<SIM_RED_BLOCKS, SIM_THREADS, 0, st>>>(V, w, n, NV - 1, m, part, tk, ctl, sel);
        else OrthDispatch<NV - 1>::norm(nv, st, V, w, n, m, part, tk, ctl, sel);
    }
    static void orth(int nv, cudaStream_t st, const double *V, double *w, long n, const double *h, double *part,
                     unsigned int *tk, double *out, const int *done, int sel) {
        // 6 blocks of 128 threads per SM keep loads in flight while tiles are reduced
        if (nv == NV) orth_dots_kernel<NV><<<2 * SIM_RED_BLOCKS, kOrthTile, 0, st>>>(V, w, n, h, part, tk, out, done, sel);
        else OrthDispatch<NV - 1>::orth(nv, st, V, w, n, h, part, tk, out, done, sel);
    }
    // batched: one launch per pass over every member (work lists of SIM_RED_BLOCKS
    // and 2 SIM_RED_BLOCKS virtual blocks per member)
    static void bdots(int nv, cudaStream_t st, const KMember *M, const int2 *wred, int nred) {
        if (nv == NV) b_dots_kernel<NV><<<nred, SIM_THREADS, 0, st>>>(M, wred);
        else OrthDispatch<NV - 1>::bdots(nv, st, M, wred, nred);
    }
    static void borth(int nv, cudaStream_t st, const KMember *M, const int2 *worth, int north, int sel) {
        if (nv == NV) b_orth_dots_kernel<NV><<<north, kOrthTile, 0, st>>>(M, worth, sel);
        else OrthDispatch<NV - 1>::borth(nv, st, M, worth, north, sel);
    }
    static void bnorm(int nv, cudaStream_t st, const KMember *M, const int2 *wred, int nred, int m, int sel) {
        if (nv == NV) b_orth_norm_kernel<NV><<<nred, SIM_THREADS, 0, st>>>(M, wred, m, sel);
        else OrthDispatch<NV - 1>::bnorm(nv, st, M, wred, nred, m, sel);
    }
};
template <>
struct OrthDispatch<0> {
    static void dots(int, cudaStream_t, const double *, const double *, long, double *, unsigned int *, double *,
                     const int *) {}
    static void orth(int, cudaStream_t, const double *, double *, long, const double *, double *, unsigned int *,
                     double *, const int *, int) {}
    static void norm(int, cudaStream_t, const double *, double *, long, int, double *, unsigned int *, KrylovCtl *,
                     int) {}
    static void bdots(int, cudaStream_t, const KMember *, const int2 *, int) {}
    static void borth(int, cudaStream_t, const KMember *, const int2 *, int, int) {}
    static void bnorm(int, cudaStream_t, const KMember *, const int2 *, int, int, int) {}
};

// ---- BiCGSTAB (right-preconditioned, van der Vorst) ---------------------
// One iteration is a fixed kernel sequence reading its scalars from the
// device control block; the last block of each reduction updates them, so a
// chunk of iterations is enqueued (or replayed as a graph) with no host
// synchronisation.  Once ctl->done is set every later kernel returns at once.
__device__ __forceinline__ bool bdone(const BicgCtl *c) { return *(volatile const int *)&c->done; }

// start or restart from the current residual: rh = r, rho = (r, r)
__global__ void __launch_bounds__(SIM_THREADS) bicg_restart_kernel(const double *__restrict__ r, double *__restrict__ rh,
                                                                   long n, double *partials, unsigned int *ticket,
                                                                   BicgCtl *ctl) {
    double acc[1] = {0.0};
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double v = r[i];
        rh[i] = v;
        acc[0] += v * v;
    }
    block_partials<1>(acc, 1, partials);
    if (last_block(ticket)) {
        __shared__ double d;
        fold(partials, 1, &d);
        __syncthreads();
        if (threadIdx.x == 0) {
            *ticket = 0u;
            ctl->rho = d;
            ctl->fresh = 1;
            ctl->flag = 0;
            ctl->half_j = -1;
            ctl->done = (d == 0.0 || !(d == d)) ? 1 : 0;
            if (ctl->done) ctl->flag = 2;
        }
    }
}

__global__ void bicg_init_kernel(BicgCtl *ctl, double tol, int max_it) {
    ctl->tol = tol; ctl->max_it = max_it; ctl->it = 0;
    ctl->rho_old = 1.0; ctl->alpha = 1.0; ctl->omega = 1.0;
}

__global__ void bicg_chunk_init_kernel(BicgCtl *ctl) { ctl->half_j = -1; }

// p = r (first iteration of a start) or r + beta (p - omega v)
__global__ void bicg_p_kernel(const double *__restrict__ r, const double *__restrict__ v, double *__restrict__ p, long n,
                              const BicgCtl *ctl) {
    if (bdone(ctl)) return;
    const bool fresh = ctl->fresh;
    const double om = ctl->omega;
    const double beta = (ctl->rho / ctl->rho_old) * (ctl->alpha / om);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        p[i] = fresh ? r[i] : r[i] + beta * (p[i] - om * v[i]);
}

// alpha = rho / (rh, v); one iteration counted
__global__ void __launch_bounds__(SIM_THREADS) bicg_alpha_kernel(const double *__restrict__ rh, const double *__restrict__ v,
                                                                 long n, double *partials, unsigned int *ticket,
                                                                 BicgCtl *ctl) {
    if (bdone(ctl)) return;
    double acc[1] = {0.0};
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) acc[0] += rh[i] * v[i];
    block_partials<1>(acc, 1, partials);
    if (last_block(ticket)) {
        __shared__ double d;
        fold(partials, 1, &d);
        __syncthreads();
        if (threadIdx.x == 0) {
            *ticket = 0u;
            ctl->it++;
            if (d == 0.0 || !(d == d)) { ctl->flag = 2; ctl->done = 1; }
            else ctl->alpha = ctl->rho / d;
        }
    }
}

// s = r - alpha v; ||s|| <= tol ends the iteration at its half step (iteration j of the chunk)
__global__ void __launch_bounds__(SIM_THREADS) bicg_s_kernel(const double *__restrict__ r, const double *__restrict__ v,
                                                             double *__restrict__ sv, long n, double *partials,
                                                             unsigned int *ticket, BicgCtl *ctl, int j) {
    if (bdone(ctl)) return;
    const double al = ctl->alpha;
    double acc[1] = {0.0};
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double t = r[i] - al * v[i];
        sv[i] = t;
        acc[0] += t * t;
    }
    block_partials<1>(acc, 1, partials);
    if (last_block(ticket)) {
        __shared__ double d;
        fold(partials, 1, &d);
        __syncthreads();
        if (threadIdx.x == 0) {
            *ticket = 0u;
            if (sqrt(d) <= ctl->tol) { ctl->half_j = j; ctl->flag = 1; ctl->done = 1; }
        }
    }
}

// x += alpha p^ when iteration j stopped at its half step (runs after done is set)
template <typename Z>
__global__ void bicg_xhalf_kernel(double *__restrict__ x, const Z *__restrict__ ph, long n, const BicgCtl *ctl, int j) {
    if (ctl->half_j != j) return;
    const double al = ctl->alpha;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        x[i] += al * (double)ph[i];
}

// omega = (t, s) / (t, t)
__global__ void __launch_bounds__(SIM_THREADS) bicg_omega_kernel(const double *__restrict__ t, const double *__restrict__ sv,
                                                                 long n, double *partials, unsigned int *ticket,
                                                                 BicgCtl *ctl) {
    if (bdone(ctl)) return;
    double acc[2] = {0.0, 0.0};
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double ti = t[i];
        acc[0] += ti * ti;
        acc[1] += ti * sv[i];
    }
    block_partials<2>(acc, 2, partials);
    if (last_block(ticket)) {
        __shared__ double d[2];
        fold(partials, 2, d);
        __syncthreads();
        if (threadIdx.x == 0) {
            *ticket = 0u;
            ctl->omega = d[0] > 0.0 ? d[1] / d[0] : 0.0;
        }
    }
}

// x += alpha p^ + omega s^; r = s - omega t; rho for the next iteration; tests
template <typename Z>
__global__ void __launch_bounds__(SIM_THREADS) bicg_xr_kernel(double *__restrict__ x, const Z *__restrict__ ph,
                                                              const Z *__restrict__ sh, const double *__restrict__ sv,
                                                              const double *__restrict__ t, double *__restrict__ r,
                                                              const double *__restrict__ rh, long n, double *partials,
                                                              unsigned int *ticket, BicgCtl *ctl) {
    if (bdone(ctl)) return;
    const double al = ctl->alpha, om = ctl->omega;
    double acc[2] = {0.0, 0.0};
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        x[i] += al * (double)ph[i] + om * (double)sh[i];
        const double ri = sv[i] - om * t[i];
        r[i] = ri;
        acc[0] += rh[i] * ri;
        acc[1] += ri * ri;
    }
    block_partials<2>(acc, 2, partials);
    if (last_block(ticket)) {
        __shared__ double d[2];
        fold(partials, 2, d);
        __syncthreads();
        if (threadIdx.x == 0) {
            *ticket = 0u;
            ctl->rho_old = ctl->rho;
            ctl->rho = d[0];
            ctl->rnorm = sqrt(d[1]);
            ctl->fresh = 0;
            if (ctl->rnorm <= ctl->tol) { ctl->flag = 1; ctl->done = 1; }
            else if (om == 0.0 || !(om == om)) { ctl->flag = 2; ctl->done = 1; }
            else if (d[0] == 0.0 || !(d[0] == d[0])) { ctl->flag = 2; ctl->done = 1; }
            else if (ctl->it >= ctl->max_it) { ctl->flag = 3; ctl->done = 1; }
        }
    }
}

// ||a - b||
__global__ void diff_norm_kernel(const double *__restrict__ a, const double *__restrict__ b, long n, double *partials,
                                 unsigned int *ticket, double *out) {
    double acc[1] = {0.0};
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double d = a[i] - b[i];
        acc[0] += d * d;
    }
    block_partials<1>(acc, 1, partials);
    if (last_block(ticket)) {
        __shared__ double nrm;
        fold(partials, 1, &nrm);
        __syncthreads();
        if (threadIdx.x == 0) { *ticket = 0u; out[0] = sqrt(nrm); }
    }
}

}  // namespace

// ===========================================================================
// y = S x: the block-stencil product, then the rate-controlled wells' Schur
// term -A_pw A_ww^-1 A_wp x (Eq. 16 with the well unknowns eliminated)
sim_status k_spmv_block(sim_t *s, const double *x, double *y, int bs) {
    if (s->b == 2) spmv_kernel<2, double><<<sim_blocks(s->N, bs), bs, 0, s->stream>>>(s->gd, s->J, x, y, nullptr);
    else spmv_kernel<3, double><<<sim_blocks(s->N, bs), bs, 0, s->stream>>>(s->gd, s->J, x, y, nullptr);
    SIM_LAUNCHED(s);
    return k_well_op<double>(s, x, y, nullptr);
}

sim_status k_spmv(sim_t *s, const double *x, double *y) { return k_spmv_block(s, x, y, s->tune_spmv); }

static sim_status spmv_done(sim_t *s, const void *x, bool xf, double *y, const int *done) {
    const int bs = s->tune_spmv;
    const int nb = sim_blocks(s->N, bs);
    if (s->b == 2) {
        if (xf) spmv_kernel<2, float><<<nb, bs, 0, s->stream>>>(s->gd, s->J, (const float *)x, y, done);
        else spmv_kernel<2, double><<<nb, bs, 0, s->stream>>>(s->gd, s->J, (const double *)x, y, done);
    } else {
        if (xf) spmv_kernel<3, float><<<nb, bs, 0, s->stream>>>(s->gd, s->J, (const float *)x, y, done);
        else spmv_kernel<3, double><<<nb, bs, 0, s->stream>>>(s->gd, s->J, (const double *)x, y, done);
    }
    SIM_LAUNCHED(s);
    return xf ? k_well_op<float>(s, (const float *)x, y, done) : k_well_op<double>(s, (const double *)x, y, done);
}

sim_status k_spmv_f(sim_t *s, const float *x, double *y) { return spmv_done(s, x, true, y, nullptr); }

sim_status k_norm2(sim_t *s, const double *v, long n, double *out) {
    norm_kernel<<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(v, n, s->red, s->ticket, s->scal);
    SIM_LAUNCHED(s);
    SIM_CK(s, cudaMemcpyAsync(s->h_pinned, s->scal, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    SIM_CK(s, cudaStreamSynchronize(s->stream));
    *out = s->h_pinned[0];
    return SIM_OK;
}

// one restart cycle of FGMRES from v0 = r / beta: m Arnoldi steps, each kernel
// skipping its work once ctl->done is set (no host synchronisation inside)
static sim_status enqueue_cycle(sim_t *s) {
    const long n = (long)s->N * s->b;
    const int m = s->m;
    const bool zf = sim_mixed(s);
    const size_t zes = zf ? sizeof(float) : sizeof(double);
    KrylovCtl *ctl = s->ctl;
    const int *done = &ctl->done;
    cycle_init_kernel<<<1, 64, 0, s->stream>>>(ctl);
    SIM_LAUNCHED(s);
    scale_kernel<<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(s->r, s->V, n, ctl, 1);
    SIM_LAUNCHED(s);
    for (int j = 0; j < m; j++) {
        double *vj = s->V + (size_t)j * n;
        void *zj = (char *)s->Z + (size_t)j * n * zes;
        if (cpr_apply(s, vj, zj, done) != SIM_OK) return s->err;
        if (spmv_done(s, zj, zf, s->w, done) != SIM_OK) return s->err;
        OrthDispatch<SIM_MAX_M>::dots(j + 1, s->stream, s->V, s->w, n, s->red, s->ticket, ctl->h, done);
        SIM_LAUNCHED(s);
        OrthDispatch<SIM_MAX_M>::orth(j + 1, s->stream, s->V, s->w, n, ctl->h, s->red, s->ticket, ctl->h2, done,
                                      s->opt.orth);
        SIM_LAUNCHED(s);
        OrthDispatch<SIM_MAX_M>::norm(j + 1, s->stream, s->V, s->w, n, m, s->red, s->ticket, ctl, s->opt.orth);
        SIM_LAUNCHED(s);
        scale_kernel<<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(s->w, s->V + (size_t)(j + 1) * n, n, ctl, 0);
        SIM_LAUNCHED(s);
    }
    return SIM_OK;
}

// One Arnoldi orthogonalisation step of w against basis vectors 0..nv-1 of V
// and the normalisation into V[nv], as inside a restart cycle (measurement
// only: sim_time_op clears ctl->done and poisons ctl->tol first, so no
// convergence test stops it).
sim_status k_orth_step(sim_t *s, int nv) {
    const long n = (long)s->N * s->b;
    KrylovCtl *ctl = s->ctl;
    const int *done = &ctl->done;
    OrthDispatch<SIM_MAX_M>::dots(nv, s->stream, s->V, s->w, n, s->red, s->ticket, ctl->h, done);
    SIM_LAUNCHED(s);
    OrthDispatch<SIM_MAX_M>::orth(nv, s->stream, s->V, s->w, n, ctl->h, s->red, s->ticket, ctl->h2, done, s->opt.orth);
    SIM_LAUNCHED(s);
    OrthDispatch<SIM_MAX_M>::norm(nv, s->stream, s->V, s->w, n, s->m, s->red, s->ticket, ctl, s->opt.orth);
    SIM_LAUNCHED(s);
    scale_kernel<<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(s->w, s->V + (size_t)nv * n, n, ctl, 0);
    SIM_LAUNCHED(s);
    return SIM_OK;
}

double k_orth_step_bytes(const sim_t *s, int nv) { return (3.0 * nv + 7) * (double)s->N * s->b * 8; }

sim_status k_fgmres(sim_t *s, const double *b, double *x, sim_linear_info *info) {
    const long n = (long)s->N * s->b;
    const bool zf = sim_mixed(s);
    sim_linear_info li = {0, 0, 0, 0.0, 0.0};
    if (!s->precond_ready) { if (cpr_setup(s) != SIM_OK) return s->err; }
    double bn;
    if (k_norm2(s, b, n, &bn) != SIM_OK) return s->err;
    li.b_norm = bn;
    SIM_CK(s, cudaMemsetAsync(x, 0, sizeof(double) * n, s->stream));
    if (bn == 0.0) {
        SIM_CK(s, cudaMemcpyAsync(s->r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
        li.converged = 1;
        if (info) *info = li;
        return SIM_OK;
    }
    if (!(bn == bn)) { if (info) *info = li; return sim_fail(s, SIM_ENAN, "non-finite right-hand side"); }
    const double tol = s->theta * bn;
    KrylovCtl *ctl = s->ctl;
    SIM_CK(s, cudaMemcpyAsync(s->r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
    SIM_CK(s, cudaMemcpyAsync(&ctl->beta, &bn, sizeof(double), cudaMemcpyHostToDevice, s->stream));
    SIM_CK(s, cudaMemcpyAsync(&ctl->tol, &tol, sizeof(double), cudaMemcpyHostToDevice, s->stream));
    s->learned_active = (s->learned_on && s->net && s->opt.precond == SIM_PRECOND_CPR) ? 1 : 0;
    const int learned_used = s->learned_active;
    for (int cyc = 0; cyc <= s->opt.gmres_max_restarts; cyc++) {
        if (s->opt.graphs) {
            // the restart cycle as one CUDA graph, captured once per preconditioner setup
            if (!s->cycle_exec || s->cycle_gen != s->setup_gen || s->cycle_learned != s->learned_active) {
                cudaGraph_t g = nullptr;
                SIM_CK(s, cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
                const int64_t l0 = s->launches;
                const sim_status st = enqueue_cycle(s);
                const cudaError_t ec = cudaStreamEndCapture(s->stream, &g);
                if (st != SIM_OK) { if (g) cudaGraphDestroy(g); return s->err; }
                if (!sim_cuda_ok(s, ec, "cudaStreamEndCapture")) return s->err;
                s->graph_nodes = s->launches - l0;
                if (s->cycle_exec) {
                    cudaGraphExecUpdateResultInfo ri;
                    if (cudaGraphExecUpdate(s->cycle_exec, g, &ri) != cudaSuccess) {
                        cudaGetLastError();
                        cudaGraphExecDestroy(s->cycle_exec);
                        s->cycle_exec = nullptr;
                    }
                }
                if (!s->cycle_exec) {
                    const cudaError_t ei = cudaGraphInstantiate(&s->cycle_exec, g, 0);
                    if (ei != cudaSuccess) { cudaGraphDestroy(g); s->cycle_exec = nullptr; sim_cuda_ok(s, ei, "cudaGraphInstantiate"); return s->err; }
                }
                cudaGraphDestroy(g);
                s->cycle_gen = s->setup_gen;
                s->cycle_learned = s->learned_active;
            } else {
                s->launches += s->graph_nodes;
            }
            SIM_CK(s, cudaGraphLaunch(s->cycle_exec, s->stream));
        } else if (enqueue_cycle(s) != SIM_OK) {
            return s->err;
        }
        backsolve_kernel<<<1, 32, 0, s->stream>>>(ctl);
        SIM_LAUNCHED(s);
        if (zf) xupdate_kernel<float><<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(x, (const float *)s->Z, n, ctl);
        else xupdate_kernel<double><<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(x, (const double *)s->Z, n, ctl);
        SIM_LAUNCHED(s);
        if (k_spmv(s, x, s->w) != SIM_OK) return s->err;
        resid_kernel<<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(b, s->w, s->r, n, s->red, s->ticket, &ctl->beta);
        SIM_LAUNCHED(s);
        SIM_CK(s, cudaMemcpyAsync(s->ctl_host, ctl, offsetof(KrylovCtl, h), cudaMemcpyDeviceToHost, s->stream));
        SIM_CK(s, cudaStreamSynchronize(s->stream));
        const int k = s->ctl_host->k;
        const double beta = s->ctl_host->beta;
        li.iterations += k;
        li.r_norm = beta;
        s->last_cycle_k = k;
        if (beta <= tol) { li.converged = 1; break; }
        if (s->learned_active && cyc == 0 && !(beta <= 0.1 * bn)) {
            // the learned stage did not pay off: redo the solve with plain CPR
            s->learned_active = 0;
            s->learned_fallbacks++;
            SIM_CK(s, cudaMemsetAsync(x, 0, sizeof(double) * n, s->stream));
            SIM_CK(s, cudaMemcpyAsync(s->r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
            SIM_CK(s, cudaMemcpyAsync(&ctl->beta, &bn, sizeof(double), cudaMemcpyHostToDevice, s->stream));
            li.restarts++;
            continue;
        }
        if (!(beta == beta)) break;
        if (cyc < s->opt.gmres_max_restarts) li.restarts++;
    }
    s->linear_total += li.iterations;
    if (info) *info = li;
    if (learned_used) {
        const int ns = net_status_word(s->net, s->stream);
        if (ns != 0) return sim_fail(s, ns < 0 ? SIM_ECUDA : SIM_ETIMEOUT, "learned stage: a convolution's bounded wait gave up");
    }
    if (!(li.r_norm == li.r_norm)) return sim_fail(s, SIM_ENAN, "non-finite linear residual");
    return SIM_OK;
}


// ---------------------------------------------------------------------------
// BiCGSTAB host driver
// ---------------------------------------------------------------------------
static constexpr int kBicgChunk = 4;   // iterations enqueued between host checks

// vectors: rh, p, v, s, t in V; p^, s^ in Z (apply precision)
static sim_status enqueue_bicg_chunk(sim_t *s, double *x) {
    const long n = (long)s->N * s->b;
    const bool zf = sim_mixed(s);
    const size_t zes = zf ? sizeof(float) : sizeof(double);
    BicgCtl *ctl = s->bctl;
    const int *done = &ctl->done;
    double *rh = s->V, *p = s->V + n, *v = s->V + 2 * n, *sv = s->V + 3 * n, *t = s->V + 4 * n;
    void *ph = s->Z, *sh = (char *)s->Z + (size_t)n * zes;
    bicg_chunk_init_kernel<<<1, 1, 0, s->stream>>>(ctl);
    SIM_LAUNCHED(s);
    for (int j = 0; j < kBicgChunk; j++) {
        bicg_p_kernel<<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(s->r, v, p, n, ctl);
        SIM_LAUNCHED(s);
        if (cpr_apply(s, p, ph, done) != SIM_OK) return s->err;
        if (spmv_done(s, ph, zf, v, done) != SIM_OK) return s->err;
        bicg_alpha_kernel<<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(rh, v, n, s->red, s->ticket, ctl);
        SIM_LAUNCHED(s);
        bicg_s_kernel<<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(s->r, v, sv, n, s->red, s->ticket, ctl, j);
        SIM_LAUNCHED(s);
        if (zf) bicg_xhalf_kernel<float><<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(x, (const float *)ph, n, ctl, j);
        else bicg_xhalf_kernel<double><<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(x, (const double *)ph, n, ctl, j);
        SIM_LAUNCHED(s);
        if (cpr_apply(s, sv, sh, done) != SIM_OK) return s->err;
        if (spmv_done(s, sh, zf, t, done) != SIM_OK) return s->err;
        bicg_omega_kernel<<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(t, sv, n, s->red, s->ticket, ctl);
        SIM_LAUNCHED(s);
        if (zf)
            bicg_xr_kernel<float><<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(x, (const float *)ph, (const float *)sh, sv, t,
                                                                                s->r, rh, n, s->red, s->ticket, ctl);
        else
            bicg_xr_kernel<double><<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(x, (const double *)ph, (const double *)sh,
                                                                                 sv, t, s->r, rh, n, s->red, s->ticket, ctl);
        SIM_LAUNCHED(s);
    }
    return SIM_OK;
}

static sim_status launch_bicg_chunk(sim_t *s, double *x) {
    if (!s->opt.graphs) return enqueue_bicg_chunk(s, x);
    // x is baked into the graph: recapture when it changes
    if (!s->bicg_exec || s->bicg_gen != s->setup_gen || s->bicg_x != x) {
        cudaGraph_t g = nullptr;
        SIM_CK(s, cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
        const int64_t l0 = s->launches;
        const sim_status st = enqueue_bicg_chunk(s, x);
        const cudaError_t ec = cudaStreamEndCapture(s->stream, &g);
        if (st != SIM_OK) { if (g) cudaGraphDestroy(g); return s->err; }
        if (!sim_cuda_ok(s, ec, "cudaStreamEndCapture")) return s->err;
        s->bicg_nodes = s->launches - l0;
        if (s->bicg_exec) {
            cudaGraphExecUpdateResultInfo ri;
            if (cudaGraphExecUpdate(s->bicg_exec, g, &ri) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphExecDestroy(s->bicg_exec);
                s->bicg_exec = nullptr;
            }
        }
        if (!s->bicg_exec) {
            const cudaError_t ei = cudaGraphInstantiate(&s->bicg_exec, g, 0);
            if (ei != cudaSuccess) { cudaGraphDestroy(g); s->bicg_exec = nullptr; sim_cuda_ok(s, ei, "cudaGraphInstantiate"); return s->err; }
        }
        cudaGraphDestroy(g);
        s->bicg_gen = s->setup_gen;
        s->bicg_x = x;
    } else {
        s->launches += s->bicg_nodes;
    }
    SIM_CK(s, cudaGraphLaunch(s->bicg_exec, s->stream));
    return SIM_OK;
}

// true residual r = b - J x into s->r, its norm into ctl->rnorm; read back
static sim_status bicg_true_residual(sim_t *s, const double *b, const double *x) {
    const long n = (long)s->N * s->b;
    if (k_spmv(s, x, s->w) != SIM_OK) return s->err;
    resid_kernel<<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(b, s->w, s->r, n, s->red, s->ticket, &s->bctl->rnorm);
    SIM_LAUNCHED(s);
    SIM_CK(s, cudaMemcpyAsync(s->bctl_host, s->bctl, sizeof(BicgCtl), cudaMemcpyDeviceToHost, s->stream));
    SIM_CK(s, cudaStreamSynchronize(s->stream));
    return SIM_OK;
}

// Right-preconditioned BiCGSTAB from x = 0.  When the recursive residual
// meets the tolerance the true residual decides; if it does not, or on a
// breakdown, the iteration restarts from the current x with rh = r.
sim_status k_bicgstab(sim_t *s, const double *b, double *x, sim_linear_info *info) {
    const long n = (long)s->N * s->b;
    sim_linear_info li = {0, 0, 0, 0.0, 0.0};
    if (!s->precond_ready) { if (cpr_setup(s) != SIM_OK) return s->err; }
    double bn;
    if (k_norm2(s, b, n, &bn) != SIM_OK) return s->err;
    li.b_norm = bn;
    SIM_CK(s, cudaMemsetAsync(x, 0, sizeof(double) * n, s->stream));
    SIM_CK(s, cudaMemcpyAsync(s->r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
    if (bn == 0.0) { li.converged = 1; if (info) *info = li; return SIM_OK; }
    if (!(bn == bn)) { if (info) *info = li; return sim_fail(s, SIM_ENAN, "non-finite right-hand side"); }
    const double tol = s->theta * bn;
    s->learned_active = 0;   // the learned stage is used with FGMRES only (a nonlinear stage)
    li.r_norm = bn;
    BicgCtl *ctl = s->bctl;
    bicg_init_kernel<<<1, 1, 0, s->stream>>>(ctl, tol, s->opt.lin_max_iter);
    SIM_LAUNCHED(s);
    bicg_restart_kernel<<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(s->r, s->V, n, s->red, s->ticket, ctl);
    SIM_LAUNCHED(s);
    for (;;) {
        if (launch_bicg_chunk(s, x) != SIM_OK) return s->err;
        SIM_CK(s, cudaMemcpyAsync(s->bctl_host, ctl, sizeof(BicgCtl), cudaMemcpyDeviceToHost, s->stream));
        SIM_CK(s, cudaStreamSynchronize(s->stream));
        if (!s->bctl_host->done) continue;     // the device caps the iterations (flag 3)
        if (bicg_true_residual(s, b, x) != SIM_OK) return s->err;
        const BicgCtl &h = *s->bctl_host;
        li.iterations = h.it;
        li.r_norm = h.rnorm;
        if (h.rnorm <= tol) { li.converged = 1; break; }
        if (!(h.rnorm == h.rnorm) || h.it >= h.max_it) break;
        bicg_restart_kernel<<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(s->r, s->V, n, s->red, s->ticket, ctl);
        SIM_LAUNCHED(s);
        li.restarts++;
    }
    s->linear_total += li.iterations;
    if (info) *info = li;
    if (!(li.r_norm == li.r_norm)) return sim_fail(s, SIM_ENAN, "non-finite linear residual");
    return SIM_OK;
}

sim_status k_linear_solve(sim_t *s, const double *b, double *x, sim_linear_info *info) {
    return s->opt.krylov == SIM_KRYLOV_BICGSTAB ? k_bicgstab(s, b, x, info) : k_fgmres(s, b, x, info);
}

sim_status k_diff_norm2(sim_t *s, const double *a, const double *b, long n, double *out) {
    diff_norm_kernel<<<SIM_RED_BLOCKS, SIM_THREADS, 0, s->stream>>>(a, b, n, s->red, s->ticket, s->scal);
    SIM_LAUNCHED(s);
    SIM_CK(s, cudaMemcpyAsync(s->h_pinned, s->scal, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    SIM_CK(s, cudaStreamSynchronize(s->stream));
    *out = s->h_pinned[0];
    return SIM_OK;
}

// ===========================================================================
// FGMRES batched over the members of an ensemble
// ===========================================================================
namespace {
// per member after a cycle: active, inner iterations so far, beta
__global__ void b_gather_kernel(const KMember *M, const int2 *work, double *out) {
    VBlk vb;
    const KMember &m = member_of(M, work, &vb, 1);
    if (threadIdx.x == 0) {
        double *o = out + 4 * (long)work[blockIdx.x].x;
        o[0] = m.ctl->active;
        o[1] = m.ctl->iters;
        o[2] = m.ctl->beta;
        o[3] = m.ctl->k;
    }
}
}  // namespace

struct KrylovBatch {
    int nm = 0, m = 0, b = 0, zf = 0, orth = 0;
    KMember *dmem = nullptr; size_t mem_cap = 0;
    int2 *dwork = nullptr; size_t work_cap = 0;
    double *dout = nullptr, *hout = nullptr; int out_cap = 0;
    long red_off = 0, orth_off = 0, one_off = 0, cell_off = 0;
    int red_n = 0, orth_n = 0, one_n = 0, cell_n = 0;
    CprBatch *cpr = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t nodes = 0, launches = 0;
};

KrylovBatch *k_batch_new() {
    KrylovBatch *kb = new KrylovBatch();
    kb->cpr = cpr_batch_new();
    return kb;
}

void k_batch_free(KrylovBatch *kb) {
    if (!kb) return;
    if (kb->exec) cudaGraphExecDestroy(kb->exec);
    if (kb->dmem) cudaFree(kb->dmem);
    if (kb->dwork) cudaFree(kb->dwork);
    if (kb->dout) cudaFree(kb->dout);
    if (kb->hout) cudaFreeHost(kb->hout);
    cpr_batch_free(kb->cpr);
    delete kb;
}

int64_t k_batch_launches(const KrylovBatch *kb) { return kb ? kb->launches : 0; }

static cudaError_t kgrow(void **p, size_t *cap, size_t bytes) {
    if (bytes <= *cap) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr; *cap = 0;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) *cap = bytes;
    return e;
}

// the kernels of one restart cycle for every member (captured as one graph)
static cudaError_t enqueue_batch_cycle(KrylovBatch *kb, cudaStream_t st, int64_t *launches) {
    const KMember *M = kb->dmem;
    const int2 *W = kb->dwork;
    int64_t n = 0;
    b_cycle_init_kernel<<<kb->one_n, 64, 0, st>>>(M, W + kb->one_off); n++;
    b_scale_kernel<<<kb->red_n, SIM_THREADS, 0, st>>>(M, W + kb->red_off, 0, 1); n++;
    for (int j = 0; j < kb->m; j++) {
        const int a = cpr_batch_apply(kb->cpr, st, j);
        if (a < 0) return cudaErrorLaunchFailure;
        n += a;
        if (kb->b == 2) {
            if (kb->zf) b_spmv_kernel<2, float><<<kb->cell_n, SIM_THREADS, 0, st>>>(M, W + kb->cell_off, j, 0);
            else b_spmv_kernel<2, double><<<kb->cell_n, SIM_THREADS, 0, st>>>(M, W + kb->cell_off, j, 0);
        } else {
            if (kb->zf) b_spmv_kernel<3, float><<<kb->cell_n, SIM_THREADS, 0, st>>>(M, W + kb->cell_off, j, 0);
            else b_spmv_kernel<3, double><<<kb->cell_n, SIM_THREADS, 0, st>>>(M, W + kb->cell_off, j, 0);
        }
        OrthDispatch<SIM_MAX_M>::bdots(j + 1, st, M, W + kb->red_off, kb->red_n);
        OrthDispatch<SIM_MAX_M>::borth(j + 1, st, M, W + kb->orth_off, kb->orth_n, kb->orth);
        OrthDispatch<SIM_MAX_M>::bnorm(j + 1, st, M, W + kb->red_off, kb->red_n, kb->m, kb->orth);
        b_scale_kernel<<<kb->red_n, SIM_THREADS, 0, st>>>(M, W + kb->red_off, j + 1, 0);
        n += 5;
    }
    *launches = n;
    return cudaGetLastError();
}

// Solve J_k x_k = rhs_k for the members ms[0..nm) (their bl -> dx, at their
// own tolerance theta * ||rhs||) by FGMRES(m) with the batched CPR
// application: every Krylov operation is one launch over all members, a
// restart cycle is one graph, and a member whose estimate meets its tolerance
// stops (its kernels return at once) while the others go on.
sim_status k_fgmres_batch(KrylovBatch *kb, sim_t *const *ms, int nm, cudaStream_t st, sim_linear_info *infos,
                          std::string *err) {
    auto fail = [&](const char *what, cudaError_t e) {
        *err = std::string("batched FGMRES: ") + what + ": " + cudaGetErrorString(e);
        return SIM_ECUDA;
    };
    const sim_t *s0 = ms[0];
    kb->nm = nm; kb->m = s0->m; kb->b = s0->b; kb->zf = sim_mixed(s0) ? 1 : 0; kb->orth = s0->opt.orth;
    std::vector<KMember> hm(nm);
    std::vector<int2> work;
    auto add = [&](long *off, int *count, int per_member_fixed, bool cells) {
        *off = (long)work.size();
        for (int k = 0; k < nm; k++) {
            const int nb = cells ? sim_blocks(ms[k]->N, SIM_THREADS) : per_member_fixed;
            for (int q = 0; q < nb; q++) work.push_back(make_int2(k, q));
        }
        *count = (int)((long)work.size() - *off);
    };
    for (int k = 0; k < nm; k++) {
        sim_t *s = ms[k];
        KMember &m = hm[k];
        m.g = s->gd; m.n = (long)s->N * s->b; m.theta = s->theta; m.J = s->J;
        m.V = s->V; m.w = s->w; m.r = s->r; m.x = s->dx; m.rhs = s->bl; m.Z = s->Z;
        m.ctl = s->ctl; m.red = s->red; m.ticket = s->ticket;
    }
    add(&kb->red_off, &kb->red_n, SIM_RED_BLOCKS, false);
    add(&kb->orth_off, &kb->orth_n, 2 * SIM_RED_BLOCKS, false);
    add(&kb->one_off, &kb->one_n, 1, false);
    add(&kb->cell_off, &kb->cell_n, 0, true);
    cudaError_t e;
    if ((e = kgrow((void **)&kb->dmem, &kb->mem_cap, sizeof(KMember) * nm)) != cudaSuccess) return fail("allocation", e);
    if ((e = kgrow((void **)&kb->dwork, &kb->work_cap, sizeof(int2) * work.size())) != cudaSuccess) return fail("allocation", e);
    if (kb->out_cap < nm) {
        if (kb->dout) cudaFree(kb->dout);
        if (kb->hout) cudaFreeHost(kb->hout);
        kb->dout = nullptr; kb->hout = nullptr; kb->out_cap = 0;
        if ((e = cudaMalloc(&kb->dout, sizeof(double) * 4 * nm)) != cudaSuccess) return fail("allocation", e);
        if ((e = cudaMallocHost(&kb->hout, sizeof(double) * 4 * nm)) != cudaSuccess) return fail("allocation", e);
        kb->out_cap = nm;
    }
    if ((e = cudaMemcpyAsync(kb->dmem, hm.data(), sizeof(KMember) * nm, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(kb->dwork, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return fail("table upload", e);
    if ((e = cpr_batch_build(kb->cpr, ms, nm, st)) != cudaSuccess) return fail("CPR tables", e);   // synchronises st
    // start: r = b, x = 0, beta = ||b||, tolerance, active
    b_start_kernel<<<kb->red_n, SIM_THREADS, 0, st>>>(kb->dmem, kb->dwork + kb->red_off);
    kb->launches++;
    b_gather_kernel<<<kb->one_n, 32, 0, st>>>(kb->dmem, kb->dwork + kb->one_off, kb->dout);
    kb->launches++;
    if ((e = cudaMemcpyAsync(kb->hout, kb->dout, sizeof(double) * 4 * nm, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail("start", e);
    std::vector<double> bnorm(nm);
    std::vector<char> stopped(nm, 0);
    int active = 0;
    for (int k = 0; k < nm; k++) {
        bnorm[k] = kb->hout[4 * k + 2];
        infos[k] = sim_linear_info{0, 0, 0, bnorm[k], bnorm[k]};
        if (bnorm[k] == 0.0) infos[k].converged = 1;
        if (kb->hout[4 * k] != 0.0) active++;
        else stopped[k] = 1;            // zero right-hand side (x = 0) or a non-finite one
    }
    // the cycle graph: captured for this call's tables (they change with every setup)
    {
        cudaGraph_t g = nullptr;
        if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return fail("capture", e);
        int64_t nl = 0;
        const cudaError_t eq = enqueue_batch_cycle(kb, st, &nl);
        const cudaError_t ec = cudaStreamEndCapture(st, &g);
        if (eq != cudaSuccess || ec != cudaSuccess) { if (g) cudaGraphDestroy(g); return fail("capture", eq != cudaSuccess ? eq : ec); }
        kb->nodes = nl;
        if (kb->exec) {
            cudaGraphExecUpdateResultInfo ri;
            if (cudaGraphExecUpdate(kb->exec, g, &ri) != cudaSuccess) {
                (void)cudaGetLastError();
                cudaGraphExecDestroy(kb->exec);
                kb->exec = nullptr;
            }
        }
        if (!kb->exec && (e = cudaGraphInstantiate(&kb->exec, g, 0)) != cudaSuccess) {
            cudaGraphDestroy(g);
            kb->exec = nullptr;
            return fail("instantiate", e);
        }
        cudaGraphDestroy(g);
    }
    const int maxr = s0->opt.gmres_max_restarts;
    for (int cyc = 0; cyc <= maxr && active > 0; cyc++) {
        if ((e = cudaGraphLaunch(kb->exec, st)) != cudaSuccess) return fail("cycle", e);
        kb->launches += kb->nodes;
        b_backsolve_kernel<<<kb->one_n, 32, 0, st>>>(kb->dmem, kb->dwork + kb->one_off);
        if (kb->zf) b_xupdate_kernel<float><<<kb->red_n, SIM_THREADS, 0, st>>>(kb->dmem, kb->dwork + kb->red_off);
        else b_xupdate_kernel<double><<<kb->red_n, SIM_THREADS, 0, st>>>(kb->dmem, kb->dwork + kb->red_off);
        if (kb->b == 2) b_spmv_kernel<2, double><<<kb->cell_n, SIM_THREADS, 0, st>>>(kb->dmem, kb->dwork + kb->cell_off, 0, 1);
        else b_spmv_kernel<3, double><<<kb->cell_n, SIM_THREADS, 0, st>>>(kb->dmem, kb->dwork + kb->cell_off, 0, 1);
        b_resid_kernel<<<kb->red_n, SIM_THREADS, 0, st>>>(kb->dmem, kb->dwork + kb->red_off);
        b_gather_kernel<<<kb->one_n, 32, 0, st>>>(kb->dmem, kb->dwork + kb->one_off, kb->dout);
        kb->launches += 5;
        if ((e = cudaGetLastError()) != cudaSuccess) return fail("launch", e);
        if ((e = cudaMemcpyAsync(kb->hout, kb->dout, sizeof(double) * 4 * nm, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return fail("cycle end", e);
        active = 0;
        for (int k = 0; k < nm; k++) {
            if (stopped[k]) continue;
            sim_linear_info &li = infos[k];
            li.iterations = (int)kb->hout[4 * k + 1];
            li.r_norm = kb->hout[4 * k + 2];
            if (kb->hout[4 * k] != 0.0) {          // still above its tolerance: another cycle
                active++;
                if (cyc < maxr) li.restarts++;
                continue;
            }
            stopped[k] = 1;                        // met its tolerance, or turned non-finite
            li.converged = li.r_norm <= ms[k]->theta * bnorm[k] ? 1 : 0;
            ms[k]->last_cycle_k = (int)kb->hout[4 * k + 3];
        }
    }
    for (int k = 0; k < nm; k++) ms[k]->linear_total += infos[k].iterations;
    return SIM_OK;
}
