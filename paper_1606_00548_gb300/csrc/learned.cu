// Learned pressure stage: a 3-D convolutional network on the grid, trained on
// the device by hand-written BF16 tensor-core kernels (FP32 accumulation).
//
// Network: 4 layers of 3x3x3 convolutions (zero padding, stride 1) with
// channels 4 -> 16 -> 16 -> 16 -> 1, ReLU between layers.  Input features per
// cell: the normalised pressure residual and three standardised log face
// transmissibility sums; output: a pressure correction (normalised).
//
// Convolution as implicit GEMM on mma.sync.m16n8k16 (BF16 x BF16 -> FP32):
//   forward / data gradient: M = 16 cells per warp, K = 16 channels per tap
//   (27 taps), N = output channels (8 or 16);
//   weight gradient: M = 16 input channels, N = output channels, K = cells.
// Activations are stored channels-innermost as BF16 [N][16] (pairs of channels
// per 32-bit word), which is also the register layout of the MMA fragments.
// Reductions over cells (weight and bias gradients, loss) are written as
// per-block partials and folded in block order: results do not depend on
// scheduling.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "sim_internal.cuh"

namespace {

constexpr int CH = 16;          // padded channel count
constexpr int NLAYER = 4;
constexpr int CIN[NLAYER] = {4, 16, 16, 16};
constexpr int COUT[NLAYER] = {16, 16, 16, 1};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return a | (b << 16);
}
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ uint32_t bf16_bits(const uint16_t *p) { return (uint32_t)(*p); }

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

struct Dims {
    int nx, ny, nz, N;
};

// neighbour of cell c through tap t (offset (t/9-1, (t/3)%3-1, t%3-1) in (z, y, x)), or -1
__device__ __forceinline__ int tap_nbr(const Dims &d, int x, int y, int z, int c, int t) {
    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
    const int X = x + dx, Y = y + dy, Z = z + dz;
    if (X < 0 || X >= d.nx || Y < 0 || Y >= d.ny || Z < 0 || Z >= d.nz) return -1;
    return c + dx + d.nx * (dy + d.ny * dz);
}

// ---------------------------------------------------------------------------
// forward convolution / data gradient (same structure, different weights)
//   MODE 0: out = bf16(relu(acc + bias))             hidden layer forward
//   MODE 1: outf[c] = acc[channel 0] + bias[0]        last layer forward
//   MODE 2: out = bf16(acc * (mask > 0))              data gradient into a ReLU layer
// wpk: packed weights [27][NT][8 n][8 k-pairs] (uint32 of two bf16)
//
// One block computes a brick of 16 x TBY x TBZ output cells: the brick and
// its one-cell halo are staged in shared memory once (zero
// outside the grid), so the 27 taps read shared memory instead of gathering
// from global memory 27 times.  An MMA row block is one x-row of 16 cells;
// cells are padded to 12 words in shared memory so that the 32 lanes of a
// fragment load hit 32 distinct banks.
// ---------------------------------------------------------------------------
constexpr int TBX = 16, TBY = 8, TBZ = 4;
constexpr int HX = TBX + 2, HY = TBY + 2, HZ = TBZ + 2, HCELLS = HX * HY * HZ;
constexpr int CW = 12;                       // words per staged cell (8 used)
constexpr int TWARPS = 16, TROWS = TBY * TBZ;   // 2 row blocks per warp

template <int NT>
constexpr int tiled_smem_bytes() { return (27 * NT * 64 + HCELLS * CW) * 4; }

template <int NT, int MODE>
__global__ void __launch_bounds__(TWARPS * 32) conv_tiled_kernel(Dims d, const uint32_t *__restrict__ in,
                                                               const uint32_t *__restrict__ wpk,
                                                               const float *__restrict__ bias,
                                                               const uint32_t *__restrict__ mask,
                                                               uint32_t *__restrict__ out, float *__restrict__ outf,
                                                               const int *done) {
    if (done != nullptr && *(volatile const int *)done) return;
    extern __shared__ uint32_t smem[];
    uint32_t *ws = smem, *hs = smem + 27 * NT * 64;
    const int bx0 = blockIdx.x * TBX, by0 = blockIdx.y * TBY, bz0 = blockIdx.z * TBZ;
    for (int k = threadIdx.x; k < 27 * NT * 64; k += blockDim.x) ws[k] = wpk[k];
    for (int k = threadIdx.x; k < HCELLS * 8; k += blockDim.x) {
        const int hc = k >> 3, w = k & 7;
        const int hx = hc % HX, hy = (hc / HX) % HY, hz = hc / (HX * HY);
        const int X = bx0 - 1 + hx, Y = by0 - 1 + hy, Z = bz0 - 1 + hz;
        uint32_t v = 0u;
        if (X >= 0 && X < d.nx && Y >= 0 && Y < d.ny && Z >= 0 && Z < d.nz)
            v = in[((long)X + (long)d.nx * (Y + (long)d.ny * Z)) * 8 + w];
        hs[hc * CW + w] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    for (int rb = warp; rb < TROWS; rb += TWARPS) {
        const int my = rb % TBY, mz = rb / TBY;
        const int Y = by0 + my, Z = bz0 + mz;
        const int X0 = bx0 + g, X1 = bx0 + g + 8;
        const bool rowok = Y < d.ny && Z < d.nz;
        const bool v0 = rowok && X0 < d.nx, v1 = rowok && X1 < d.nx;
        float acc[NT][4];
#pragma unroll
        for (int nt = 0; nt < NT; nt++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[nt][q] = 0.0f;
#pragma unroll 3
        for (int tap = 0; tap < 27; tap++) {
            const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;      // halo offsets 0..2
            const int h0 = (g + dx) + HX * ((my + dy) + HY * (mz + dz));
            const uint32_t *c0 = hs + h0 * CW, *c1 = hs + (h0 + 8) * CW;
            const uint32_t a0 = c0[t4], a1 = c1[t4], a2 = c0[4 + t4], a3 = c1[4 + t4];
#pragma unroll
            for (int nt = 0; nt < NT; nt++) {
                const uint32_t *wb = ws + ((tap * NT + nt) * 8 + g) * 8;
                mma_bf16(acc[nt], a0, a1, a2, a3, wb[t4], wb[t4 + 4]);
            }
        }
        const long r0 = (long)X0 + (long)d.nx * (Y + (long)d.ny * Z), r1 = r0 + 8;
#pragma unroll
        for (int nt = 0; nt < NT; nt++) {
            const int col = nt * 8 + 2 * t4;
            if (MODE == 0) {
                const float b0 = bias[col], b1 = bias[col + 1];
                if (v0) out[r0 * 8 + nt * 4 + t4] = pack_bf16(fmaxf(acc[nt][0] + b0, 0.f), fmaxf(acc[nt][1] + b1, 0.f));
                if (v1) out[r1 * 8 + nt * 4 + t4] = pack_bf16(fmaxf(acc[nt][2] + b0, 0.f), fmaxf(acc[nt][3] + b1, 0.f));
            } else if (MODE == 1) {
                if (nt == 0 && t4 == 0) {
                    if (v0) outf[r0] = acc[0][0] + bias[0];
                    if (v1) outf[r1] = acc[0][2] + bias[0];
                }
            } else {
                if (v0) {
                    const uint32_t mk = mask[r0 * 8 + nt * 4 + t4];
                    out[r0 * 8 + nt * 4 + t4] =
                        pack_bf16(bf16_lo(mk) > 0.f ? acc[nt][0] : 0.f, bf16_hi(mk) > 0.f ? acc[nt][1] : 0.f);
                }
                if (v1) {
                    const uint32_t mk = mask[r1 * 8 + nt * 4 + t4];
                    out[r1 * 8 + nt * 4 + t4] =
                        pack_bf16(bf16_lo(mk) > 0.f ? acc[nt][2] : 0.f, bf16_hi(mk) > 0.f ? acc[nt][3] : 0.f);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// weight gradient: dW[tap][ci][co] = sum_c in[nbr(c, tap)][ci] * dout[c][co]
// block (chunk, tap); 4 warps stride over 16-cell k-steps; per-block partials
// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(128) wgrad_kernel(Dims d, const uint16_t *__restrict__ in,
                                                    const uint16_t *__restrict__ dout, int cells_per_block,
                                                    float *__restrict__ part) {
    const int tap = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int c_begin = blockIdx.x * cells_per_block;
    const int c_end = min(d.N, c_begin + cells_per_block);
    float acc[NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; nt++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[nt][q] = 0.0f;
    for (int k0 = c_begin + warp * 16; k0 < c_end; k0 += 64) {
        int cell[4], nb[4];
        const int kk[4] = {2 * t4, 2 * t4 + 1, 2 * t4 + 8, 2 * t4 + 9};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            cell[q] = k0 + kk[q];
            nb[q] = -1;
            if (cell[q] < c_end) {
                const int c = cell[q];
                const int x = c % d.nx, qq = c / d.nx, y = qq % d.ny, z = qq / d.ny;
                nb[q] = tap_nbr(d, x, y, z, c, tap);
            } else {
                cell[q] = -1;
            }
        }
        auto A = [&](int q, int ci) -> uint32_t { return nb[q] >= 0 ? bf16_bits(in + (long)nb[q] * CH + ci) : 0u; };
        const uint32_t a0 = A(0, g) | (A(1, g) << 16);
        const uint32_t a1 = A(0, g + 8) | (A(1, g + 8) << 16);
        const uint32_t a2 = A(2, g) | (A(3, g) << 16);
        const uint32_t a3 = A(2, g + 8) | (A(3, g + 8) << 16);
#pragma unroll
        for (int nt = 0; nt < NT; nt++) {
            auto Bv = [&](int q) -> uint32_t { return cell[q] >= 0 ? bf16_bits(dout + (long)cell[q] * CH + nt * 8 + g) : 0u; };
            const uint32_t b0 = Bv(0) | (Bv(1) << 16);
            const uint32_t b1 = Bv(2) | (Bv(3) << 16);
            mma_bf16(acc[nt], a0, a1, a2, a3, b0, b1);
        }
    }
    // fold the 4 warps in shared memory, then write the block partial [16][NT*8]
    __shared__ float red[4][16 * 16];
#pragma unroll
    for (int nt = 0; nt < NT; nt++) {
        const int col = nt * 8 + 2 * t4;
        red[warp][g * 16 + col] = acc[nt][0];
        red[warp][g * 16 + col + 1] = acc[nt][1];
        red[warp][(g + 8) * 16 + col] = acc[nt][2];
        red[warp][(g + 8) * 16 + col + 1] = acc[nt][3];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 16 * NT * 8; e += blockDim.x) {
        const int ci = e / (NT * 8), co = e % (NT * 8);
        const float s = red[0][ci * 16 + co] + red[1][ci * 16 + co] + red[2][ci * 16 + co] + red[3][ci * 16 + co];
        part[(((long)tap * gridDim.x + blockIdx.x) * 16 + ci) * (NT * 8) + co] = s;
    }
}

// dW[tap][ci][co] (FP32, logical cin x cout) = sum over chunks of the partials
template <int NT>
__global__ void wgrad_fold_kernel(int nchunk, int cin, int cout, const float *__restrict__ part, float *__restrict__ dW) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 27 * cin * cout) return;
    const int tap = e / (cin * cout), r = e % (cin * cout), ci = r / cout, co = r % cout;
    float s = 0.f;
    for (int b = 0; b < nchunk; b++) s += part[(((long)tap * nchunk + b) * 16 + ci) * (NT * 8) + co];
    dW[e] = s;
}

// bias gradient partials: per block sums of dout channels
__global__ void bgrad_kernel(int N, int cout, const uint16_t *__restrict__ dout, float *__restrict__ part) {
    __shared__ float sh[128][16];
    float s[16];
    for (int c = 0; c < 16; c++) s[c] = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        for (int c = 0; c < cout; c++) s[c] += __uint_as_float(bf16_bits(dout + (long)i * CH + c) << 16);
    for (int c = 0; c < 16; c++) sh[threadIdx.x][c] = s[c];
    __syncthreads();
    if (threadIdx.x < 16) {
        float t = 0.f;
        for (int k = 0; k < (int)blockDim.x; k++) t += sh[k][threadIdx.x];
        part[blockIdx.x * 16 + threadIdx.x] = t;
    }
}
__global__ void bgrad_fold_kernel(int nblk, int cout, const float *__restrict__ part, float *__restrict__ db) {
    const int c = threadIdx.x;
    if (c >= cout) return;
    float t = 0.f;
    for (int b = 0; b < nblk; b++) t += part[b * 16 + c];
    db[c] = t;
}

// MSE loss partials and dL/dy = 2 (y - target) / N into channel 0 of a BF16 [N][16] buffer
__global__ void mse_kernel(int N, const float *__restrict__ y, const float *__restrict__ target, uint16_t *__restrict__ dout,
                           double *__restrict__ part) {
    __shared__ double sh[128];
    double s = 0.0;
    const float scale = 2.0f / (float)N;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const float e = y[i] - target[i];
        s += (double)e * e;
        uint32_t *o = (uint32_t *)(dout + (long)i * CH);
        o[0] = pack_bf16(e * scale, 0.f);
        for (int k = 1; k < 8; k++) o[k] = 0u;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)blockDim.x; k++) t += sh[k];
        part[blockIdx.x] = t;
    }
}
__global__ void mse_fold_kernel(int nblk, int N, const double *__restrict__ part, double *__restrict__ loss) {
    if (threadIdx.x != 0) return;
    double t = 0.0;
    for (int b = 0; b < nblk; b++) t += part[b];
    *loss = t / N;
}

// FP32 features [N][4] -> BF16 [N][16] (channels 4..15 zero)
__global__ void features_kernel(int N, const float *__restrict__ x, uint32_t *__restrict__ out, const int *done) {
    if (done != nullptr && *(volatile const int *)done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    out[(long)i * 8 + 0] = pack_bf16(x[(long)i * 4 + 0], x[(long)i * 4 + 1]);
    out[(long)i * 8 + 1] = pack_bf16(x[(long)i * 4 + 2], x[(long)i * 4 + 3]);
    for (int k = 2; k < 8; k++) out[(long)i * 8 + k] = 0u;
}

// pack FP32 weights W[27][cin][cout] into MMA B-fragment order.
// transpose = 0: forward  B[k = ci][n = co], tap t
// transpose = 1: data grad B[k = co][n = ci], tap 26 - t (offsets negated)
__global__ void pack_kernel(int cin, int cout, int NT, int transpose, const float *__restrict__ W, uint32_t *__restrict__ wpk) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;   // over 27 * NT * 8 * 8
    if (e >= 27 * NT * 64) return;
    const int tap = e / (NT * 64), r = e % (NT * 64), nt = r / 64, n = (r / 8) % 8, kp = r % 8;
    const int nn = nt * 8 + n, k0 = 2 * kp, k1 = 2 * kp + 1;
    float lo = 0.f, hi = 0.f;
    if (!transpose) {
        if (nn < cout) {
            if (k0 < cin) lo = W[((long)tap * cin + k0) * cout + nn];
            if (k1 < cin) hi = W[((long)tap * cin + k1) * cout + nn];
        }
    } else {
        const int st = 26 - tap;
        if (nn < cin) {
            if (k0 < cout) lo = W[((long)st * cin + nn) * cout + k0];
            if (k1 < cout) hi = W[((long)st * cin + nn) * cout + k1];
        }
    }
    wpk[e] = pack_bf16(lo, hi);
}

// Adam (bias-corrected) on FP32 master parameters
__global__ void adam_kernel(int n, float *__restrict__ p, const float *__restrict__ gr, float *__restrict__ m,
                            float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = gr[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi; v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

// ===========================================================================
struct sim_net {
    Dims d;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string msg;
    sim_status err = SIM_OK;
    std::vector<void *> allocs;
    int64_t nparam = 0;
    int64_t off_w[NLAYER], off_b[NLAYER];
    float *param = nullptr, *grad = nullptr, *adam_m = nullptr, *adam_v = nullptr;   // flat FP32
    uint32_t *wf[NLAYER], *wb[NLAYER];   // packed forward / data-gradient weights
    uint32_t *act[NLAYER + 1];           // BF16 [N][16]: input features, hidden activations
    float *out = nullptr;                // [N]
    uint32_t *g0 = nullptr, *g1 = nullptr;   // BF16 [N][16] gradient buffers
    float *wpart = nullptr, *bpart = nullptr;
    double *lpart = nullptr, *dloss = nullptr;
    int chunk = 0, nchunk = 0, bblk = 0, lblk = 0;
    int adam_t = 0;
    int64_t launches = 0;
};

static sim_status net_fail(sim_net_t *n, sim_status st, const std::string &m) {
    if (n && n->err == SIM_OK) { n->err = st; n->msg = m; }
    return n ? n->err : st;
}
static bool net_ok(sim_net_t *n, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return true;
    net_fail(n, SIM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return false;
}
#define NET_CK(n, call) do { if (!net_ok((n), (call), #call)) return (n)->err; } while (0)
#define NET_LAUNCHED(n) do { (n)->launches++; if (!net_ok((n), cudaGetLastError(), "kernel launch")) return (n)->err; } while (0)

static void *net_alloc(sim_net_t *n, size_t bytes) {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) { net_fail(n, SIM_ENOMEM, "cudaMalloc failed"); return nullptr; }
    n->allocs.push_back(p);
    return p;
}

static sim_status pack_all(sim_net_t *n) {
    for (int l = 0; l < NLAYER; l++) {
        const int NT = COUT[l] > 8 ? 2 : 1;
        const int NTb = CIN[l] > 8 ? 2 : 1;
        pack_kernel<<<sim_blocks(27 * NT * 64), SIM_THREADS, 0, n->stream>>>(CIN[l], COUT[l], NT, 0, n->param + n->off_w[l],
                                                                           n->wf[l]);
        NET_LAUNCHED(n);
        pack_kernel<<<sim_blocks(27 * NTb * 64), SIM_THREADS, 0, n->stream>>>(CIN[l], COUT[l], NTb, 1,
                                                                            n->param + n->off_w[l], n->wb[l]);
        NET_LAUNCHED(n);
    }
    return SIM_OK;
}

static dim3 tiled_grid(const Dims &d) {
    return dim3((d.nx + TBX - 1) / TBX, (d.ny + TBY - 1) / TBY, (d.nz + TBZ - 1) / TBZ);
}

// once per process: the tiled kernels need more than the default 48 KB of shared memory
static bool tiled_attrs() {
    static const bool ok = [] {
        return cudaFuncSetAttribute(conv_tiled_kernel<2, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    tiled_smem_bytes<2>()) == cudaSuccess &&
               cudaFuncSetAttribute(conv_tiled_kernel<2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    tiled_smem_bytes<2>()) == cudaSuccess &&
               cudaFuncSetAttribute(conv_tiled_kernel<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    tiled_smem_bytes<1>()) == cudaSuccess;
    }();
    return ok;
}

static sim_status net_forward(sim_net_t *n, const int *done = nullptr) {
    if (!tiled_attrs()) return SIM_ECUDA;
    const dim3 grid = tiled_grid(n->d);
    for (int l = 0; l < NLAYER; l++) {
        const float *bias = n->param + n->off_b[l];
        if (l + 1 < NLAYER)
            conv_tiled_kernel<2, 0><<<grid, TWARPS * 32, tiled_smem_bytes<2>(), n->stream>>>(
                n->d, n->act[l], n->wf[l], bias, nullptr, n->act[l + 1], nullptr, done);
        else
            conv_tiled_kernel<1, 1><<<grid, TWARPS * 32, tiled_smem_bytes<1>(), n->stream>>>(
                n->d, n->act[l], n->wf[l], bias, nullptr, nullptr, n->out, done);
        NET_LAUNCHED(n);
    }
    return SIM_OK;
}

// gradients of the MSE loss of the last forward pass into n->grad; loss into n->dloss
static sim_status net_backward(sim_net_t *n, const float *target) {
    const int N = n->d.N;
    mse_kernel<<<n->lblk, 128, 0, n->stream>>>(N, n->out, target, (uint16_t *)n->g0, n->lpart);
    NET_LAUNCHED(n);
    mse_fold_kernel<<<1, 32, 0, n->stream>>>(n->lblk, N, n->lpart, n->dloss);
    NET_LAUNCHED(n);
    uint32_t *gcur = n->g0, *gnext = n->g1;
    for (int l = NLAYER - 1; l >= 0; l--) {
        const int NT = COUT[l] > 8 ? 2 : 1;
        dim3 grid(n->nchunk, 27);
        if (NT == 2) wgrad_kernel<2><<<grid, 128, 0, n->stream>>>(n->d, (const uint16_t *)n->act[l], (const uint16_t *)gcur, n->chunk, n->wpart);
        else wgrad_kernel<1><<<grid, 128, 0, n->stream>>>(n->d, (const uint16_t *)n->act[l], (const uint16_t *)gcur, n->chunk, n->wpart);
        NET_LAUNCHED(n);
        const int ne = 27 * CIN[l] * COUT[l];
        if (NT == 2) wgrad_fold_kernel<2><<<sim_blocks(ne), SIM_THREADS, 0, n->stream>>>(n->nchunk, CIN[l], COUT[l], n->wpart, n->grad + n->off_w[l]);
        else wgrad_fold_kernel<1><<<sim_blocks(ne), SIM_THREADS, 0, n->stream>>>(n->nchunk, CIN[l], COUT[l], n->wpart, n->grad + n->off_w[l]);
        NET_LAUNCHED(n);
        bgrad_kernel<<<n->bblk, 128, 0, n->stream>>>(N, COUT[l], (const uint16_t *)gcur, n->bpart);
        NET_LAUNCHED(n);
        bgrad_fold_kernel<<<1, 32, 0, n->stream>>>(n->bblk, COUT[l], n->bpart, n->grad + n->off_b[l]);
        NET_LAUNCHED(n);
        if (l > 0) {   // data gradient through layer l into the ReLU output of layer l-1
            conv_tiled_kernel<2, 2><<<tiled_grid(n->d), TWARPS * 32, tiled_smem_bytes<2>(), n->stream>>>(
                n->d, gcur, n->wb[l], nullptr, n->act[l], gnext, nullptr, nullptr);
            NET_LAUNCHED(n);
            uint32_t *t = gcur; gcur = gnext; gnext = t;
        }
    }
    return SIM_OK;
}

extern "C" {

sim_status sim_net_create(int32_t nx, int32_t ny, int32_t nz, uint64_t seed, void *cuda_stream, sim_net_t **out) {
    if (!out) return SIM_EINVAL;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz > 0x7fffffffLL / 32)
        return sim_fail(nullptr, SIM_EINVAL, "sim_net_create: bad grid");
    sim_net_t *n = new sim_net_t();
    n->d.nx = nx; n->d.ny = ny; n->d.nz = nz; n->d.N = nx * ny * nz;
    if (cuda_stream) n->stream = (cudaStream_t)cuda_stream;
    else {
        if (cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete n;
            return sim_fail(nullptr, SIM_ECUDA, "sim_net_create: cannot create a stream");
        }
        n->own_stream = true;
    }
    int64_t off = 0;
    for (int l = 0; l < NLAYER; l++) {
        n->off_w[l] = off; off += 27LL * CIN[l] * COUT[l];
        n->off_b[l] = off; off += COUT[l];
    }
    n->nparam = off;
    const int N = n->d.N;
    bool ok = true;
    auto A = [&](size_t b) -> void * { void *p = ok ? net_alloc(n, b) : nullptr; if (!p) ok = false; return p; };
    n->param = (float *)A(sizeof(float) * off);
    n->grad = (float *)A(sizeof(float) * off);
    n->adam_m = (float *)A(sizeof(float) * off);
    n->adam_v = (float *)A(sizeof(float) * off);
    for (int l = 0; l < NLAYER; l++) {
        n->wf[l] = (uint32_t *)A(sizeof(uint32_t) * 27 * 2 * 64);
        n->wb[l] = (uint32_t *)A(sizeof(uint32_t) * 27 * 2 * 64);
    }
    for (int l = 0; l <= NLAYER; l++) n->act[l] = (uint32_t *)A(sizeof(uint32_t) * 8 * (size_t)N);
    n->out = (float *)A(sizeof(float) * N);
    n->g0 = (uint32_t *)A(sizeof(uint32_t) * 8 * (size_t)N);
    n->g1 = (uint32_t *)A(sizeof(uint32_t) * 8 * (size_t)N);
    n->chunk = 4096;
    n->nchunk = (N + n->chunk - 1) / n->chunk;
    n->wpart = (float *)A(sizeof(float) * 27 * (size_t)n->nchunk * 16 * 16);
    n->bblk = 256;
    n->bpart = (float *)A(sizeof(float) * n->bblk * 16);
    n->lblk = 256;
    n->lpart = (double *)A(sizeof(double) * n->lblk);
    n->dloss = (double *)A(sizeof(double) * 2);
    if (!ok) {
        std::string m = n->msg;
        sim_net_destroy(n);
        return sim_fail(nullptr, SIM_ENOMEM, "sim_net_create: " + m);
    }
    // He-normal initial weights from a splitmix64 stream (host), zero biases
    std::vector<float> h(off, 0.f);
    uint64_t st = seed;
    auto next = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ULL);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return ((z ^ (z >> 31)) >> 11) * (1.0 / 9007199254740992.0) + 0.5 / 9007199254740992.0;
    };
    for (int l = 0; l < NLAYER; l++) {
        const double sd = std::sqrt(2.0 / (27.0 * CIN[l]));
        for (int64_t k = 0; k < 27LL * CIN[l] * COUT[l]; k++) {
            const double u1 = next(), u2 = next();
            h[n->off_w[l] + k] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2));
        }
    }
    if (cudaMemcpy(n->param, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(n->adam_m, 0, sizeof(float) * off) != cudaSuccess ||
        cudaMemset(n->adam_v, 0, sizeof(float) * off) != cudaSuccess || pack_all(n) != SIM_OK) {
        sim_net_destroy(n);
        return sim_fail(nullptr, SIM_ECUDA, "sim_net_create: initialisation failed");
    }
    *out = n;
    return SIM_OK;
}

void sim_net_destroy(sim_net_t *n) {
    if (!n) return;
    if (n->stream) cudaStreamSynchronize(n->stream);
    for (void *p : n->allocs) cudaFree(p);
    if (n->own_stream && n->stream) cudaStreamDestroy(n->stream);
    delete n;
}

int64_t sim_net_param_count(sim_net_t *n) { return n ? n->nparam : 0; }
const char *sim_net_last_error(sim_net_t *n) { return n ? n->msg.c_str() : ""; }

sim_status sim_net_set_params(sim_net_t *n, const float *params) {
    if (!n || !params) return SIM_EINVAL;
    NET_CK(n, cudaMemcpyAsync(n->param, params, sizeof(float) * n->nparam, cudaMemcpyHostToDevice, n->stream));
    if (pack_all(n) != SIM_OK) return n->err;
    NET_CK(n, cudaStreamSynchronize(n->stream));
    return SIM_OK;
}

sim_status sim_net_get_params(sim_net_t *n, float *params) {
    if (!n || !params) return SIM_EINVAL;
    NET_CK(n, cudaMemcpyAsync(params, n->param, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost, n->stream));
    NET_CK(n, cudaStreamSynchronize(n->stream));
    return SIM_OK;
}

sim_status sim_net_forward(sim_net_t *n, const float *x_dev, float *y_dev) {
    if (!n || !x_dev || !y_dev) return SIM_EINVAL;
    if (n->err != SIM_OK) return n->err;
    features_kernel<<<sim_blocks(n->d.N), SIM_THREADS, 0, n->stream>>>(n->d.N, x_dev, n->act[0], nullptr);
    NET_LAUNCHED(n);
    if (net_forward(n) != SIM_OK) return n->err;
    NET_CK(n, cudaMemcpyAsync(y_dev, n->out, sizeof(float) * n->d.N, cudaMemcpyDeviceToDevice, n->stream));
    return SIM_OK;
}

sim_status sim_net_loss_grad(sim_net_t *n, const float *x_dev, const float *target_dev, double *loss, float *grads) {
    if (!n || !x_dev || !target_dev) return SIM_EINVAL;
    if (n->err != SIM_OK) return n->err;
    features_kernel<<<sim_blocks(n->d.N), SIM_THREADS, 0, n->stream>>>(n->d.N, x_dev, n->act[0], nullptr);
    NET_LAUNCHED(n);
    if (net_forward(n) != SIM_OK || net_backward(n, target_dev) != SIM_OK) return n->err;
    double l = 0.0;
    NET_CK(n, cudaMemcpyAsync(&l, n->dloss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    if (grads) NET_CK(n, cudaMemcpyAsync(grads, n->grad, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost, n->stream));
    NET_CK(n, cudaStreamSynchronize(n->stream));
    if (loss) *loss = l;
    return SIM_OK;
}

sim_status sim_net_train_step(sim_net_t *n, const float *x_dev, const float *target_dev, float lr, double *loss) {
    if (!n || !x_dev || !target_dev) return SIM_EINVAL;
    if (n->err != SIM_OK) return n->err;
    features_kernel<<<sim_blocks(n->d.N), SIM_THREADS, 0, n->stream>>>(n->d.N, x_dev, n->act[0], nullptr);
    NET_LAUNCHED(n);
    if (net_forward(n) != SIM_OK || net_backward(n, target_dev) != SIM_OK) return n->err;
    n->adam_t++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)n->adam_t), c2 = 1.f - std::pow(b2, (float)n->adam_t);
    adam_kernel<<<sim_blocks(n->nparam), SIM_THREADS, 0, n->stream>>>((int)n->nparam, n->param, n->grad, n->adam_m,
                                                                      n->adam_v, lr, b1, b2, 1e-8f, c1, c2);
    NET_LAUNCHED(n);
    if (pack_all(n) != SIM_OK) return n->err;
    if (loss) {
        NET_CK(n, cudaMemcpyAsync(loss, n->dloss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
        NET_CK(n, cudaStreamSynchronize(n->stream));
    }
    return SIM_OK;
}

}  // extern "C"

// inference inside the CPR preconditioner: features x [N][4] -> y [N], on the
// caller's stream, every kernel skipping its work once *done is set
sim_status net_infer(sim_net_t *n, const float *x_dev, float *y_dev, cudaStream_t st, const int *done) {
    cudaStream_t keep = n->stream;
    n->stream = st;
    features_kernel<<<sim_blocks(n->d.N), SIM_THREADS, 0, st>>>(n->d.N, x_dev, n->act[0], done);
    n->launches++;
    sim_status r = net_forward(n, done);
    if (r == SIM_OK && cudaMemcpyAsync(y_dev, n->out, sizeof(float) * n->d.N, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        r = SIM_ECUDA;
    n->stream = keep;
    return r;
}
int64_t net_launches(sim_net_t *n) { return n ? n->launches : 0; }
int net_cells(sim_net_t *n) { return n ? n->d.N : 0; }
