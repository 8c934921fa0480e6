// Learned pressure stage: a 3-D convolutional network on the grid, trained on
// the device by hand-written BF16 tensor-core kernels (FP32 accumulation).
//
// Network: 4 layers of 3x3x3 convolutions (zero padding, stride 1) with
// channels 4 -> 16 -> 16 -> 16 -> 1, ReLU between layers.  Input features per
// cell: the normalised pressure residual and three standardised log face
// transmissibility sums; output: a pressure correction (normalised).
//
// Convolution as implicit GEMM, BF16 x BF16 -> FP32:
//   forward / data gradient on tcgen05.mma with the accumulators in tensor
//   memory and the input staged by TMA (conv_tc_kernel): M = 128 cells of an
//   x-row, K = 16 channels of one tap, N = 16 outputs x up to 3 taps along z;
//   weight gradient on mma.sync.m16n8k16: M = 16 input channels, N = output
//   channels, K = cells (a training-only kernel; its (tap, channel) rows have
//   no uniform shared-memory stride, which the tcgen05 operand layouts need).
// Activations are stored channels-innermost as BF16 [N][16] (pairs of channels
// per 32-bit word).
// Reductions over cells (weight and bias gradients, loss) are written as
// per-block partials and folded in block order: results do not depend on
// scheduling.
#include <cuda.h>
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
// forward convolution / data gradient on the 5th-generation tensor cores
// (tcgen05.mma kind::f16, BF16 x BF16 -> FP32 accumulators in tensor memory)
//   MODE 0: out = bf16(relu(acc))        hidden layer forward (acc starts at the bias)
//   MODE 1: outf[c] = acc[channel 0]     last layer forward (acc starts at bias[0])
//   MODE 2: out = bf16(acc * (mask > 0)) data gradient into a ReLU layer
//
// Implicit GEMM per output line (an x-row of 128 cells at fixed y, z):
//   D[x][o] += sum_k In[x + dx, y + dy, z + dz][k] * B_t[k][o]   over 27 taps t.
// One CTA owns 128 x TC_TY x TC_TZ output cells.  TMA stages the input lines
// (y0-1 .. y0+TC_TY, z0-1 .. z0+TC_TZ, x0-1 .. x0+128) into shared memory as two
// planes, channels 0-7 and 8-15, 16 bytes per cell: that is the no-swizzle
// K-major core-matrix layout (8 rows x 16 bytes per core matrix, the two
// K halves one plane apart), so the A operand for any x-shift dx is the same
// lines read from a start address 16 (dx + 1) bytes further on.  Out-of-grid
// cells come in as zeros from the TMA bounds fill (the zero padding).
// One staged line (y_s, z_s) with fixed (dy, dx) feeds the three output lines
// z' = z_s - dz, dz = +1, 0, -1, whose accumulators sit side by side in tensor
// memory: a single MMA with N = 48 (fewer at the z edges) does all three taps,
// its B operand the three tap matrices stacked along N.
// One thread issues the TMA copies and the MMAs; all four warps initialise the
// accumulators and run the epilogue (lane = cell).  Every wait is bounded: on a
// timeout the kernel sets bit 0 (staging) or bit 1 (MMA) of *status, waits
// once more, bounded, for its copies and MMAs, frees its tensor memory and
// skips the epilogue; a staging buffer off the 128-byte alignment the TMA
// needs sets bit 2, and nothing is copied or multiplied.
// ---------------------------------------------------------------------------
constexpr int TC_M = 128;                                  // cells along x per output line
constexpr int TC_TY = 2, TC_TZ = 8;                        // output lines per CTA (y, z)
constexpr int TC_SY = TC_TY + 2, TC_SZ = TC_TZ + 2;        // staged lines (y, z)
constexpr int TC_LINE = (TC_M + 2) * 16;                   // bytes of one staged line, one channel half
constexpr int TC_BOX = TC_SZ * TC_LINE;                    // bytes of one TMA box: one staged y, TC_SZ lines
constexpr int TC_SLAB = (TC_BOX + 127) / 128 * 128;        // its stride: TMA destinations are 128-byte aligned
constexpr int TC_PLANE = TC_SY * TC_SLAB;                  // one channel half of the staged brick
constexpr int TC_WROWS = 48;                               // B rows per (dy, dx): 3 taps x 16 outputs
constexpr int TC_WELEMS = 9 * 2 * TC_WROWS * 8;            // BF16 elements of the packed weights
constexpr int TC_WBYTES = TC_WELEMS * 2;
constexpr int TC_COLS = TC_TY * TC_TZ * 16;                // FP32 accumulator columns in tensor memory
constexpr int TC_SMEM = 2 * TC_PLANE + TC_WBYTES + 128;    // + alignment slack
static_assert(TC_COLS == 256, "tensor-memory allocation must be a power of two >= 32");
static_assert(TC_SMEM <= 227 * 1024, "shared memory per CTA");
static_assert((TC_LINE % 16) == 0 && (TC_SLAB % 128) == 0 && (TC_PLANE % 128) == 0 && (TC_PLANE >> 4) < (1 << 14),
              "TMA destination alignment and descriptor fields");

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major; lbo = byte distance of
// the two K halves (core matrices adjacent in K), sbo = distance of 8-row groups
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor, kind::f16: FP32 accumulate, A and B BF16, both K-major
__device__ __forceinline__ uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc) {
    asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;\n" ::"r"(d), "l"(a), "l"(b), "r"(idesc));
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// bounded wait for phase `parity` of an mbarrier (about 2 s of SM clock)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > 4000000000LL) return false;
    }
}
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_addr(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

template <int MODE>
__global__ void __launch_bounds__(128, 1) conv_tc_kernel(const __grid_constant__ CUtensorMap tin, Dims d,
                                                         const uint16_t *__restrict__ wtc,
                                                         const float *__restrict__ bias,
                                                         const uint32_t *__restrict__ mask, uint32_t *__restrict__ out,
                                                         float *__restrict__ outf, const int *done,
                                                         int *__restrict__ status) {
    if (done != nullptr && *(volatile const int *)done) return;
    extern __shared__ uint8_t tc_raw[];
    __shared__ uint64_t bar_slab[TC_SY];
    __shared__ uint64_t bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ int issue_ok;
    uint8_t *sA = tc_raw + ((128u - (smem_addr(tc_raw) & 127u)) & 127u);
    uint8_t *sW = sA + 2 * TC_PLANE;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.x * TC_M, y0 = blockIdx.y * TC_TY, z0 = blockIdx.z * TC_TZ;
    if (tid == 0) {
        for (int s = 0; s < TC_SY; s++) mbar_init(&bar_slab[s], 1);
        mbar_init(&bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        issue_ok = 1;
    }
    __syncthreads();
    if (tid == 0) {   // staged y slab s = y0 - 1 + s, both channel halves, lines z0-1 .. z0+TC_TZ, cells x0-1 ..
        if ((smem_addr(sA) & 127u) != 0u) {   // TMA destinations must be 128-byte aligned: copy nothing
            atomicOr(status, 4);
            issue_ok = 0;
        } else {
            for (int s = 0; s < TC_SY; s++) {
                mbar_expect(&bar_slab[s], 2 * TC_BOX);
                for (int h = 0; h < 2; h++)
                    tma_load_4d(sA + h * TC_PLANE + s * TC_SLAB, &tin, 8 * h, x0 - 1, y0 - 1 + s, z0 - 1, &bar_slab[s]);
            }
        }
    }
    for (int i = tid; i < TC_WBYTES / 16; i += 128) ((uint4 *)sW)[i] = ((const uint4 *)wtc)[i];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // weights: generic writes -> tensor-core reads
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(TC_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tb = tmem_base;
    const uint32_t lane_base = tb + ((uint32_t)(warp * 32) << 16);
    {   // accumulators start at the bias (forward) or zero (data gradient)
        uint32_t v[16];
#pragma unroll
        for (int j = 0; j < 16; j++)
            v[j] = __float_as_uint(MODE == 0 ? bias[j] : (MODE == 1 && j == 0 ? bias[0] : 0.0f));
        for (int l = 0; l < TC_TY * TC_TZ; l++) tc_st16(lane_base + l * 16, v);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_addr(sA), w0 = smem_addr(sW);
        int s = issue_ok ? 0 : TC_SY;
        for (; s < TC_SY; s++) {
            if (!mbar_wait(&bar_slab[s], 0)) break;
            const int ys = s - 1;   // staged y relative to y0
            for (int dy = -1; dy <= 1; dy++) {
                const int yo = ys - dy;   // output line it feeds
                if (yo < 0 || yo >= TC_TY) continue;
                for (int dx = -1; dx <= 1; dx++) {
                    const uint32_t wcb = w0 + ((dy + 1) * 3 + (dx + 1)) * (2 * TC_WROWS * 16);
                    for (int zs = -1; zs <= TC_TZ; zs++) {
                        const int zlo = max(0, zs - 1), zhi = min(TC_TZ - 1, zs + 1);
                        const int j0 = zlo - zs + 1;   // B block of the first output line: 0 dz=+1, 1 dz=0, 2 dz=-1
                        const uint64_t ad =
                            tc_sdesc(a0 + s * TC_SLAB + ((zs + 1) * (TC_M + 2) + dx + 1) * 16, TC_PLANE, 128);
                        const uint64_t bd = tc_sdesc(wcb + j0 * 256, TC_WROWS * 16, 128);
                        tc_mma(tb + (uint32_t)((yo * TC_TZ + zlo) * 16), ad, bd, tc_idesc(TC_M, (zhi - zlo + 1) * 16));
                    }
                }
            }
        }
        tc_commit(&bar_mma);   // arrives once every MMA issued above has completed
        if (issue_ok && s < TC_SY) {   // staging timed out: let the copies in flight land before the CTA exits
            issue_ok = 0;
            atomicOr(status, 1);
            for (; s < TC_SY; s++) mbar_wait(&bar_slab[s], 0);
        }
    }
    __syncwarp();
    bool ok = mbar_wait(&bar_mma, 0);
    if (!ok) {
        atomicOr(status, 2);
        mbar_wait(&bar_mma, 0);
    }
    __syncthreads();
    tc_fence_after();
    if (ok && issue_ok) {
        const int x = x0 + warp * 32 + lane;
        for (int l = 0; l < TC_TY * TC_TZ; l++) {
            uint32_t r[16];
            tc_ld16(lane_base + l * 16, r);
            const int Y = y0 + l / TC_TZ, Z = z0 + l % TC_TZ;
            if (x >= d.nx || Y >= d.ny || Z >= d.nz) continue;
            const long c = (long)x + (long)d.nx * (Y + (long)d.ny * Z);
            if (MODE == 1) {
                outf[c] = __uint_as_float(r[0]);
                continue;
            }
            uint32_t o[8];
            if (MODE == 0) {
#pragma unroll
                for (int k = 0; k < 8; k++)
                    o[k] = pack_bf16(fmaxf(__uint_as_float(r[2 * k]), 0.f), fmaxf(__uint_as_float(r[2 * k + 1]), 0.f));
            } else {
                const uint4 m0 = ((const uint4 *)(mask + c * 8))[0], m1 = ((const uint4 *)(mask + c * 8))[1];
                const uint32_t mk[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
                for (int k = 0; k < 8; k++)
                    o[k] = pack_bf16(bf16_lo(mk[k]) > 0.f ? __uint_as_float(r[2 * k]) : 0.f,
                                     bf16_hi(mk[k]) > 0.f ? __uint_as_float(r[2 * k + 1]) : 0.f);
            }
            uint4 *dst = (uint4 *)(out + c * 8);
            dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
            dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tb), "r"(TC_COLS) : "memory");
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

// pack FP32 weights W[27][cin][cout] into the B operand of conv_tc_kernel:
// BF16 [9 (dy, dx)][2 K halves][48 rows n = 16 j + o][8 k], rows j = 0, 1, 2
// holding the taps dz = +1, 0, -1 of that (dy, dx); tap t = 9 (dz + 1) + 3 (dy + 1) + (dx + 1).
// transpose = 0: forward        B_t[k = ci][o = co] = W[t][ci][co]
// transpose = 1: data gradient  B_t[k = co][o = ci] = W[26 - t][ci][co]   (offsets negated)
__global__ void pack_tc_kernel(int cin, int cout, int transpose, const float *__restrict__ W, uint16_t *__restrict__ wtc) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= TC_WELEMS) return;
    const int kk = e % 8, n = (e / 8) % TC_WROWS, h = (e / (8 * TC_WROWS)) % 2, cb = e / (16 * TC_WROWS);
    const int j = n / 16, o = n % 16, k = 8 * h + kk;
    const int t = 9 * (2 - j) + cb;   // dz + 1 = 2 - j
    float v = 0.f;
    if (!transpose) {
        if (k < cin && o < cout) v = W[((long)t * cin + k) * cout + o];
    } else {
        if (o < cin && k < cout) v = W[((long)(26 - t) * cin + o) * cout + k];
    }
    wtc[e] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
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
    uint16_t *wf[NLAYER], *wb[NLAYER];   // packed forward / data-gradient weights (conv_tc_kernel B operand)
    uint32_t *act[NLAYER + 1];           // BF16 [N][16]: input features, hidden activations
    CUtensorMap map_act[NLAYER];         // TMA maps of act[0..3] (inputs of the forward layers)
    CUtensorMap map_g[2];                // TMA maps of g0, g1 (inputs of the data gradients)
    int *dstat = nullptr;                // device status word of the convolutions (bounded waits)
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

// the convolutions' status word, read after the stream has drained: non-zero
// means a bounded wait inside a convolution gave up (its output was skipped)
static sim_status net_status(sim_net_t *n) {
    int st = 0;
    NET_CK(n, cudaMemcpyAsync(&st, n->dstat, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
    NET_CK(n, cudaStreamSynchronize(n->stream));
    if (st != 0) return net_fail(n, SIM_ETIMEOUT, "convolution: a bounded wait gave up (status " + std::to_string(st) + ")");
    return SIM_OK;
}

static void *net_alloc(sim_net_t *n, size_t bytes) {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) { net_fail(n, SIM_ENOMEM, "cudaMalloc failed"); return nullptr; }
    n->allocs.push_back(p);
    return p;
}

static sim_status pack_all(sim_net_t *n) {
    for (int l = 0; l < NLAYER; l++) {
        pack_tc_kernel<<<sim_blocks(TC_WELEMS), SIM_THREADS, 0, n->stream>>>(CIN[l], COUT[l], 0, n->param + n->off_w[l], n->wf[l]);
        NET_LAUNCHED(n);
        pack_tc_kernel<<<sim_blocks(TC_WELEMS), SIM_THREADS, 0, n->stream>>>(CIN[l], COUT[l], 1, n->param + n->off_w[l], n->wb[l]);
        NET_LAUNCHED(n);
    }
    return SIM_OK;
}

// TMA map of a BF16 [N][16] activation buffer as the 4-D tensor (channel, x, y, z);
// one box is one channel half of a staged y slab: 8 x (128 + 2) x 1 x (TC_TZ + 2)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return (EncodeTiledFn)f;
    }();
    return fn;
}
static bool act_map(const Dims &d, void *buf, CUtensorMap *map) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t dims[4] = {16, (cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz};
    const cuuint64_t strides[3] = {32, (cuuint64_t)d.nx * 32, (cuuint64_t)d.nx * d.ny * 32};
    const cuuint32_t box[4] = {8, TC_M + 2, 1, TC_SZ}, estr[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

static dim3 tc_grid(const Dims &d) {
    return dim3((d.nx + TC_M - 1) / TC_M, (d.ny + TC_TY - 1) / TC_TY, (d.nz + TC_TZ - 1) / TC_TZ);
}

// once per process: the convolution needs more than the default 48 KB of shared memory
static bool tc_attrs() {
    static const bool ok = [] {
        return cudaFuncSetAttribute(conv_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM) == cudaSuccess &&
               cudaFuncSetAttribute(conv_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM) == cudaSuccess &&
               cudaFuncSetAttribute(conv_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM) == cudaSuccess;
    }();
    return ok;
}

static sim_status net_forward(sim_net_t *n, const int *done = nullptr) {
    if (!tc_attrs()) return net_fail(n, SIM_ECUDA, "convolution kernel attributes");
    const dim3 grid = tc_grid(n->d);
    for (int l = 0; l < NLAYER; l++) {
        const float *bias = n->param + n->off_b[l];
        if (l + 1 < NLAYER)
            conv_tc_kernel<0><<<grid, 128, TC_SMEM, n->stream>>>(n->map_act[l], n->d, n->wf[l], bias, nullptr,
                                                                 n->act[l + 1], nullptr, done, n->dstat);
        else
            conv_tc_kernel<1><<<grid, 128, TC_SMEM, n->stream>>>(n->map_act[l], n->d, n->wf[l], bias, nullptr, nullptr,
                                                                 n->out, done, n->dstat);
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
    if (!tc_attrs()) return net_fail(n, SIM_ECUDA, "convolution kernel attributes");
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
            conv_tc_kernel<2><<<tc_grid(n->d), 128, TC_SMEM, n->stream>>>(n->map_g[gcur == n->g0 ? 0 : 1], n->d, n->wb[l],
                                                                          nullptr, n->act[l], gnext, nullptr, nullptr, n->dstat);
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
        n->wf[l] = (uint16_t *)A(TC_WBYTES);
        n->wb[l] = (uint16_t *)A(TC_WBYTES);
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
    n->dstat = (int *)A(sizeof(int));
    if (!ok) {
        std::string m = n->msg;
        sim_net_destroy(n);
        return sim_fail(nullptr, SIM_ENOMEM, "sim_net_create: " + m);
    }
    bool maps = true;
    for (int l = 0; l < NLAYER; l++) maps = maps && act_map(n->d, n->act[l], &n->map_act[l]);
    maps = maps && act_map(n->d, n->g0, &n->map_g[0]) && act_map(n->d, n->g1, &n->map_g[1]);
    if (!maps) {
        sim_net_destroy(n);
        return sim_fail(nullptr, SIM_ECUDA, "sim_net_create: cannot encode the TMA maps of the activations");
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
        cudaMemset(n->adam_v, 0, sizeof(float) * off) != cudaSuccess || cudaMemset(n->dstat, 0, sizeof(int)) != cudaSuccess ||
        pack_all(n) != SIM_OK) {
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
    return net_status(n);
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
    return net_status(n);
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
    if (loss) NET_CK(n, cudaMemcpyAsync(loss, n->dloss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    return net_status(n);
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
int net_status_word(sim_net_t *n, cudaStream_t st) {
    int v = 0;
    if (!n) return 0;
    if (cudaMemcpyAsync(&v, n->dstat, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return -1;
    return v;
}
int net_cells(sim_net_t *n) { return n ? n->d.N : 0; }
