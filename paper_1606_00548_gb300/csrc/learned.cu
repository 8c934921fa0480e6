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
// Activations are BF16, 16 channels per cell, stored as two planes of 8
// channels (16 bytes per cell; see Dims).
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

// Grid and activation layout.  Activations (and their gradients) are BF16,
// 16 channels per cell, stored as two planes -- channels 0-7, then 8-15 --
// of nxp x ny x nz cells, 16 bytes per cell, x padded to nxp (a multiple of 8)
// with cells that stay zero: a TMA box row is then 8 cells (128 bytes), and a
// plane is the shared-memory operand layout of the convolution as it stands.
struct Dims {
    int nx, ny, nz, N;
    int nxp;    // nx rounded up to a multiple of 8
    long P;     // cells of one plane: nxp * ny * nz
};
// BF16 element offset of channel ch of cell (x, y, z)
__device__ __forceinline__ long act_elem(const Dims &d, int x, int y, int z, int ch) {
    return ((long)(ch >> 3) * d.P + (long)x + (long)d.nxp * (y + (long)d.ny * z)) * 8 + (ch & 7);
}
// the same for the cell of compact index c = x + nx (y + ny z)
__device__ __forceinline__ long act_elem_c(const Dims &d, int c, int ch) {
    const int x = c % d.nx, q = c / d.nx;
    return act_elem(d, x, q % d.ny, q / d.ny, ch);
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
// Work unit: a brick of 128 x TC_TY x TC_TZ output cells.  Its input is TC_SY
// staged slabs (one y each: lines z0-1 .. z0+TC_TZ, cells x0-8 .. x0+135),
// each loaded by TMA from the two activation planes (rows of 8 cells, 128
// bytes): in shared memory a plane is the no-swizzle K-major core-matrix layout
// (8 rows x 16 bytes per core matrix, the two K halves one plane apart), so the
// A operand for any x-shift dx is the same lines read from a start address
// 16 (dx + 8) bytes further on.  Out-of-grid cells are zeros: the TMA bounds
// fill, and the zero cells that pad x to a multiple of 8.
// One staged line (y_s, z_s) with fixed (dy, dx) feeds the three output lines
// z' = z_s - dz, dz = +1, 0, -1, whose accumulators sit side by side in tensor
// memory: a single MMA with N = 48 (fewer at the z edges) does all three taps,
// its B operand the three tap matrices stacked along N.
//
// Persistent and warp-specialised, one CTA per SM, bricks dealt round-robin:
//   warp 0     TMA producer: slabs into a ring of TC_RING buffers
//   warp 1     tensor-memory owner and MMA issuer: 180 MMAs per brick from
//              precomputed descriptors; each slab's buffer is released by a
//              tcgen05.commit once the MMAs reading it are done
//   warps 2-5  epilogue (one lane = one cell of the 128): drains a brick's
//              accumulators, writes the outputs, and re-seeds the columns with
//              the bias for the brick after next
// Two accumulator buffers of TC_ACC columns let the epilogue of one brick
// overlap the MMAs of the next.  Every wait is bounded: on a timeout the CTA
// sets bit 0 (producer), 1 (MMA) or 3 (epilogue) of *status, stops all its
// roles, lets its copies and MMAs in flight land, frees its tensor memory and
// exits; a staging ring off the 128-byte alignment the TMA needs sets bit 2,
// and nothing is copied or multiplied.  stall_slab >= 0 (a testing hook, -1
// otherwise) makes CTA 0 skip the copy of that slab of its sequence without
// arming its barrier, so that the MMA thread's bounded wait runs out.
// ---------------------------------------------------------------------------
constexpr int TC_M = 128;                                  // cells along x per output line
constexpr int TC_TY = 2, TC_TZ = 8;                        // output lines per brick (y, z)
constexpr int TC_SY = TC_TY + 2, TC_SZ = TC_TZ + 2;        // staged slabs per brick, lines per slab
constexpr int TC_XS = TC_M + 16;                           // staged cells per line: x0-8 .. x0+135 (8-cell units)
constexpr int TC_LINE = TC_XS * 16;                        // bytes of one staged line, one channel half
constexpr int TC_BOX = TC_SZ * TC_LINE;                    // bytes of one TMA box: one slab, one half
constexpr int TC_HALF = (TC_BOX + 127) / 128 * 128;        // its stride: TMA destinations are 128-byte aligned
constexpr int TC_SLOT = 2 * TC_HALF;                       // one ring buffer: a slab, both halves
constexpr int TC_RING = 4;                                 // ring buffers
constexpr int TC_WROWS = 48;                               // B rows per (dy, dx): 3 taps x 16 outputs
constexpr int TC_WELEMS = 9 * 2 * TC_WROWS * 8;            // BF16 elements of the packed weights
constexpr int TC_WBYTES = TC_WELEMS * 2;
constexpr int TC_ACC = TC_TY * TC_TZ * 16;                 // FP32 accumulator columns of one brick
constexpr int TC_COLS = 2 * TC_ACC;                        // two bricks in flight
constexpr int TC_THREADS = 192;
constexpr int TC_SMEM = TC_RING * TC_SLOT + TC_WBYTES + 128;   // + alignment slack
static_assert(TC_COLS == 512, "tensor-memory allocation: a power of two >= 32, at most 512");
static_assert((TC_TY * TC_TZ) % 4 == 0, "the epilogue reads four output lines per tensor-memory load");
static_assert(TC_SMEM <= 227 * 1024, "shared memory per CTA");
static_assert((TC_LINE % 128) == 0 && (TC_HALF % 128) == 0 && (TC_SLOT % 128) == 0 && (TC_HALF >> 4) < (1 << 14),
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
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// bounded wait for phase `parity` of an mbarrier (about 2 s of SM clock).  It
// gives up early once *abort is set; on its own timeout it sets *abort and
// the status bit, so that every role of the CTA stops.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort, int *status, int bit) {
    const long long t0 = clock64();
    for (;;) {
        if (mbar_test(bar, parity)) return true;
        if (*abort) return false;
        if (clock64() - t0 > 4000000000LL) {
            *abort = 1;
            atomicOr(status, bit);
            return false;
        }
    }
}
// the same without the early exit: used to let copies and MMAs in flight land
// before the CTA frees its tensor memory and exits
__device__ __forceinline__ bool mbar_drain(uint64_t *bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > 4000000000LL) return false;
    return true;
}
__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(smem_addr(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 64 consecutive columns (four output lines) of this warp's 32 lanes in one load
__device__ __forceinline__ void tc_ld64(uint32_t taddr, uint32_t (&r)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,"
        "%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,"
        "%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]),
          "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]),
          "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]),
          "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]),
          "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
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

struct TcBars {
    uint64_t full[TC_RING], empty[TC_RING];   // slab buffer: loaded / released
    uint64_t acc_full[2], acc_empty[2];       // accumulator buffer: MMAs done / drained and re-seeded
    uint64_t drain;                           // every MMA of the CTA done
};

template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1) conv_tc_kernel(const __grid_constant__ CUtensorMap tin, Dims d,
                                                                int nbricks, const uint16_t *__restrict__ wtc,
                                                                const float *__restrict__ bias,
                                                                const uint32_t *__restrict__ mask,
                                                                uint32_t *__restrict__ out, float *__restrict__ outf,
                                                                const int *done, int *__restrict__ status,
                                                                int stall_slab) {
    if (done != nullptr && *(volatile const int *)done) return;
    extern __shared__ uint8_t tc_raw[];
    __shared__ TcBars bars;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    volatile int *abort = &abort_flag;
    uint8_t *ring = tc_raw + ((128u - (smem_addr(tc_raw) & 127u)) & 127u);
    uint8_t *sW = ring + TC_RING * TC_SLOT;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gx = (d.nx + TC_M - 1) / TC_M, gy = (d.ny + TC_TY - 1) / TC_TY;
    if (tid == 0) {
        for (int i = 0; i < TC_RING; i++) {
            mbar_init(&bars.full[i], 1);
            mbar_init(&bars.empty[i], 1);
        }
        for (int i = 0; i < 2; i++) {
            mbar_init(&bars.acc_full[i], 1);
            mbar_init(&bars.acc_empty[i], 4);   // one arrival per epilogue warp
        }
        mbar_init(&bars.drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
        if ((smem_addr(ring) & 127u) != 0u) {   // TMA destinations must be 128-byte aligned: do nothing
            abort_flag = 1;
            atomicOr(status, 4);
        }
    }
    for (int i = tid; i < TC_WBYTES / 16; i += TC_THREADS) ((uint4 *)sW)[i] = ((const uint4 *)wtc)[i];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // weights: generic writes -> tensor-core reads
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(TC_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tb = tmem_base;
    int issued = 0;   // producer: slabs whose copies were started
    if (!*abort && warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        for (int br = blockIdx.x; br < nbricks && !*abort; br += gridDim.x) {
            const int bx = br % gx, r = br / gx, by = r % gy, bz = r / gy;
            const int x0 = bx * TC_M, y0 = by * TC_TY, z0 = bz * TC_TZ;
            for (int s = 0; s < TC_SY; s++) {
                const int slot = issued % TC_RING;
                if (!mbar_wait(&bars.empty[slot], ((issued / TC_RING) & 1) ^ 1, abort, status, 1)) break;
                if (blockIdx.x == 0 && issued == stall_slab) {   // testing hook: this slab is never copied
                    issued++;
                    continue;
                }
                mbar_expect(&bars.full[slot], 2 * TC_BOX);
                for (int h = 0; h < 2; h++)
                    tma_load_5d(ring + slot * TC_SLOT + h * TC_HALF, &tin, 0, x0 / 8 - 1, y0 - 1 + s, z0 - 1, h,
                                &bars.full[slot]);
                issued++;
            }
        }
    } else if (!*abort && warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint64_t a_desc0 = tc_sdesc(smem_addr(ring), TC_HALF, 128);
        const uint64_t w_desc0 = tc_sdesc(smem_addr(sW), TC_WROWS * 16, 128);
        const uint32_t id16 = tc_idesc(TC_M, 16), id32 = tc_idesc(TC_M, 32), id48 = tc_idesc(TC_M, 48);
        int q = 0, i = 0;
        for (int br = blockIdx.x; br < nbricks && !*abort; br += gridDim.x, i++) {
            const int ab = i & 1;
            if (!mbar_wait(&bars.acc_empty[ab], (i >> 1) & 1, abort, status, 2)) break;
            tc_fence_after();
            const uint32_t dbase = tb + (uint32_t)(ab * TC_ACC);
            for (int s = 0; s < TC_SY; s++, q++) {
                const int slot = q % TC_RING;
                if (!mbar_wait(&bars.full[slot], (q / TC_RING) & 1, abort, status, 2)) break;
                tc_fence_after();
                const uint64_t abase = a_desc0 + (uint64_t)((slot * TC_SLOT) >> 4);
                const int ys = s - 1;   // staged y relative to the brick
#pragma unroll
                for (int dy = -1; dy <= 1; dy++) {
                    const int yo = ys - dy;   // output line it feeds
                    if (yo < 0 || yo >= TC_TY) continue;
                    const uint32_t dline = dbase + (uint32_t)(yo * TC_TZ * 16);
#pragma unroll
                    for (int dx = -1; dx <= 1; dx++) {
                        const uint64_t bb = w_desc0 + (uint64_t)((((dy + 1) * 3 + (dx + 1)) * (2 * TC_WROWS * 16)) >> 4);
                        const uint64_t aa = abase + (uint64_t)(dx + 8);
#pragma unroll
                        for (int zs = -1; zs <= TC_TZ; zs++) {
                            const int zlo = zs - 1 < 0 ? 0 : zs - 1, zhi = zs + 1 > TC_TZ - 1 ? TC_TZ - 1 : zs + 1;
                            const int nl = zhi - zlo + 1, j0 = zlo - zs + 1;   // B block of z' = zlo: 0 dz=+1, 1 dz=0, 2 dz=-1
                            tc_mma(dline + (uint32_t)(zlo * 16), aa + (uint64_t)((zs + 1) * TC_XS),
                                   bb + (uint64_t)(j0 * 16), nl == 3 ? id48 : nl == 2 ? id32 : id16);
                        }
                    }
                }
                tc_commit(&bars.empty[slot]);   // the buffer is free once these MMAs have read it
            }
            tc_commit(&bars.acc_full[ab]);
        }
    } else if (warp >= 2) {
        // ---------------- epilogue: warps 2-5, lane quarter (warp % 4) ----------------
        const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
        uint32_t seed[16];
#pragma unroll
        for (int j = 0; j < 16; j++)
            seed[j] = __float_as_uint(MODE == 0 ? bias[j] : (MODE == 1 && j == 0 ? bias[0] : 0.0f));
        for (int ab = 0; ab < 2; ab++) {
            for (int l = 0; l < TC_TY * TC_TZ; l++) tc_st16(tb + lane_off + (uint32_t)(ab * TC_ACC + l * 16), seed);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars.acc_empty[ab]);
        }
        int i = 0;
        for (int br = blockIdx.x; br < nbricks && !*abort; br += gridDim.x, i++) {
            const int ab = i & 1;
            const int bx = br % gx, r = br / gx, by = r % gy, bz = r / gy;
            const int x = bx * TC_M + (warp & 3) * 32 + lane, y0 = by * TC_TY, z0 = bz * TC_TZ;
            if (MODE == 2 && x < d.nx) {   // the brick's ReLU masks into L2 while its MMAs run
                for (int l = 0; l < TC_TY * TC_TZ; l++) {
                    const int Y = y0 + l / TC_TZ, Z = z0 + l % TC_TZ;
                    if (Y >= d.ny || Z >= d.nz) continue;
                    const long pc = (long)x + (long)d.nxp * (Y + (long)d.ny * Z);
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(mask + pc * 4));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(mask + (d.P + pc) * 4));
                }
            }
            const bool okw = mbar_wait(&bars.acc_full[ab], (i >> 1) & 1, abort, status, 8);
            if (!__all_sync(0xffffffffu, okw)) break;   // the warp's lanes leave together
            tc_fence_after();
            const uint32_t acc = tb + lane_off + (uint32_t)(ab * TC_ACC);
            for (int l4 = 0; l4 < TC_TY * TC_TZ; l4 += 4) {
                uint4 mk4[4][2];   // data gradient: the group's masks, loaded before the accumulators
                if (MODE == 2) {
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        const int l = l4 + k, Y = y0 + l / TC_TZ, Z = z0 + l % TC_TZ;
                        mk4[k][0] = mk4[k][1] = make_uint4(0u, 0u, 0u, 0u);
                        if (x < d.nx && Y < d.ny && Z < d.nz) {
                            const long pc = (long)x + (long)d.nxp * (Y + (long)d.ny * Z);
                            mk4[k][0] = *(const uint4 *)(mask + pc * 4);
                            mk4[k][1] = *(const uint4 *)(mask + (d.P + pc) * 4);
                        }
                    }
                }
                uint32_t v4[64];
                tc_ld64(acc + (uint32_t)(l4 * 16), v4);   // four lines, one wait
#pragma unroll
                for (int k = 0; k < 4; k++) tc_st16(acc + (uint32_t)((l4 + k) * 16), seed);
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int l = l4 + k;
                    const uint32_t *v = v4 + 16 * k;
                    const int Y = y0 + l / TC_TZ, Z = z0 + l % TC_TZ;
                    if (x >= d.nx || Y >= d.ny || Z >= d.nz) continue;
                    if (MODE == 1) {
                        outf[(long)x + (long)d.nx * (Y + (long)d.ny * Z)] = __uint_as_float(v[0]);
                        continue;
                    }
                    const long pc = (long)x + (long)d.nxp * (Y + (long)d.ny * Z);   // plane cell index
                    uint32_t o[8];
                    if (MODE == 0) {
#pragma unroll
                        for (int w = 0; w < 8; w++)
                            o[w] = pack_bf16(fmaxf(__uint_as_float(v[2 * w]), 0.f), fmaxf(__uint_as_float(v[2 * w + 1]), 0.f));
                    } else {
                        const uint4 m0 = mk4[k][0], m1 = mk4[k][1];
                        const uint32_t mk[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
                        for (int w = 0; w < 8; w++)
                            o[w] = pack_bf16(bf16_lo(mk[w]) > 0.f ? __uint_as_float(v[2 * w]) : 0.f,
                                             bf16_hi(mk[w]) > 0.f ? __uint_as_float(v[2 * w + 1]) : 0.f);
                    }
                    *(uint4 *)(out + pc * 4) = make_uint4(o[0], o[1], o[2], o[3]);
                    *(uint4 *)(out + (d.P + pc) * 4) = make_uint4(o[4], o[5], o[6], o[7]);
                }
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars.acc_empty[ab]);
        }
    }
    __syncwarp();
    // ---------------- drain: nothing in flight when tensor memory is freed ----------------
    if (warp == 1 && lane == 0) {
        tc_commit(&bars.drain);
        if (!mbar_drain(&bars.drain, 0)) atomicOr(status, 2);
    }
    if (warp == 0 && lane == 0 && *abort) {
        for (int k = issued - TC_RING < 0 ? 0 : issued - TC_RING; k < issued; k++)
            if (!(blockIdx.x == 0 && k == stall_slab) && !mbar_drain(&bars.full[k % TC_RING], (k / TC_RING) & 1))
                atomicOr(status, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tb), "r"(TC_COLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// weight gradient: dW[t][ci][co] = sum over cells c of In[c + off(t)][ci] * G[c][co]
// (mma.sync.m16n8k16 BF16 -> FP32; per tap a 16 x 16 product with the cells
// as the contraction: too narrow for the 128-row tcgen05 tile).
// Persistent, two CTAs per SM, bricks of 128 x 1 x WG_TZ cells dealt
// round-robin.  Per brick one thread stages by TMA the three input slabs
// (y-1, y, y+1; lines z0-1 .. z0+WG_TZ; cells x0-8 .. x0+135) and the brick's
// output-gradient lines, both activation planes each, in the rows of 16 bytes
// the activations have; out-of-grid cells arrive as zeros (bounds fill and x
// padding), so no cell is masked.  Warp w owns taps w, w+8, w+16, w+24; per
// 16-cell step it loads the gradient fragment once (ldmatrix.trans: rows are
// cells) and, per tap, the input fragment of the shifted cells, and issues two
// MMAs (output channels 0-7, 8-15).  Accumulators stay in registers across the
// CTA's bricks; each CTA writes one partial [27][16][16], folded in CTA order
// (deterministic).  Waits are bounded (status bit 4 on a timeout).
// ---------------------------------------------------------------------------
constexpr int WG_TZ = 4;                                   // output lines per brick (z)
constexpr int WG_SZ = WG_TZ + 2;                           // staged lines per input slab
constexpr int WG_IBOX = WG_SZ * TC_LINE;                   // one input slab, one plane (TMA box)
constexpr int WG_GBOX = WG_TZ * TC_M * 16;                 // output-gradient lines of a brick, one plane
constexpr int WG_IN = 6 * WG_IBOX;                         // 3 slabs x 2 planes
constexpr int WG_SMEM = WG_IN + 2 * WG_GBOX + 128;
constexpr int WG_THREADS = 256;
static_assert(WG_IBOX % 128 == 0 && WG_GBOX % 128 == 0, "TMA destinations 128-byte aligned");
static_assert(2 * (WG_SMEM + 1024) <= 228 * 1024, "two CTAs per SM");

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__global__ void __launch_bounds__(WG_THREADS, 2) wgrad_tc_kernel(const __grid_constant__ CUtensorMap tin,
                                                                 const __grid_constant__ CUtensorMap tg, Dims d,
                                                                 int nbricks, float *__restrict__ part,
                                                                 int *__restrict__ status) {
    extern __shared__ uint8_t wg_raw[];
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    volatile int *abort = &abort_flag;
    uint8_t *sin = wg_raw + ((128u - (smem_addr(wg_raw) & 127u)) & 127u);
    uint8_t *sg = sin + WG_IN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gx = (d.nx + TC_M - 1) / TC_M;
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = (smem_addr(sin) & 127u) != 0u;
        if (abort_flag) atomicOr(status, 4);
    }
    __syncthreads();
    float acc[4][2][4];
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int h = 0; h < 2; h++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[j][h][q] = 0.f;
    // ldmatrix row of this lane: lanes 8m .. 8m+7 address the rows (cells) of matrix m
    const int mrow = lane & 7, mat = lane >> 3;
    const uint32_t s_in = smem_addr(sin), s_g = smem_addr(sg);
    int it = 0;
    bool in_flight = false;   // thread 0: the current brick's copies were started and not yet waited for
    for (int br = blockIdx.x; br < nbricks && !*abort; br += gridDim.x, it++) {
        const int bx = br % gx, r = br / gx, y = r % d.ny, bz = r / d.ny;
        const int x0 = bx * TC_M, z0 = bz * WG_TZ;
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect(&bar, WG_IN + 2 * WG_GBOX);
            for (int s = 0; s < 3; s++)
                for (int h = 0; h < 2; h++)
                    tma_load_5d(sin + (s * 2 + h) * WG_IBOX, &tin, 0, x0 / 8 - 1, y - 1 + s, z0 - 1, h, &bar);
            for (int h = 0; h < 2; h++) tma_load_5d(sg + h * WG_GBOX, &tg, 0, x0 / 8, y, z0, h, &bar);
            in_flight = true;
        }
        const bool ok = mbar_wait(&bar, it & 1, abort, status, 16);
        if (tid == 0 && ok) in_flight = false;
        if (__syncthreads_or(!ok)) break;   // every thread leaves together: no barrier below waits on one that left
        for (int zo = 0; zo < WG_TZ; zo++) {
            for (int xk = 0; xk < TC_M; xk += 16) {
                // gradient fragment (B, 16 cells x 16 outputs): matrices (plane 0, cells 0-7), (0, 8-15), (1, 0-7), (1, 8-15)
                uint32_t b[4];
                ldsm_x4_t(s_g + (uint32_t)((mat >> 1) * WG_GBOX + ((zo * TC_M + xk + (mat & 1) * 8 + mrow) * 16)), b[0], b[1],
                          b[2], b[3]);
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int t = warp + 8 * j;
                    if (t < 27) {
                        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
                        // input fragment (A, 16 channels x 16 cells) at the shifted cells:
                        // matrices (plane 0, cells 0-7), (1, 0-7), (0, 8-15), (1, 8-15)
                        const int cell = (zo + dz + 1) * TC_XS + xk + dx + 8 + (mat >> 1) * 8 + mrow;
                        uint32_t a[4];
                        ldsm_x4_t(s_in + (uint32_t)(((dy + 1) * 2 + (mat & 1)) * WG_IBOX + cell * 16), a[0], a[1], a[2], a[3]);
                        mma_bf16(acc[j][0], a[0], a[1], a[2], a[3], b[0], b[1]);
                        mma_bf16(acc[j][1], a[0], a[1], a[2], a[3], b[2], b[3]);
                    }
                }
            }
        }
        __syncthreads();   // every warp is done with the buffers before the next brick's copies
    }
    if (tid == 0 && in_flight && !mbar_drain(&bar, it & 1)) atomicOr(status, 16);
    // partial of this CTA: [27][16 ci][16 co]
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int t = warp + 8 * j;
        if (t >= 27) continue;
        float *o = part + ((long)blockIdx.x * 27 + t) * 256;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int co = 8 * h + 2 * t4;
            o[g * 16 + co] = acc[j][h][0];
            o[g * 16 + co + 1] = acc[j][h][1];
            o[(g + 8) * 16 + co] = acc[j][h][2];
            o[(g + 8) * 16 + co + 1] = acc[j][h][3];
        }
    }
}

// dW[t][ci][co] (FP32, logical cin x cout) = sum of the CTAs' partials, in CTA order
__global__ void wgrad_fold_kernel(int nblk, int cin, int cout, const float *__restrict__ part, float *__restrict__ dW) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 27 * cin * cout) return;
    const int tap = e / (cin * cout), r = e % (cin * cout), ci = r / cout, co = r % cout;
    float s = 0.f;
    for (int b = 0; b < nblk; b++) s += part[((long)b * 27 + tap) * 256 + ci * 16 + co];
    dW[e] = s;
}

// bias gradient partials: per block sums of dout channels
__global__ void bgrad_kernel(Dims d, int cout, const uint16_t *__restrict__ dout, float *__restrict__ part) {
    __shared__ float sh[128][16];
    float s[16];
    for (int c = 0; c < 16; c++) s[c] = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += gridDim.x * blockDim.x)
        for (int c = 0; c < cout; c++) s[c] += __uint_as_float(bf16_bits(dout + act_elem_c(d, i, c)) << 16);
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

// MSE loss partials and dL/dy = 2 (y - target) / N into channel 0 of a planar BF16 buffer
__global__ void mse_kernel(Dims d, const float *__restrict__ y, const float *__restrict__ target, uint16_t *__restrict__ dout,
                           double *__restrict__ part) {
    __shared__ double sh[128];
    double s = 0.0;
    const int N = d.N;
    const float scale = 2.0f / (float)N;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const float e = y[i] - target[i];
        s += (double)e * e;
        uint4 *o0 = (uint4 *)(dout + act_elem_c(d, i, 0)), *o1 = (uint4 *)(dout + act_elem_c(d, i, 8));
        *o0 = make_uint4(pack_bf16(e * scale, 0.f), 0u, 0u, 0u);
        *o1 = make_uint4(0u, 0u, 0u, 0u);
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

// FP32 features [N][4] -> planar BF16 activations (channels 4..15 zero)
__global__ void features_kernel(Dims d, const float *__restrict__ x, uint16_t *__restrict__ out, const int *done) {
    if (done != nullptr && *(volatile const int *)done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    uint4 *o0 = (uint4 *)(out + act_elem_c(d, i, 0)), *o1 = (uint4 *)(out + act_elem_c(d, i, 8));
    *o0 = make_uint4(pack_bf16(x[(long)i * 4 + 0], x[(long)i * 4 + 1]), pack_bf16(x[(long)i * 4 + 2], x[(long)i * 4 + 3]), 0u, 0u);
    *o1 = make_uint4(0u, 0u, 0u, 0u);
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
    CUtensorMap map_win[NLAYER];         // act[0..3] with the weight gradient's input box
    CUtensorMap map_wg[2];               // g0, g1 with the weight gradient's output-gradient box
    int *dstat = nullptr;                // device status word of the convolutions (bounded waits)
    int stall_once = -1;                 // testing hook: slab whose copy the next forward pass skips
    float *out = nullptr;                // [N]
    uint32_t *g0 = nullptr, *g1 = nullptr;   // BF16 [N][16] gradient buffers
    float *wpart = nullptr, *bpart = nullptr;
    double *lpart = nullptr, *dloss = nullptr;
    int wg_ctas = 0, bblk = 0, lblk = 0;
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

// activations and gradients start at zero: the cells that pad x are never written
static bool zero_acts(sim_net_t *n, size_t bytes) {
    bool ok = true;
    for (int l = 0; l <= NLAYER; l++) ok = ok && cudaMemset(n->act[l], 0, bytes) == cudaSuccess;
    return ok && cudaMemset(n->g0, 0, bytes) == cudaSuccess && cudaMemset(n->g1, 0, bytes) == cudaSuccess;
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

// TMA map of a planar activation buffer as the 5-D tensor (8 cells x 8 channels,
// x / 8, y, z, plane); one box is one plane of a staged slab: rows of 8 cells
// (128 bytes), TC_XS / 8 rows per line, TC_SZ lines
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
static bool act_map(const Dims &d, void *buf, CUtensorMap *map, int box_x8 = TC_XS / 8, int box_z = TC_SZ) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t dims[5] = {64, (cuuint64_t)d.nxp / 8, (cuuint64_t)d.ny, (cuuint64_t)d.nz, 2};
    const cuuint64_t strides[4] = {128, (cuuint64_t)d.nxp * 16, (cuuint64_t)d.nxp * d.ny * 16, (cuuint64_t)d.P * 16};
    const cuuint32_t box[5] = {64, (cuuint32_t)box_x8, 1, (cuuint32_t)box_z, 1}, estr[5] = {1, 1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

static int tc_bricks(const Dims &d) {
    return ((d.nx + TC_M - 1) / TC_M) * ((d.ny + TC_TY - 1) / TC_TY) * ((d.nz + TC_TZ - 1) / TC_TZ);
}
static int tc_grid_sms() {
    static const int sms = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            v = 1;
        return v > 0 ? v : 1;
    }();
    return sms;
}
// persistent grid: one CTA per SM (the kernel's shared memory admits no second), at most one per brick
static int tc_grid(const Dims &d) {
    const int nb = tc_bricks(d), sms = tc_grid_sms();
    return nb < sms ? nb : sms;
}

static int wg_bricks(const Dims &d) { return ((d.nx + TC_M - 1) / TC_M) * d.ny * ((d.nz + WG_TZ - 1) / WG_TZ); }
// persistent weight-gradient grid: two CTAs per SM, at most one per brick
static int wg_grid(const Dims &d) {
    const int nb = wg_bricks(d), two = 2 * tc_grid_sms();
    return nb < two ? nb : two;
}

// once per process: the convolution needs more than the default 48 KB of shared memory
static bool tc_attrs() {
    static const bool ok = [] {
        return cudaFuncSetAttribute(conv_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM) == cudaSuccess &&
               cudaFuncSetAttribute(conv_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM) == cudaSuccess &&
               cudaFuncSetAttribute(conv_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM) == cudaSuccess &&
               cudaFuncSetAttribute(wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, WG_SMEM) == cudaSuccess;
    }();
    return ok;
}

static sim_status net_forward(sim_net_t *n, const int *done = nullptr) {
    if (!tc_attrs()) return net_fail(n, SIM_ECUDA, "convolution kernel attributes");
    const int grid = tc_grid(n->d), nb = tc_bricks(n->d);
    const int stall = n->stall_once;
    n->stall_once = -1;
    for (int l = 0; l < NLAYER; l++) {
        const float *bias = n->param + n->off_b[l];
        if (l + 1 < NLAYER)
            conv_tc_kernel<0><<<grid, TC_THREADS, TC_SMEM, n->stream>>>(n->map_act[l], n->d, nb, n->wf[l], bias, nullptr,
                                                                        n->act[l + 1], nullptr, done, n->dstat,
                                                                        l == 0 ? stall : -1);
        else
            conv_tc_kernel<1><<<grid, TC_THREADS, TC_SMEM, n->stream>>>(n->map_act[l], n->d, nb, n->wf[l], bias, nullptr,
                                                                        nullptr, n->out, done, n->dstat, -1);
        NET_LAUNCHED(n);
    }
    return SIM_OK;
}

// gradients of the MSE loss of the last forward pass into n->grad; loss into n->dloss
static sim_status net_backward(sim_net_t *n, const float *target) {
    const int N = n->d.N;
    mse_kernel<<<n->lblk, 128, 0, n->stream>>>(n->d, n->out, target, (uint16_t *)n->g0, n->lpart);
    NET_LAUNCHED(n);
    mse_fold_kernel<<<1, 32, 0, n->stream>>>(n->lblk, N, n->lpart, n->dloss);
    NET_LAUNCHED(n);
    if (!tc_attrs()) return net_fail(n, SIM_ECUDA, "convolution kernel attributes");
    uint32_t *gcur = n->g0, *gnext = n->g1;
    for (int l = NLAYER - 1; l >= 0; l--) {
        const int gi = gcur == n->g0 ? 0 : 1;
        wgrad_tc_kernel<<<n->wg_ctas, WG_THREADS, WG_SMEM, n->stream>>>(n->map_win[l], n->map_wg[gi], n->d, wg_bricks(n->d),
                                                                       n->wpart, n->dstat);
        NET_LAUNCHED(n);
        const int ne = 27 * CIN[l] * COUT[l];
        wgrad_fold_kernel<<<sim_blocks(ne), SIM_THREADS, 0, n->stream>>>(n->wg_ctas, CIN[l], COUT[l], n->wpart,
                                                                          n->grad + n->off_w[l]);
        NET_LAUNCHED(n);
        bgrad_kernel<<<n->bblk, 128, 0, n->stream>>>(n->d, COUT[l], (const uint16_t *)gcur, n->bpart);
        NET_LAUNCHED(n);
        bgrad_fold_kernel<<<1, 32, 0, n->stream>>>(n->bblk, COUT[l], n->bpart, n->grad + n->off_b[l]);
        NET_LAUNCHED(n);
        if (l > 0) {   // data gradient through layer l into the ReLU output of layer l-1
            conv_tc_kernel<2><<<tc_grid(n->d), TC_THREADS, TC_SMEM, n->stream>>>(
                n->map_g[gcur == n->g0 ? 0 : 1], n->d, tc_bricks(n->d), n->wb[l], nullptr, n->act[l], gnext, nullptr,
                nullptr, n->dstat, -1);
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
    n->d.nxp = (nx + 7) / 8 * 8;
    n->d.P = (long)n->d.nxp * ny * nz;
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
    const size_t act_bytes = 32 * (size_t)n->d.P;   // two planes of 16 bytes per (padded) cell
    for (int l = 0; l <= NLAYER; l++) n->act[l] = (uint32_t *)A(act_bytes);
    n->out = (float *)A(sizeof(float) * N);
    n->g0 = (uint32_t *)A(act_bytes);
    n->g1 = (uint32_t *)A(act_bytes);
    n->wg_ctas = wg_grid(n->d);
    n->wpart = (float *)A(sizeof(float) * 27 * 256 * (size_t)n->wg_ctas);
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
    for (int l = 0; l < NLAYER; l++)
        maps = maps && act_map(n->d, n->act[l], &n->map_act[l]) && act_map(n->d, n->act[l], &n->map_win[l], TC_XS / 8, WG_SZ);
    maps = maps && act_map(n->d, n->g0, &n->map_g[0]) && act_map(n->d, n->g1, &n->map_g[1]) &&
           act_map(n->d, n->g0, &n->map_wg[0], TC_M / 8, WG_TZ) && act_map(n->d, n->g1, &n->map_wg[1], TC_M / 8, WG_TZ);
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
        !zero_acts(n, act_bytes) || pack_all(n) != SIM_OK) {
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
    features_kernel<<<sim_blocks(n->d.N), SIM_THREADS, 0, n->stream>>>(n->d, x_dev, (uint16_t *)n->act[0], nullptr);
    NET_LAUNCHED(n);
    if (net_forward(n) != SIM_OK) return n->err;
    NET_CK(n, cudaMemcpyAsync(y_dev, n->out, sizeof(float) * n->d.N, cudaMemcpyDeviceToDevice, n->stream));
    return net_status(n);
}

sim_status sim_net_loss_grad(sim_net_t *n, const float *x_dev, const float *target_dev, double *loss, float *grads) {
    if (!n || !x_dev || !target_dev) return SIM_EINVAL;
    if (n->err != SIM_OK) return n->err;
    features_kernel<<<sim_blocks(n->d.N), SIM_THREADS, 0, n->stream>>>(n->d, x_dev, (uint16_t *)n->act[0], nullptr);
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
    features_kernel<<<sim_blocks(n->d.N), SIM_THREADS, 0, n->stream>>>(n->d, x_dev, (uint16_t *)n->act[0], nullptr);
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

sim_status sim_net_inject_stall(sim_net_t *n, int32_t slab) {
    if (!n || slab < 0) return SIM_EINVAL;
    n->stall_once = slab;
    return SIM_OK;
}

sim_status sim_net_time_conv(sim_net_t *n, int32_t which, int32_t reps, double *us) {
    if (!n || !us || which < 0 || which > 2 || reps < 1) return SIM_EINVAL;
    if (n->err != SIM_OK) return n->err;
    if (!tc_attrs()) return net_fail(n, SIM_ECUDA, "convolution kernel attributes");
    const size_t flush_bytes = 256u << 20;
    void *flush = nullptr;
    NET_CK(n, cudaMalloc(&flush, flush_bytes));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sim_status st = SIM_OK;
    double total = 0.0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = SIM_ECUDA;
    const int l = 1;   // hidden layer 2: act[1] -> act[2]
    for (int r = 0; r < reps && st == SIM_OK; r++) {
        if (cudaMemsetAsync(flush, r & 0xff, flush_bytes, n->stream) != cudaSuccess ||
            cudaEventRecord(e0, n->stream) != cudaSuccess) { st = SIM_ECUDA; break; }
        if (which == 0) {
            conv_tc_kernel<0><<<tc_grid(n->d), TC_THREADS, TC_SMEM, n->stream>>>(
                n->map_act[l], n->d, tc_bricks(n->d), n->wf[l], n->param + n->off_b[l], nullptr, n->act[l + 1], nullptr,
                nullptr, n->dstat, -1);
        } else if (which == 1) {
            wgrad_tc_kernel<<<n->wg_ctas, WG_THREADS, WG_SMEM, n->stream>>>(n->map_win[l], n->map_wg[0], n->d,
                                                                           wg_bricks(n->d), n->wpart, n->dstat);
            n->launches++;
            wgrad_fold_kernel<<<sim_blocks(27 * 256), SIM_THREADS, 0, n->stream>>>(n->wg_ctas, CIN[l], COUT[l], n->wpart,
                                                                                    n->grad + n->off_w[l]);
        } else {
            conv_tc_kernel<2><<<tc_grid(n->d), TC_THREADS, TC_SMEM, n->stream>>>(
                n->map_g[0], n->d, tc_bricks(n->d), n->wb[l], nullptr, n->act[l], n->g1, nullptr, nullptr, n->dstat, -1);
        }
        n->launches++;
        float ms = 0.f;
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, n->stream) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            st = SIM_ECUDA;
            break;
        }
        total += ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(n->stream);
    cudaFree(flush);
    if (st != SIM_OK) return net_fail(n, st, "sim_net_time_conv: CUDA error");
    *us = 1e3 * total / reps;
    return net_status(n);
}

}  // extern "C"

// inference inside the CPR preconditioner: features x [N][4] -> y [N], on the
// caller's stream, every kernel skipping its work once *done is set
sim_status net_infer(sim_net_t *n, const float *x_dev, float *y_dev, cudaStream_t st, const int *done) {
    cudaStream_t keep = n->stream;
    n->stream = st;
    features_kernel<<<sim_blocks(n->d.N), SIM_THREADS, 0, st>>>(n->d, x_dev, (uint16_t *)n->act[0], done);
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
