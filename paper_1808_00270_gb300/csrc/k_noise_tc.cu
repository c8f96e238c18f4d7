// k_noise_tc.cu -- the moving-average filter of the colored noise on the
// tensor cores (tcgen05, TMEM accumulators, TMA tile loads).
//
// For a block of T = 64 steps starting at n0, Eq. noise_production gives per
// stream j (a particle's component) and t < 64
//     F^R[t][j] = sum_{s=-H}^{H} A_s W[n0 + t + s][j],          H = m_max - 1.
// Over a window of times t_lo + k (t_lo = n0 - H rounded down to a multiple
// of 64, a = n0 - H - t_lo) this is the product
//     F^R[t][j] = sum_k W[t_lo + k][j] B[k][t],   B[k][t] = A_{k - a - t - H},
// a GEMM with M = streams (128 per tile), N = 64 outputs and K = window rows,
// whose B operand is a Toeplitz matrix of the taps (zero outside |s| <= H).
//
// Precision: the products run in FP16 (kind::f16, K = 16 per MMA, FP32
// accumulation); FP16 keeps 11 significant bits, so each operand is split into
// an FP16 part and its remainder scaled by 2^11 (again FP16), and
//     F = D1 + 2^-11 D2,   D1 = W_hi A_hi,   D2 = W_hi A_lo + W_lo A_hi,
// which drops only W_lo A_lo (2^-22 of a product).  The taps are first scaled
// by a power of two that puts the largest one in [2^14, 2^15) (FP16 range;
// undone exactly at the end).  The tensor cores' FP32 accumulation rounds
// toward zero; summed over a whole window (hundreds of MMAs) that bias reached
// 1.2e-5 of F^R, so each 64-row group (four K steps) accumulates into fresh
// TMEM accumulators and the groups are added on the FP32 pipes with
// round-to-nearest (about 1e-7 to 2e-7 of the FP32 sum with 32-row groups at
// m_max = 200 ... 1000, measured and emulated on the CPU; 64-row groups double
// the terms each rounding-toward-zero sum takes).  A 16-bit MMA costs the same
// tensor-pipe time as a TF32 one with half the K (about 96 cycles for
// N <= 128, measured), so this takes half the MMAs of a TF32 split.  Every
// group starts at a time that is a multiple of 64, so an output's sum does not
// depend on where its 64-step block started.
//
// B is never materialised per K step: shared memory holds the scaled taps as
// overlapping FP16 rows R[u] = (Acp[u - 126 + e], e < 8) (hi and lo parts),
// and the K-major descriptor of K step k0 starts at row k0 - a + 63, with
// 8-row groups 128 bytes apart (SBO) and the second 8-column group 128 bytes
// on (LBO).  With output column n standing for t = 63 - n, both offsets are
// positive.
//
// The white-noise ring is stored in that split form already (the generator
// writes an FP16 plane of W_hi and one of W_lo, the same bytes as FP32), so the
// A operands come straight from shared memory: per 32-row chunk four TMA boxes
// {64 streams, 32 rows} with 128-byte swizzle, the MN-major canonical layout
// (64-stream atoms 4 KB apart: LBO; 8-row groups 1024 bytes apart: SBO).  Rows
// outside the real window meet zero taps; the ring holds finite values only
// (zeros until generated), so they add exact zeros.
//
// One persistent CTA per SM (all 512 TMEM columns), warp-specialized and
// linked by mbarriers, so that loads, MMAs and accumulation of different
// chunks overlap:
//   warp 0, one thread  TMA loads of a chunk's four boxes into a ring of
//                       16 KB shared-memory stages;
//   warp 1, one thread  the MMAs of a chunk (2 K steps x 3 products) into the
//                       TMEM accumulator pair (D1, D2) of its 64-row group, one
//                       of four; owns the TMEM allocation; its commit frees the
//                       stage, and at a group's second chunk the pair;
//   warps 2-5           accumulators: a group's D read back and added in FP32
//                       registers (thread = stream = TMEM lane); at the last
//                       group of a tile, F^R written out.
// The single-thread roles step their chunk, stage, parity and ring-slot
// counters by increments: computed from the chunk index by 64-bit division
// and remainder (software routines, a long dependent chain in one thread) they
// took longer than a chunk's copies and halved the filter's rate.
// Every wait is bounded: a wait that runs out sets kErrTimeout and a shared
// abort flag that ends every role's loop; the CTA then lets its copies and
// MMAs finish (bounded again), frees its TMEM and returns.
#include <algorithm>

#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include "launch.h"

namespace gld {

namespace {

constexpr int kTcThreads = 192;                            // 6 warps (roles above)
constexpr int kTcMaxStages = 12;
constexpr int kTcChunk = 32;                               // window rows per stage (2 K steps)
constexpr int kTcBoxBytes = kTcChunk * 64 * 2;             // {64 streams, 32 rows} FP16: 4 KB
constexpr int kTcStageBytes = 4 * kTcBoxBytes;             // hi and lo parts of 128 streams
constexpr int kTcND = 4;                                   // TMEM accumulator pairs
constexpr uint32_t kTcCols = 512;                          // pair d: D1 at 128 d, D2 at 128 d + 64
constexpr int kTcRowOff = 126;                             // R[u] holds Acp[u - kTcRowOff + e]
constexpr long long kTcWaitCycles = 2000000000LL;          // about one second

// Instruction descriptor of tcgen05.mma kind::f16: D FP32, A and B FP16,
// A MN-major (bit 15), B K-major, N = 64, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 15) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

// Waits until the phase with the given parity has completed; false after
// about a second.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity)
{
    const uint32_t a = smem_u32(b);
    long long t0 = 0;
    for (int it = 0;; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
        if (it == 0) t0 = clock64();
        else if (clock64() - t0 > kTcWaitCycles) return false;
    }
}

// As mbar_wait, but also gives up when another role raised the CTA's abort
// flag; raises it on a timeout.
__device__ __forceinline__ bool mbar_wait_ab(uint64_t* b, uint32_t parity, volatile int* abort_flag)
{
    const uint32_t a = smem_u32(b);
    long long t0 = 0;
    for (int it = 0;; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
        if (*abort_flag) return false;
        if (it == 0) t0 = clock64();
        else if (clock64() - t0 > kTcWaitCycles) {
            *abort_flag = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_u32(bar))
                 : "memory");
}

// Shared-memory matrix descriptor (tcgen05 version 1): start address, leading
// and stride byte offsets, layout (0: no swizzle, 2: 128-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t layout)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)layout << 61);
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d), "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate)
                 : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15}, [%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15])
                 : "r"(taddr)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Chunks of the window: real rows [a, a + 2H + T) from the time t_lo.
__host__ __device__ inline int tc_nch_max(int H, int T) { return 2 * ((63 + 2 * H + T + 63) / 64); }
// Rows of the overlapping tap array: every K-step tile of any window offset.
__host__ __device__ inline int tc_rows(int H, int T) { return kTcChunk * tc_nch_max(H, T) + 127; }

constexpr size_t kTcBarBytes = 8 * (2 * kTcMaxStages + 2 * kTcND) + 16;

// Load stages that fit beside the taps (at most 12, at least 2).
int tc_stages(int H, int T)
{
    const long long room = 227LL * 1024 - 1024 - 2LL * tc_rows(H, T) * 16 - (long long)kTcBarBytes;
    return (int)std::max(0LL, std::min<long long>(kTcMaxStages, room / kTcStageBytes));
}

size_t tc_smem_bytes(int H, int T)
{
    const size_t b = 1024 + (size_t)tc_stages(H, T) * kTcStageBytes + 2 * (size_t)tc_rows(H, T) * 16 + kTcBarBytes;
    // at least 116 KB: a second CTA (which would wait for the TMEM) never shares an SM
    return std::max<size_t>(b, 116 * 1024);
}

__global__ void __launch_bounds__(kTcThreads, 1) fir_tc(const __grid_constant__ CUtensorMap wmap, const StepParams P,
                                                        Ctrl* __restrict__ ctrl, const float* __restrict__ taps,
                                                        float* __restrict__ out, int nrows, int nst)
{
    extern __shared__ unsigned char sm_raw[];
    const uint32_t raw = smem_u32(sm_raw);
    unsigned char* sm = sm_raw + (((raw + 1023u) & ~1023u) - raw);
    unsigned char* stage = sm;                                       // [nst][4 boxes of 4 KB]
    __half* Rhi = (__half*)(sm + (size_t)nst * kTcStageBytes);       // [nrows][8]
    __half* Rlo = Rhi + 8 * (size_t)nrows;
    uint64_t* full = (uint64_t*)(Rlo + 8 * (size_t)nrows);           // [nst]  stage loaded
    uint64_t* empty = full + kTcMaxStages;                           // [nst]  stage read by the MMAs
    uint64_t* dfull = empty + kTcMaxStages;                          // [ND]   accumulator complete
    uint64_t* dempty = dfull + kTcND;                                // [ND]   accumulator read back
    uint32_t* misc = (uint32_t*)(dempty + kTcND);                    // TMEM base
    volatile int* abort_flag = (volatile int*)(misc + 1);
    int* red = (int*)(misc + 2);                                     // largest tap (bit pattern)

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        // the layout must fit the dynamic shared memory of the launch
        uint32_t dyn;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        const size_t used = (size_t)(sm - sm_raw) + (size_t)nst * kTcStageBytes + 32 * (size_t)nrows + kTcBarBytes;
        if (used > dyn || nst < 2 || nst > kTcMaxStages) {
            if (tid == 0) atomicOr(&ctrl->err, kErrCheck);
            return;  // uniform: before any barrier or tensor-memory use
        }
    }
    const int H = P.H, T = P.T;
    const long long n0 = ctrl->step;
    const long long np3 = 3LL * P.n_pad;
    const int ntiles = (int)((np3 + 127) / 128);
    const long long w0 = n0 - H;
    const long long t_lo = w0 >= 0 ? (w0 & ~63LL) : -((-w0 + 63) & ~63LL);
    const int a = (int)(w0 - t_lo);
    const int nk = 2 * H + T;                       // real window rows [a, a + nk)
    const int nch = 2 * ((a + nk + 63) / 64);       // 32-row chunks, in pairs (64-row groups)
    const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const long long G = (long long)my_tiles * nch;  // chunks this CTA streams

    // the taps scaled by 2^ks (largest in [2^14, 2^15)) as overlapping FP16
    // rows, FP16 part and 2^11-scaled remainder
    if (tid == 0) *red = 0;
    __syncthreads();
    {
        float mx = 0.f;
        for (int sig = tid; sig <= 2 * H; sig += kTcThreads) mx = fmaxf(mx, fabsf(__ldg(taps + sig)));
        if (mx > 0.f) atomicMax(red, __float_as_int(mx));  // non-negative floats order as ints
    }
    __syncthreads();
    const float amax = __int_as_float(*red);
    const int ks = amax > 0.f ? max(-60, min(60, 14 - ilogbf(amax))) : 0;
    for (int idx = tid; idx < 8 * nrows; idx += kTcThreads) {
        const int sig = (idx >> 3) - kTcRowOff + (idx & 7);
        const float v = (sig >= 0 && sig <= 2 * H) ? ldexpf(__ldg(taps + sig), ks) : 0.f;
        unsigned short hb, lb;
        split_f16(v, hb, lb);
        Rhi[idx] = __ushort_as_half(hb);
        Rlo[idx] = __ushort_as_half(lb);
    }
    if (tid == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int d = 0; d < kTcND; ++d) {
            mbar_init(&dfull[d], 1);
            mbar_init(&dempty[d], 4);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the taps, for the tensor cores
    __syncwarp();  // .sync.aligned tcgen05 instructions need the whole warp converged
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&misc[0])),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = misc[0];
    // the allocation must start at lane 0 and column 0 (all 512 columns)
    if ((tm & 0xFFFF0000u) != 0 || (tm & 0xFFFFu) != 0) {
        if (tid == 0) atomicOr(&ctrl->err, kErrCheck);
        *abort_flag = 1;
    }
    __syncthreads();
    const bool ok0 = *abort_flag == 0;

    int committed = -1;  // MMA thread: last 64-row group whose MMAs were committed
    if (ok0 && warp == 0 && lane == 0) {
        // ---- producer: TMA loads of the window's chunks, hi and lo planes ------
        // (chunk, tile, stage, phase and ring slot advance as counters: 64-bit
        // divisions in this single thread's loop cost more than a chunk's copy)
        long long slot0 = t_lo % P.lw;
        if (slot0 < 0) slot0 += P.lw;
        const int lw = (int)P.lw;
        int c = 0, s = 0, slot = (int)slot0;
        uint32_t ph = 0;  // parity of the stage's current fill
        long long x = (long long)blockIdx.x * 128;
        for (int g = 0; g < (int)G; ++g) {
            if (g >= nst && !mbar_wait_ab(&empty[s], ph ^ 1u, abort_flag)) break;
            if (x >= np3 || (slot & 31) || slot + kTcChunk > lw) {  // never for a valid launch
                atomicOr(&ctrl->err, kErrCheck);
                *abort_flag = 1;
                break;
            }
            unsigned char* st = stage + (size_t)s * kTcStageBytes;
            mbar_expect_tx(&full[s], kTcStageBytes);
            tma_load_2d(st, &wmap, (int)x, slot, &full[s]);
            tma_load_2d(st + kTcBoxBytes, &wmap, (int)x + 64, slot, &full[s]);
            tma_load_2d(st + 2 * kTcBoxBytes, &wmap, (int)x, lw + slot, &full[s]);
            tma_load_2d(st + 3 * kTcBoxBytes, &wmap, (int)x + 64, lw + slot, &full[s]);
            if (++s == nst) {
                s = 0;
                ph ^= 1u;
            }
            slot += kTcChunk;
            if (slot >= lw) slot -= lw;
            if (++c == nch) {  // the next tile
                c = 0;
                slot = (int)slot0;
                x += (long long)gridDim.x * 128;
            }
        }
    } else if (ok0 && warp == 1 && lane == 0) {
        // ---- MMA issuer ---------------------------------------------------------
        const uint32_t rhi = smem_u32(Rhi), rlo = smem_u32(Rlo), st0 = smem_u32(stage);
        int c = 0, s = 0, d = 0;
        uint32_t ph = 0, dph = 0;  // parities of the stage's fill and of the accumulator pair's use
        for (int g = 0; g < (int)G; ++g) {
            if (!mbar_wait_ab(&full[s], ph, abort_flag)) break;
            // a 64-row group (chunks c, c + 1) accumulates into pair d
            if (!(c & 1) && g >= 2 * kTcND && !mbar_wait_ab(&dempty[d], dph ^ 1u, abort_flag)) break;
            tc_fence_after();
            const uint32_t d1 = tm + 128u * (uint32_t)d, d2 = d1 + 64u;
            const uint32_t sa = st0 + (uint32_t)s * kTcStageBytes;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k0 = kTcChunk * c + 16 * h;
                const uint32_t u0 = (uint32_t)(k0 - a - 63 + kTcRowOff);
                if (u0 + 72u > (uint32_t)nrows) {  // never for a valid launch
                    atomicOr(&ctrl->err, kErrCheck);
                    continue;
                }
                const uint64_t bh = smem_desc(rhi + 16u * u0, 128u, 128u, 0u);
                const uint64_t bl = smem_desc(rlo + 16u * u0, 128u, 128u, 0u);
                // rows 16 h .. 16 h + 15 of the hi boxes and of the lo boxes
                const uint64_t ah = smem_desc(sa + 2048u * (uint32_t)h, 4096u, 1024u, 2u);
                const uint64_t al = smem_desc(sa + 2u * kTcBoxBytes + 2048u * (uint32_t)h, 4096u, 1024u, 2u);
                const uint32_t acc0 = (c & 1) || h > 0 ? 1u : 0u;
                mma_f16(d1, ah, bh, acc0);
                mma_f16(d2, ah, bl, acc0);
                mma_f16(d2, al, bh, 1u);
            }
            mma_commit(&empty[s]);
            if (c & 1) {
                mma_commit(&dfull[d]);
                committed = g >> 1;
                if (++d == kTcND) {
                    d = 0;
                    dph ^= 1u;
                }
            }
            if (++s == nst) {
                s = 0;
                ph ^= 1u;
            }
            if (++c == nch) c = 0;
        }
    } else if (ok0 && warp >= 2) {
        // ---- accumulators: D -> FP32 registers, F^R at the end of a tile -------
        const int q4 = warp & 3;  // TMEM lanes 32 q4 .. 32 q4 + 31 (warps 2-5 cover all four)
        const int ft = 32 * q4 + lane;
        const uint32_t lane_base = (uint32_t)(32 * q4) << 16;
        float acc[64];
#pragma unroll
        for (int q = 0; q < 64; ++q) acc[q] = 0.f;
        int c = 0, i = 0, d = 0;  // c: 64-row group of the tile
        uint32_t dph = 0;
        for (int g = 0; g < (int)G / 2; ++g) {
            const bool okw = mbar_wait_ab(&dfull[d], dph, abort_flag);
            if (!__all_sync(0xffffffffu, okw)) break;
            tc_fence_after();
            {  // all 128 columns of the pair in flight, one wait
                uint32_t dv1[4][16], dv2[4][16];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    tmem_ld16(tm + lane_base + 128u * (uint32_t)d + 16u * (uint32_t)h, dv1[h]);
                    tmem_ld16(tm + lane_base + 128u * (uint32_t)d + 64u + 16u * (uint32_t)h, dv2[h]);
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int h = 0; h < 4; ++h)
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int o = 16 * h + q;
                        acc[o] = __fadd_rn(acc[o], __fmaf_rn(__uint_as_float(dv2[h][q]), 1.0f / 2048.0f,
                                                             __uint_as_float(dv1[h][q])));
                    }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&dempty[d]);
            if (c == nch / 2 - 1) {  // the tile is complete: to F^R (column n is t = 63 - n)
                const long long j = ((long long)blockIdx.x + (long long)i * gridDim.x) * 128 + ft;
                if (j < np3)
#pragma unroll
                    for (int q = 0; q < 64; ++q) out[(size_t)(63 - q) * np3 + j] = ldexpf(acc[q], -ks);
#pragma unroll
                for (int q = 0; q < 64; ++q) acc[q] = 0.f;
            }
            if (++d == kTcND) {
                d = 0;
                dph ^= 1u;
            }
            if (++c == nch / 2) {
                c = 0;
                ++i;
            }
        }
    }
    __syncthreads();
    if (*abort_flag) {
        if (tid == 0) atomicOr(&ctrl->err, kErrTimeout);
        // let copies and MMAs still in flight finish before the memory goes
        if (warp == 1 && lane == 0 && committed >= 0)
            mbar_wait(&dfull[committed % kTcND], (uint32_t)((committed / kTcND) & 1));
        if (tid == 0) {
            const long long t0 = clock64();
            while (clock64() - t0 < 200000) {
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kTcCols) : "memory");
    }
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&ctrl->done_fir, 1u) == gridDim.x - 1) {
            ctrl->noise_n0 = n0;
            ctrl->w_lo = n0 - P.H;
            ctrl->w_hi = n0 + P.T + P.H;
            ctrl->done_fir = 0u;
            __threadfence();
        }
    }
}

}  // namespace

bool noise_filter_tc_ok(const StepParams& P)
{
    return P.T == 64 && P.lw % kTcChunk == 0 && P.lw >= 2LL * P.H + P.T + 31 && tc_stages(P.H, P.T) >= 2 &&
           tc_smem_bytes(P.H, P.T) <= 227 * 1024;
}

cudaError_t make_noise_ring_map(void* W, const StepParams& P, CUtensorMap* map)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return e != cudaSuccess ? e : cudaErrorNotSupported;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    // the split ring: rows [0, lw) hold the FP16 hi parts, rows [lw, 2 lw) the lo parts
    const cuuint64_t dims[2] = {(cuuint64_t)3 * P.n_pad, 2 * (cuuint64_t)P.lw};
    const cuuint64_t strides[1] = {(cuuint64_t)3 * P.n_pad * sizeof(__half)};
    const cuuint32_t box[2] = {64u, (cuuint32_t)kTcChunk};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, W, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_noise_filter_tc(const StepParams& P, Ctrl* ctrl, const CUtensorMap* wmap, const float* taps,
                                   float* out, int num_sms, cudaStream_t st)
{
    if (!noise_filter_tc_ok(P) || !P.wsplit) return cudaErrorInvalidValue;  // it reads the split ring
    const size_t smem = tc_smem_bytes(P.H, P.T);
    cudaError_t e = cudaFuncSetAttribute(fir_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long ntiles = (3LL * P.n_pad + 127) / 128;
    const int grid = (int)std::min<long long>(ntiles, std::max(num_sms, 1));
    fir_tc<<<grid, kTcThreads, smem, st>>>(*wmap, P, ctrl, taps, out, tc_rows(P.H, P.T), tc_stages(P.H, P.T));
    return cudaGetLastError();
}

}  // namespace gld
