// k_noise_tc.cu -- the moving-average filter of the colored noise on the
// tensor cores (tcgen05, TMEM accumulators, TMA tile loads).
//
// For a block of T = 64 steps starting at n0, Eq. noise_production gives per
// stream j (a particle's component) and t < 64
//     F^R[t][j] = sum_{s=-H}^{H} A_s W[n0 + t + s][j],          H = m_max - 1.
// Over a window of times t_lo + k (t_lo = n0 - H rounded down to a multiple
// of 32, a = n0 - H - t_lo) this is the product
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
// 1.2e-5 of F^R, so each 32-row chunk accumulates into fresh TMEM accumulators
// and the chunks are added on the FP32 pipes with round-to-nearest: about
// 1e-7 to 2e-7 of the FP32 sum at m_max = 200 ... 1000 (measured, and emulated
// on the CPU).  A 16-bit MMA costs the same tensor-pipe time as a TF32 one
// with half the K (about 96 cycles for N <= 128, measured), so this takes half
// the MMAs of a TF32 split.  Every 32-row chunk starts at a time that is a
// multiple of 32, so an output's sum does not depend on where its 64-step
// block started.
//
// B is never materialised per K step: shared memory holds the scaled taps as
// overlapping FP16 rows R[u] = (Acp[u - 94 + e], e < 8) (hi and lo parts),
// and the K-major descriptor of K step k0 starts at row k0 - a + 31, with
// 8-row groups 128 bytes apart (SBO) and the second 8-column group 128 bytes
// on (LBO).  With output column n standing for t = 63 - n, both offsets are
// positive.
//
// One persistent CTA per SM (all 512 TMEM columns), warp-specialized and
// linked by mbarriers, so that loads, conversions, MMAs and accumulation of
// different chunks overlap:
//   warp 0, one thread  TMA loads of W tiles [32 rows][128 streams] into a
//                       ring of shared-memory stages;
//   warp 1, one thread  the MMAs of a chunk (2 K steps x 3 products) into one
//                       of three TMEM accumulator pairs (D1, D2), from one of
//                       four TMEM A buffers; owns the TMEM allocation;
//   warps 4-7           converters: a stage's rows (zero outside the real
//                       window) split into FP16 parts and stored into an A
//                       buffer (thread = stream = TMEM lane);
//   warps 8-11          accumulators: D read back and added in FP32 registers;
//                       at the last chunk of a tile, F^R written out.
// Measured on GB300 (262144 particles, m_max = 400, one 64-step block): 1.3 ms
// including the white-noise generation, against 2.2 ms for the FP32-pipe
// filter.  The bulk-tensor copies are the limit: with every other role idle
// they stream the ring at about 3.6 TB/s (0.90 ms; the same from L2-resident
// tiles, and the same with the stage split into 2 or 4 smaller boxes), about
// 12 bytes per cycle per SM.  Loading with 16-byte cp.async copies issued by
// the converter warps instead (completion on the same mbarriers) took 2.2 ms.
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

constexpr int kTcThreads = 384;                            // 12 warps (roles above)
constexpr int kTcMaxStages = 8;
constexpr int kTcChunk = 32;                               // window rows per stage (4 K steps)
constexpr int kTcStageFloats = kTcChunk * 128;
constexpr int kTcStageBytes = kTcStageFloats * 4;          // 16 KB
constexpr int kTcNA = 4, kTcND = 3;                        // TMEM A buffers and accumulator pairs
constexpr uint32_t kTcCols = 512;                          // D pairs [0, 384), A [384, 512)
constexpr uint32_t kTcAcol = 128u * kTcND;
constexpr int kTcRowOff = 94;                              // R[u] holds Acp[u - kTcRowOff + e]
constexpr long long kTcWaitCycles = 2000000000LL;          // about one second

// Instruction descriptor of tcgen05.mma kind::f16: D FP32, A and B FP16,
// both K-major, N = 64, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (0u << 7) | (0u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

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

// K-major, no-swizzle shared-memory matrix descriptor (tcgen05 version 1).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
                 ::"r"(d), "r"(a), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate)
                 : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15, %16};"
                 ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                 "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
                 "r"(v[15])
                 : "memory");
}

// FP16 part of v and its remainder scaled by 2^11 (as FP16 bit patterns)
__device__ __forceinline__ void split_f16(float v, uint32_t& hi, uint32_t& lo)
{
    const __half h = __float2half_rn(v);
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(__float2half_rn((v - __half2float(h)) * 2048.0f));
}

// The same for two values at once with packed conversions: v0 in the low
// halves (bit for bit split_f16 of each).
__device__ __forceinline__ void split2_f16(float v0, float v1, uint32_t& hi, uint32_t& lo)
{
    const __half2 h = __floats2half2_rn(v0, v1);
    const float2 f = __half22float2(h);
    const __half2 l = __floats2half2_rn((v0 - f.x) * 2048.0f, (v1 - f.y) * 2048.0f);
    hi = (uint32_t)__half_as_ushort(__low2half(h)) | ((uint32_t)__half_as_ushort(__high2half(h)) << 16);
    lo = (uint32_t)__half_as_ushort(__low2half(l)) | ((uint32_t)__half_as_ushort(__high2half(l)) << 16);
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
__host__ __device__ inline int tc_nch_max(int H, int T) { return (31 + 2 * H + T + 31) / kTcChunk; }
// Rows of the overlapping tap array: every K-step tile of any window offset.
__host__ __device__ inline int tc_rows(int H, int T) { return kTcChunk * tc_nch_max(H, T) + 91; }

constexpr size_t kTcBarBytes = 8 * (2 * kTcMaxStages + 2 * kTcNA + 2 * kTcND) + 16;

// Load stages that fit beside the taps (at most 8, at least 2).
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
    float* stage = (float*)sm;                                       // [nst][32][128]
    __half* Rhi = (__half*)(sm + (size_t)nst * kTcStageBytes);       // [nrows][8]
    __half* Rlo = Rhi + 8 * (size_t)nrows;
    uint64_t* full = (uint64_t*)(Rlo + 8 * (size_t)nrows);           // [nst]  stage loaded
    uint64_t* empty = full + kTcMaxStages;                           // [nst]  stage read
    uint64_t* afull = empty + kTcMaxStages;                          // [NA]   A buffer written
    uint64_t* aempty = afull + kTcNA;                                // [NA]   A buffer read by the MMAs
    uint64_t* dfull = aempty + kTcNA;                                // [ND]   accumulator complete
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
    const long long t_lo = w0 >= 0 ? (w0 & ~31LL) : -((-w0 + 31) & ~31LL);
    const int a = (int)(w0 - t_lo);
    const int nk = 2 * H + T;                       // real window rows [a, a + nk)
    const int nch = (a + nk + kTcChunk - 1) / kTcChunk;
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
        uint32_t hb, lb;
        split_f16(v, hb, lb);
        Rhi[idx] = __ushort_as_half((unsigned short)hb);
        Rlo[idx] = __ushort_as_half((unsigned short)lb);
    }
    if (tid == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 4);
        }
        for (int b = 0; b < kTcNA; ++b) {
            mbar_init(&afull[b], 4);
            mbar_init(&aempty[b], 1);
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

    long long committed = -1;  // MMA thread: last chunk whose MMAs were committed
    if (ok0 && warp == 0 && lane == 0) {
        // ---- producer: TMA loads of the window's 32-row tiles ---------------
        for (long long g = 0; g < G; ++g) {
            const int i = (int)(g / nch), c = (int)(g - (long long)i * nch);
            const int s = (int)(g % nst);
            if (g >= nst && !mbar_wait_ab(&empty[s], (uint32_t)((g / nst - 1) & 1), abort_flag)) break;
            long long slot = (t_lo + (long long)kTcChunk * c) % P.lw;
            if (slot < 0) slot += P.lw;
            const long long x = ((long long)blockIdx.x + (long long)i * gridDim.x) * 128;
            if (x >= np3 || (slot & 31) || slot + kTcChunk > P.lw) {  // never for a valid launch
                atomicOr(&ctrl->err, kErrCheck);
                *abort_flag = 1;
                break;
            }
            mbar_expect_tx(&full[s], kTcStageBytes);
            tma_load_2d(stage + (size_t)s * kTcStageFloats, &wmap, (int)x, (int)slot, &full[s]);
        }
    } else if (ok0 && warp == 1 && lane == 0) {
        // ---- MMA issuer ---------------------------------------------------------
        const uint32_t rhi = smem_u32(Rhi), rlo = smem_u32(Rlo);
        for (long long g = 0; g < G; ++g) {
            const int c = (int)(g % nch);
            const int b = (int)(g % kTcNA), d = (int)(g % kTcND);
            if (!mbar_wait_ab(&afull[b], (uint32_t)((g / kTcNA) & 1), abort_flag)) break;
            if (g >= kTcND && !mbar_wait_ab(&dempty[d], (uint32_t)((g / kTcND - 1) & 1), abort_flag)) break;
            tc_fence_after();
            const uint32_t d1 = tm + 128u * (uint32_t)d, d2 = d1 + 64u;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int k0 = kTcChunk * c + 16 * s;
                const uint32_t u0 = (uint32_t)(k0 - a - 63 + kTcRowOff);
                if (u0 + 72u > (uint32_t)nrows) {  // never for a valid launch
                    atomicOr(&ctrl->err, kErrCheck);
                    continue;
                }
                const uint64_t dh = smem_desc(rhi + 16u * u0, 128u, 128u);
                const uint64_t dl = smem_desc(rlo + 16u * u0, 128u, 128u);
                const uint32_t ah = tm + kTcAcol + 32u * (uint32_t)b + 8u * (uint32_t)s, al = ah + 16u;
                mma_f16(d1, ah, dh, s > 0 ? 1u : 0u);
                mma_f16(d2, ah, dl, s > 0 ? 1u : 0u);
                mma_f16(d2, al, dh, 1u);
            }
            mma_commit(&aempty[b]);
            mma_commit(&dfull[d]);
            committed = g;
        }
    } else if (ok0 && warp >= 4 && warp < 8) {
        // ---- converters: stage rows -> TF32 part / remainder in TMEM ------------
        const int ct = tid - 128;  // stream within the tile = TMEM lane
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        int b_prev = -1;  // A buffer whose stores are still in flight
        for (long long g = 0; g < G; ++g) {
            const int c = (int)(g % nch);
            const int s = (int)(g % nst), b = (int)(g % kTcNA);
            bool okw = mbar_wait_ab(&full[s], (uint32_t)((g / nst) & 1), abort_flag);
            if (okw && g >= kTcNA) okw = mbar_wait_ab(&aempty[b], (uint32_t)((g / kTcNA - 1) & 1), abort_flag);
            if (!__all_sync(0xffffffffu, okw)) break;  // the same decision in every lane
            uint32_t hv[16], lv[16];  // two FP16 per column, the earlier row in the low half
            const float* sp = stage + (size_t)s * kTcStageFloats + ct;
            const int k0 = kTcChunk * c;
            if (k0 >= a && k0 + kTcChunk <= a + nk) {  // (uniform) a chunk inside the window
#pragma unroll
                for (int r = 0; r < 32; r += 2) split2_f16(sp[r * 128], sp[(r + 1) * 128], hv[r >> 1], lv[r >> 1]);
            } else {  // rows outside the window are zero
#pragma unroll
                for (int r = 0; r < 32; r += 2) {
                    const int k = k0 + r;
                    const float v0 = (k >= a && k < a + nk) ? sp[r * 128] : 0.f;
                    const float v1 = (k + 1 >= a && k + 1 < a + nk) ? sp[(r + 1) * 128] : 0.f;
                    split2_f16(v0, v1, hv[r >> 1], lv[r >> 1]);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);  // the stage may be loaded again
            __syncwarp();  // converged for the aligned TMEM operations
            // the previous chunk's stores completed while this one was split
            // (chunk g waited only for the MMAs of chunk g - 4)
            if (b_prev >= 0) {
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&afull[b_prev]);
                __syncwarp();
            }
            const uint32_t ta = tm + lane_base + kTcAcol + 32u * (uint32_t)b;
            tmem_st16(ta, hv);
            tmem_st16(ta + 16u, lv);
            b_prev = b;
        }
        __syncwarp();
        if (b_prev >= 0) {  // uniform: every lane ran the same rounds; the stores end before TMEM is freed
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0 && !*abort_flag) mbar_arrive(&afull[b_prev]);
        }
    } else if (ok0 && warp >= 8) {
        // ---- accumulators: D -> FP32 registers, F^R at the end of a tile -------
        const int ft = tid - 256;
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        float acc[64];
#pragma unroll
        for (int q = 0; q < 64; ++q) acc[q] = 0.f;
        for (long long g = 0; g < G; ++g) {
            const int i = (int)(g / nch), c = (int)(g - (long long)i * nch);
            const int d = (int)(g % kTcND);
            const bool okw = mbar_wait_ab(&dfull[d], (uint32_t)((g / kTcND) & 1), abort_flag);
            if (!__all_sync(0xffffffffu, okw)) break;
            tc_fence_after();
#pragma unroll
            for (int half = 0; half < 2; ++half) {  // two column groups per wait for the loads
                uint32_t dv1[2][16], dv2[2][16];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t col = 16u * (uint32_t)(2 * half + h);
                    tmem_ld16(tm + lane_base + 128u * (uint32_t)d + col, dv1[h]);
                    tmem_ld16(tm + lane_base + 128u * (uint32_t)d + 64u + col, dv2[h]);
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int o = 16 * (2 * half + h) + q;
                        acc[o] = __fadd_rn(acc[o], __fmaf_rn(__uint_as_float(dv2[h][q]), 1.0f / 2048.0f,
                                                             __uint_as_float(dv1[h][q])));
                    }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&dempty[d]);
            if (c == nch - 1) {  // the tile is complete: to F^R (column n is t = 63 - n)
                const long long j = ((long long)blockIdx.x + (long long)i * gridDim.x) * 128 + ft;
                if (j < np3)
#pragma unroll
                    for (int q = 0; q < 64; ++q) out[(size_t)(63 - q) * np3 + j] = ldexpf(acc[q], -ks);
#pragma unroll
                for (int q = 0; q < 64; ++q) acc[q] = 0.f;
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
    const cuuint64_t dims[2] = {(cuuint64_t)3 * P.n_pad, (cuuint64_t)P.lw};
    const cuuint64_t strides[1] = {(cuuint64_t)3 * P.n_pad * sizeof(float)};
    const cuuint32_t box[2] = {128u, (cuuint32_t)kTcChunk};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, W, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_noise_filter_tc(const StepParams& P, Ctrl* ctrl, const CUtensorMap* wmap, const float* taps,
                                   float* out, int num_sms, cudaStream_t st)
{
    if (!noise_filter_tc_ok(P)) return cudaErrorInvalidValue;
    const size_t smem = tc_smem_bytes(P.H, P.T);
    cudaError_t e = cudaFuncSetAttribute(fir_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long ntiles = (3LL * P.n_pad + 127) / 128;
    const int grid = (int)std::min<long long>(ntiles, std::max(num_sms, 1));
    fir_tc<<<grid, kTcThreads, smem, st>>>(*wmap, P, ctrl, taps, out, tc_rows(P.H, P.T), tc_stages(P.H, P.T));
    return cudaGetLastError();
}

}  // namespace gld
