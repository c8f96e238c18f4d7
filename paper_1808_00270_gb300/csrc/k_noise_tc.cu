// k_noise_tc.cu -- the moving-average filter of the colored noise on the
// tensor cores (tcgen05, TMEM accumulators, TMA tile loads).
//
// For a block of T = 64 steps starting at n0, Eq. noise_production gives per
// stream j (a particle's component) and t < 64
//     F^R[t][j] = sum_{s=-H}^{H} A_s W[n0 + t + s][j],          H = m_max - 1.
// Over a window of times t_lo + k (k < 32 nch, t_lo = n0 - H rounded down to a
// multiple of 32, a = n0 - H - t_lo) this is the product
//     F^R[t][j] = sum_k W[t_lo + k][j] B[k][t],   B[k][t] = A_{k - a - t - H},
// a GEMM with M = streams (128 per tile), N = 64 outputs and K = window rows,
// whose B operand is a Toeplitz matrix of the taps (zero outside |s| <= H).
//
// Precision: the tensor cores read FP32 operands as TF32 (the low 13 mantissa
// bits dropped).  Each operand is split into a TF32 part and the FP32
// remainder, and three products are accumulated,
//     W_hi A_hi + W_hi A_lo + W_lo A_hi
// (the dropped W_lo A_lo term and the remainders' own truncation are below
// 2^-21 of each product).  The tensor cores' FP32 accumulation rounds toward
// zero; summed over a whole window (up to 750 MMAs at m_max = 1000) that bias
// reached 1.2e-5 of F^R, so each 32-row chunk accumulates into a fresh TMEM
// accumulator and the chunks are added on the FP32 pipes with round-to-
// nearest: about 4e-7 of the FP32 sum at any m_max (measured, and emulated
// on the CPU).
//
// Layout, per CTA (128 threads, one stream per thread and TMEM lane):
//   * W tiles [32 rows][128 streams] arrive by TMA (cp.async.bulk.tensor,
//     three stages, mbarrier completion); rows outside the real window are
//     replaced by zero, the rest split into hi / lo and stored into TMEM
//     (A buffers of 64 columns at 128 and 192: hi in the first 32, lo in the
//     last 32).
//   * B is never materialised per K step: shared memory holds the taps as
//     overlapping rows R[u] = (Acp[u - 94 + e], e < 4) (hi and lo copies),
//     and the K-major descriptor of K step k0 starts at row k0 - a + 31, with
//     8-row groups 128 bytes apart (SBO) and the second 4-column group 64
//     bytes on (LBO).  With output column n standing for t = 63 - n, both
//     offsets are positive.
//   * Chunk g accumulates into D[g & 1] [128 lanes][64 columns] FP32 in TMEM
//     (columns 0 and 64); one thread issues the MMAs and commits them to an
//     mbarrier; two chunks later the threads add D into registers.
// CTAs are persistent over tiles (two per SM: 256 TMEM columns each).
// Every wait is bounded: a wait that runs out sets kErrTimeout, and the CTA
// drains its copies and MMAs (bounded again), frees its TMEM and returns.
#include <algorithm>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "launch.h"

namespace gld {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTcStages = 3;
constexpr int kTcChunk = 32;                               // window rows per stage (4 K steps)
constexpr int kTcStageFloats = kTcChunk * 128;
constexpr int kTcStageBytes = kTcStageFloats * 4;          // 16 KB
constexpr uint32_t kTcCols = 256;                          // D buffers [0, 128), A buffers [128, 256)
constexpr int kTcRowOff = 94;                              // R[u] holds Acp[u - kTcRowOff + e]
constexpr long long kTcWaitCycles = 2000000000LL;          // about one second

// Instruction descriptor of tcgen05.mma kind::tf32: D FP32, A and B TF32,
// both K-major, N = 64, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t tf32_rna(float v)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}

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

__device__ __forceinline__ void mma_tf32(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}"
                 ::"r"(d), "r"(a), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate)
                 : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
                 ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                 "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
                 "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]),
                 "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]),
                 "r"(v[31])
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                   "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                   "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Chunks of the window: real rows [a, a + 2H + T) from the time t_lo.
__host__ __device__ inline int tc_nch_max(int H, int T) { return (31 + 2 * H + T + 31) / kTcChunk; }
// Rows of the overlapping tap array: every K-step tile of any window offset.
__host__ __device__ inline int tc_rows(int H, int T) { return kTcChunk * tc_nch_max(H, T) + 91; }

size_t tc_smem_bytes(int H, int T)
{
    const size_t b = 1024 + (size_t)kTcStages * kTcStageBytes + 2 * (size_t)tc_rows(H, T) * 16 + 64;
    // at least 80 KB: at most two CTAs (2 x 256 TMEM columns) share an SM
    return b < 80 * 1024 ? 80 * 1024 : b;
}

__global__ void __launch_bounds__(kTcThreads) fir_tc(const __grid_constant__ CUtensorMap wmap, const StepParams P,
                                                     Ctrl* __restrict__ ctrl, const float* __restrict__ taps,
                                                     float* __restrict__ out, int nrows)
{
    extern __shared__ unsigned char sm_raw[];
    const uint32_t raw = smem_u32(sm_raw);
    unsigned char* sm = sm_raw + (((raw + 1023u) & ~1023u) - raw);
    float* stage = (float*)sm;                                   // [kTcStages][32][128]
    float* Rhi = (float*)(sm + (size_t)kTcStages * kTcStageBytes);  // [nrows][4]
    float* Rlo = Rhi + 4 * (size_t)nrows;
    uint64_t* full = (uint64_t*)(Rlo + 4 * (size_t)nrows);       // [kTcStages]
    uint64_t* mdone = full + kTcStages;                          // [2]: MMAs of A buffer b done
    uint32_t* misc = (uint32_t*)(mdone + 2);                     // TMEM base

    const int tid = threadIdx.x, warp = tid >> 5;
    {
        // the layout below must fit the dynamic shared memory of the launch
        uint32_t dyn;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        const size_t used = (size_t)(sm - sm_raw) + (size_t)kTcStages * kTcStageBytes + 32 * (size_t)nrows + 64;
        if (used > dyn) {
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

    // taps as overlapping rows, TF32 part and remainder
    for (int idx = tid; idx < 4 * nrows; idx += kTcThreads) {
        const int sig = (idx >> 2) - kTcRowOff + (idx & 3);
        const float v = (sig >= 0 && sig <= 2 * H) ? __ldg(taps + sig) : 0.f;
        const float hi = __uint_as_float(tf32_rna(v));
        Rhi[idx] = hi;
        Rlo[idx] = v - hi;
    }
    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) mbar_init(&full[s], 1);
        mbar_init(&mdone[0], 1);
        mbar_init(&mdone[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the taps, for the tensor cores
    __syncwarp();  // .sync.aligned tcgen05 instructions need the whole warp converged
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&misc[0])),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = misc[0];
    // the allocation must start at lane 0 and hold the columns used
    const bool tm_ok = (tm >> 16) == 0 && (tm & 0xFFFFu) + kTcCols <= 512u;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const uint32_t rhi = smem_u32(Rhi), rlo = smem_u32(Rlo);

    long long issued = 0;     // chunks whose tile load was issued (thread 0)
    long long committed = -1; // last chunk whose MMAs were committed (thread 0)
    auto issue = [&](long long g) {
        const int i = (int)(g / nch), c = (int)(g - (long long)i * nch);
        const int tile = (int)blockIdx.x + i * (int)gridDim.x;
        const int st = (int)(g % kTcStages);
        long long slot = (t_lo + (long long)kTcChunk * c) % P.lw;
        if (slot < 0) slot += P.lw;
        const long long x = (long long)tile * 128;
        if (x >= np3 || (slot & 31) || slot + kTcChunk > P.lw) {  // never for a valid launch
            atomicOr(&ctrl->err, kErrCheck);
            mbar_expect_tx(&full[st], 0);  // completes the phase without a copy
            return;
        }
        mbar_expect_tx(&full[st], kTcStageBytes);
        tma_load_2d(stage + (size_t)st * kTcStageFloats, &wmap, (int)x, (int)slot, &full[st]);
    };
    if (tid == 0)
        for (; issued < G && issued < kTcStages - 1; ++issued) issue(issued);

    // Chunk g accumulates into a fresh D[g & 1] from A[g & 1]; two iterations
    // later (when both buffers are needed again) the threads add D into FP32
    // registers with round-to-nearest.  The tensor cores' own accumulation
    // rounds toward zero, and over the ~100-750 MMAs of a whole window that
    // bias reaches 1e-5 of the result; per chunk it stays near 4e-7.
    float acc[64];
#pragma unroll
    for (int q = 0; q < 64; ++q) acc[q] = 0.f;
    auto fold = [&](long long gg) {  // all threads; D[gg & 1] holds chunk gg
        const int fi = (int)(gg / nch), fc = (int)(gg - (long long)fi * nch);
        __syncwarp();
        tc_fence_after();
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            uint32_t d[32];
            tmem_ld32(tm + lane_base + 64u * (uint32_t)(gg & 1) + 32u * (uint32_t)half, d);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 32; ++q) acc[32 * half + q] = __fadd_rn(acc[32 * half + q], __uint_as_float(d[q]));
        }
        if (fc == nch - 1) {  // the tile is complete: to F^R (column n is t = 63 - n)
            const long long j = ((long long)blockIdx.x + (long long)fi * gridDim.x) * 128 + tid;
            if (j < np3)
#pragma unroll
                for (int q = 0; q < 64; ++q) out[(size_t)(63 - q) * np3 + j] = acc[q];
#pragma unroll
            for (int q = 0; q < 64; ++q) acc[q] = 0.f;
        }
    };

    // A wait that runs out makes this thread `bad`; the CTA learns of it at the
    // next barrier (__syncthreads_or: the same answer in every thread) and
    // stops streaming.
    bool bad = !tm_ok, aborted = false;
    long long g_stop = G;
    if (!tm_ok && tid == 0) atomicOr(&ctrl->err, kErrCheck);
    for (long long g = 0; g < G; ++g) {
        const int i = (int)(g / nch), c = (int)(g - (long long)i * nch);
        const int st = (int)(g % kTcStages), ab = (int)(g & 1);
        (void)i;
        if (tid == 0 && issued < G && issued <= g + kTcStages - 1) issue(issued++);
        if (!mbar_wait(&full[st], (uint32_t)((g / kTcStages) & 1))) bad = true;
        // A[ab] and D[ab] are free once the MMAs of chunk g - 2 are done
        if (g >= 2) {
            if (!mbar_wait(&mdone[ab], (uint32_t)(((g - 2) >> 1) & 1))) bad = true;
            if (tm_ok) fold(g - 2);
        }
        // this thread's stream: 32 window rows, zero outside the real window
        if (tm_ok) {
            uint32_t hv[32], lv[32];
            const float* sp = stage + (size_t)st * kTcStageFloats + tid;
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const int k = kTcChunk * c + r;
                float v = sp[r * 128];
                v = (k >= a && k < a + nk) ? v : 0.f;
                hv[r] = tf32_rna(v);
                lv[r] = __float_as_uint(v - __uint_as_float(hv[r]));
            }
            const uint32_t ta = tm + lane_base + 128u + 64u * (uint32_t)ab;
            __syncwarp();  // lanes leave the waits above at different times
            tmem_st32(ta, hv);
            tmem_st32(ta + 32u, lv);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        tc_fence_before();
        if (__syncthreads_or(bad)) {
            aborted = true;
            g_stop = g;
            break;
        }
        if (tid == 0) {
            tc_fence_after();
            const uint32_t dd = tm + 64u * (uint32_t)ab;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int k0 = kTcChunk * c + 8 * s;
                const uint32_t u0 = (uint32_t)(k0 - a - 63 + kTcRowOff);
                if (u0 + 68u > (uint32_t)nrows) {  // never for a valid launch
                    atomicOr(&ctrl->err, kErrCheck);
                    continue;
                }
                const uint64_t dh = smem_desc(rhi + 16u * u0, 64u, 128u);
                const uint64_t dl = smem_desc(rlo + 16u * u0, 64u, 128u);
                const uint32_t ah = tm + 128u + 64u * (uint32_t)ab + 8u * (uint32_t)s, al = ah + 32u;
                mma_tf32(dd, ah, dh, s > 0 ? 1u : 0u);
                mma_tf32(dd, ah, dl, 1u);
                mma_tf32(dd, al, dh, 1u);
            }
            mma_commit(&mdone[ab]);
            committed = g;
        }
    }
    // the last two chunks: wait for their MMAs, agree on the outcome, fold
    const long long g_last0 = G >= 2 ? G - 2 : 0;
    if (!aborted)
        for (long long gg = g_last0; gg < G; ++gg)
            if (!mbar_wait(&mdone[gg & 1], (uint32_t)((gg >> 1) & 1))) bad = true;
    if (__syncthreads_or(bad)) aborted = true;
    if (!aborted && tm_ok)
        for (long long gg = g_last0; gg < G; ++gg) fold(gg);
    tc_fence_before();
    if (aborted && tid == 0) {
        atomicOr(&ctrl->err, kErrTimeout);
        // drain (bounded): tile loads still in flight, then the last MMAs
        for (long long gg = g_stop; gg < issued; ++gg)
            mbar_wait(&full[gg % kTcStages], (uint32_t)((gg / kTcStages) & 1));
        if (committed >= 0) mbar_wait(&mdone[committed & 1], (uint32_t)((committed >> 1) & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
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
    return P.T == 64 && P.lw % kTcChunk == 0 && P.lw >= 2LL * P.H + P.T + 31 && tc_smem_bytes(P.H, P.T) <= 227 * 1024;
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
    const int grid = (int)std::min<long long>(ntiles, 2LL * std::max(num_sms, 1));
    fir_tc<<<grid, kTcThreads, smem, st>>>(*wmap, P, ctrl, taps, out, tc_rows(P.H, P.T));
    return cudaGetLastError();
}

}  // namespace gld
