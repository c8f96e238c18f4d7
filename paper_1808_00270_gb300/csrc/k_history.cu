// k_history.cu -- the history convolution of Eq. dissipative_force2.
//
// For every particle i and component c the dissipative force needs
//   S_i      = sum_{m=1}^{m_max-1} K^s_m       dR_{i,n-m}     (self term)
//   P_{i,q}  = sum_{m=1}^{m_max-1} g_q[m]      dR_{i,n-m}     (pair terms)
//   Ps_{i,q} = sum_{m=1}^{m_max-1} gs_q[m]     dR_{i,n-m}     (dK^s terms)
// With separable kernels K^p_m(r) = sum_q f_q(r) g_q[m] the pair sums of
// Eq. dissipative_force2 become sum_j f_q(r_ij) e e^T P_{j,q}, so the history
// ring is streamed exactly once per step, here.  This is the step that sets
// the cost: 12 (m_max-1) bytes per particle (FP32) against ~2 flops per
// byte per accumulator -- bound by HBM bandwidth, so no tensor cores.
//
// Layout: ring[slot][3][n_pad], slot = k mod (m_max-1) for dR_k.  Every slot
// is one contiguous row of 3 n_pad values; a thread owns one 16-byte column
// (4 consecutive values) and walks all slots with 8 loads in flight, so each
// warp reads 512 contiguous bytes per slot.  The ring is never rotated: the
// coefficients are (slot s holds m = ((n - s - 1) mod (m_max-1)) + 1),
// staged in shared memory.
//
// Launch shape: the block size is picked from the occupancy of the
// instantiation so that every column gets its own thread in ONE wave; a
// second partial wave would leave a handful of CTAs streaming alone at the
// end (measured: 768 CTAs on 760 resident slots cost +50 % at 262144
// particles).  Only when the columns exceed one full wave does the grid
// become persistent, each thread taking columns q, q + grid, ...
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include <cuda_bf16.h>

#include "launch.h"

namespace gld {

namespace {

constexpr int kThreads = 256;     // largest block; the launch picks 64 .. 256
constexpr int kUnroll = 8;         // loads issued together per thread

template <bool KAHAN>
__device__ __forceinline__ void acc1(float& s, float& comp, float c, float v)
{
    if (KAHAN) {
        const float y = fmaf(c, v, -comp);
        const float t = s + y;
        comp = (t - s) - y;
        s = t;
    } else {
        s = fmaf(c, v, s);
    }
}

template <int NACC>
__device__ __forceinline__ void stage_coefs(float* cs, const float* __restrict__ coef, int M, int H,
                                            long long n)
{
    int r0 = (int)((n - 1) % H);  // slot s holds m = ((n - 1 - s) mod H) + 1
    if (r0 < 0) r0 += H;
    for (int s = threadIdx.x; s < H; s += blockDim.x) {
        const int r = r0 - s;
        const int m = (r < 0 ? r + H : r) + 1;
#pragma unroll
        for (int a = 0; a < NACC; ++a) cs[s * NACC + a] = __ldg(coef + a * M + m);
    }
    __syncthreads();
}

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

template <bool BF16>
struct Col {
    using V = typename std::conditional<BF16, uint4, float4>::type;
    static constexpr int W = BF16 ? 8 : 4;  // values per 16-byte column
};

template <bool BF16>
__device__ __forceinline__ void unpack(const typename Col<BF16>::V v, float (&x)[Col<BF16>::W])
{
    if constexpr (BF16) {
        x[0] = bf_lo(v.x); x[1] = bf_hi(v.x); x[2] = bf_lo(v.y); x[3] = bf_hi(v.y);
        x[4] = bf_lo(v.z); x[5] = bf_hi(v.z); x[6] = bf_lo(v.w); x[7] = bf_hi(v.w);
    } else {
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
}

// One 16-byte column per thread over all slots, one wave (the common case;
// the lean form keeps the register count at 44 for two FP32 accumulators).
// Two FP32 accumulators fit in 40 registers: 6 CTAs of 256 threads per SM,
// enough for one wave of the 262144-particle suspension (768 CTAs).
template <int NACC, bool KAHAN, bool BF16>
__global__ void __launch_bounds__(kThreads, (NACC * Col<BF16>::W * (KAHAN ? 2 : 1) <= 8) ? 6 : 1)
    hist_conv_col(const typename Col<BF16>::V* __restrict__ ring, long long cols, int H,
                  const float* __restrict__ coef, int M, const long long* __restrict__ nstep, long long step,
                  float* __restrict__ out)
{
    using V = typename Col<BF16>::V;
    constexpr int VW = Col<BF16>::W;
    extern __shared__ float cs[];
    const long long n = nstep ? *nstep : step;
    stage_coefs<NACC>(cs, coef, M, H, n);
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cols) return;
    float acc[NACC][VW];
    float cmp[KAHAN ? NACC : 1][VW];
#pragma unroll
    for (int a = 0; a < NACC; ++a)
#pragma unroll
        for (int e = 0; e < VW; ++e) acc[a][e] = 0.f;
#pragma unroll
    for (int a = 0; a < (KAHAN ? NACC : 1); ++a)
#pragma unroll
        for (int e = 0; e < VW; ++e) cmp[a][e] = 0.f;
    const V* p = ring + q;
    int s = 0;
    for (; s + kUnroll <= H; s += kUnroll) {
        V v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) v[u] = __ldcs(p + (long long)(s + u) * cols);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            float x[VW];
            unpack<BF16>(v[u], x);
#pragma unroll
            for (int a = 0; a < NACC; ++a) {
                const float cf = cs[(s + u) * NACC + a];
#pragma unroll
                for (int e = 0; e < VW; ++e) acc1<KAHAN>(acc[a][e], cmp[KAHAN ? a : 0][e], cf, x[e]);
            }
        }
    }
    for (; s < H; ++s) {
        float x[VW];
        unpack<BF16>(__ldcs(p + (long long)s * cols), x);
#pragma unroll
        for (int a = 0; a < NACC; ++a) {
            const float cf = cs[s * NACC + a];
#pragma unroll
            for (int e = 0; e < VW; ++e) acc1<KAHAN>(acc[a][e], cmp[KAHAN ? a : 0][e], cf, x[e]);
        }
    }
    float4* o = (float4*)out;
    const long long cols4 = cols * (VW / 4);
#pragma unroll
    for (int a = 0; a < NACC; ++a)
#pragma unroll
        for (int h = 0; h < VW / 4; ++h) {
            float r[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) r[e] = KAHAN ? acc[a][4 * h + e] - cmp[KAHAN ? a : 0][4 * h + e] : acc[a][4 * h + e];
            o[a * cols4 + q * (VW / 4) + h] = make_float4(r[0], r[1], r[2], r[3]);
        }
}

// One 16-byte column (4 FP32 or 8 BF16 values) per thread and slot group.
// The G threads of a column split its slots into G contiguous ranges and are
// combined in shared memory in a fixed order.  Loads run as a rolling
// pipeline: a register is refilled with the slot kUnroll ahead as soon as it
// is consumed, so kUnroll loads per thread stay in flight.
template <int NACC, bool KAHAN, bool BF16>
__global__ void __launch_bounds__(kThreads)
    hist_conv(const typename Col<BF16>::V* __restrict__ ring, long long cols, int H, const float* __restrict__ coef,
              int M, const long long* __restrict__ nstep, long long step, float* __restrict__ out, int G)
{
    using V = typename Col<BF16>::V;
    constexpr int VW = Col<BF16>::W;
    extern __shared__ float cs[];
    __shared__ float4 red[kThreads * (BF16 ? 2 : 1)];
    const long long n = nstep ? *nstep : step;
    stage_coefs<NACC>(cs, coef, M, H, n);
    const int per = blockDim.x / G;  // columns per block
    const int g = threadIdx.x / per, c = threadIdx.x - g * per;
    const int s_lo = (int)((long long)g * H / G), s_hi = (int)((long long)(g + 1) * H / G);
    for (long long qb = (long long)blockIdx.x * per; qb < cols; qb += (long long)gridDim.x * per) {
        const long long q = qb + c;
        float acc[NACC][VW];
        float cmp[KAHAN ? NACC : 1][VW];
#pragma unroll
        for (int a = 0; a < NACC; ++a)
#pragma unroll
            for (int e = 0; e < VW; ++e) acc[a][e] = 0.f;
#pragma unroll
        for (int a = 0; a < (KAHAN ? NACC : 1); ++a)
#pragma unroll
            for (int e = 0; e < VW; ++e) cmp[a][e] = 0.f;
        if (q < cols) {
            const V* p = ring + q;
            int s = s_lo;
            for (; s + kUnroll <= s_hi; s += kUnroll) {
                V v[kUnroll];
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) v[u] = __ldcs(p + (long long)(s + u) * cols);
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    float x[VW];
                    unpack<BF16>(v[u], x);
#pragma unroll
                    for (int a = 0; a < NACC; ++a) {
                        const float cf = cs[(s + u) * NACC + a];
#pragma unroll
                        for (int e = 0; e < VW; ++e) acc1<KAHAN>(acc[a][e], cmp[KAHAN ? a : 0][e], cf, x[e]);
                    }
                }
            }
            for (; s < s_hi; ++s) {
                float x[VW];
                unpack<BF16>(__ldcs(p + (long long)s * cols), x);
#pragma unroll
                for (int a = 0; a < NACC; ++a) {
                    const float cf = cs[s * NACC + a];
#pragma unroll
                    for (int e = 0; e < VW; ++e) acc1<KAHAN>(acc[a][e], cmp[KAHAN ? a : 0][e], cf, x[e]);
                }
            }
            if constexpr (KAHAN) {
#pragma unroll
                for (int a = 0; a < NACC; ++a)
#pragma unroll
                    for (int e = 0; e < VW; ++e) acc[a][e] -= cmp[a][e];  // compensated value
            }
        }
        float4* o = (float4*)out;
        const long long cols4 = cols * (VW / 4);  // float4 per accumulator row
        if (G == 1) {
            if (q < cols)
#pragma unroll
                for (int a = 0; a < NACC; ++a)
#pragma unroll
                    for (int h = 0; h < VW / 4; ++h)
                        o[a * cols4 + q * (VW / 4) + h] =
                            make_float4(acc[a][4 * h], acc[a][4 * h + 1], acc[a][4 * h + 2], acc[a][4 * h + 3]);
        } else {
            // fixed-order combine of the G slot ranges, one accumulator at a time
#pragma unroll
            for (int a = 0; a < NACC; ++a) {
#pragma unroll
                for (int h = 0; h < VW / 4; ++h)
                    red[threadIdx.x * (VW / 4) + h] =
                        make_float4(acc[a][4 * h], acc[a][4 * h + 1], acc[a][4 * h + 2], acc[a][4 * h + 3]);
                __syncthreads();
                if (g == 0 && q < cols) {
#pragma unroll
                    for (int h = 0; h < VW / 4; ++h) {
                        float4 t = red[c * (VW / 4) + h];
                        for (int gg = 1; gg < G; ++gg) {
                            const float4 y = red[(gg * per + c) * (VW / 4) + h];
                            t.x += y.x; t.y += y.y; t.z += y.z; t.w += y.w;
                        }
                        o[a * cols4 + q * (VW / 4) + h] = t;
                    }
                }
                __syncthreads();
            }
        }
    }
}

// Launch shape (see the header).  Registers are allocated per warp, so small
// blocks can use every warp slot the registers allow (44 registers: 42 warps
// per SM, but only 40 in 128-thread blocks).  Returns the largest block size
// among 256..64 with which one wave of `kern` covers `items` threads, or 0.
template <class K>
cudaError_t one_wave_block(K kern, long long items, size_t smem, int* block, long long* best_cap, int* best_b)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    *block = 0;
    for (int b : {256, 128, 96, 64}) {
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, b, smem);
        if (e != cudaSuccess) return e;
        const long long cap = (long long)occ * sms * b;  // resident threads
        if (cap > *best_cap) {
            *best_cap = cap;
            *best_b = b;
        }
        if (cap >= items && *block == 0) *block = b;
    }
    return cudaSuccess;
}

// A launch decision, cached per (device, columns, slots) for each
// instantiation: the occupancy queries cost far more host time than a launch.
struct Shape {
    int kind;  // 0: one column per thread, 1: general kernel
    int block, G;
    unsigned grid;
};

template <int NACC, bool KAHAN, bool BF16>
cudaError_t choose_shape(long long cols, int H, size_t smem, Shape* out);

template <int NACC, bool KAHAN, bool BF16>
cudaError_t launch_tb(const void* ring, int n_pad, int M, const long long* nstep, long long step, const float* coef,
                      float* out, cudaStream_t st)
{
    using V = typename Col<BF16>::V;
    static std::mutex mu;
    static std::map<std::tuple<int, long long, int>, Shape> cache;
    const int H = M - 1;
    const size_t smem = sizeof(float) * (size_t)H * NACC;
    const long long cols = 3LL * n_pad / Col<BF16>::W;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    Shape sh{};
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find({dev, cols, H});
        if (it != cache.end()) {
            sh = it->second;
        } else {
            if ((e = choose_shape<NACC, KAHAN, BF16>(cols, H, smem, &sh)) != cudaSuccess) return e;
            cache[{dev, cols, H}] = sh;
        }
    }
    if (sh.kind == 0)
        hist_conv_col<NACC, KAHAN, BF16><<<sh.grid, sh.block, smem, st>>>((const V*)ring, cols, H, coef, M, nstep, step,
                                                                          out);
    else
        hist_conv<NACC, KAHAN, BF16><<<sh.grid, sh.block, smem, st>>>((const V*)ring, cols, H, coef, M, nstep, step,
                                                                      out, sh.G);
    return cudaGetLastError();
}

template <int NACC, bool KAHAN, bool BF16>
cudaError_t choose_shape(long long cols, int H, size_t smem, Shape* out)
{
    auto kc = hist_conv_col<NACC, KAHAN, BF16>;
    auto kg = hist_conv<NACC, KAHAN, BF16>;
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(kg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    int b1 = 0, bcap_b = kThreads;
    long long bcap = 0;
    cudaError_t e = one_wave_block(kc, cols, smem, &b1, &bcap, &bcap_b);
    if (e != cudaSuccess) return e;
    // Room for twice the threads in one wave: split each column's slots (not
    // with compensated sums, which stay one sequence over all m).
    int G = 1, bg = 0, gcap_b = kThreads;
    long long gcap = 0;
    for (int g = 4; g >= 2 && b1 && !KAHAN; g /= 2) {
        if (H < 16 * g) continue;
        int b = 0;
        gcap = 0;
        if ((e = one_wave_block(kg, cols * g, smem, &b, &gcap, &gcap_b)) != cudaSuccess) return e;
        if (b && b / g >= 32) {
            G = g;
            bg = b;
            break;
        }
    }
    if (G > 1) {
        const int per = bg / G;
        *out = Shape{1, bg, G, (unsigned)((cols + per - 1) / per)};
    } else if (b1) {
        *out = Shape{0, b1, 1, (unsigned)((cols + b1 - 1) / b1)};
    } else {
        // more columns than one wave: a persistent grid of the resident CTAs
        long long cap = 0;
        int b = 0, cb = kThreads;
        if ((e = one_wave_block(kg, cols, smem, &b, &cap, &cb)) != cudaSuccess) return e;
        *out = Shape{1, cb, 1, (unsigned)std::max(1LL, cap / cb)};
    }
    return cudaSuccess;
}

template <int NACC, bool KAHAN>
cudaError_t launch_t(const void* ring, int bf16, int n_pad, int M, const long long* nstep, long long step,
                     const float* coef, float* out, cudaStream_t st)
{
    return bf16 ? launch_tb<NACC, KAHAN, true>(ring, n_pad, M, nstep, step, coef, out, st)
                : launch_tb<NACC, KAHAN, false>(ring, n_pad, M, nstep, step, coef, out, st);
}

template <bool KAHAN>
cudaError_t dispatch(int nacc, const void* ring, int bf16, int n_pad, int M, const long long* nstep,
                     long long step, const float* coef, float* out, cudaStream_t st)
{
    switch (nacc) {
    case 1: return launch_t<1, KAHAN>(ring, bf16, n_pad, M, nstep, step, coef, out, st);
    case 2: return launch_t<2, KAHAN>(ring, bf16, n_pad, M, nstep, step, coef, out, st);
    case 3: return launch_t<3, KAHAN>(ring, bf16, n_pad, M, nstep, step, coef, out, st);
    case 4: return launch_t<4, KAHAN>(ring, bf16, n_pad, M, nstep, step, coef, out, st);
    case 5: return launch_t<5, KAHAN>(ring, bf16, n_pad, M, nstep, step, coef, out, st);
    case 6: return launch_t<6, KAHAN>(ring, bf16, n_pad, M, nstep, step, coef, out, st);
    case 7: return launch_t<7, KAHAN>(ring, bf16, n_pad, M, nstep, step, coef, out, st);
    case 8: return launch_t<8, KAHAN>(ring, bf16, n_pad, M, nstep, step, coef, out, st);
    case 9: return launch_t<9, KAHAN>(ring, bf16, n_pad, M, nstep, step, coef, out, st);
    default: return cudaErrorInvalidValue;
    }
}

// Batch convolution: tile (member, 256-column block); the member's
// coefficients are staged for its own step and memory length.
template <int NACC, bool KAHAN, bool BF16>
__global__ void __launch_bounds__(kBatchConvCols)
    b_conv(const SysDesc* __restrict__ D, const Tile* __restrict__ tiles)
{
    using V = typename Col<BF16>::V;
    constexpr int VW = Col<BF16>::W;
    extern __shared__ float cs[];
    const Tile t = tiles[blockIdx.x];
    const SysDesc& d = D[t.m];
    const int H = d.P.H, M = d.P.m_max;
    stage_coefs<NACC>(cs, d.coef, M, H, d.B.ctrl->step);
    const long long cols = 3LL * d.P.n_pad / VW;
    // columns b*bd + tid, then strided by the member's tiles in this schedule
    for (long long q = (long long)t.b * blockDim.x + threadIdx.x; q < cols; q += (long long)t.nb * blockDim.x) {
    const V* p = (const V*)d.B.ring + q;
    float acc[NACC][VW];
    float cmp[KAHAN ? NACC : 1][VW];
#pragma unroll
    for (int a = 0; a < NACC; ++a)
#pragma unroll
        for (int e = 0; e < VW; ++e) acc[a][e] = 0.f;
#pragma unroll
    for (int a = 0; a < (KAHAN ? NACC : 1); ++a)
#pragma unroll
        for (int e = 0; e < VW; ++e) cmp[a][e] = 0.f;
    int s = 0;
    for (; s + kUnroll <= H; s += kUnroll) {
        V v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) v[u] = __ldcs(p + (long long)(s + u) * cols);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            float x[VW];
            unpack<BF16>(v[u], x);
#pragma unroll
            for (int a = 0; a < NACC; ++a) {
                const float cf = cs[(s + u) * NACC + a];
#pragma unroll
                for (int e = 0; e < VW; ++e) acc1<KAHAN>(acc[a][e], cmp[KAHAN ? a : 0][e], cf, x[e]);
            }
        }
    }
    for (; s < H; ++s) {
        float x[VW];
        unpack<BF16>(__ldcs(p + (long long)s * cols), x);
#pragma unroll
        for (int a = 0; a < NACC; ++a) {
            const float cf = cs[s * NACC + a];
#pragma unroll
            for (int e = 0; e < VW; ++e) acc1<KAHAN>(acc[a][e], cmp[KAHAN ? a : 0][e], cf, x[e]);
        }
    }
    float4* o = (float4*)d.B.conv;
    const long long cols4 = cols * (VW / 4);
#pragma unroll
    for (int a = 0; a < NACC; ++a)
#pragma unroll
        for (int h = 0; h < VW / 4; ++h) {
            float r[4];
#pragma unroll
            for (int e = 0; e < 4; ++e)
                r[e] = KAHAN ? acc[a][4 * h + e] - cmp[KAHAN ? a : 0][4 * h + e] : acc[a][4 * h + e];
            o[a * cols4 + q * (VW / 4) + h] = make_float4(r[0], r[1], r[2], r[3]);
        }
    }
}

template <int NACC, bool KAHAN>
cudaError_t launch_b_conv_t(const BatchPlan& bp, cudaStream_t st)
{
    const size_t smem = sizeof(float) * (size_t)bp.max_H * NACC;
    auto k = bp.bf16 ? b_conv<NACC, KAHAN, true> : b_conv<NACC, KAHAN, false>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<bp.n_conv, bp.conv_block, smem, st>>>(bp.desc, bp.conv);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_batch_conv(const BatchPlan& bp, cudaStream_t st)
{
    if (!bp.n_conv) return cudaSuccess;
    const bool k = bp.kahan != 0;
    switch (bp.nacc) {
    case 1: return k ? launch_b_conv_t<1, true>(bp, st) : launch_b_conv_t<1, false>(bp, st);
    case 2: return k ? launch_b_conv_t<2, true>(bp, st) : launch_b_conv_t<2, false>(bp, st);
    case 3: return k ? launch_b_conv_t<3, true>(bp, st) : launch_b_conv_t<3, false>(bp, st);
    case 4: return k ? launch_b_conv_t<4, true>(bp, st) : launch_b_conv_t<4, false>(bp, st);
    case 5: return k ? launch_b_conv_t<5, true>(bp, st) : launch_b_conv_t<5, false>(bp, st);
    case 6: return k ? launch_b_conv_t<6, true>(bp, st) : launch_b_conv_t<6, false>(bp, st);
    case 7: return k ? launch_b_conv_t<7, true>(bp, st) : launch_b_conv_t<7, false>(bp, st);
    case 8: return k ? launch_b_conv_t<8, true>(bp, st) : launch_b_conv_t<8, false>(bp, st);
    case 9: return k ? launch_b_conv_t<9, true>(bp, st) : launch_b_conv_t<9, false>(bp, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_hist_conv(const void* ring, int bf16, int n_pad, int m_max, const Ctrl* ctrl,
                             long long step, const float* coef, int nacc, float* out, int kahan,
                             cudaStream_t st)
{
    if (m_max < 2 || n_pad <= 0 || n_pad % 32 != 0 || nacc < 1 || nacc > kMaxAcc) return cudaErrorInvalidValue;
    const long long* nstep = ctrl ? &ctrl->step : nullptr;
    return kahan ? dispatch<true>(nacc, ring, bf16, n_pad, m_max, nstep, step, coef, out, st)
                 : dispatch<false>(nacc, ring, bf16, n_pad, m_max, nstep, step, coef, out, st);
}

cudaError_t launch_hist_conv_next(const void* ring, int bf16, int n_pad, int m_max, const Ctrl* ctrl,
                                  const float* coef, int nacc, float* out, int kahan, cudaStream_t st)
{
    if (m_max < 2 || n_pad <= 0 || n_pad % 32 != 0 || nacc < 1 || nacc > kMaxAcc || !ctrl) return cudaErrorInvalidValue;
    return kahan ? dispatch<true>(nacc, ring, bf16, n_pad, m_max, &ctrl->conv_step, 0, coef, out, st)
                 : dispatch<false>(nacc, ring, bf16, n_pad, m_max, &ctrl->conv_step, 0, coef, out, st);
}

}  // namespace gld
