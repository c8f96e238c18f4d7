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
// (4 consecutive values) and walks all slots, so each warp reads 512
// contiguous bytes per slot.  The ring is never rotated: the coefficients are
// (slot s holds m = ((n - s - 1) mod (m_max-1)) + 1), staged in shared memory.
#include <cuda_bf16.h>

#include "launch.h"

namespace gld {

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 8;

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
    for (int s = threadIdx.x; s < H; s += blockDim.x) {
        long long r = (n - s - 1) % H;
        if (r < 0) r += H;
        const int m = (int)r + 1;
#pragma unroll
        for (int a = 0; a < NACC; ++a) cs[s * NACC + a] = __ldg(coef + a * M + m);
    }
    __syncthreads();
}

// FP32 ring: one float4 column per thread.
template <int NACC, bool KAHAN>
__global__ void __launch_bounds__(kThreads) hist_conv_f32(const float4* __restrict__ ring, long long cols,
                                                          int H, const float* __restrict__ coef, int M,
                                                          const Ctrl* __restrict__ ctrl, long long step,
                                                          float4* __restrict__ out)
{
    extern __shared__ float cs[];
    const long long n = ctrl ? ctrl->step : step;
    stage_coefs<NACC>(cs, coef, M, H, n);
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cols) return;
    float4 acc[NACC], cmp[NACC];
#pragma unroll
    for (int a = 0; a < NACC; ++a) acc[a] = cmp[a] = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4* p = ring + q;
    int s = 0;
    for (; s + kUnroll <= H; s += kUnroll) {
        float4 v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) v[u] = __ldcs(p + (long long)(s + u) * cols);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int a = 0; a < NACC; ++a) {
                const float c = cs[(s + u) * NACC + a];
                acc1<KAHAN>(acc[a].x, cmp[a].x, c, v[u].x);
                acc1<KAHAN>(acc[a].y, cmp[a].y, c, v[u].y);
                acc1<KAHAN>(acc[a].z, cmp[a].z, c, v[u].z);
                acc1<KAHAN>(acc[a].w, cmp[a].w, c, v[u].w);
            }
        }
    }
    for (; s < H; ++s) {
        const float4 v = __ldcs(p + (long long)s * cols);
#pragma unroll
        for (int a = 0; a < NACC; ++a) {
            const float c = cs[s * NACC + a];
            acc1<KAHAN>(acc[a].x, cmp[a].x, c, v.x);
            acc1<KAHAN>(acc[a].y, cmp[a].y, c, v.y);
            acc1<KAHAN>(acc[a].z, cmp[a].z, c, v.z);
            acc1<KAHAN>(acc[a].w, cmp[a].w, c, v.w);
        }
    }
#pragma unroll
    for (int a = 0; a < NACC; ++a) out[a * cols + q] = acc[a];
}

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// BF16 ring: one 16-byte column of 8 values per thread, FP32 accumulation.
template <int NACC, bool KAHAN>
__global__ void __launch_bounds__(kThreads) hist_conv_bf16(const uint4* __restrict__ ring, long long cols,
                                                           int H, const float* __restrict__ coef, int M,
                                                           const Ctrl* __restrict__ ctrl, long long step,
                                                           float4* __restrict__ out)
{
    extern __shared__ float cs[];
    const long long n = ctrl ? ctrl->step : step;
    stage_coefs<NACC>(cs, coef, M, H, n);
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cols) return;
    float acc[NACC][8], cmp[NACC][8];
#pragma unroll
    for (int a = 0; a < NACC; ++a)
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[a][e] = cmp[a][e] = 0.f;
    const uint4* p = ring + q;
    int s = 0;
    for (; s + kUnroll <= H; s += kUnroll) {
        uint4 v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) v[u] = __ldcs(p + (long long)(s + u) * cols);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const float x[8] = {bf_lo(v[u].x), bf_hi(v[u].x), bf_lo(v[u].y), bf_hi(v[u].y),
                                bf_lo(v[u].z), bf_hi(v[u].z), bf_lo(v[u].w), bf_hi(v[u].w)};
#pragma unroll
            for (int a = 0; a < NACC; ++a) {
                const float c = cs[(s + u) * NACC + a];
#pragma unroll
                for (int e = 0; e < 8; ++e) acc1<KAHAN>(acc[a][e], cmp[a][e], c, x[e]);
            }
        }
    }
    for (; s < H; ++s) {
        const uint4 w = __ldcs(p + (long long)s * cols);
        const float x[8] = {bf_lo(w.x), bf_hi(w.x), bf_lo(w.y), bf_hi(w.y),
                            bf_lo(w.z), bf_hi(w.z), bf_lo(w.w), bf_hi(w.w)};
#pragma unroll
        for (int a = 0; a < NACC; ++a) {
            const float c = cs[s * NACC + a];
#pragma unroll
            for (int e = 0; e < 8; ++e) acc1<KAHAN>(acc[a][e], cmp[a][e], c, x[e]);
        }
    }
    const long long cols4 = 2 * cols;
#pragma unroll
    for (int a = 0; a < NACC; ++a) {
        out[a * cols4 + 2 * q] = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
        out[a * cols4 + 2 * q + 1] = make_float4(acc[a][4], acc[a][5], acc[a][6], acc[a][7]);
    }
}

template <int NACC, bool KAHAN>
cudaError_t launch_t(const void* ring, int bf16, int n_pad, int M, const Ctrl* ctrl, long long step,
                     const float* coef, float* out, cudaStream_t st)
{
    const int H = M - 1;
    const size_t smem = sizeof(float) * (size_t)H * NACC;
    const long long vals = 3LL * n_pad;
    if (bf16) {
        const long long cols = vals / 8;
        const unsigned grid = (unsigned)((cols + kThreads - 1) / kThreads);
        auto k = hist_conv_bf16<NACC, KAHAN>;
        if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, kThreads, smem, st>>>((const uint4*)ring, cols, H, coef, M, ctrl, step, (float4*)out);
    } else {
        const long long cols = vals / 4;
        const unsigned grid = (unsigned)((cols + kThreads - 1) / kThreads);
        auto k = hist_conv_f32<NACC, KAHAN>;
        if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, kThreads, smem, st>>>((const float4*)ring, cols, H, coef, M, ctrl, step, (float4*)out);
    }
    return cudaGetLastError();
}

template <bool KAHAN>
cudaError_t dispatch(int nacc, const void* ring, int bf16, int n_pad, int M, const Ctrl* ctrl,
                     long long step, const float* coef, float* out, cudaStream_t st)
{
    switch (nacc) {
    case 1: return launch_t<1, KAHAN>(ring, bf16, n_pad, M, ctrl, step, coef, out, st);
    case 2: return launch_t<2, KAHAN>(ring, bf16, n_pad, M, ctrl, step, coef, out, st);
    case 3: return launch_t<3, KAHAN>(ring, bf16, n_pad, M, ctrl, step, coef, out, st);
    case 4: return launch_t<4, KAHAN>(ring, bf16, n_pad, M, ctrl, step, coef, out, st);
    case 5: return launch_t<5, KAHAN>(ring, bf16, n_pad, M, ctrl, step, coef, out, st);
    case 6: return launch_t<6, KAHAN>(ring, bf16, n_pad, M, ctrl, step, coef, out, st);
    case 7: return launch_t<7, KAHAN>(ring, bf16, n_pad, M, ctrl, step, coef, out, st);
    case 8: return launch_t<8, KAHAN>(ring, bf16, n_pad, M, ctrl, step, coef, out, st);
    case 9: return launch_t<9, KAHAN>(ring, bf16, n_pad, M, ctrl, step, coef, out, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_hist_conv(const void* ring, int bf16, int n_pad, int m_max, const Ctrl* ctrl,
                             long long step, const float* coef, int nacc, float* out, int kahan,
                             cudaStream_t st)
{
    if (m_max < 2 || n_pad <= 0 || n_pad % 32 != 0 || nacc < 1 || nacc > kMaxAcc) return cudaErrorInvalidValue;
    return kahan ? dispatch<true>(nacc, ring, bf16, n_pad, m_max, ctrl, step, coef, out, st)
                 : dispatch<false>(nacc, ring, bf16, n_pad, m_max, ctrl, step, coef, out, st);
}

}  // namespace gld
