// k_modes.cu -- the memory sums of Eq. dissipative_force2 in auxiliary-
// variable form, for kernels that are sums of damped exponentials and
// cosines (the alternative to the history ring discussed in App. C).
//
// With modes z_k = exp((-rate_k + i omega_k) dt), the weights of every
// accumulator a (self kernel, pair and self-difference terms) for m >= 1 are
//   w_a[m] = sum_k ( x_ak Re z_k^m + y_ak Im z_k^m ),
// so with the per-particle, per-component auxiliary sums
//   Y_k(n) = sum_{m=1}^{H} z_k^m dR_{n-m}          (H = m_max - 1)
// the history projections are S_a(n) = sum_k x_ak Re Y_k(n) + y_ak Im Y_k(n)
// -- the same truncated convolution, now O(1) per particle and step in m_max:
//   Y_k(n+1) = z_k ( dR_n + Y_k(n) - z_k^H dR_{n-H} ).
// The kernel of step n runs where the convolution ran (before the pair kernel,
// which overwrites the ring slot of dR_{n-H} with dR_n), so it stores
//   Y'_k(n) = Y_k(n) - z_k^H dR_{n-H}   (slot n mod H still holds dR_{n-H})
// and the next step completes Y_k(n+1) = z_k (dR_n + Y'_k(n)).
#include <cuda_bf16.h>

#include "launch.h"

namespace gld {
namespace {

constexpr int kModeThreads = 256;

__device__ __forceinline__ float ring_at(const void* ring, int bf16, long long slot, long long plane_off)
{
    if (bf16) return __bfloat162float(((const __nv_bfloat16*)ring)[slot * plane_off]);
    return ((const float*)ring)[slot * plane_off];
}

// Thread (c, i): component c of particle i.  coef[k] = {zr, zi, zHr, zHi};
// w[a * nm + k] = {x_ak, y_ak}.
__global__ void __launch_bounds__(kModeThreads)
    modes_step(const StepParams P, const Ctrl* __restrict__ ctrl, const void* __restrict__ ring,
               const float4* __restrict__ coef, const float2* __restrict__ w, float2* __restrict__ Y,
               float* __restrict__ conv)
{
    const long long np = P.n_pad, cols = 3 * np;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cols) return;
    const long long hs = ctrl->hslot;                    // n mod H: holds dR_{n-H}
    const long long prev = hs == 0 ? P.H - 1 : hs - 1;   // holds dR_{n-1}
    const float x1 = ring_at((const char*)ring + (P.hist_bf16 ? 2 : 4) * t, P.hist_bf16, prev, cols);
    const float xH = ring_at((const char*)ring + (P.hist_bf16 ? 2 : 4) * t, P.hist_bf16, hs, cols);
    float s[kMaxAcc];
#pragma unroll
    for (int a = 0; a < kMaxAcc; ++a) s[a] = 0.f;
    for (int k = 0; k < P.nmodes; ++k) {
        const float4 z = __ldg(coef + k);
        const float2 yp = Y[(size_t)k * cols + t];
        const float ur = x1 + yp.x;
        const float yr = ur * z.x - yp.y * z.y;  // Y_k(n) = z (dR_{n-1} + Y'_k(n-1))
        const float yi = ur * z.y + yp.y * z.x;
#pragma unroll
        for (int a = 0; a < kMaxAcc; ++a)
            if (a < P.nacc) {
                const float2 c = __ldg(w + a * P.nmodes + k);
                s[a] = fmaf(c.x, yr, fmaf(c.y, yi, s[a]));
            }
        Y[(size_t)k * cols + t] = make_float2(yr - z.z * xH, yi - z.w * xH);  // Y'_k(n)
    }
#pragma unroll
    for (int a = 0; a < kMaxAcc; ++a)
        if (a < P.nacc) conv[(size_t)a * cols + t] = s[a];
}

// Y'_k(n0 - 1) = Y_k(n0) / z_k - dR_{n0-1} from the ring as it stands, with
// Y_k(n0) = sum_{m=1}^{H} z^m dR_{n0-m} by Horner's rule in FP64 (one-off).
__global__ void __launch_bounds__(kModeThreads)
    modes_init(const StepParams P, const Ctrl* __restrict__ ctrl, const void* __restrict__ ring,
               const double* __restrict__ zd, float2* __restrict__ Y)
{
    const long long np = P.n_pad, cols = 3 * np;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cols) return;
    const long long hs = ctrl->hslot;
    const char* base = (const char*)ring + (P.hist_bf16 ? 2 : 4) * t;
    for (int k = 0; k < P.nmodes; ++k) {
        const double zr = zd[2 * k], zi = zd[2 * k + 1];
        double ar = 0.0, ai = 0.0;
        for (int m = P.H; m >= 1; --m) {
            long long slot = (hs - m) % P.H;
            slot = slot < 0 ? slot + P.H : slot;
            const double x = ring_at(base, P.hist_bf16, slot, cols);
            const double ur = ar + x;
            ar = ur * zr - ai * zi;
            ai = ur * zi + ai * zr;
        }
        long long s1 = hs - 1;
        s1 = s1 < 0 ? s1 + P.H : s1;
        const double x1 = ring_at(base, P.hist_bf16, s1, cols);
        const double den = zr * zr + zi * zi;  // Y / z
        const double qr = (ar * zr + ai * zi) / den, qi = (ai * zr - ar * zi) / den;
        Y[(size_t)k * cols + t] = make_float2((float)(qr - x1), (float)qi);
    }
}

}  // namespace

cudaError_t launch_modes_step(const StepParams& P, const Ctrl* ctrl, const void* ring, const float4* coef,
                              const float2* w, float2* Y, float* conv, cudaStream_t st)
{
    const long long cols = 3LL * P.n_pad;
    const unsigned grid = (unsigned)((cols + kModeThreads - 1) / kModeThreads);
    modes_step<<<grid, kModeThreads, 0, st>>>(P, ctrl, ring, coef, w, Y, conv);
    return cudaGetLastError();
}

cudaError_t launch_modes_init(const StepParams& P, const Ctrl* ctrl, const void* ring, const double* zd, float2* Y,
                              cudaStream_t st)
{
    const long long cols = 3LL * P.n_pad;
    const unsigned grid = (unsigned)((cols + kModeThreads - 1) / kModeThreads);
    modes_init<<<grid, kModeThreads, 0, st>>>(P, ctrl, ring, zd, Y);
    return cudaGetLastError();
}

}  // namespace gld
