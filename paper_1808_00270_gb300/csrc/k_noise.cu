// k_noise.cu -- kernel preparation and the colored random force.
//
// prep (one block, FP64): discrete kernels of Eq. k-discrete, the noise target
//   C_m = kT a_m K^s_m / dt (Eq. FDT_discretized, a_0 = 2), its transform over
//   the 2 m_max - 1 points of Eq. FT, the positive-semi-definiteness check,
//   A_s = inverse transform of sqrt(hat C) (Sec. II C, with 1/(2 m_max - 1)),
//   and the integrator factors a, b of Eq. aa-bb.
// wgen: white noise W_{i,k} from Philox4x32-10 into a ring of times, each
//   (particle, time) drawn exactly once over the whole run.
// fir:  F^R_{i,n+t} = sum_{s=-(m_max-1)}^{m_max-1} A_s W_{i,n+t+s} for a block
//   of T steps at once (the windowed generation remarked on in Sec. II C):
//   one thread per (particle, component) keeps T outputs in registers and
//   streams its W window once; the taps come from shared memory as 16-byte
//   broadcasts out of four shifted, zero-padded copies of A.
#include "launch.h"

namespace gld {

namespace {

constexpr int kPrepThreads = 1024;

__device__ double cos_frac(long long w, long long m, long long L)
{
    long long r = (w * m) % L;
    if (r < 0) r += L;
    return cospi(2.0 * (double)r / (double)L);
}

__device__ double block_reduce(double v, double* sh, bool is_max)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            sh[threadIdx.x] = is_max ? fmax(sh[threadIdx.x], sh[threadIdx.x + w]) : sh[threadIdx.x] + sh[threadIdx.x + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__device__ double discretize(const double* s, int m, double dt, int discrete)
{
    if (discrete) return s[m];
    return m == 0 ? 0.5 * dt * s[0] : dt * s[m];
}

__global__ void __launch_bounds__(kPrepThreads) prep(const PrepArgs a)
{
    extern __shared__ double Ahat[];  // [m_max]
    __shared__ double red[kPrepThreads];
    const int M = a.m_max, H = M - 1;
    const long long L = 2LL * M - 1;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const double k = discretize(a.Ks, m, a.dt, a.discrete);
        a.Kd[m] = k;
        a.coef[m] = (float)k;
        a.C[m] = a.kT * (m == 0 ? 2.0 : 1.0) * k / a.dt;
        for (int q = 0; q < a.Q; ++q) {
            const double g = discretize(a.g + (size_t)q * M, m, a.dt, a.discrete);
            a.coef[(size_t)(1 + q) * M + m] = (float)g;
            if (m == 0) a.g0[q] = (float)g;
        }
        for (int q = 0; q < a.Qs; ++q) {
            const double g = discretize(a.gs + (size_t)q * M, m, a.dt, a.discrete);
            a.coef[(size_t)(1 + a.Q + q) * M + m] = (float)g;
            if (m == 0) a.g0[a.Q + q] = (float)g;
        }
    }
    __syncthreads();
    double lmax = 0.0, lmin = 1e300;
    for (int w = threadIdx.x; w < M; w += blockDim.x) {
        double s = a.C[0];
        for (int m = 1; m < M; ++m) s += 2.0 * a.C[m] * cos_frac(w, m, L);
        a.Chat[w] = s;
        lmax = fmax(lmax, fabs(s));
        lmin = fmin(lmin, s);
    }
    __syncthreads();
    const double cmax = block_reduce(lmax, red, true);
    const double cmin = -block_reduce(-lmin, red, true);
    double neg = 0.0;
    int bad = 0;
    for (int w = threadIdx.x; w < M; w += blockDim.x) {
        double c = a.Chat[w];
        if (c < 0.0) {
            if (c < -1e-12 * cmax && !a.clamp) bad = 1;
            neg += -c * (w == 0 ? 1.0 : 2.0);
            c = 0.0;
        }
        Ahat[w] = sqrt(c);
    }
    const double negsum = block_reduce(neg, red, false);
    const double anybad = block_reduce((double)bad, red, true);
    __syncthreads();
    for (int s = threadIdx.x; s < 2 * M - 1; s += blockDim.x) {
        const long long sh = s - H;
        double v = Ahat[0];
        for (int w = 1; w < M; ++w) v += 2.0 * Ahat[w] * cos_frac(w, sh, L);
        a.A[s] = v / (double)L;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double c = a.dt * a.Kd[0] / (2.0 * a.mass);
        const double b = 1.0 / (1.0 + c);
        a.scal[0] = b * (1.0 - c);
        a.scal[1] = b;
        a.scal[2] = cmin;
        a.scal[3] = negsum / (double)L;
        *a.status = anybad > 0.0 ? -3 : 0;
    }
    // Four copies of the zero-padded taps, copy r shifted right by r entries:
    // Apad[u] = A_{u - T - H} for T <= u <= T + 2H, else 0.
    for (int idx = threadIdx.x; idx < 4 * a.la; idx += blockDim.x) {
        const int r = idx / a.la, u = idx % a.la - r;
        a.Acp[idx] = (u >= a.T && u <= a.T + 2 * H) ? (float)a.A[u - a.T] : 0.0f;
    }
}

constexpr int kGenThreads = 256;

__global__ void __launch_bounds__(kGenThreads)
    wgen(const StepParams P, const Ctrl* __restrict__ ctrl, float* __restrict__ W, uint32_t k0, uint32_t k1)
{
    const long long n0 = ctrl->step;
    const long long need_lo = n0 - P.H, hi = n0 + P.T + P.H;
    const long long wl = ctrl->w_lo, wh = ctrl->w_hi;
    const bool valid = wl <= wh && wl <= need_lo && wh >= need_lo && wh <= hi;
    const long long lo = valid ? wh : need_lo;
    const long long count = hi - lo;
    const long long np = P.n_pad;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    for (long long kk = blockIdx.y; kk < count; kk += gridDim.y) {
        const long long time = lo + kk;
        long long slot = time % P.lw;
        if (slot < 0) slot += P.lw;
        const float3 z = gauss3(k0, k1, (uint32_t)i, time, 0u);
        float* w = W + (size_t)slot * 3 * np + i;
        w[0] = z.x;
        w[np] = z.y;
        w[2 * np] = z.z;
    }
}

constexpr int kFirThreads = 128;

template <int T>
__global__ void __launch_bounds__(kFirThreads)
    fir(const StepParams P, Ctrl* __restrict__ ctrl, const float* __restrict__ W, const float* __restrict__ Acp,
        int la, float* __restrict__ out)
{
    extern __shared__ float4 As4[];
    float* As = (float*)As4;
    for (int idx = threadIdx.x; idx < 4 * la; idx += blockDim.x) As[idx] = Acp[idx];
    __syncthreads();
    const long long n0 = ctrl->step;
    const long long np = P.n_pad, nstreams = 3 * np;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nstreams) {
        float acc[T];
#pragma unroll
        for (int t = 0; t < T; ++t) acc[t] = 0.f;
        const int nk = T + 2 * P.H;
        const int nk4 = (nk + 3) & ~3;
        long long slot = (n0 - P.H) % P.lw;
        if (slot < 0) slot += P.lw;
        for (int kk0 = 0; kk0 < nk4; kk0 += 4) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int kk = kk0 + e;
                const float w = kk < nk ? __ldcs(W + (size_t)slot * nstreams + j) : 0.f;
                slot = slot + 1 == P.lw ? 0 : slot + 1;
                const int r = 3 - e;  // copy whose shift makes the 16-byte loads aligned
#pragma unroll
                for (int j4 = 0; j4 < T / 4; ++j4) {
                    // taps for t = 4 j4 + 3 .. 4 j4 at Apad[kk + T - t]
                    const float4 a4 = *(const float4*)(As + r * la + (kk - e) + T - 4 * j4);
                    acc[4 * j4 + 3] = fmaf(a4.x, w, acc[4 * j4 + 3]);
                    acc[4 * j4 + 2] = fmaf(a4.y, w, acc[4 * j4 + 2]);
                    acc[4 * j4 + 1] = fmaf(a4.z, w, acc[4 * j4 + 1]);
                    acc[4 * j4 + 0] = fmaf(a4.w, w, acc[4 * j4 + 0]);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < T; ++t) out[(size_t)t * nstreams + j] = acc[t];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
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

__global__ void philox_k(const uint4* __restrict__ ctr, uint32_t k0, uint32_t k1, uint4* __restrict__ out, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c4 = ctr[i];
    uint32_t c[4] = {c4.x, c4.y, c4.z, c4.w};
    philox4x32_10(c, k0, k1);
    out[i] = make_uint4(c[0], c[1], c[2], c[3]);
}

__global__ void gauss3_k(uint32_t k0, uint32_t k1, const uint32_t* __restrict__ particle,
                         const long long* __restrict__ time, uint32_t stream_id, float* __restrict__ out, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float3 z = gauss3(k0, k1, particle[i], time[i], stream_id);
    out[3 * i] = z.x;
    out[3 * i + 1] = z.y;
    out[3 * i + 2] = z.z;
}

}  // namespace

int fir_copy_len(int T, int H) { return (2 * T + 2 * H + 4 + 3) & ~3; }

cudaError_t launch_prep(const PrepArgs& a, cudaStream_t st)
{
    const size_t smem = sizeof(double) * (size_t)a.m_max;
    if (smem > 48 * 1024) cudaFuncSetAttribute(prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    prep<<<1, kPrepThreads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_noise_block(const StepParams& P, Ctrl* ctrl, float* W, const float* Acp, int la, float* frblock,
                               unsigned long long seed, int num_sms, cudaStream_t st)
{
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    dim3 g((P.n + kGenThreads - 1) / kGenThreads, (unsigned)P.T);
    wgen<<<g, kGenThreads, 0, st>>>(P, ctrl, W, k0, k1);
    const long long streams = 3LL * P.n_pad;
    const unsigned grid = (unsigned)((streams + kFirThreads - 1) / kFirThreads);
    const size_t smem = sizeof(float) * 4 * (size_t)la;
    (void)num_sms;
    switch (P.T) {
    case 16:
        if (smem > 48 * 1024) cudaFuncSetAttribute(fir<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fir<16><<<grid, kFirThreads, smem, st>>>(P, ctrl, W, Acp, la, frblock);
        break;
    case 32:
        if (smem > 48 * 1024) cudaFuncSetAttribute(fir<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fir<32><<<grid, kFirThreads, smem, st>>>(P, ctrl, W, Acp, la, frblock);
        break;
    case 64:
        if (smem > 48 * 1024) cudaFuncSetAttribute(fir<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fir<64><<<grid, kFirThreads, smem, st>>>(P, ctrl, W, Acp, la, frblock);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out, long long n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    philox_k<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const uint4*)ctr, k0, k1, (uint4*)out, n);
    return cudaGetLastError();
}

cudaError_t launch_gauss3(uint32_t k0, uint32_t k1, const uint32_t* particle, const long long* time,
                          uint32_t stream_id, float* out, long long n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    gauss3_k<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(k0, k1, particle, time, stream_id, out, n);
    return cudaGetLastError();
}

}  // namespace gld
