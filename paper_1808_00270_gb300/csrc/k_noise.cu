// k_noise.cu -- kernel preparation and the colored random force.
//
// prep (one block, FP64): discrete kernels of Eq. k-discrete, the noise target
//   C_m = kT a_m K^s_m / dt (Eq. FDT_discretized, a_0 = 2), its transform over
//   the 2 m_max - 1 points of Eq. FT, the positive-semi-definiteness check,
//   A_s = inverse transform of sqrt(hat C) (Sec. II C, with 1/(2 m_max - 1)),
//   and the integrator factors a, b of Eq. aa-bb.
// wgen: white noise W_{i,k} from Philox4x32-10 into a ring of times, each
//   (particle, time) drawn exactly once over the whole run; FP32, or split
//   into the FP16 parts the tensor-core filter multiplies.
// fir:  F^R_{i,n+t} = sum_{s=-(m_max-1)}^{m_max-1} A_s W_{i,n+t+s} for a block
//   of T = 64 steps at once (the windowed generation remarked on in Sec. II C),
//   from a shared-memory tile of W with a sliding register window.
#include <algorithm>

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
    // Filter taps in FP32: Acp[sigma] = A_{sigma - H}, zero past sigma = 2H.
    for (int idx = threadIdx.x; idx < a.la; idx += blockDim.x) a.Acp[idx] = idx <= 2 * H ? (float)a.A[idx] : 0.0f;
}

constexpr int kGenThreads = 256;

__device__ __forceinline__ void wgen_body(const StepParams& P, const Ctrl* __restrict__ ctrl, float* __restrict__ W,
                                          uint32_t k0, uint32_t k1, const int* __restrict__ int2ext, int blk)
{
    const long long n0 = ctrl->step;
    const long long need_lo = n0 - P.H, hi = n0 + P.T + P.H;
    const long long wl = ctrl->w_lo, wh = ctrl->w_hi;
    const bool valid = wl <= wh && wl <= need_lo && wh >= need_lo && wh <= hi;
    const long long lo = valid ? wh : need_lo;
    const long long count = hi - lo;
    const long long np = P.n_pad;
    const int i = blk * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const uint32_t ext = (uint32_t)__ldg(int2ext + i);
    auto put = [&](long long time, float3 z) {
        long long slot = time % P.lw;
        if (slot < 0) slot += P.lw;
        if (P.wsplit) {  // FP16 planes: hi parts, then lo parts
            unsigned short* h = (unsigned short*)W + (size_t)slot * 3 * np + i;
            unsigned short* l = h + (size_t)P.lw * 3 * np;
            split_f16(z.x, h[0], l[0]);
            split_f16(z.y, h[np], l[np]);
            split_f16(z.z, h[2 * np], l[2 * np]);
        } else {
            float* w = W + (size_t)slot * 3 * np + i;
            w[0] = z.x;
            w[np] = z.y;
            w[2 * np] = z.z;
        }
    };
    // two independent draws per round (times kk and kk + gridDim.y), so that
    // their Philox rounds and transcendental functions overlap
    for (long long kk = blockIdx.y; kk < count; kk += 2LL * gridDim.y) {
        const long long kk2 = kk + gridDim.y;
        const float3 z0 = gauss3(k0, k1, ext, lo + kk, 0u);
        const float3 z1 = gauss3(k0, k1, ext, lo + (kk2 < count ? kk2 : kk), 0u);
        put(lo + kk, z0);
        if (kk2 < count) put(lo + kk2, z1);
    }
}

__global__ void __launch_bounds__(kGenThreads)
    wgen(const StepParams P, const Ctrl* __restrict__ ctrl, float* __restrict__ W, uint32_t k0, uint32_t k1,
         const int* __restrict__ int2ext)
{
    wgen_body(P, ctrl, W, k0, k1, int2ext, blockIdx.x);
}

constexpr int kFirThreads = 128;  // 4 warps x 16 outputs = one 64-step block
constexpr int kFirR = 16;         // outputs per thread (register window)
constexpr int kFirStreams = 32;   // streams per CTA (one per lane)
// Taps per shared-memory stage: 41 KB, five CTAs (20 warps) per SM.  More
// resident warps beat fewer re-read overlap rows: on the 262144-particle
// workload 768 / 384 / 256 / 128 took 2.65 / 2.36 / 2.17 / 2.22 ms per block,
// and a double-buffered variant (two stages in flight, fewer CTAs) was slower.
constexpr int kFirChunk = 256;

// F^R[t][j] = sum_{sigma=0}^{2H} A_{sigma-H} W[n0 - H + t + sigma][j], t < 64.
// The taps are taken in chunks of `chunk` (a multiple of 16): the CTA stages
// the chunk's taps and the W rows they touch for its 32 streams in shared
// memory; warp w produces outputs 16 w .. 16 w + 15, 16 taps at a time from
// 31 W rows and 16 taps held in registers (256 FMAs per 31 + 4 shared loads,
// taps in the same order as a plain loop over sigma).
__device__ __forceinline__ void fir_body(const StepParams& P, Ctrl* __restrict__ ctrl, const float* __restrict__ W,
                                         const float* __restrict__ taps, int ntaps, int chunk, float* __restrict__ out,
                                         int blk, int nblk)
{
    extern __shared__ float4 sm4[];
    float* At = (float*)sm4;               // [chunk]
    float* Wt = At + chunk;                // [chunk + 64][32]
    const long long n0 = ctrl->step;
    const long long np = P.n_pad, nstreams = 3 * np;
    const long long j = (long long)blk * kFirStreams + (threadIdx.x & 31);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    (void)lane;
    const int nk = 64 + 2 * P.H;           // rows holding real W
    const int t0 = warp * kFirR;
    float acc[kFirR];
#pragma unroll
    for (int r = 0; r < kFirR; ++r) acc[r] = 0.f;
    for (int c0 = 0; c0 < ntaps; c0 += chunk) {
        const int cn = min(chunk, ntaps - c0);
        __syncthreads();  // the previous chunk is consumed
        for (int k = threadIdx.x; k < cn; k += blockDim.x) At[k] = taps[c0 + k];
        // W rows of this chunk: 8 threads copy one 128-byte row as 16-byte
        // asynchronous copies, all in flight together; rows past the window
        // are zero-filled.
        const long long jb = (long long)blk * kFirStreams;
        for (int idx = threadIdx.x; idx < (cn + 64) * 8; idx += blockDim.x) {
            const int k = idx >> 3, part = idx & 7;
            const int row = c0 + k;
            const bool real = row < nk && jb + 4 * part < nstreams;
            long long slot = real ? (n0 - P.H + row) % P.lw : 0;
            if (slot < 0) slot += P.lw;
            const float* src = W + (size_t)slot * nstreams + jb + 4 * part;
            const unsigned dst = (unsigned)__cvta_generic_to_shared(Wt + k * 32 + 4 * part);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(real ? 16 : 0)
                         : "memory");
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
        // 16 taps at a time: the 31 W rows they touch and the taps are loaded
        // into registers, so every index below is static (no window to rotate)
        const float* wl = Wt + t0 * 32 + lane;
        for (int sg = 0; sg < cn; sg += kFirR) {
            float win[2 * kFirR - 1], tap[kFirR];
#pragma unroll
            for (int k = 0; k < 2 * kFirR - 1; ++k) win[k] = wl[(sg + k) * 32];
#pragma unroll
            for (int u = 0; u < kFirR; u += 4) {
                const float4 t4 = *(const float4*)(At + sg + u);
                tap[u] = t4.x; tap[u + 1] = t4.y; tap[u + 2] = t4.z; tap[u + 3] = t4.w;
            }
#pragma unroll
            for (int u = 0; u < kFirR; ++u)
#pragma unroll
                for (int r = 0; r < kFirR; ++r) acc[r] = fmaf(tap[u], win[u + r], acc[r]);
        }
    }
    if (j < nstreams)
#pragma unroll
        for (int r = 0; r < kFirR; ++r) out[(size_t)(t0 + r) * nstreams + j] = acc[r];
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&ctrl->done_fir, 1u) == nblk - 1) {
            ctrl->noise_n0 = n0;
            ctrl->w_lo = n0 - P.H;
            ctrl->w_hi = n0 + P.T + P.H;
            ctrl->done_fir = 0u;
            __threadfence();
        }
    }
}

size_t fir_smem(int chunk) { return sizeof(float) * ((size_t)chunk + (size_t)(64 + chunk) * kFirStreams); }

__global__ void __launch_bounds__(kFirThreads)
    fir(const StepParams P, Ctrl* __restrict__ ctrl, const float* __restrict__ W, const float* __restrict__ taps,
        int ntaps, int chunk, float* __restrict__ out)
{
    fir_body(P, ctrl, W, taps, ntaps, chunk, out, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kGenThreads) b_wgen(const SysDesc* __restrict__ D, const Tile* __restrict__ tiles)
{
    const Tile t = tiles[blockIdx.x];
    const SysDesc& d = D[t.m];
    wgen_body(d.P, d.B.ctrl, d.W, d.k0, d.k1, d.int2ext, t.b);
}

__global__ void __launch_bounds__(kFirThreads)
    b_fir(const SysDesc* __restrict__ D, const Tile* __restrict__ tiles, int chunk)
{
    const Tile t = tiles[blockIdx.x];
    const SysDesc& d = D[t.m];
    fir_body(d.P, d.B.ctrl, d.W, d.taps, d.ntaps, chunk, d.B.frblock, t.b, d.nb_fir);
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
int fir_taps_len(int H) { return (2 * H + 1 + 15) & ~15; }

cudaError_t launch_prep(const PrepArgs& a, cudaStream_t st)
{
    const size_t smem = sizeof(double) * (size_t)a.m_max;
    if (smem > 48 * 1024) cudaFuncSetAttribute(prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    prep<<<1, kPrepThreads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_noise_block(const StepParams& P, Ctrl* ctrl, float* W, const float* Acp, int la, float* frblock,
                               unsigned long long seed, const int* int2ext, const CUtensorMap* wmap, int num_sms,
                               cudaStream_t st)
{
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    dim3 g((P.n + kGenThreads - 1) / kGenThreads, (unsigned)(P.T / 2));  // two times per thread and round
    wgen<<<g, kGenThreads, 0, st>>>(P, ctrl, W, k0, k1, int2ext);
    const long long streams = 3LL * P.n_pad;
    (void)la;
    if (P.T != 64) return cudaErrorInvalidValue;
    // the split ring is read by the tensor-core filter, FP32 by the FP32-pipe one
    if (P.wsplit) return wmap ? launch_noise_filter_tc(P, ctrl, wmap, Acp, frblock, num_sms, st) : cudaErrorInvalidValue;
    const int ntaps = fir_taps_len(P.H);
    const int chunk = std::min(ntaps, kFirChunk);
    const size_t smem = fir_smem(chunk);
    cudaError_t e = cudaFuncSetAttribute(fir, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((streams + kFirStreams - 1) / kFirStreams);
    fir<<<grid, kFirThreads, smem, st>>>(P, ctrl, W, Acp, ntaps, chunk, frblock);
    return cudaGetLastError();
}

cudaError_t launch_noise_filter(const StepParams& P, Ctrl* ctrl, const float* W, const float* taps, float* out,
                                const CUtensorMap* wmap, int num_sms, cudaStream_t st)
{
    if (P.T != 64) return cudaErrorInvalidValue;
    if (P.wsplit) return wmap ? launch_noise_filter_tc(P, ctrl, wmap, taps, out, num_sms, st) : cudaErrorInvalidValue;
    const int ntaps = fir_taps_len(P.H);
    const int chunk = std::min(ntaps, kFirChunk);
    const size_t smem = fir_smem(chunk);
    cudaError_t e = cudaFuncSetAttribute(fir, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((3LL * P.n_pad + kFirStreams - 1) / kFirStreams);
    fir<<<grid, kFirThreads, smem, st>>>(P, ctrl, W, taps, ntaps, chunk, out);
    return cudaGetLastError();
}

// Pass k >= 1 of the pair-noise filters: Z_k of the members whose degree
// reaches k (the others' tiles return at once).
__global__ void __launch_bounds__(kFirThreads)
    b_fir_pn(const SysDesc* __restrict__ D, const Tile* __restrict__ tiles, int chunk, int k)
{
    const Tile t = tiles[blockIdx.x];
    const SysDesc& d = D[t.m];
    if (k > d.P.pn_deg) return;  // uniform over the block
    fir_body(d.P, d.B.ctrl, d.W, d.pntaps + (size_t)k * d.pn_la, d.ntaps, chunk,
             d.zblk + (size_t)(k - 1) * d.P.T * 3 * d.P.n_pad, t.b, d.nb_fir);
}

cudaError_t launch_batch_noise(const BatchPlan& bp, cudaStream_t st)
{
    static_assert(kGenThreads == kBatchPartBlock, "white-noise tiles use the particle tiles");
    static_assert(kFirStreams == kBatchFirStreams, "filter tiles");
    if (!bp.n_part || !bp.n_fir) return cudaSuccess;
    dim3 g((unsigned)bp.n_part, 32u);  // two times per thread and round
    b_wgen<<<g, kGenThreads, 0, st>>>(bp.desc, bp.part);
    const int chunk = std::min(bp.max_ntaps, kFirChunk);
    const size_t smem = fir_smem(chunk);
    cudaError_t e = cudaFuncSetAttribute(b_fir, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    b_fir<<<bp.n_fir, kFirThreads, smem, st>>>(bp.desc, bp.fir, chunk);
    if (bp.pn_kmax > 0) {
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(b_fir_pn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        for (int k = 1; k <= bp.pn_kmax; ++k) b_fir_pn<<<bp.n_fir, kFirThreads, smem, st>>>(bp.desc, bp.fir, chunk, k);
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
