// k_pn_krylov.cu -- the pair-correlated random force of Sec. II C by Algorithm
// 1: a Lanczos iteration per frequency.
//
// With the kernels taken at the current configuration (the time-scale
// separation remarked on after Algorithm 1), the transformed correlation
// matrix of frequency w is
//     hat K_w = a_w 1 + sum_q g_qw M_q + sum_q gs_qw D_q,
// M_q the 3N x 3N pair matrices (blocks f_q e e^T + fp_q (1 - e e^T) between
// neighbours), D_q the self-difference matrices (diagonal blocks summed over
// neighbours) and a_w, g_qw, gs_qw the transforms (Eq. FT) of kT a_m / dt
// times the discrete time factors.  For every w = 0 .. m_max - 1 the
// iteration builds the Krylov basis V of hat K_w from the transformed white
// noise hat W_w (its real part, hat K_w being real) and approximates
// sqrt(hat K_w) hat W_w = |hat W_w| V sqrt(H) e_1 (H the tridiagonal Lanczos
// matrix); F_n = (x_0 + 2 sum_{w >= 1} x_w) / (2 m_max - 1).
//
// All frequencies run together: vectors are stored [3 n_pad][Mp] with the
// frequency the fast index (Mp = m_max rounded up to 32), so one warp handles
// 32 frequencies of one vector entry and every neighbour sweep reads 128
// contiguous bytes per entry; one sweep applies hat K_w for all w.  Products
// are FP32, every dot product and norm is summed in FP64 in a fixed order
// (block partials folded by one thread per frequency).  The square roots of
// the small tridiagonal matrices and the stopping test (Algorithm 1's Delta)
// run on the host.
#include "launch.h"

namespace gld {

namespace {

constexpr int kKryWarps = 8;  // vector entries (one per warp) per block; 32 frequencies per warp

// V0[I][w] = sum_{s=-H}^{H} W_{n+s}[I] cos(2 pi w s / L), I = c n_pad + i, L = 2H + 1.
__global__ void __launch_bounds__(32 * kKryWarps)
    pnk_ft(const StepParams P, const Ctrl* __restrict__ ctrl, const float* __restrict__ W, int M, int Mp,
           float* __restrict__ V0)
{
    extern __shared__ float cosL[];  // cos(2 pi t / L), t < L
    const int H = P.H, L = 2 * H + 1;
    for (int t = threadIdx.x; t < L; t += blockDim.x) cosL[t] = (float)cospi(2.0 * t / (double)L);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long np3 = 3LL * P.n_pad;
    const long long I = (long long)blockIdx.x * kKryWarps + warp;
    const int w = blockIdx.y * 32 + lane;
    if (I >= np3) return;
    const long long n = ctrl->step;
    int t = (int)((((long long)w * -H) % L + L) % L);  // (w s) mod L at s = -H
    const int dw = w % L;
    float acc = 0.f;
    for (int s = -H; s <= H; ++s) {
        long long slot = (n + s) % P.lw;
        if (slot < 0) slot += P.lw;
        acc = fmaf(__ldg(W + (size_t)slot * np3 + I), cosL[t], acc);
        t += dw;
        if (t >= L) t -= L;
    }
    V0[(size_t)I * Mp + w] = w < M ? acc : 0.f;
}

// part[b][w] = sum over the entries of block-row b of a[I][w] * b[I][w] (FP64).
__global__ void __launch_bounds__(32 * kKryWarps)
    pnk_dot(const float* __restrict__ a, const float* __restrict__ b, long long np3, int Mp,
            double* __restrict__ part)
{
    __shared__ double red[kKryWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int w = blockIdx.y * 32 + lane;
    double acc = 0.0;
    for (long long I = (long long)blockIdx.x * kKryWarps + warp; I < np3; I += (long long)gridDim.x * kKryWarps)
        acc += (double)a[(size_t)I * Mp + w] * (double)b[(size_t)I * Mp + w];
    red[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
        double s = 0.0;
        for (int k = 0; k < kKryWarps; ++k) s += red[k][lane];
        part[(size_t)blockIdx.x * Mp + w] = s;
    }
}

// out[w] = sum_b part[b][w] in block order; mode 0: the sum; mode 1: its
// square root, and alive[w] = 0 (the vector of that frequency is set to zero
// from then on) when the root is below 1e-6 |ref[w]| (a Krylov space
// exhausted to the precision of FP32 vectors: the result is exact to that
// precision already); mode 2: the square root.
__global__ void pnk_fold(const double* __restrict__ part, int nblk, int Mp, double* __restrict__ out, int mode,
                         const double* __restrict__ ref, int* __restrict__ alive)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= Mp) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * Mp + w];
    if (mode == 0) {
        out[w] = s;
        return;
    }
    double r = sqrt(fmax(s, 0.0));
    if (mode == 1 && !(r > 1e-6 * fabs(ref[w]))) {
        alive[w] = 0;
        r = 0.0;
    }
    out[w] = r;
}

// dst[I][w] = src[I][w] / d[w] (zero where d[w] is zero or the frequency is done).
__global__ void __launch_bounds__(32 * kKryWarps)
    pnk_scale(const float* __restrict__ src, float* __restrict__ dst, long long np3, int Mp,
              const double* __restrict__ d, const int* __restrict__ alive)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int w = blockIdx.y * 32 + lane;
    const double dd = d[w];
    const float inv = (alive[w] && dd > 0.0) ? (float)(1.0 / dd) : 0.f;
    for (long long I = (long long)blockIdx.x * kKryWarps + warp; I < np3; I += (long long)gridDim.x * kKryWarps)
        dst[(size_t)I * Mp + w] = src[(size_t)I * Mp + w] * inv;
}

// r = Y - alpha_k v_k - beta_{k-1} v_{k-1} (v_{k-1} may be null).
__global__ void __launch_bounds__(32 * kKryWarps)
    pnk_resid(const float* __restrict__ Y, const float* __restrict__ vk, const float* __restrict__ vkm1,
              const double* __restrict__ alpha, const double* __restrict__ beta, long long np3, int Mp,
              float* __restrict__ r)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int w = blockIdx.y * 32 + lane;
    const float a = (float)alpha[w], b = vkm1 ? (float)beta[w] : 0.f;
    for (long long I = (long long)blockIdx.x * kKryWarps + warp; I < np3; I += (long long)gridDim.x * kKryWarps) {
        const size_t k = (size_t)I * Mp + w;
        float v = fmaf(-a, vk[k], Y[k]);
        if (vkm1) v = fmaf(-b, vkm1[k], v);
        r[k] = v;
    }
}

__device__ __forceinline__ float kdot3(float ax, float ay, float az, float bx, float by, float bz)
{
    return fmaf(ax, bx, fmaf(ay, by, az * bz));
}

// Y = hat K_w V for every frequency: a_w v_i + sum_q g_qw sum_j B_q(ij) v_j
// + sum_q gs_qw sum_j Bs_q(ij) v_i, B = f e e^T + fp (1 - e e^T) at
// max(r, r_c,min), neighbours within r_c from the lists.  wc[a][w]: row 0 a_w,
// rows 1..Q g_qw, rows 1+Q.. gs_qw.
__global__ void __launch_bounds__(32 * kKryWarps)
    pnk_matvec(const StepParams P, const float4* __restrict__ pos, const int* __restrict__ nbr,
               const int* __restrict__ nbr_cnt, const float* __restrict__ ftab, const float* __restrict__ fptab,
               const double* __restrict__ wc, int Mp, const float* __restrict__ V, float* __restrict__ Y)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * kKryWarps + warp;
    const int w = blockIdx.y * 32 + lane;
    if (i >= P.n) return;  // uniform over the warp
    const long long np = P.n_pad;
    float gq[kMaxQ], gsq[kMaxQ];
#pragma unroll
    for (int q = 0; q < kMaxQ; ++q) {
        gq[q] = q < P.Q ? (float)wc[(size_t)(1 + q) * Mp + w] : 0.f;
        gsq[q] = q < P.Qs ? (float)wc[(size_t)(1 + P.Q + q) * Mp + w] : 0.f;
    }
    const float aw = (float)wc[w];
    const float vix = V[(size_t)i * Mp + w], viy = V[(size_t)(np + i) * Mp + w], viz = V[(size_t)(2 * np + i) * Mp + w];
    float yx = aw * vix, yy = aw * viy, yz = aw * viz;
    const float4 pi = pos[i];
    for_each_listed(pi, i, nbr, nbr_cnt[i], P.n_pad, pos, P, [&](int jd, float dx, float dy, float dz, float r2) {
        const float r = sqrtf(r2);
        const float inv_r = 1.0f / r;
        const float ex = dx * inv_r, ey = dy * inv_r, ez = dz * inv_r;
        const float xr = fmaxf(r, P.rc_min) * P.inv_dr;
        const float vjx = V[(size_t)jd * Mp + w], vjy = V[(size_t)(np + jd) * Mp + w],
                    vjz = V[(size_t)(2 * np + jd) * Mp + w];
        const float ej = kdot3(ex, ey, ez, vjx, vjy, vjz), ei = kdot3(ex, ey, ez, vix, viy, viz);
        float cpar = 0.f, cperp = 0.f, spar = 0.f, sperp = 0.f;  // combined radial factors of this pair
        for (int q = 0; q < P.Q; ++q) {
            const float f = table_at(ftab + q * P.nr, P.nr, xr);
            const float fp = P.perp ? table_at(fptab + q * P.nr, P.nr, xr) : 0.f;
            cpar = fmaf(gq[q], f, cpar);
            cperp = fmaf(gq[q], fp, cperp);
        }
        for (int q = 0; q < P.Qs; ++q) {
            const float f = table_at(ftab + (P.Q + q) * P.nr, P.nr, xr);
            const float fp = P.perp ? table_at(fptab + (P.Q + q) * P.nr, P.nr, xr) : 0.f;
            spar = fmaf(gsq[q], f, spar);
            sperp = fmaf(gsq[q], fp, sperp);
        }
        // (par - perp) (e.x) e + perp x, for x = v_j (pair) and x = v_i (self-difference)
        const float pj = (cpar - cperp) * ej, si = (spar - sperp) * ei;
        yx += fmaf(pj + si, ex, fmaf(cperp, vjx, sperp * vix));
        yy += fmaf(pj + si, ey, fmaf(cperp, vjy, sperp * viy));
        yz += fmaf(pj + si, ez, fmaf(cperp, vjz, sperp * viz));
    });
    Y[(size_t)i * Mp + w] = yx;
    Y[(size_t)(np + i) * Mp + w] = yy;
    Y[(size_t)(2 * np + i) * Mp + w] = yz;
}

// out[I] = (sum_w c_w sum_p cf[w][p] V_p[I][w]) / L, c_0 = 1, c_w = 2: one
// warp per entry, lanes over frequencies, a fixed-order warp sum.
__global__ void __launch_bounds__(32 * kKryWarps)
    pnk_combine(const float* __restrict__ V, const float* __restrict__ cf, int kp, int M, int Mp, long long np3,
                float inv_L, float* __restrict__ out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long I = (long long)blockIdx.x * kKryWarps + warp;
    if (I >= np3) return;
    const size_t stride = (size_t)np3 * Mp;
    float acc = 0.f;
    for (int w = lane; w < M; w += 32) {
        float x = 0.f;
        for (int p = 0; p < kp; ++p) x = fmaf(cf[(size_t)w * kp + p], V[p * stride + (size_t)I * Mp + w], x);
        acc = fmaf(w == 0 ? 1.f : 2.f, x, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[I] = acc * inv_L;
}

unsigned blocks_for(long long np3) { return (unsigned)std::min<long long>((np3 + kKryWarps - 1) / kKryWarps, 1024); }

}  // namespace

cudaError_t kry_ft(const StepParams& P, const Ctrl* ctrl, const float* W, int M, int Mp, float* V0, cudaStream_t st)
{
    const long long np3 = 3LL * P.n_pad;
    const dim3 g((unsigned)((np3 + kKryWarps - 1) / kKryWarps), (unsigned)(Mp / 32));
    const size_t smem = sizeof(float) * (size_t)(2 * P.H + 1);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(pnk_ft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    pnk_ft<<<g, 32 * kKryWarps, smem, st>>>(P, ctrl, W, M, Mp, V0);
    return cudaGetLastError();
}

int kry_dot_blocks(const StepParams& P) { return (int)blocks_for(3LL * P.n_pad); }

cudaError_t kry_dot(const StepParams& P, const float* a, const float* b, int Mp, double* part, double* out, int mode,
                    const double* ref, int* alive, cudaStream_t st)
{
    const long long np3 = 3LL * P.n_pad;
    const unsigned nb = blocks_for(np3);
    pnk_dot<<<dim3(nb, (unsigned)(Mp / 32)), 32 * kKryWarps, 0, st>>>(a, b, np3, Mp, part);
    pnk_fold<<<(Mp + 127) / 128, 128, 0, st>>>(part, (int)nb, Mp, out, mode, ref, alive);
    return cudaGetLastError();
}

cudaError_t kry_scale(const StepParams& P, const float* src, float* dst, int Mp, const double* d, const int* alive,
                      cudaStream_t st)
{
    const long long np3 = 3LL * P.n_pad;
    pnk_scale<<<dim3(blocks_for(np3), (unsigned)(Mp / 32)), 32 * kKryWarps, 0, st>>>(src, dst, np3, Mp, d, alive);
    return cudaGetLastError();
}

cudaError_t kry_resid(const StepParams& P, const float* Y, const float* vk, const float* vkm1, const double* alpha,
                      const double* beta, int Mp, float* r, cudaStream_t st)
{
    const long long np3 = 3LL * P.n_pad;
    pnk_resid<<<dim3(blocks_for(np3), (unsigned)(Mp / 32)), 32 * kKryWarps, 0, st>>>(Y, vk, vkm1, alpha, beta, np3,
                                                                                     Mp, r);
    return cudaGetLastError();
}

cudaError_t kry_matvec(const StepParams& P, const ParticleBuffers& B, const double* wc, int Mp, const float* V,
                       float* Y, cudaStream_t st)
{
    const dim3 g((unsigned)((P.n + kKryWarps - 1) / kKryWarps), (unsigned)(Mp / 32));
    pnk_matvec<<<g, 32 * kKryWarps, 0, st>>>(P, B.pos, B.nbr, B.nbr_cnt, B.ftab, B.fptab, wc, Mp, V, Y);
    return cudaGetLastError();
}

cudaError_t kry_combine(const StepParams& P, const float* V, const float* cf, int kp, int M, int Mp, float* out,
                        cudaStream_t st)
{
    const long long np3 = 3LL * P.n_pad;
    pnk_combine<<<(unsigned)((np3 + kKryWarps - 1) / kKryWarps), 32 * kKryWarps, 0, st>>>(
        V, cf, kp, M, Mp, np3, 1.0f / (float)(2 * P.H + 1), out);
    return cudaGetLastError();
}

}  // namespace gld
