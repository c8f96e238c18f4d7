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
// iteration builds the Krylov basis of hat K_w from the transformed white
// noise hat W_w (its real part, hat K_w being real) and approximates
// sqrt(hat K_w) hat W_w = |hat W_w| V sqrt(H) e_1 (H the tridiagonal Lanczos
// matrix); F_n = (x_0 + 2 sum_{w >= 1} x_w) / (2 m_max - 1).
//
// All frequencies run together: vectors are stored [3 n_pad][Mp] with the
// frequency the fast index (Mp = m_max rounded up to 32), so a warp reads 128
// contiguous bytes per vector entry and one neighbour sweep applies hat K_w
// for every w.  The Lanczos vectors are kept unnormalised (R_k, with
// v_k = R_k / beta_k and beta_k = |R_k|), so no pass only rescales; the
// sweep also sums the partials of alpha_k = v_k . hat K v_k, the residual
// kernel those of |R_{k+1}|^2.  Products are FP32; sums are FP32 over at most
// 16 terms and FP64 beyond, folded in a fixed order, so a run is
// deterministic.  The square roots of the small tridiagonal matrices and the
// stopping test (Algorithm 1's Delta) run on the host.
#include "launch.h"

namespace gld {

namespace {

constexpr int kKryWarps = 8;    // warps per block of the elementwise kernels and the sweep
constexpr int kFtThreads = 256; // entries per block of the transform
constexpr int kMvGroups = 8;    // frequency groups (of 32) per neighbour pass of the sweep
constexpr int kChunk = 16;      // FP32 terms summed before an FP64 addition

// V0[I][w] = W_n[I] + sum_{s=1}^{H} (W_{n+s}[I] + W_{n-s}[I]) cos(2 pi w s / L)
// (cos is even in s), I = c n_pad + i, L = 2H + 1.  Block (g, y) takes the
// frequencies 32g .. 32g + 31 of the entries 256y .. 256y + 255, one entry
// per thread with 32 accumulators; the group's 32 columns of the cosine
// table (cosT[s][w], s = 0..H) are staged in shared memory, where all lanes of
// a warp read the same row (a broadcast).  The frequency groups of one entry
// chunk are adjacent in the grid, so they share the W window through L2.
// With the time window (Mc < Mp): columns Mc + w hold the sine transform
// S_w = sum_{s=1}^{H} (W_{n+s} - W_{n-s}) sin(2 pi w s / L) (no s = 0 term),
// their table columns the sines.
__global__ void __launch_bounds__(kFtThreads)
    pnk_ft(const StepParams P, const Ctrl* __restrict__ ctrl, const float* __restrict__ W,
           const float* __restrict__ cosT, int M, int Mp, int Mc, float* __restrict__ V0)
{
    extern __shared__ float4 cs4[];  // [H + 1][8]
    const int H = P.H, g = blockIdx.x;
    const bool sine = g * 32 >= Mc;  // uniform over the block
    const float sg = sine ? -1.f : 1.f;
    for (int e = threadIdx.x; e < (H + 1) * 8; e += blockDim.x)
        cs4[e] = reinterpret_cast<const float4*>(cosT + (size_t)(e >> 3) * Mp + g * 32)[e & 7];
    __syncthreads();
    const long long np3 = 3LL * P.n_pad;
    const long long I = (long long)blockIdx.y * blockDim.x + threadIdx.x;
    if (I >= np3) return;  // after the only barrier
    const long long n = ctrl->step, lw = P.lw;
    long long s0 = n % lw;
    if (s0 < 0) s0 += lw;
    float acc[32];
    const float w0 = ring_w(P, W, (size_t)s0 * np3 + I);
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = sine ? 0.f : w0;  // s = 0: cos 0 = 1, sin 0 = 0
    long long sp = s0 + 1 == lw ? 0 : s0 + 1, sm = s0 == 0 ? lw - 1 : s0 - 1;
    auto term = [&](float p, int s) {
        const float4* c = cs4 + s * 8;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float4 cc = c[k];
            acc[4 * k] = fmaf(p, cc.x, acc[4 * k]);
            acc[4 * k + 1] = fmaf(p, cc.y, acc[4 * k + 1]);
            acc[4 * k + 2] = fmaf(p, cc.z, acc[4 * k + 2]);
            acc[4 * k + 3] = fmaf(p, cc.w, acc[4 * k + 3]);
        }
    };
    int s = 1;
    for (; s + 3 <= H; s += 4) {  // the loads of four window pairs in flight together
        float a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a[u] = ring_w(P, W, (size_t)sp * np3 + I);
            b[u] = ring_w(P, W, (size_t)sm * np3 + I);
            sp = sp + 1 == lw ? 0 : sp + 1;
            sm = sm == 0 ? lw - 1 : sm - 1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) term(fmaf(sg, b[u], a[u]), s + u);
    }
    for (; s <= H; ++s) {
        term(fmaf(sg, ring_w(P, W, (size_t)sm * np3 + I), ring_w(P, W, (size_t)sp * np3 + I)), s);
        sp = sp + 1 == lw ? 0 : sp + 1;
        sm = sm == 0 ? lw - 1 : sm - 1;
    }
    float4* out = reinterpret_cast<float4*>(V0 + (size_t)I * Mp + g * 32);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int col = g * 32 + 4 * k + e;
            v[e] = (sine ? col - Mc : col) < M ? acc[4 * k + e] : 0.f;  // padding frequencies
        }
        out[k] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

// part[b][w] = sum over the entries of block-row b of a[I][w] * b[I][w]:
// FP32 over chunks of kChunk entries, FP64 beyond.
__global__ void __launch_bounds__(32 * kKryWarps)
    pnk_dot(const float* __restrict__ a, const float* __restrict__ b, long long np3, int Mp,
            double* __restrict__ part)
{
    __shared__ double red[kKryWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int w = blockIdx.y * 32 + lane;
    double acc = 0.0;
    float c = 0.f;
    int t = 0;
    for (long long I = (long long)blockIdx.x * kKryWarps + warp; I < np3; I += (long long)gridDim.x * kKryWarps) {
        c = fmaf(a[(size_t)I * Mp + w], b[(size_t)I * Mp + w], c);
        if (++t == kChunk) {
            acc += (double)c;
            c = 0.f;
            t = 0;
        }
    }
    acc += (double)c;
    red[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
        double s = 0.0;
        for (int k = 0; k < kKryWarps; ++k) s += red[k][lane];
        part[(size_t)blockIdx.x * Mp + w] = s;
    }
}

// out[w] = sum_b part[b][w] in block order (8 warps split the blocks, then
// their sums in warp order); mode 0: the sum; mode 1: its square root, and
// alive[w] = 0 (that frequency's vectors are zero from then on) when the root
// is below 1e-6 |ref[w]| (a Krylov space exhausted to the precision of FP32
// vectors: the result is exact to that precision already); mode 2: the
// square root.  Block x takes the frequencies 32x .. 32x + 31.
__global__ void __launch_bounds__(32 * kKryWarps)
    pnk_fold(const double* __restrict__ part, int nblk, int Mp, double* __restrict__ out, int mode,
             const double* __restrict__ ref, int* __restrict__ alive)
{
    __shared__ double red[kKryWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int w = blockIdx.x * 32 + lane;
    double s = 0.0;
    for (int b = warp; b < nblk; b += kKryWarps) s += part[(size_t)b * Mp + w];
    red[warp][lane] = s;
    __syncthreads();
    if (warp != 0) return;
    s = 0.0;
    for (int k = 0; k < kKryWarps; ++k) s += red[k][lane];
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

__device__ __forceinline__ float kdot3(float ax, float ay, float az, float bx, float by, float bz)
{
    return fmaf(ax, bx, fmaf(ay, by, az * bz));
}

// Z = hat K_w v_k for every frequency (v_k = R_k / beta_k), and the block
// partials of alpha_k = v_k . Z.  One warp per particle (particles
// blk * 8 + warp, then strided by the grid), lanes over the 32 frequencies
// of a group; a neighbour's geometry and radial factors are computed once
// per pass over kMvGroups groups.  Blocks f e e^T + fp (1 - e e^T) at
// max(r, r_c,min) for pairs within r_c, from the lists.  wc rows: a_w, g_qw
// (q < Q), gs_qw (q < Qs), staged in shared memory as FP32 with 1 / beta_k
// (0 for exhausted frequencies); alpha partials per warp in FP64 there.
__global__ void __launch_bounds__(32 * kKryWarps, 2)
    pnk_matvec(const StepParams P, const float4* __restrict__ pos, const int* __restrict__ nbr,
               const int* __restrict__ nbr_cnt, const float* __restrict__ ftab, const float* __restrict__ fptab,
               const double* __restrict__ wc, const double* __restrict__ beta, const int* __restrict__ alive, int Mp,
               const float* __restrict__ R, float* __restrict__ Z, double* __restrict__ part)
{
    extern __shared__ double smd[];
    const int nrow = 1 + P.Q + P.Qs;
    double* red = smd;                          // [kKryWarps][Mp]
    float* wcs = (float*)(smd + kKryWarps * Mp); // [nrow][Mp]
    float* ib = wcs + (size_t)nrow * Mp;         // [Mp]
    for (int e = threadIdx.x; e < nrow * Mp; e += blockDim.x) wcs[e] = (float)wc[e];
    for (int w = threadIdx.x; w < Mp; w += blockDim.x) ib[w] = (alive[w] && beta[w] > 0.0) ? (float)(1.0 / beta[w]) : 0.f;
    for (int e = threadIdx.x; e < kKryWarps * Mp; e += blockDim.x) red[e] = 0.0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ng = Mp / 32;
    const long long np = P.n_pad;
    double* myred = red + (size_t)warp * Mp;
    for (int i = blockIdx.x * kKryWarps + warp; i < P.n; i += gridDim.x * kKryWarps) {
        const float4 pi = pos[i];
        for (int g0 = 0; g0 < ng; g0 += kMvGroups) {
            float vi[kMvGroups][3], y[kMvGroups][3];
#pragma unroll
            for (int gg = 0; gg < kMvGroups; ++gg) {
                const int w = (g0 + gg) * 32 + lane;
                const bool in = g0 + gg < ng;
                const float b = in ? ib[w] : 0.f, aw = in ? wcs[w] : 0.f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    vi[gg][c] = in ? b * R[((size_t)c * np + i) * Mp + w] : 0.f;
                    y[gg][c] = aw * vi[gg][c];
                }
            }
            // the list in order, one neighbour at a time with the next one's
            // index and position in flight; the pair test of the list walkers
            const int cnt = nbr_cnt[i];
            int jn = cnt > 0 ? __ldg(nbr + i) : 0;
            float4 pn = cnt > 0 ? __ldg(pos + jn) : pi;
            for (int sl = 0; sl < cnt; ++sl) {
                const int jd = jn;
                const float4 pj = pn;
                if (sl + 1 < cnt) {
                    jn = __ldg(nbr + (size_t)(sl + 1) * P.n_pad + i);
                    pn = __ldg(pos + jn);
                }
                const float dx = min_image(pi.x, pj.x, P.box, P.half_box);
                const float dy = min_image(pi.y, pj.y, P.box, P.half_box);
                const float dz = min_image(pi.z, pj.z, P.box, P.half_box);
                const float r2 = dist2(dx, dy, dz);
                if (!(r2 < P.rc2)) continue;
                const float r = sqrtf(r2);
                const float inv_r = 1.0f / r;
                const float ex = dx * inv_r, ey = dy * inv_r, ez = dz * inv_r;
                const float xr = fmaxf(r, P.rc_min) * P.inv_dr;
                float fq[kMaxQ], fpq[kMaxQ], fs[kMaxQ], fsp[kMaxQ];
#pragma unroll
                for (int q = 0; q < kMaxQ; ++q) {
                    fq[q] = q < P.Q ? table_at(ftab + q * P.nr, P.nr, xr) : 0.f;
                    fpq[q] = (q < P.Q && P.perp) ? table_at(fptab + q * P.nr, P.nr, xr) : 0.f;
                    fs[q] = q < P.Qs ? table_at(ftab + (P.Q + q) * P.nr, P.nr, xr) : 0.f;
                    fsp[q] = (q < P.Qs && P.perp) ? table_at(fptab + (P.Q + q) * P.nr, P.nr, xr) : 0.f;
                }
#pragma unroll
                for (int gg = 0; gg < kMvGroups; ++gg) {
                    if (g0 + gg >= ng) break;  // uniform over the warp
                    const int w = (g0 + gg) * 32 + lane;
                    float cpar = 0.f, cperp = 0.f, spar = 0.f, sperp = 0.f;  // the pair's combined radial factors
#pragma unroll
                    for (int q = 0; q < kMaxQ; ++q) {
                        if (q < P.Q) {
                            const float gq = wcs[(1 + q) * Mp + w];
                            cpar = fmaf(gq, fq[q], cpar);
                            cperp = fmaf(gq, fpq[q], cperp);
                        }
                        if (q < P.Qs) {
                            const float gs = wcs[(1 + P.Q + q) * Mp + w];
                            spar = fmaf(gs, fs[q], spar);
                            sperp = fmaf(gs, fsp[q], sperp);
                        }
                    }
                    const float b = ib[w];
                    const float vjx = b * R[(size_t)jd * Mp + w], vjy = b * R[((size_t)np + jd) * Mp + w],
                                vjz = b * R[((size_t)2 * np + jd) * Mp + w];
                    const float ej = kdot3(ex, ey, ez, vjx, vjy, vjz);
                    const float ei = kdot3(ex, ey, ez, vi[gg][0], vi[gg][1], vi[gg][2]);
                    // (par - perp) (e.x) e + perp x, for x = v_j (pair) and x = v_i (self-difference)
                    const float pj = (cpar - cperp) * ej, si = (spar - sperp) * ei;
                    y[gg][0] += fmaf(pj + si, ex, fmaf(cperp, vjx, sperp * vi[gg][0]));
                    y[gg][1] += fmaf(pj + si, ey, fmaf(cperp, vjy, sperp * vi[gg][1]));
                    y[gg][2] += fmaf(pj + si, ez, fmaf(cperp, vjz, sperp * vi[gg][2]));
                }
            }
#pragma unroll
            for (int gg = 0; gg < kMvGroups; ++gg) {
                if (g0 + gg >= ng) break;
                const int w = (g0 + gg) * 32 + lane;
#pragma unroll
                for (int c = 0; c < 3; ++c) Z[((size_t)c * np + i) * Mp + w] = y[gg][c];
                myred[w] += (double)kdot3(vi[gg][0], vi[gg][1], vi[gg][2], y[gg][0], y[gg][1], y[gg][2]);
            }
        }
    }
    __syncthreads();
    for (int w = threadIdx.x; w < Mp; w += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < kKryWarps; ++k) s += red[(size_t)k * Mp + w];
        part[(size_t)blockIdx.x * Mp + w] = s;
    }
}

// R_{k+1} = Z - (alpha_k / beta_k) R_k - (beta_k / beta_{k-1}) R_{k-1} (the
// last term when R_{k-1} is given), zero for exhausted frequencies; block
// partials of |R_{k+1}|^2 (FP32 over kChunk entries, FP64 beyond).
__global__ void __launch_bounds__(32 * kKryWarps)
    pnk_resid(const float* __restrict__ Z, const float* __restrict__ Rk, const float* __restrict__ Rkm1,
              const double* __restrict__ alpha_k, const double* __restrict__ beta_k,
              const double* __restrict__ beta_km1, const int* __restrict__ alive, long long np3, int Mp,
              float* __restrict__ Rkp1, double* __restrict__ part)
{
    __shared__ double red[kKryWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int w = blockIdx.y * 32 + lane;
    const bool on = alive[w] && beta_k[w] > 0.0;
    const float a = on ? (float)(alpha_k[w] / beta_k[w]) : 0.f;
    const float b = (on && Rkm1 && beta_km1[w] > 0.0) ? (float)(beta_k[w] / beta_km1[w]) : 0.f;
    double acc = 0.0;
    float c = 0.f;
    int t = 0;
    const long long st = (long long)gridDim.x * kKryWarps;
    // four entries per round with their loads in flight together (summed in
    // the order of the entries, as one at a time)
    for (long long I0 = (long long)blockIdx.x * kKryWarps + warp; I0 < np3; I0 += 4 * st) {
        float z[4], rk[4], rm[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long I = I0 + u * st;
            const bool in = I < np3;
            const size_t e = (size_t)(in ? I : I0) * Mp + w;
            z[u] = in && on ? Z[e] : 0.f;
            rk[u] = in && on ? Rk[e] : 0.f;
            rm[u] = in && on && Rkm1 ? Rkm1[e] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long I = I0 + u * st;
            if (I >= np3) break;
            float r = 0.f;
            if (on) {
                r = fmaf(-a, rk[u], z[u]);
                if (Rkm1) r = fmaf(-b, rm[u], r);
            }
            Rkp1[(size_t)I * Mp + w] = r;
            c = fmaf(r, r, c);
            if (++t == kChunk) {
                acc += (double)c;
                c = 0.f;
                t = 0;
            }
        }
    }
    acc += (double)c;
    red[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
        double s = 0.0;
        for (int k = 0; k < kKryWarps; ++k) s += red[k][lane];
        part[(size_t)blockIdx.x * Mp + w] = s;
    }
}

// out[I] = (sum_w c_w sum_p cf[w][p] R_p[I][w]) / L, c_0 = 1, c_w = 2 (cf
// includes 1 / beta_p): one warp per entry, lanes over frequencies, a
// fixed-order warp sum.
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
        int p = 0;
        for (; p + 4 <= kp; p += 4) {  // four vectors' loads in flight, summed in order
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = V[(p + u) * stride + (size_t)I * Mp + w];
#pragma unroll
            for (int u = 0; u < 4; ++u) x = fmaf(cf[(size_t)w * kp + p + u], v[u], x);
        }
        for (; p < kp; ++p) x = fmaf(cf[(size_t)w * kp + p], V[p * stride + (size_t)I * Mp + w], x);
        acc = fmaf(w == 0 ? 1.f : 2.f, x, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[I] = acc * inv_L;
}

// Y[I][c] = sum_p cf[c][p] R_p[I][c] (cf includes 1 / beta_p): warps over
// entries, lanes over columns, four vectors' loads in flight, in order.
__global__ void __launch_bounds__(32 * kKryWarps)
    pnk_combine_y(const float* __restrict__ V, const float* __restrict__ cf, int kp, int Mp, long long np3,
                  float* __restrict__ Y)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.y * 32 + lane;
    const size_t stride = (size_t)np3 * Mp;
    for (long long I = (long long)blockIdx.x * kKryWarps + warp; I < np3; I += (long long)gridDim.x * kKryWarps) {
        float x = 0.f;
        int p = 0;
        for (; p + 4 <= kp; p += 4) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = V[(p + u) * stride + (size_t)I * Mp + c];
#pragma unroll
            for (int u = 0; u < 4; ++u) x = fmaf(cf[(size_t)c * kp + p + u], v[u], x);
        }
        for (; p < kp; ++p) x = fmaf(cf[(size_t)c * kp + p], V[p * stride + (size_t)I * Mp + c], x);
        Y[(size_t)I * Mp + c] = x;
    }
}

constexpr int kRowsChunk = 64;  // columns of the row weights staged at a time

// out[m][I] = inv_L sum_c wgt[c][m] Y[I][c] for the T rows m of a block: one
// entry per thread with T accumulators; the weights of kRowsChunk columns at a
// time in shared memory (all lanes read the same column: a broadcast).
__global__ void __launch_bounds__(256)
    pnk_rows(const float* __restrict__ Y, const float* __restrict__ wgt, int ncol, int Mp, long long np3,
             float inv_L, float* __restrict__ out)
{
    constexpr int T = kMaxNoiseBlock;
    __shared__ float4 ws4[kRowsChunk][T / 4];
    const long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float acc[T];
#pragma unroll
    for (int m = 0; m < T; ++m) acc[m] = 0.f;
    for (int c0 = 0; c0 < ncol; c0 += kRowsChunk) {
        const int nc = min(kRowsChunk, ncol - c0);
        __syncthreads();
        for (int e = threadIdx.x; e < nc * (T / 4); e += blockDim.x)
            ws4[e / (T / 4)][e % (T / 4)] = reinterpret_cast<const float4*>(wgt + (size_t)(c0 + e / (T / 4)) * T)[e % (T / 4)];
        __syncthreads();
        if (I < np3)
            for (int c = 0; c < nc; ++c) {
                const float y = Y[(size_t)I * Mp + c0 + c];
#pragma unroll
                for (int k = 0; k < T / 4; ++k) {
                    const float4 w = ws4[c][k];
                    acc[4 * k] = fmaf(w.x, y, acc[4 * k]);
                    acc[4 * k + 1] = fmaf(w.y, y, acc[4 * k + 1]);
                    acc[4 * k + 2] = fmaf(w.z, y, acc[4 * k + 2]);
                    acc[4 * k + 3] = fmaf(w.w, y, acc[4 * k + 3]);
                }
            }
    }
    if (I < np3)
#pragma unroll
        for (int m = 0; m < T; ++m) out[(size_t)m * np3 + I] = acc[m] * inv_L;
}

unsigned elem_blocks(long long np3) { return (unsigned)std::min<long long>((np3 + kKryWarps - 1) / kKryWarps, 1024); }
unsigned sweep_blocks(int n) { return (unsigned)std::min<long long>((n + kKryWarps - 1) / kKryWarps, 1024); }

size_t sweep_smem(const StepParams& P, int Mp)
{
    return sizeof(double) * kKryWarps * Mp + sizeof(float) * (size_t)(1 + P.Q + P.Qs + 1) * Mp;
}

cudaError_t set_smem(const void* f, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

bool kry_fits(const StepParams& P, int Mp)
{
    return (size_t)(P.H + 1) * 8 * sizeof(float4) <= 227 * 1024 && sweep_smem(P, Mp) <= 227 * 1024;
}

int kry_part_blocks(const StepParams& P)
{
    return (int)std::max(elem_blocks(3LL * P.n_pad), sweep_blocks(P.n));
}

cudaError_t kry_ft(const StepParams& P, const Ctrl* ctrl, const float* W, const float* cosT, int M, int Mp, int Mc,
                   float* V0, cudaStream_t st)
{
    const long long np3 = 3LL * P.n_pad;
    const dim3 g((unsigned)(Mp / 32), (unsigned)((np3 + kFtThreads - 1) / kFtThreads));
    const size_t smem = (size_t)(P.H + 1) * 8 * sizeof(float4);
    cudaError_t e = set_smem((const void*)pnk_ft, smem);
    if (e != cudaSuccess) return e;
    pnk_ft<<<g, kFtThreads, smem, st>>>(P, ctrl, W, cosT, M, Mp, Mc, V0);
    return cudaGetLastError();
}

cudaError_t kry_rows(const StepParams& P, const float* V, const float* cf, int kp, int Mp, const float* wgt, float* Y,
                     float* out, cudaStream_t st)
{
    if (P.T != kMaxNoiseBlock) return cudaErrorInvalidValue;
    const long long np3 = 3LL * P.n_pad;
    pnk_combine_y<<<dim3(elem_blocks(np3), (unsigned)(Mp / 32)), 32 * kKryWarps, 0, st>>>(V, cf, kp, Mp, np3, Y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    pnk_rows<<<(unsigned)((np3 + 255) / 256), 256, 0, st>>>(Y, wgt, Mp, Mp, np3, 1.0f / (float)(2 * P.H + 1), out);
    return cudaGetLastError();
}

cudaError_t kry_fold(const double* part, int nblk, int Mp, double* out, int mode, const double* ref, int* alive,
                     cudaStream_t st)
{
    pnk_fold<<<(unsigned)(Mp / 32), 32 * kKryWarps, 0, st>>>(part, nblk, Mp, out, mode, ref, alive);
    return cudaGetLastError();
}

cudaError_t kry_dot(const StepParams& P, const float* a, const float* b, int Mp, double* part, double* out, int mode,
                    const double* ref, int* alive, cudaStream_t st)
{
    const long long np3 = 3LL * P.n_pad;
    const unsigned nb = elem_blocks(np3);
    pnk_dot<<<dim3(nb, (unsigned)(Mp / 32)), 32 * kKryWarps, 0, st>>>(a, b, np3, Mp, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return kry_fold(part, (int)nb, Mp, out, mode, ref, alive, st);
}

cudaError_t kry_matvec(const StepParams& P, const ParticleBuffers& B, const double* wc, const double* beta_k,
                       const int* alive, int Mp, const float* R, float* Z, double* part, double* alpha_k,
                       cudaStream_t st)
{
    const unsigned nb = sweep_blocks(P.n);
    const size_t smem = sweep_smem(P, Mp);
    cudaError_t e = set_smem((const void*)pnk_matvec, smem);
    if (e != cudaSuccess) return e;
    pnk_matvec<<<nb, 32 * kKryWarps, smem, st>>>(P, B.pos, B.nbr, B.nbr_cnt, B.ftab, B.fptab, wc, beta_k, alive, Mp,
                                                 R, Z, part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return kry_fold(part, (int)nb, Mp, alpha_k, 0, nullptr, nullptr, st);
}

cudaError_t kry_resid(const StepParams& P, const float* Z, const float* Rk, const float* Rkm1, const double* alpha_k,
                      const double* beta_k, const double* beta_km1, int* alive, const double* ref, int Mp,
                      float* Rkp1, double* part, double* beta_kp1, cudaStream_t st)
{
    const long long np3 = 3LL * P.n_pad;
    const unsigned nb = elem_blocks(np3);
    pnk_resid<<<dim3(nb, (unsigned)(Mp / 32)), 32 * kKryWarps, 0, st>>>(Z, Rk, Rkm1, alpha_k, beta_k, beta_km1,
                                                                         alive, np3, Mp, Rkp1, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return kry_fold(part, (int)nb, Mp, beta_kp1, 1, ref, alive, st);
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
