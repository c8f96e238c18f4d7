// gld_internal.cuh -- device-side building blocks shared by the GLD kernels.
//
// Contents: the device control block, the by-value parameter block of a step,
// Philox4x32-10 with the Box-Muller map of the white noise W (Sec. II C asks
// for uncorrelated unit Gaussians; the generator is Salmon et al., SC'11),
// cell geometry and the 27-cell stencil traversal (Sec. II C: the method
// iterates over all neighbours within the cutoff), and the FP32 distance test
// whose exact operation order include/gld.h states.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace gld {

constexpr int kMaxQ = 4;            // separable terms per pair-kernel family
constexpr int kMaxAcc = 1 + 2 * kMaxQ;
constexpr int kMaxModes = 8;         // damped-exponential modes of the recursive memory form
constexpr int kPcMaxOriginBins = 2048;  // origins x bins of the pair correlations (48 KB of shared sums)
constexpr int kMaxNoiseBlock = 64;  // register-resident outputs per FIR thread
constexpr int kMaxPnDegree = 16;    // Chebyshev degree of the pair-correlated noise
constexpr int kPnLanczosSteps = 32;  // Lanczos steps for the pair matrix's extreme eigenvalues

// Latched device error bits.
enum : unsigned { kErrNonFinite = 1u, kErrTimeout = 2u, kErrNoise = 4u, kErrNbrOverflow = 8u, kErrPnBound = 16u,
                  kErrCheck = 32u };

// Device control block: the step counter lives on the device so that a
// captured graph of several steps can be replayed without new arguments.
struct Ctrl {
    long long step;      // n: time index of R_n
    long long noise_n0;  // first step covered by the current F^R block
    long long w_hi;      // W generated for times [w_lo, w_hi)
    long long w_lo;
    unsigned err;
    unsigned done_cforce;  // last-block counters (reset by the last block)
    unsigned done_scan;
    unsigned done_fir;
    int rebuild;           // != 0: rebuild cells and neighbour lists after this step's move
    int pad_;
    long long rebuilds;    // neighbour-list builds so far
    long long hslot;       // step mod H: the history slot this step writes
    long long conv_step;   // n + 1, written by the pair kernel of step n
    // VACF schedule at the step the next VACF kernel sees (written by the
    // pair kernel): active, origins in flight, slot of the newest origin, a
    // new origin at this step, lag of the newest origin, partial buffer
    int vacf_on, vacf_nact, vacf_slot0, vacf_origin, vacf_lag0, vacf_buf;
    // partials of an earlier VACF launch not yet added to the sums: set by
    // the VACF kernel, consumed by the next VACF kernel or by a flush
    int vacf_pending;
    // the previous launch's schedule as the next VACF kernel must fold it
    int pv_nact, pv_lag0, pv_buf;
    // the same bookkeeping for the distance-binned pair correlations
    int pc_pending, pc_buf, pc_pv_nact, pc_pv_lag0, pc_pv_buf, pad3_;
};

// Everything a step kernel needs, passed by value.
struct StepParams {
    int n, n_pad, m_max, H;   // H = m_max - 1 history slots
    int Q, Qs, nacc, nr;
    int nc;                   // cells per dimension (1 or >= 3)
    int T;                    // noise block length
    long long lw;             // W ring length (times)
    float box, half_box, inv_box, inv_cell, rc2, rc_min, inv_dr, inv_dt;
    float pos_v, pos_f;       // b dt, b dt^2 / (2M)
    float vh_v, vh_fc, vh_f;  // a, a dt/(2M), b dt/M
    float vf_fc;              // dt/(2M)
    float fc_mag, inv_rc;     // 2A/r_c, 1/r_c
    float rl2;                // (r_c + skin)^2: neighbour-list radius
    float trig2;              // rebuild when a particle moved more than sqrt(trig2)
    int maxnb;                // neighbour-list capacity per particle
    int hist_bf16;
    // VACF
    int vacf_len, vacf_stride, n_os;
    long long vacf_burnin;
    // memory sums in recursive (auxiliary-variable) form: modes (0: ring convolution)
    int nmodes;
    // tabulated conservative force -dU/dr on r = k / fc_inv_dr (0 rows: soft repulsion)
    int fc_nr;
    float fc_inv_dr;
    // distance-binned pair correlations (0 bins: off)
    int pc_nbins;
    float pc_rmax2, pc_inv_dr;  // r_max^2, nbins / r_max
    // pair-correlated noise: Chebyshev degree (0: self-kernel noise only) and
    // the interval [pn_cen - pn_lambda, pn_cen + pn_lambda] holding the
    // spectrum of the pair matrix (pn_cen = 0: the symmetric bound lambda),
    // with 1 / pn_lambda; pn_iv: the interval comes from Ritz values and is
    // checked by a Lanczos run at each noise block (else Gershgorin, each step)
    int pn_deg;
    float pn_lambda, pn_inv_lambda, pn_cen;
    int pn_iv;
    float pn_cs;  // self-difference time factor = pn_cs x the pair term's (when Qs = 1)
    // perpendicular factors of the pair and self-difference terms are set
    // (rows of ParticleBuffers::fptab)
    int perp;
    // pair-correlated noise by a Lanczos iteration per frequency (Algorithm 1)
    int pn_kry;
    // the white-noise ring holds the FP16 split of each value (the form the
    // tensor-core filter multiplies) instead of FP32
    int wsplit;
};

// ---------------------------------------------------------------- Philox --
__host__ __device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
#ifdef __CUDA_ARCH__
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
#else
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
#endif
        const uint32_t n0 = hi1 ^ c[1] ^ k0;
        const uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// u in (0, 1) from the top 23 bits: (x >> 9) + 1/2 needs 24 significant
// bits, so u is exact in FP32.
__device__ inline float u01(uint32_t x) { return ((float)(x >> 9) + 0.5f) * (1.0f / 8388608.0f); }

// W_{i,k} for particle i at time k: counter (i, (k + 2^62) lo, hi, stream).
__device__ inline float3 gauss3(uint32_t k0, uint32_t k1, uint32_t particle, long long time,
                                uint32_t stream)
{
    const unsigned long long t = (unsigned long long)(time + (1LL << 62));
    uint32_t c[4] = {particle, (uint32_t)t, (uint32_t)(t >> 32), stream};
    philox4x32_10(c, k0, k1);
    const float r01 = sqrtf(-2.0f * logf(u01(c[0])));
    const float r23 = sqrtf(-2.0f * logf(u01(c[2])));
    float s1, c1, s3, c3;
    sincospif(2.0f * u01(c[1]), &s1, &c1);
    sincospif(2.0f * u01(c[3]), &s3, &c3);
    return make_float3(r01 * c1, r01 * s1, r23 * c3);
}

// White noise w as the FP16 pair the tensor-core filter multiplies:
// hi = fp16(w), lo = fp16((w - hi) 2^11) (round to nearest each); hi + 2^-11 lo
// is w to 2^-22 of |w|.
__device__ __forceinline__ void split_f16(float v, unsigned short& hi, unsigned short& lo)
{
    const __half h = __float2half_rn(v);
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(__float2half_rn((v - __half2float(h)) * 2048.0f));
}

// Entry idx = slot * 3 n_pad + stream of the white-noise ring, in either form:
// FP32, or (wsplit) an FP16 plane of hi parts followed by one of lo parts.
__device__ __forceinline__ float ring_w(const StepParams& P, const float* __restrict__ W, size_t idx)
{
    if (P.wsplit) {
        const __half* h = (const __half*)W;
        const size_t plane = (size_t)P.lw * 3 * P.n_pad;
        return fmaf(__half2float(__ldg(h + plane + idx)), 1.0f / 2048.0f, __half2float(__ldg(h + idx)));
    }
    return __ldg(W + idx);
}

// ------------------------------------------------------------ geometry --
__device__ inline int cell_coord(float x, float inv_cell, int nc)
{
    int c = (int)(x * inv_cell);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__device__ inline int cell_of(float4 p, const StepParams& P)
{
    const int cx = cell_coord(p.x, P.inv_cell, P.nc), cy = cell_coord(p.y, P.inv_cell, P.nc),
              cz = cell_coord(p.z, P.inv_cell, P.nc);
    return (cz * P.nc + cy) * P.nc + cx;
}

// Minimum-image difference in the operation order stated in gld.h.
__device__ inline float min_image(float a, float b, float L, float half)
{
    float d = __fsub_rn(a, b);
    if (d > half) d = __fsub_rn(d, L);
    else if (d < -half) d = __fadd_rn(d, L);
    return d;
}

// The same without branches: d - L rint(d / L), one rounding like the
// subtraction above, so the same bits whenever |d| is not within rounding of
// L / 2 (every pair inside a cutoff below half the box).
__device__ inline float min_image_fma(float a, float b, float L, float inv_L)
{
    const float d = __fsub_rn(a, b);
    return fmaf(-L, rintf(__fmul_rn(d, inv_L)), d);
}

__device__ inline float dist2(float dx, float dy, float dz)
{
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ inline float wrap_box(float x, float L)
{
    if (x < 0.0f) x = __fadd_rn(x, L);
    else if (x >= L) x = __fsub_rn(x, L);
    if (x >= L) x = 0.0f;
    return x;
}

// Visits every particle j != i with r_ij^2 < r2max over the 27-cell stencil,
// cells in a fixed order and particles of a cell by increasing id:
// f(j, dx, dy, dz, r2) with d = R_i - R_j.
template <class F>
__device__ inline void for_each_in_stencil(const float4 pi, const int id, const float4* __restrict__ pos_sorted,
                                           const int* __restrict__ cell_start, const StepParams& P, float r2max,
                                           F&& f)
{
    const int nc = P.nc;
    const int span = nc == 1 ? 0 : 1;
    const int cx = cell_coord(pi.x, P.inv_cell, nc), cy = cell_coord(pi.y, P.inv_cell, nc),
              cz = cell_coord(pi.z, P.inv_cell, nc);
    for (int oz = -span; oz <= span; ++oz) {
        int z = cz + oz;
        z = z < 0 ? z + nc : (z >= nc ? z - nc : z);
        for (int oy = -span; oy <= span; ++oy) {
            int y = cy + oy;
            y = y < 0 ? y + nc : (y >= nc ? y - nc : y);
            for (int ox = -span; ox <= span; ++ox) {
                int x = cx + ox;
                x = x < 0 ? x + nc : (x >= nc ? x - nc : x);
                const int c = (z * nc + y) * nc + x;
                const int beg = __ldg(cell_start + c), end = __ldg(cell_start + c + 1);
                for (int k = beg; k < end; ++k) {
                    const float4 pj = __ldg(pos_sorted + k);
                    const int jd = __float_as_int(pj.w);
                    if (jd == id) continue;
                    const float dx = min_image(pi.x, pj.x, P.box, P.half_box);
                    const float dy = min_image(pi.y, pj.y, P.box, P.half_box);
                    const float dz = min_image(pi.z, pj.z, P.box, P.half_box);
                    const float r2 = dist2(dx, dy, dz);
                    if (r2 < r2max) f(jd, dx, dy, dz, r2);
                }
            }
        }
    }
}

// Visits every j != i with r_ij < r_c from i's neighbour list (a superset built
// with r_c + skin, in stencil order): f(j, dx, dy, dz, r2) with d = R_i - R_j.
// The distance test is the same as the stencil's, so the pairs are the same.
template <class F>
__device__ inline void for_each_listed(const float4 pi, const int k, const int* __restrict__ nbr,
                                       const int cnt, const int stride, const float4* __restrict__ pos,
                                       const StepParams& P, F&& f)
{
    // four entries per round with their loads in flight together; the next
    // round's entries load during this round's gathers, and the last round is
    // masked (entries past the list stand for i itself, never listed)
    int jn[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) jn[u] = u < cnt ? __ldg(nbr + (size_t)u * stride + k) : k;
    for (int s = 0; s < cnt; s += 4) {
        int j[4];
        float4 pj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) j[u] = jn[u];
#pragma unroll
        for (int u = 0; u < 4; ++u) pj[u] = __ldg(pos + j[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) jn[u] = s + 4 + u < cnt ? __ldg(nbr + (size_t)(s + 4 + u) * stride + k) : k;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (j[u] == k) continue;
            const float dx = min_image_fma(pi.x, pj[u].x, P.box, P.inv_box);
            const float dy = min_image_fma(pi.y, pj[u].y, P.box, P.inv_box);
            const float dz = min_image_fma(pi.z, pj[u].z, P.box, P.inv_box);
            const float r2 = dist2(dx, dy, dz);
            if (r2 < P.rc2) f(j[u], dx, dy, dz, r2);
        }
    }
}

// Linear interpolation of a radial table on r = k dr; constant past the end.
__device__ inline float table_at(const float* __restrict__ t, int nr, float x /* r / dr */)
{
    if (x <= 0.0f) return __ldg(t);
    const int k = (int)x;
    if (k >= nr - 1) return __ldg(t + nr - 1);
    const float w = x - (float)k;
    return fmaf(w, __ldg(t + k + 1) - __ldg(t + k), __ldg(t + k));
}

}  // namespace gld
