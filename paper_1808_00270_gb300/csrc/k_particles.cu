// k_particles.cu -- the per-particle kernels of one GLD step.
//
//   pair_force_integrate  F^D_n (Eq. dissipative_force2) from the history
//                         projections and the neighbours at R_n, then the
//                         position half of Eq. GLD_integrator (with b, App. A),
//                         the new displacement into the history ring, and the
//                         velocity terms that do not need F^C_{n+1}.  Requests
//                         a neighbour-list rebuild when a particle has moved
//                         more than half the skin since the last build.
//   cell build + nbr_build (only when a rebuild was requested): cell list at
//                         R_{n+1} (per-cell linked lists, chunked scan, cells
//                         filled in id order), then per particle the ids within
//                         r_c + skin in the (fixed) stencil traversal order.
//   cforce                F^C_{n+1} = sum_j 2A/r_c (1 - r/r_c) e_ij and the
//                         rest of the velocity update; advances n.
//   vacf                  FP64 accumulation of <V(t0+tau) V(t0)> (Sec. III A).
//
// Every neighbour sum runs over a Verlet list with the exact FP32 r < r_c test
// of the cell traversal, so the pair set is the same; lists are sorted by
// neighbour id at each build, so the order of every sum does not depend on
// when the list was built.  Particles are stored in the Morton order of their cells at creation
// and a thread handles one particle id, so own loads are coalesced and
// neighbours lie close in memory; ids never change, so the displacement
// history is never permuted.
#include <algorithm>

#include <cuda_bf16.h>

#include "launch.h"

namespace gld {

namespace {

constexpr int kPairThreads = kBatchPairBlock;
constexpr int kPairLanes = kBatchPairLanes;  // lanes per particle in the one-term pair kernel
constexpr int kPairBatch = 4;                 // list entries per round of the one-term pair kernel
constexpr int kCforceLanes = kBatchCforceLanes;  // lanes per particle in the F^C kernel
constexpr int kCellThreads = kBatchCellChunk;
constexpr int kThreads = kBatchPartBlock;
constexpr int kNbrSortCap = 128;  // list entries sorted by id at each build
static_assert(kBatchVacfBlock == kThreads, "vacf blocks share the particle block size");

__device__ __forceinline__ float dot3(float ax, float ay, float az, float bx, float by, float bz)
{
    return fmaf(ax, bx, fmaf(ay, by, az * bz));
}

// The VACF kernel's view of step t (once per step, by one thread): origins
// start at vacf_burnin and every vacf_stride steps; the origin of age j is
// active while its lag t - t_j is below vacf_len.
__device__ __forceinline__ void vacf_schedule(const StepParams& P, Ctrl* __restrict__ ctrl, long long t)
{
    // the partials of the last VACF launch are folded by the next one; the
    // same for the pair correlations' per-step sums
    ctrl->pc_pv_nact = ctrl->pc_pending ? ctrl->vacf_nact : 0;
    ctrl->pc_pv_lag0 = ctrl->vacf_lag0;
    ctrl->pc_pv_buf = ctrl->pc_buf;
    ctrl->pc_pending = 0;
    ctrl->pc_buf ^= 1;
    ctrl->pv_nact = ctrl->vacf_pending ? ctrl->vacf_nact : 0;
    ctrl->pv_lag0 = ctrl->vacf_lag0;
    ctrl->pv_buf = ctrl->vacf_buf;
    ctrl->vacf_pending = 0;
    ctrl->vacf_buf ^= 1;
    if (t < P.vacf_burnin) {
        ctrl->vacf_on = 0;
        return;
    }
    const long long rel = t - P.vacf_burnin;
    const long long o_now = rel / P.vacf_stride;
    const int lag0 = (int)(rel - o_now * P.vacf_stride);
    int n_act = 0;
    for (int j = 0; j < P.n_os; ++j)
        if (o_now - j >= 0 && lag0 + (long long)j * P.vacf_stride < P.vacf_len) n_act = j + 1;
    ctrl->vacf_on = 1;
    ctrl->vacf_nact = n_act;
    ctrl->vacf_slot0 = (int)(o_now % P.n_os);
    ctrl->vacf_origin = lag0 == 0;
    ctrl->vacf_lag0 = lag0;
}

// FAST: exactly one separable pair term and no self-difference term.
template <bool FAST>
__device__ __forceinline__ void pair_force_integrate_body(const StepParams& P, Ctrl* __restrict__ ctrl, const float4* __restrict__ pos,
                         const int* __restrict__ perm, const int* __restrict__ nbr, const int* __restrict__ nbr_cnt,
                         const float4* __restrict__ vel, const float4* __restrict__ fc, const float* __restrict__ conv,
                         const float* __restrict__ frblock, const float* __restrict__ ftab,
                         const float* __restrict__ fptab,
                         const float* __restrict__ g0, void* __restrict__ ring, float4* __restrict__ pos_next,
                         float4* __restrict__ vhalf, float4* __restrict__ fd_out, float4* __restrict__ disp,
                         const float4* __restrict__ disp_build, int blk, int nblk)
{
    unsigned* err = &ctrl->err;
    // FAST: kPairLanes consecutive lanes share a particle and split its list
    constexpr int LANES = FAST ? kPairLanes : 1;
    const int k = (blk * blockDim.x + threadIdx.x) / LANES;
    const int lr = threadIdx.x & (LANES - 1);
    if (k >= P.n) return;  // uniform over the lanes of a particle
    const long long n = ctrl->step;
    const long long np = P.n_pad;
    const int id = k;  // particles in storage (Morton) order; lists are by id
    if (blk == 0 && threadIdx.x == 0) {
        ctrl->conv_step = n + 1;  // for a convolution of the next step that overlaps this one's tail
        if (P.vacf_len > 0) vacf_schedule(P, ctrl, n + 1);
    }
    const float4 pi = pos[id];
    const float4 vi = vel[id];

    float ps[FAST ? 1 : kMaxQ][3];
#pragma unroll
    for (int q = 0; q < (FAST ? 1 : kMaxQ); ++q) {
        if (q < P.Qs) {
            const float* p = conv + (size_t)(1 + P.Q + q) * 3 * np + id;
            ps[q][0] = p[0];
            ps[q][1] = p[np];
            ps[q][2] = p[2 * np];
        } else {
            ps[q][0] = ps[q][1] = ps[q][2] = 0.f;
        }
    }
    float f0x = 0.f, f0y = 0.f, f0z = 0.f;  // instantaneous (m = 0) pair terms
    float fhx = 0.f, fhy = 0.f, fhz = 0.f;  // history pair terms (times -1, before 1/dt)
    if (FAST) {
        // one separable pair term (the common case): the neighbour's V_j and
        // P_j are fetched together with its position, four candidates at a
        // time, so that one memory latency covers the whole batch; the
        // arithmetic is the general loop's below, term for term
        const float* pj0 = conv + 3 * (size_t)np;
        const float g00 = __ldg(g0);
        const int cnt = nbr_cnt[id];
        auto term = [&](int jd, float4 pj, float4 vj, float qx, float qy, float qz) {
            const float dx = min_image_fma(pi.x, pj.x, P.box, P.inv_box);
            const float dy = min_image_fma(pi.y, pj.y, P.box, P.inv_box);
            const float dz = min_image_fma(pi.z, pj.z, P.box, P.inv_box);
            const float r2 = dist2(dx, dy, dz);
            if (!(r2 < P.rc2)) return;
            const float inv_r = rsqrtf(r2);  // listed pairs are distinct particles: r2 > 0
            const float r = r2 * inv_r;
            const float ex = dx * inv_r, ey = dy * inv_r, ez = dz * inv_r;
            const float x = fmaxf(r, P.rc_min) * P.inv_dr;
            const float evj = dot3(ex, ey, ez, vj.x, vj.y, vj.z);
            const float fq = table_at(ftab, P.nr, x);
            const float epj = dot3(ex, ey, ez, qx, qy, qz);
            const float inst = fmaf(fq * g00, evj, 0.f);
            const float hist = fmaf(fq, epj, 0.f);
            f0x = fmaf(-inst, ex, f0x); f0y = fmaf(-inst, ey, f0y); f0z = fmaf(-inst, ez, f0z);
            fhx = fmaf(-hist, ex, fhx); fhy = fmaf(-hist, ey, fhy); fhz = fmaf(-hist, ez, fhz);
        };
        // lane lr takes the entries lr, lr + LANES, ...: kPairBatch of them
        // per round with all their loads in flight together
        // (the last round is masked: entries past the list stand for the
        // particle itself, whose loads hit cache, and add nothing)
        // (the last round is masked: entries past the list stand for the
        // particle itself, whose loads hit cache, and add nothing; the next
        // round's list entries load while this round's gathers are in flight)
        constexpr int NB = kPairBatch;
        int jn[NB];
#pragma unroll
        for (int u = 0; u < NB; ++u) jn[u] = lr + u * LANES < cnt ? __ldg(nbr + (size_t)(lr + u * LANES) * P.n_pad + id) : id;
        for (int base = lr; base < cnt; base += NB * LANES) {
            int j[NB];
            float4 pj[NB], vj[NB];
            float qx[NB], qy[NB], qz[NB];
#pragma unroll
            for (int u = 0; u < NB; ++u) j[u] = jn[u];
#pragma unroll
            for (int u = 0; u < NB; ++u) {
                pj[u] = __ldg(pos + j[u]);
                vj[u] = __ldg(vel + j[u]);
                qx[u] = __ldg(pj0 + j[u]);
                qy[u] = __ldg(pj0 + np + j[u]);
                qz[u] = __ldg(pj0 + 2 * np + j[u]);
            }
            const int nb = base + NB * LANES;
#pragma unroll
            for (int u = 0; u < NB; ++u)
                jn[u] = nb + u * LANES < cnt ? __ldg(nbr + (size_t)(nb + u * LANES) * P.n_pad + id) : id;
#pragma unroll
            for (int u = 0; u < NB; ++u)
                if (j[u] != id) term(j[u], pj[u], vj[u], qx[u], qy[u], qz[u]);
        }
        if (LANES > 1) {  // sum over the lanes of the particle (same result in each)
            const unsigned grp = ((1u << LANES) - 1u) << ((threadIdx.x & 31) & ~(LANES - 1));
#pragma unroll
            for (int o = 1; o < LANES; o <<= 1) {
                f0x += __shfl_xor_sync(grp, f0x, o); f0y += __shfl_xor_sync(grp, f0y, o);
                f0z += __shfl_xor_sync(grp, f0z, o); fhx += __shfl_xor_sync(grp, fhx, o);
                fhy += __shfl_xor_sync(grp, fhy, o); fhz += __shfl_xor_sync(grp, fhz, o);
            }
        }
        if (lr != 0) return;  // one lane finishes the particle
    } else if (!FAST && P.Q + P.Qs > 0) {
        for_each_listed(pi, id, nbr, nbr_cnt[id], P.n_pad, pos, P, [&](int jd, float dx, float dy, float dz, float r2) {
            const float r = sqrtf(r2);
            const float inv_r = 1.0f / r;
            const float ex = dx * inv_r, ey = dy * inv_r, ez = dz * inv_r;
            const float x = fmaxf(r, P.rc_min) * P.inv_dr;
            const float4 vj = __ldg(vel + jd);
            const float evj = dot3(ex, ey, ez, vj.x, vj.y, vj.z);
            const float evi = dot3(ex, ey, ez, vi.x, vi.y, vi.z);
            float inst = 0.f, hist = 0.f;
            for (int q = 0; q < P.Q; ++q) {
                const float fq = table_at(ftab + q * P.nr, P.nr, x);
                const float* pj = conv + (size_t)(1 + q) * 3 * np + jd;
                const float epj = dot3(ex, ey, ez, __ldg(pj), __ldg(pj + np), __ldg(pj + 2 * np));
                inst = fmaf(fq * __ldg(g0 + q), evj, inst);
                hist = fmaf(fq, epj, hist);
            }
            for (int q = 0; q < P.Qs; ++q) {
                const float fq = table_at(ftab + (P.Q + q) * P.nr, P.nr, x);
                const float epi = dot3(ex, ey, ez, ps[q][0], ps[q][1], ps[q][2]);
                inst = fmaf(fq * __ldg(g0 + P.Q + q), evi, inst);
                hist = fmaf(fq, epi, hist);
            }
            f0x = fmaf(-inst, ex, f0x); f0y = fmaf(-inst, ey, f0y); f0z = fmaf(-inst, ez, f0z);
            fhx = fmaf(-hist, ex, fhx); fhy = fmaf(-hist, ey, fhy); fhz = fmaf(-hist, ez, fhz);
            if (P.perp) {
                // perpendicular parts act through 1 - e e^T: on X they give
                // fp (X - (e.X) e), X = V_j, P_j (pair) or V_i, P_i (self-difference)
                float cvj = 0.f, cvi = 0.f, hpe = 0.f, hpx = 0.f, hpy = 0.f, hpz = 0.f;
                for (int q = 0; q < P.Q; ++q) {
                    const float fp = table_at(fptab + q * P.nr, P.nr, x);
                    const float* pj = conv + (size_t)(1 + q) * 3 * np + jd;
                    const float px = __ldg(pj), py = __ldg(pj + np), pz = __ldg(pj + 2 * np);
                    cvj = fmaf(fp, __ldg(g0 + q), cvj);
                    hpe = fmaf(fp, dot3(ex, ey, ez, px, py, pz), hpe);
                    hpx = fmaf(fp, px, hpx); hpy = fmaf(fp, py, hpy); hpz = fmaf(fp, pz, hpz);
                }
                for (int q = 0; q < P.Qs; ++q) {
                    const float fp = table_at(fptab + (P.Q + q) * P.nr, P.nr, x);
                    cvi = fmaf(fp, __ldg(g0 + P.Q + q), cvi);
                    hpe = fmaf(fp, dot3(ex, ey, ez, ps[q][0], ps[q][1], ps[q][2]), hpe);
                    hpx = fmaf(fp, ps[q][0], hpx); hpy = fmaf(fp, ps[q][1], hpy); hpz = fmaf(fp, ps[q][2], hpz);
                }
                const float ipe = fmaf(cvj, evj, cvi * evi);
                f0x += fmaf(ipe, ex, -fmaf(cvj, vj.x, cvi * vi.x));
                f0y += fmaf(ipe, ey, -fmaf(cvj, vj.y, cvi * vi.y));
                f0z += fmaf(ipe, ez, -fmaf(cvj, vj.z, cvi * vi.z));
                fhx += fmaf(hpe, ex, -hpx); fhy += fmaf(hpe, ey, -hpy); fhz += fmaf(hpe, ez, -hpz);
            }
        });
    }
    // F^D = -sum_j (K^p_0 V_j + dK^s_0 V_i) - (1/dt) (S_i + sum_j ...)
    const float sx = conv[id], sy = conv[np + id], sz = conv[2 * np + id];
    const float fdx = fmaf(fhx - sx, P.inv_dt, f0x);
    const float fdy = fmaf(fhy - sy, P.inv_dt, f0y);
    const float fdz = fmaf(fhz - sz, P.inv_dt, f0z);
    const long long row = n - ctrl->noise_n0;
    float frx = 0.f, fry = 0.f, frz = 0.f;
    if (row >= 0 && row < P.T) {
        const float* fr = frblock + (size_t)row * 3 * np + id;
        frx = fr[0];
        fry = fr[np];
        frz = fr[2 * np];
    } else if (k == 0) {
        atomicOr(err, kErrNoise);  // the host scheduled a step outside the noise block
    }
    const float4 fci = fc[id];
    // Eq. GLD_integrator, position: dR = b dt V + b dt^2/(2M) (F^C + F^D + F^R)
    const float dRx = fmaf(P.pos_f, fci.x + fdx + frx, P.pos_v * vi.x);
    const float dRy = fmaf(P.pos_f, fci.y + fdy + fry, P.pos_v * vi.y);
    const float dRz = fmaf(P.pos_f, fci.z + fdz + frz, P.pos_v * vi.z);
    const long long slot = ctrl->hslot;  // n mod H
    if (P.hist_bf16) {
        __nv_bfloat16* h = (__nv_bfloat16*)ring + (size_t)slot * 3 * np + id;
        h[0] = __float2bfloat16_rn(dRx);
        h[np] = __float2bfloat16_rn(dRy);
        h[2 * np] = __float2bfloat16_rn(dRz);
    } else {
        float* h = (float*)ring + (size_t)slot * 3 * np + id;
        h[0] = dRx;
        h[np] = dRy;
        h[2 * np] = dRz;
    }
    pos_next[id] = make_float4(wrap_box(__fadd_rn(pi.x, dRx), P.box), wrap_box(__fadd_rn(pi.y, dRy), P.box),
                               wrap_box(__fadd_rn(pi.z, dRz), P.box), 0.f);
    // velocity part known now: a V + a dt/(2M) F^C_n + b dt/M (F^D + F^R)
    vhalf[id] = make_float4(fmaf(P.vh_f, fdx + frx, fmaf(P.vh_fc, fci.x, P.vh_v * vi.x)),
                            fmaf(P.vh_f, fdy + fry, fmaf(P.vh_fc, fci.y, P.vh_v * vi.y)),
                            fmaf(P.vh_f, fdz + frz, fmaf(P.vh_fc, fci.z, P.vh_v * vi.z)), 0.f);
    fd_out[id] = make_float4(fdx, fdy, fdz, 0.f);
    const float4 d = disp[id];
    const float4 dn = make_float4(d.x + dRx, d.y + dRy, d.z + dRz, 0.f);
    disp[id] = dn;
    // Verlet criterion: a particle moved more than half the skin since the build.
    const float4 db = disp_build[id];
    const float mx = dn.x - db.x, my = dn.y - db.y, mz = dn.z - db.z;
    if (mx * mx + my * my + mz * mz > P.trig2) atomicOr(&ctrl->rebuild, 1);
    if (!(isfinite(dRx) && isfinite(dRy) && isfinite(dRz))) {
        atomicOr(err, kErrNonFinite);
        atomicOr(&ctrl->rebuild, 1);
    }
}

template <bool FAST>
__global__ void __launch_bounds__(kPairThreads) pair_force_integrate(const StepParams P, Ctrl* __restrict__ ctrl, const float4* __restrict__ pos,
                         const int* __restrict__ perm, const int* __restrict__ nbr, const int* __restrict__ nbr_cnt,
                         const float4* __restrict__ vel, const float4* __restrict__ fc, const float* __restrict__ conv,
                         const float* __restrict__ frblock, const float* __restrict__ ftab,
                         const float* __restrict__ fptab,
                         const float* __restrict__ g0, void* __restrict__ ring, float4* __restrict__ pos_next,
                         float4* __restrict__ vhalf, float4* __restrict__ fd_out, float4* __restrict__ disp,
                         const float4* __restrict__ disp_build)
{
    pair_force_integrate_body<FAST>(P, ctrl, pos, perm, nbr, nbr_cnt, vel, fc, conv, frblock, ftab, fptab, g0, ring, pos_next, vhalf, fd_out, disp, disp_build, blockIdx.x, gridDim.x);
}

// ---- cell list --------------------------------------------------------------
__device__ __forceinline__ void cell_assign_body(const StepParams& P, const int* __restrict__ gate, const float4* __restrict__ pos,
                            int* __restrict__ head, int* __restrict__ next, int* __restrict__ count, int blk, int nblk)
{
    if (gate && *gate == 0) return;
    const int i = blk * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const int c = cell_of(pos[i], P);
    atomicAdd(count + c, 1);
    next[i] = atomicExch(head + c, i);
}

__global__ void cell_assign(const StepParams P, const int* __restrict__ gate, const float4* __restrict__ pos,
                            int* __restrict__ head, int* __restrict__ next, int* __restrict__ count)
{
    cell_assign_body(P, gate, pos, head, next, count, blockIdx.x, gridDim.x);
}

// Exclusive block scan of one int per thread; returns the block total.
__device__ int block_exclusive_scan(int v, int* out_excl)
{
    __shared__ int warp_tot[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        int t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;
    }
    __syncthreads();
    const int base = w > 0 ? warp_tot[w - 1] : 0;
    *out_excl = base + x - v;
    const int total = warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
    return total;
}

// Chunk sums of the cell counts; the last block to finish scans them.
__device__ __forceinline__ void cell_scan_body(const int* __restrict__ gate, const int* __restrict__ count, int ncells, int* __restrict__ chunk_sum,
              int* __restrict__ chunk_off, unsigned* __restrict__ done, int blk, int nblk)
{
    if (gate && *gate == 0) return;  // uniform over the grid
    const int c = blk * blockDim.x + threadIdx.x;
    int excl;
    const int tot = block_exclusive_scan(c < ncells ? count[c] : 0, &excl);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        chunk_sum[blk] = tot;
        __threadfence();
        last = atomicAdd(done, 1u) == nblk - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    int carry = 0;
    for (int base = 0; base < (int)nblk; base += blockDim.x) {
        const int b = base + threadIdx.x;
        const int v = b < (int)nblk ? ((volatile int*)chunk_sum)[b] : 0;
        int e;
        const int t = block_exclusive_scan(v, &e);
        if (b < (int)nblk) chunk_off[b] = carry + e;
        carry += t;
    }
    if (threadIdx.x == 0) *done = 0u;
}

__global__ void __launch_bounds__(kCellThreads) cell_scan(const int* __restrict__ gate, const int* __restrict__ count, int ncells, int* __restrict__ chunk_sum,
              int* __restrict__ chunk_off, unsigned* __restrict__ done)
{
    cell_scan_body(gate, count, ncells, chunk_sum, chunk_off, done, blockIdx.x, gridDim.x);
}

// Cell starts, and each cell's particles in increasing id order.
__device__ __forceinline__ void cell_fill_body(const StepParams& P, const int* __restrict__ gate, int ncells, const float4* __restrict__ pos,
              int* __restrict__ count, int* __restrict__ head, const int* __restrict__ next,
              const int* __restrict__ chunk_off, int* __restrict__ cell_start, float4* __restrict__ pos_sorted, int blk, int nblk)
{
    if (gate && *gate == 0) return;
    const int c = blk * blockDim.x + threadIdx.x;
    const int cnt = c < ncells ? count[c] : 0;
    int excl;
    block_exclusive_scan(cnt, &excl);
    if (c >= ncells) return;
    const int start = chunk_off[blk] + excl;
    cell_start[c] = start;
    int j = head[c];
    for (int r = 0; r < cnt && j >= 0; ++r) {
        // insertion by id into [start, start + r)
        int p = start + r;
        while (p > start && __float_as_int(pos_sorted[p - 1].w) > j) {
            pos_sorted[p] = pos_sorted[p - 1];
            --p;
        }
        const float4 x = pos[j];
        pos_sorted[p] = make_float4(x.x, x.y, x.z, __int_as_float(j));
        j = next[j];
    }
    head[c] = -1;
    count[c] = 0;
}

__global__ void __launch_bounds__(kCellThreads) cell_fill(const StepParams P, const int* __restrict__ gate, int ncells, const float4* __restrict__ pos,
              int* __restrict__ count, int* __restrict__ head, const int* __restrict__ next,
              const int* __restrict__ chunk_off, int* __restrict__ cell_start, float4* __restrict__ pos_sorted)
{
    cell_fill_body(P, gate, ncells, pos, count, head, next, chunk_off, cell_start, pos_sorted, blockIdx.x, gridDim.x);
}

// Per particle, in cell order: the ids within r_c + skin in traversal order.
__device__ __forceinline__ void nbr_build_body(const StepParams& P, Ctrl* __restrict__ ctrl, const float4* __restrict__ pos_sorted,
              const int* __restrict__ cell_start, int* __restrict__ nbr, int* __restrict__ nbr_cnt,
              int* __restrict__ perm, const float4* __restrict__ disp, float4* __restrict__ disp_build, int blk, int nblk)
{
    if (ctrl->rebuild == 0) return;
    const int k = blk * blockDim.x + threadIdx.x;
    if (k == 0) ctrl->rebuilds += 1;
    if (k >= P.n) return;
    const float4 pi = pos_sorted[k];
    const int id = __float_as_int(pi.w);
    const int stride = P.n_pad, cap = P.maxnb;
    int c = 0;
    // Candidates are collected in traversal order and sorted by id, so the
    // order of every sum over a list does not depend on the cell layout at
    // the time the list was built (a run resumed from a checkpoint, which
    // builds its lists at the resume step, gives the same bits).  Entries
    // beyond the first kNbrSortCap (far above any workload's lists) keep the
    // traversal order.
    int loc[kNbrSortCap];
    for_each_in_stencil(pi, id, pos_sorted, cell_start, P, P.rl2, [&](int jd, float, float, float, float) {
        if (c < kNbrSortCap) loc[c] = jd;
        else if (c < cap) nbr[(size_t)c * stride + id] = jd;
        ++c;
    });
    if (c > cap) {
        atomicOr(&ctrl->err, kErrNbrOverflow);
        c = cap;
    }
    const int ns = c < kNbrSortCap ? c : kNbrSortCap;
    for (int s = 1; s < ns; ++s) {
        const int v = loc[s];
        int q = s;
        for (; q > 0 && loc[q - 1] > v; --q) loc[q] = loc[q - 1];
        loc[q] = v;
    }
    for (int s = 0; s < ns; ++s) nbr[(size_t)s * stride + id] = loc[s];
    nbr_cnt[id] = c;
    perm[k] = id;
    disp_build[id] = disp[id];
}

__global__ void __launch_bounds__(kThreads) nbr_build(const StepParams P, Ctrl* __restrict__ ctrl, const float4* __restrict__ pos_sorted,
              const int* __restrict__ cell_start, int* __restrict__ nbr, int* __restrict__ nbr_cnt,
              int* __restrict__ perm, const float4* __restrict__ disp, float4* __restrict__ disp_build)
{
    nbr_build_body(P, ctrl, pos_sorted, cell_start, nbr, nbr_cnt, perm, disp, disp_build, blockIdx.x, gridDim.x);
}

// ---- velocity autocorrelation ------------------------------------------------
constexpr int kVacfMaxOrigins = 32;  // origins in flight (vacf_len / vacf_stride)
constexpr int kVacfGroup = 4;        // origins per block row of the VACF grid

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Knuth's two-sum: s + e equals a + b exactly (no contraction: additions only).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) += (bhi, blo) in double-float arithmetic on the FP32 pipes.
__device__ __forceinline__ void df_add(float& hi, float& lo, float bhi, float blo)
{
    float s, e;
    two_sum(hi, bhi, s, e);
    e += lo + blo;
    hi = s + e;
    lo = e - (hi - s);
}

// Adds the block partials of origins q = first, first + step, ... (buffer
// buf, nblk partials each) to C(lag0 + q*stride): double-float sums on the
// FP32 pipes in a fixed order, one FP64 addition per origin.
__device__ __forceinline__ void vacf_fold(const StepParams& P, const float* __restrict__ partial, double* __restrict__ csum,
                                          long long* __restrict__ ccnt, int buf, int nact, int lag0, int nblk, int first,
                                          int step)
{
    __shared__ float sh[kThreads / 32][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float* base = partial + (size_t)buf * P.n_os * nblk;
    for (int q = first; q < nact; q += step) {
        float hi = 0.f, lo = 0.f;
        for (int b = threadIdx.x; b < nblk; b += blockDim.x)
            df_add(hi, lo, __ldcg(base + (size_t)q * nblk + b), 0.f);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
            df_add(hi, lo, h2, l2);
        }
        if (lane == 0) {
            sh[warp][0] = hi;
            sh[warp][1] = lo;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float h = 0.f, l = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) df_add(h, l, sh[w][0], sh[w][1]);
            const int lg = lag0 + q * P.vacf_stride;  // < vacf_len for q < nact
            csum[lg] += (double)h + (double)l;
            ccnt[lg] += 1;
        }
        __syncthreads();
    }
}

// The VACF terms of V_{n+1}, fused into the F^C kernel that computes it:
// blocks b < (origins of the previous step) first fold that step's partials
// (one origin each), then every block writes its partial sums of
// V_{n+1} . V(t0) for each active origin (particle i is thread i of the
// grid; FP32 warp and block sums in a fixed order) and stores the new origin.
// All threads of the block take part (valid: thread i holds particle i).
__device__ __forceinline__ void cforce_vacf(const StepParams& P, Ctrl* __restrict__ ctrl, const float4 v, bool valid,
                                            int i, float4* __restrict__ vorig, float* __restrict__ partial,
                                            double* __restrict__ csum, long long* __restrict__ ccnt,
                                            long long* __restrict__ norig, int blk, int nblk)
{
    if (ctrl->pv_nact > 0)  // uniform over the block
        vacf_fold(P, partial, csum, ccnt, ctrl->pv_buf, ctrl->pv_nact, ctrl->pv_lag0, nblk, blk, nblk);
    if (!ctrl->vacf_on) return;  // uniform over the grid
    const int n_act = ctrl->vacf_nact;
    const bool is_origin = ctrl->vacf_origin != 0;
    const int slot0 = ctrl->vacf_slot0;  // slot of age j: (slot0 - j) mod n_os
    if (blk == 0 && threadIdx.x == 0) {
        ctrl->vacf_pending = 1;
        if (is_origin) *norig += 1;
    }
    __shared__ float wsum[kThreads / 32][kVacfGroup];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* out = partial + (size_t)ctrl->vacf_buf * P.n_os * nblk;
    for (int q0 = 0; q0 < n_act; q0 += kVacfGroup) {
        float4 w[kVacfGroup];
#pragma unroll
        for (int q = 0; q < kVacfGroup; ++q) {
            const int j = q0 + q;
            const int sl = slot0 - j < 0 ? slot0 - j + P.n_os : slot0 - j;
            // the origin of age 0 on an origin step is V_{n+1} itself
            const bool use = valid && j < n_act && !(j == 0 && is_origin);
            w[q] = use ? __ldcs(vorig + (size_t)sl * P.n + i) : v;
        }
#pragma unroll
        for (int q = 0; q < kVacfGroup; ++q) {
            const float d = (valid && q0 + q < n_act) ? fmaf(v.x, w[q].x, fmaf(v.y, w[q].y, v.z * w[q].z)) : 0.f;
            const float sq = warp_sum_f(d);
            if (lane == 0) wsum[warp][q] = sq;
        }
        __syncthreads();
        if (threadIdx.x < kVacfGroup && q0 + (int)threadIdx.x < n_act) {
            float sb = 0.f;
            for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) sb += wsum[w2][threadIdx.x];
            out[(size_t)(q0 + threadIdx.x) * nblk + blk] = sb;
        }
        __syncthreads();
    }
    if (is_origin && valid) vorig[(size_t)slot0 * P.n + i] = v;
}

// ---- conservative force and velocity finish --------------------------------
// R_{n+1} is read from pos_next (every thread reads neighbours there) and
// copied into pos for the next step.
// VACF (with STEP): the VACF terms of V_{n+1} too (cforce_vacf; one lane per
// particle, blocks of kThreads particles, nblk = the VACF partial count).
template <bool STEP, bool VACF = false>
__device__ __forceinline__ void cforce_body(const StepParams& P, Ctrl* __restrict__ ctrl, const float4* __restrict__ pos_next,
           float4* __restrict__ pos, const int* __restrict__ perm, const int* __restrict__ nbr,
           const int* __restrict__ nbr_cnt, const float4* __restrict__ vhalf, float4* __restrict__ vel,
           float4* __restrict__ fc, const float* __restrict__ fctab, int blk, int nblk,
           float4* __restrict__ vorig = nullptr, float* __restrict__ vpartial = nullptr,
           double* __restrict__ csum = nullptr, long long* __restrict__ ccnt = nullptr,
           long long* __restrict__ norig = nullptr)
{
    static_assert(!VACF || kCforceLanes == 1, "the fused VACF takes one particle per thread");
    float4 vnew = make_float4(0.f, 0.f, 0.f, 0.f);
    // kCforceLanes consecutive lanes share a particle and split its list
    const int k = (blk * blockDim.x + threadIdx.x) / kCforceLanes;
    const int lr = threadIdx.x & (kCforceLanes - 1);
    if (blk == 0 && threadIdx.x == 0) ctrl->rebuild = 0;  // the lists are current for R_{n+1}
    if (k < P.n) {  // uniform over the lanes of a particle
        const int id = k;
        const float4 pi = pos_next[id];
        const int cnt = nbr_cnt[id];
        float fx = 0.f, fy = 0.f, fz = 0.f;
        for (int base = lr; base < cnt; base += 4 * kCforceLanes) {
            int j[4];
            float4 pj[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int s = base + u * kCforceLanes;
                j[u] = s < cnt ? __ldg(nbr + (size_t)s * P.n_pad + id) : -1;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) pj[u] = __ldg(pos_next + (j[u] < 0 ? id : j[u]));
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float dx = min_image_fma(pi.x, pj[u].x, P.box, P.inv_box);
                const float dy = min_image_fma(pi.y, pj[u].y, P.box, P.inv_box);
                const float dz = min_image_fma(pi.z, pj[u].z, P.box, P.inv_box);
                const float r2 = dist2(dx, dy, dz);
                if (j[u] >= 0 && r2 < P.rc2) {
                    const float inv_r = rsqrtf(r2);  // listed pairs are distinct particles: r2 > 0
                    const float r = r2 * inv_r;
                    // -dU/dr e_ij with U = A (1 - r/r_c)^2, e_ij = (R_i - R_j)/r
                    // -dU/dr: a table (P.fc_nr > 0) or the soft repulsion A (1 - r/r_c)^2
                    const float sc = (P.fc_nr > 0 ? table_at(fctab, P.fc_nr, r * P.fc_inv_dr)
                                                   : P.fc_mag * (1.0f - r * P.inv_rc)) * inv_r;
                    fx = fmaf(sc, dx, fx);
                    fy = fmaf(sc, dy, fy);
                    fz = fmaf(sc, dz, fz);
                }
            }
        }
        const unsigned grp = ((1u << kCforceLanes) - 1u) << ((threadIdx.x & 31) & ~(kCforceLanes - 1));
#pragma unroll
        for (int o = 1; o < kCforceLanes; o <<= 1) {
            fx += __shfl_xor_sync(grp, fx, o);
            fy += __shfl_xor_sync(grp, fy, o);
            fz += __shfl_xor_sync(grp, fz, o);
        }
        if (lr == 0) {
            pos[id] = pi;
            fc[id] = make_float4(fx, fy, fz, 0.f);
            if (STEP) {
                const float4 vh = vhalf[id];
                vnew = make_float4(fmaf(P.vf_fc, fx, vh.x), fmaf(P.vf_fc, fy, vh.y), fmaf(P.vf_fc, fz, vh.z), 0.f);
                vel[id] = vnew;
            }
        }
    }
    if (STEP && VACF)
        cforce_vacf(P, ctrl, vnew, k < P.n, k, vorig, vpartial, csum, ccnt, norig, blk, nblk);
    if (STEP) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(&ctrl->done_cforce, 1u) == nblk - 1) {
                ctrl->step += 1;
                ctrl->hslot = ctrl->hslot + 1 == P.H ? 0 : ctrl->hslot + 1;
                ctrl->done_cforce = 0u;
                __threadfence();
            }
        }
    }
}

template <bool STEP, bool VACF>
__global__ void __launch_bounds__(kThreads) cforce(const StepParams P, Ctrl* __restrict__ ctrl, const float4* __restrict__ pos_next,
           float4* __restrict__ pos, const int* __restrict__ perm, const int* __restrict__ nbr,
           const int* __restrict__ nbr_cnt, const float4* __restrict__ vhalf, float4* __restrict__ vel,
           float4* __restrict__ fc, const float* __restrict__ fctab, float4* __restrict__ vorig,
           float* __restrict__ vpartial, double* __restrict__ csum, long long* __restrict__ ccnt,
           long long* __restrict__ norig)
{
    cforce_body<STEP, VACF>(P, ctrl, pos_next, pos, perm, nbr, nbr_cnt, vhalf, vel, fc, fctab, blockIdx.x, gridDim.x,
                            vorig, vpartial, csum, ccnt, norig);
}

// Block (x, y) of the grid (gx <= 256 = blockDim) takes the particles
// x*256 + tid, x*256 + tid + gx*256, ... and the origins of ages 4y .. 4y+3
// (age j = 0 is the newest): dot products in FP32 registers, warp and block
// sums in FP32 (at most 256 x a few terms) written as per-block partials.
// The partials of a step are added to C(lag) by the next VACF launch (blocks
// (x < origins, 0) fold the previous step's buffer while the rest of the grid
// streams) or by vacf_flush before the sums are read: no grid-wide wait.
// GB300's FP64 pipes are slow, so FP64 is one addition per origin and step.
__device__ __forceinline__ void vacf_body(const StepParams& P, Ctrl* __restrict__ ctrl,
                                          const float4* __restrict__ vel, float4* __restrict__ vorig,
                                          float* __restrict__ partial, double* __restrict__ csum,
                                          long long* __restrict__ ccnt, long long* __restrict__ norig, int blk,
                                          int nblk, int grp)
{
    // V_t was completed by the previous kernel; the pair kernel of this step
    // wrote the schedule of t and moved the last one to pv_*
    if (grp == 0 && ctrl->pv_nact > 0)
        vacf_fold(P, partial, csum, ccnt, ctrl->pv_buf, ctrl->pv_nact, ctrl->pv_lag0, nblk, blk, nblk);
    if (!ctrl->vacf_on) return;  // uniform over the grid
    const int n_act = ctrl->vacf_nact;
    const bool is_origin = ctrl->vacf_origin != 0;
    const int slot0 = ctrl->vacf_slot0;  // slot of age j: (slot0 - j) mod n_os
    if (blk == 0 && grp == 0 && threadIdx.x == 0) {
        ctrl->vacf_pending = 1;
        if (is_origin) *norig += 1;
    }
    const int q0 = grp * kVacfGroup;
    float acc[kVacfGroup];
#pragma unroll
    for (int q = 0; q < kVacfGroup; ++q) acc[q] = 0.f;
    if (q0 < n_act || (grp == 0 && is_origin)) {
        // two particles per round, all their loads issued before the sums (the
        // particles are still summed in the order i, i + stride, ...)
        const int stride = nblk * blockDim.x;
        int sl[kVacfGroup];
        bool use[kVacfGroup];
#pragma unroll
        for (int q = 0; q < kVacfGroup; ++q) {
            const int j = q0 + q;
            sl[q] = slot0 - j < 0 ? slot0 - j + P.n_os : slot0 - j;
            use[q] = j < n_act && !(j == 0 && is_origin);
        }
        for (int i = blk * blockDim.x + threadIdx.x; i < P.n; i += 2 * stride) {
            const int i2 = i + stride;
            const bool two = i2 < P.n;
            const float4 v = vel[i];
            const float4 v2 = two ? vel[i2] : v;
            float4 w[kVacfGroup], w2[kVacfGroup];
#pragma unroll
            for (int q = 0; q < kVacfGroup; ++q) {
                w[q] = use[q] ? __ldcs(vorig + (size_t)sl[q] * P.n + i) : v;
                w2[q] = use[q] && two ? __ldcs(vorig + (size_t)sl[q] * P.n + i2) : v2;
            }
#pragma unroll
            for (int q = 0; q < kVacfGroup; ++q)
                if (q0 + q < n_act) acc[q] = fmaf(v.x, w[q].x, fmaf(v.y, w[q].y, fmaf(v.z, w[q].z, acc[q])));
            if (two)
#pragma unroll
                for (int q = 0; q < kVacfGroup; ++q)
                    if (q0 + q < n_act)
                        acc[q] = fmaf(v2.x, w2[q].x, fmaf(v2.y, w2[q].y, fmaf(v2.z, w2[q].z, acc[q])));
            if (grp == 0 && is_origin) {
                vorig[(size_t)slot0 * P.n + i] = v;
                if (two) vorig[(size_t)slot0 * P.n + i2] = v2;
            }
        }
    }
    __shared__ float wsum[kThreads / 32][kVacfGroup];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kVacfGroup; ++q) {
        const float sq = warp_sum_f(acc[q]);
        if (lane == 0) wsum[warp][q] = sq;
    }
    __syncthreads();
    if (threadIdx.x < kVacfGroup && q0 + (int)threadIdx.x < n_act) {
        float sb = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sb += wsum[w][threadIdx.x];
        partial[((size_t)ctrl->vacf_buf * P.n_os + q0 + threadIdx.x) * nblk + blk] = sb;
    }
}

__global__ void __launch_bounds__(kThreads) vacf(const StepParams P, Ctrl* __restrict__ ctrl, const float4* __restrict__ vel,
         float4* __restrict__ vorig, float* __restrict__ partial, double* __restrict__ csum,
         long long* __restrict__ ccnt, long long* __restrict__ norig)
{
    vacf_body(P, ctrl, vel, vorig, partial, csum, ccnt, norig, blockIdx.x, gridDim.x, blockIdx.y);
}

// Adds the partials of the last VACF launch to the sums (before a read).
__global__ void __launch_bounds__(kThreads) vacf_flush(const StepParams P, Ctrl* __restrict__ ctrl,
                                                       const float* __restrict__ partial, double* __restrict__ csum,
                                                       long long* __restrict__ ccnt, int nblk)
{
    if (!ctrl->vacf_pending) return;
    vacf_fold(P, partial, csum, ccnt, ctrl->vacf_buf, ctrl->vacf_nact, ctrl->vacf_lag0, nblk, 0, 1);
    if (threadIdx.x == 0) ctrl->vacf_pending = 0;
}

// ---- distance-binned pair correlations C^a(R,t), C^c(R,t) (Sec. III A) -----
constexpr float kPcScale = 268435456.0f;       // 2^28: fixed point of the per-step sums
constexpr double kPcUnscale = 1.0 / 268435456.0;

__device__ __forceinline__ long long pc_fixed(float x) { return __float2ll_rn(x * kPcScale); }

// Adds per-step sums (buffer buf, origins q < nact) to the FP64 sums of their
// lags and clears them; entry k of the grid-wide range by one thread each.
__device__ __forceinline__ void pcorr_fold(const StepParams& P, long long* __restrict__ step_sums, int buf, int nact,
                                           int lag0, double* __restrict__ sa, double* __restrict__ sc,
                                           long long* __restrict__ sn, long long k0, long long kstep)
{
    long long* b = step_sums + (size_t)buf * P.n_os * P.pc_nbins * 3;
    for (long long k = k0; k < (long long)nact * P.pc_nbins; k += kstep) {
        const int q = (int)(k / P.pc_nbins), bin = (int)(k - (long long)q * P.pc_nbins);
        long long* e = b + 3 * k;
        const size_t at = (size_t)(lag0 + q * P.vacf_stride) * P.pc_nbins + bin;
        sa[at] += (double)e[0] * kPcUnscale;
        sc[at] += (double)e[1] * kPcUnscale;
        sn[at] += e[2];
        e[0] = e[1] = e[2] = 0;
    }
}

// At time t (after the VACF kernel stored this step's origin): for every
// unordered pair i < j of the neighbour lists with r_ij(t) < r_max and every
// active origin t0, with e = (R_i - R_j)/r and velocity components along e,
// a = v_i(t) v_i(t0) + v_j(t) v_j(t0) and c = v_i(t) v_j(t0) + v_j(t) v_i(t0)
// are added to the bin of r_ij(t) in 2^-28 fixed point (integer sums do not
// depend on the order of the atomics, so results are reproducible bit for
// bit).  The previous launch's sums are folded into the FP64 sums meanwhile.
// Each warp scans its 32 particles' lists and queues the pairs that count
// (about a quarter of the entries: j > i and r < r_max) in shared memory;
// the origin loop then runs over full warps of queued pairs.
struct PcPair {
    int i, j, bin;
    float ex, ey, ez, vit, vjt;
};
constexpr int kPcQueue = 64;  // queued pairs per warp (processed 32 at a time)

__device__ __forceinline__ void pcorr_pairs(const StepParams& P, const PcPair& e, const float4* __restrict__ vorig,
                                            long long* __restrict__ hs, long long* __restrict__ hn, int n_act,
                                            bool is_origin, int slot0, int nb)
{
    atomicAdd((unsigned long long*)(hn + e.bin), 1ull);  // the same pairs for every origin
    // lanes start at different origins, so that the shared-memory atomics of
    // one instruction seldom meet on the same (origin, bin)
    const int q0 = (threadIdx.x & 31) % n_act;
    for (int qq = 0; qq < n_act; ++qq) {
        const int q = qq + q0 < n_act ? qq + q0 : qq + q0 - n_act;
        float vi0 = e.vit, vj0 = e.vjt;
        if (!(q == 0 && is_origin)) {
            int sl = slot0 - q;
            sl = sl < 0 ? sl + P.n_os : sl;
            const float4 oi = __ldg(vorig + (size_t)sl * P.n + e.i), oj = __ldg(vorig + (size_t)sl * P.n + e.j);
            vi0 = oi.x * e.ex + oi.y * e.ey + oi.z * e.ez;
            vj0 = oj.x * e.ex + oj.y * e.ey + oj.z * e.ez;
        }
        long long* h = hs + 3 * (q * nb + e.bin);
        atomicAdd((unsigned long long*)h, (unsigned long long)pc_fixed(e.vit * vi0 + e.vjt * vj0));
        atomicAdd((unsigned long long*)(h + 1), (unsigned long long)pc_fixed(e.vit * vj0 + e.vjt * vi0));
    }
}

__global__ void __launch_bounds__(kThreads) pcorr(const StepParams P, Ctrl* __restrict__ ctrl,
                                                  const float4* __restrict__ pos, const float4* __restrict__ vel,
                                                  const float4* __restrict__ vorig, const int* __restrict__ nbr,
                                                  const int* __restrict__ nbr_cnt, long long* __restrict__ step_sums,
                                                  double* __restrict__ sa, double* __restrict__ sc,
                                                  long long* __restrict__ sn)
{
    if (ctrl->pc_pv_nact > 0)
        pcorr_fold(P, step_sums, ctrl->pc_pv_buf, ctrl->pc_pv_nact, ctrl->pc_pv_lag0, sa, sc, sn,
                   (long long)blockIdx.x * blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
    if (!ctrl->vacf_on) return;  // uniform over the grid
    const int n_act = ctrl->vacf_nact;
    const bool is_origin = ctrl->vacf_origin != 0;
    const int slot0 = ctrl->vacf_slot0;
    const int nb = P.pc_nbins;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->pc_pending = 1;
    extern __shared__ long long hs[];  // [n_act][nbins][3] (a, c, unused) then [nbins] pair counts
    long long* hn = hs + 3 * P.n_os * nb;
    __shared__ PcPair queue[kThreads / 32][kPcQueue];
    for (int k = threadIdx.x; k < n_act * nb * 3; k += blockDim.x) hs[k] = 0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) hn[k] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    PcPair* qw = queue[warp];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool own = i < P.n;
    float4 pi = make_float4(0.f, 0.f, 0.f, 0.f), vi = pi;
    int cnt = 0;
    if (own) {
        pi = pos[i];
        vi = vel[i];
        cnt = nbr_cnt[i];
    }
    int count = 0;  // queued pairs (uniform over the warp)
    for (int s = 0; __any_sync(0xffffffffu, s < cnt); ++s) {
        bool take = false;
        PcPair e;
        if (s < cnt) {
            const int j = __ldg(nbr + (size_t)s * P.n_pad + i);
            if (j > i) {
                const float4 pj = __ldg(pos + j);
                const float dx = min_image(pi.x, pj.x, P.box, P.half_box);
                const float dy = min_image(pi.y, pj.y, P.box, P.half_box);
                const float dz = min_image(pi.z, pj.z, P.box, P.half_box);
                const float r2 = dist2(dx, dy, dz);
                if (r2 < P.pc_rmax2) {
                    const float r = sqrtf(r2);
                    const float inv = 1.0f / r;
                    e.i = i;
                    e.j = j;
                    e.ex = dx * inv;
                    e.ey = dy * inv;
                    e.ez = dz * inv;
                    e.bin = min((int)(r * P.pc_inv_dr), nb - 1);
                    const float4 vj = __ldg(vel + j);
                    e.vit = vi.x * e.ex + vi.y * e.ey + vi.z * e.ez;
                    e.vjt = vj.x * e.ex + vj.y * e.ey + vj.z * e.ez;
                    take = true;
                }
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, take);
        if (take) qw[count + __popc(m & ((1u << lane) - 1u))] = e;
        count += __popc(m);  // <= 31 + 32 < kPcQueue
        __syncwarp();
        if (count >= 32) {  // a full warp of pairs; the rest moves to the front
            pcorr_pairs(P, qw[lane], vorig, hs, hn, n_act, is_origin, slot0, nb);
            __syncwarp();
            const PcPair rest = qw[32 + lane];
            __syncwarp();
            if (lane < count - 32) qw[lane] = rest;
            count -= 32;
            __syncwarp();
        }
    }
    if (lane < count) pcorr_pairs(P, qw[lane], vorig, hs, hn, n_act, is_origin, slot0, nb);
    __syncthreads();
    long long* out = step_sums + (size_t)ctrl->pc_buf * P.n_os * nb * 3;
    for (int k = threadIdx.x; k < n_act * nb * 3; k += blockDim.x) {
        const long long v = (k % 3 == 2) ? hn[(k / 3) % nb] : hs[k];
        if (v != 0) atomicAdd((unsigned long long*)(out + k), (unsigned long long)v);
    }
}

// Folds the last launch's sums (before they are read).
__global__ void __launch_bounds__(kThreads) pcorr_flush(const StepParams P, Ctrl* __restrict__ ctrl,
                                                        long long* __restrict__ step_sums, double* __restrict__ sa,
                                                        double* __restrict__ sc, long long* __restrict__ sn)
{
    if (!ctrl->pc_pending) return;
    pcorr_fold(P, step_sums, ctrl->pc_buf, ctrl->vacf_nact, ctrl->vacf_lag0, sa, sc, sn, threadIdx.x, blockDim.x);
    __syncthreads();
    if (threadIdx.x == 0) ctrl->pc_pending = 0;
}

// ---- explicit pair lists (checks of the traversals) -------------------------
__device__ __forceinline__ void emit_pair(int id, int jd, int* __restrict__ pairs, long long cap,
                                          unsigned long long* __restrict__ count)
{
    if (jd > id) {
        const unsigned long long slot = atomicAdd(count, 1ull);
        if ((long long)slot < cap) {
            pairs[2 * slot] = id;
            pairs[2 * slot + 1] = jd;
        }
    }
}

// The pairs the force kernels use: from the neighbour lists at R_n.
__global__ void list_pair_list(const StepParams P, const float4* __restrict__ pos, const int* __restrict__ perm,
                               const int* __restrict__ nbr, const int* __restrict__ nbr_cnt, int* __restrict__ pairs,
                               long long cap, unsigned long long* __restrict__ count)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.n) return;
    const int id = k;
    for_each_listed(pos[id], id, nbr, nbr_cnt[id], P.n_pad, pos, P,
                    [&](int jd, float, float, float, float) { emit_pair(id, jd, pairs, cap, count); });
}

// The pairs of a fresh cell traversal (no lists).
__global__ void pair_list(const StepParams P, const float4* __restrict__ pos_sorted, const int* __restrict__ cell_start,
                          int* __restrict__ pairs, long long cap, unsigned long long* __restrict__ count)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.n) return;
    const float4 pi = pos_sorted[k];
    const int id = __float_as_int(pi.w);
    for_each_in_stencil(pi, id, pos_sorted, cell_start, P, P.rc2, [&](int jd, float, float, float, float) {
        if (jd > id) {
            const unsigned long long slot = atomicAdd(count, 1ull);
            if ((long long)slot < cap) {
                pairs[2 * slot] = id;
                pairs[2 * slot + 1] = jd;
            }
        }
    });
}

// Sets the graph condition that guards the rebuild kernels.
__global__ void rebuild_decide(cudaGraphConditionalHandle h, const Ctrl* __restrict__ ctrl)
{
    cudaGraphSetConditional(h, ctrl->rebuild != 0 ? 1u : 0u);
}

// A bounded idle wait of one thread (lets the host run ahead of the device
// before a timed sequence of launches).
__global__ void delay_kernel(unsigned long long ns)
{
    unsigned long long t0, t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    do {
        __nanosleep(1000);
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    } while (t1 - t0 < ns);
}

// ---- batch kernels: tile -> member descriptor -> the bodies above ----------
template <bool FAST>
__global__ void __launch_bounds__(kPairThreads) b_pair(const SysDesc* __restrict__ D, const Tile* __restrict__ tiles)
{
    const Tile t = tiles[blockIdx.x];
    const SysDesc& d = D[t.m];
    const ParticleBuffers& B = d.B;
    pair_force_integrate_body<FAST>(d.P, B.ctrl, B.pos, B.perm, B.nbr, B.nbr_cnt, B.vel, B.fc, B.conv, B.frblock, B.ftab,
                              B.fptab, B.g0, B.ring, B.pos_next, B.vhalf, B.fd, B.disp, B.disp_build, t.b, d.nb_pair);
}

__global__ void b_cell_assign(const SysDesc* __restrict__ D, const Tile* __restrict__ tiles)
{
    const Tile t = tiles[blockIdx.x];
    const SysDesc& d = D[t.m];
    const ParticleBuffers& B = d.B;
    cell_assign_body(d.P, &B.ctrl->rebuild, B.pos_next, B.cell_head, B.cell_next, B.cell_count, t.b, d.nb_part);
}

__global__ void __launch_bounds__(kCellThreads) b_cell_scan(const SysDesc* __restrict__ D, const Tile* __restrict__ tiles)
{
    const Tile t = tiles[blockIdx.x];
    const SysDesc& d = D[t.m];
    const ParticleBuffers& B = d.B;
    cell_scan_body(&B.ctrl->rebuild, B.cell_count, B.ncells, B.chunk_sum, B.chunk_off, &B.ctrl->done_scan, t.b,
                   d.nb_cell);
}

__global__ void __launch_bounds__(kCellThreads) b_cell_fill(const SysDesc* __restrict__ D, const Tile* __restrict__ tiles)
{
    const Tile t = tiles[blockIdx.x];
    const SysDesc& d = D[t.m];
    const ParticleBuffers& B = d.B;
    cell_fill_body(d.P, &B.ctrl->rebuild, B.ncells, B.pos_next, B.cell_count, B.cell_head, B.cell_next, B.chunk_off,
                   B.cell_start, B.pos_sorted, t.b, d.nb_cell);
}

__global__ void __launch_bounds__(kThreads) b_nbr_build(const SysDesc* __restrict__ D, const Tile* __restrict__ tiles)
{
    const Tile t = tiles[blockIdx.x];
    const SysDesc& d = D[t.m];
    const ParticleBuffers& B = d.B;
    nbr_build_body(d.P, B.ctrl, B.pos_sorted, B.cell_start, B.nbr, B.nbr_cnt, B.perm, B.disp, B.disp_build, t.b,
                   d.nb_part);
}

__global__ void __launch_bounds__(kThreads) b_cforce(const SysDesc* __restrict__ D, const Tile* __restrict__ tiles)
{
    const Tile t = tiles[blockIdx.x];
    const SysDesc& d = D[t.m];
    const ParticleBuffers& B = d.B;
    cforce_body<true>(d.P, B.ctrl, B.pos_next, B.pos, B.perm, B.nbr, B.nbr_cnt, B.vhalf, B.vel, B.fc, B.fctab, t.b,
                      d.nb_cf);
}

__global__ void __launch_bounds__(kThreads) b_vacf(const SysDesc* __restrict__ D, const Tile* __restrict__ tiles)
{
    const Tile t = tiles[blockIdx.x];
    const SysDesc& d = D[t.m];
    const ParticleBuffers& B = d.B;
    vacf_body(d.P, B.ctrl, B.vel, B.vorig, B.vpartial, B.csum, B.ccnt, B.norig, t.b, d.nb_vacf, blockIdx.y);
}

// ---- pair-correlated noise (Sec. II C, Algorithm 1's matrix square root) --
// With one separable pair term the transformed correlation matrix of every
// frequency w is hat K_w = h_w 1 + g_w M, M the 3N x 3N pair matrix with
// off-diagonal blocks f(r_ij) e_ij e_ij^T (+ fp(r_ij) (1 - e_ij e_ij^T)) and,
// with a self-difference term of time factor c g, diagonal blocks
// c sum_k fs(r_ik) e_ik e_ik^T (+ perpendicular part); its square root is the same function of M for
// all w, so sqrt(hat K_w) ~ sum_k c_wk T_k(M / lambda) (Chebyshev), and after
// the inverse transform F_n = sum_k T_k(M / lambda) Z_k with Z_k moving
// averages of W (filters built on the host).  One stage of Clenshaw's
// recurrence:  out = Z_k + coef (M / lambda) b1 - b2  (coef 2; 1 for the last).
struct PnStage {
    const float* z;    // Z_k block [T][3][n_pad]
    const float* b1;   // b_{k+1}: a Z block (rows) or a vector [3][n_pad]
    const float* b2;   // b_{k+2} likewise, or null
    float* out;        // b_k vector, or (last stage) the Z_0 block rows
    int b1_rows, b2_rows, out_rows, last;
};

// (M b)_i for the vector b [3][n_pad]: the pair blocks f e e^T + fp (1 - e e^T)
// on the neighbours' entries and, with a self-difference term, the diagonal
// blocks pn_cs (fs e e^T + fsp (1 - e e^T)) on the own entry; rowsum: the
// Gershgorin row sum of the blocks' spectral norms.
__device__ __forceinline__ void pn_apply(const StepParams& P, const float4* __restrict__ pos,
                                         const int* __restrict__ nbr, const int* __restrict__ nbr_cnt,
                                         const float* __restrict__ ftab, const float* __restrict__ fptab, int id,
                                         const float* __restrict__ b, float& mx, float& my, float& mz, float& rowsum)
{
    const long long np = P.n_pad;
    const float4 pi = pos[id];
    const float bix = b[id], biy = b[np + id], biz = b[2 * np + id];  // own entry, for the self-difference blocks
    mx = my = mz = rowsum = 0.f;
    for_each_listed(pi, id, nbr, nbr_cnt[id], P.n_pad, pos, P, [&](int jd, float dx, float dy, float dz, float r2) {
        const float r = sqrtf(r2);
        const float inv_r = 1.0f / r;
        const float ex = dx * inv_r, ey = dy * inv_r, ez = dz * inv_r;
        const float xr = fmaxf(r, P.rc_min) * P.inv_dr;
        const float f = table_at(ftab, P.nr, xr);
        const float fp = P.perp ? table_at(fptab, P.nr, xr) : 0.f;  // block f e e^T + fp (1 - e e^T)
        const float bx = __ldg(b + jd), by = __ldg(b + np + jd), bz = __ldg(b + 2 * np + jd);
        const float eb = (f - fp) * dot3(ex, ey, ez, bx, by, bz);
        mx = fmaf(eb, ex, fmaf(fp, bx, mx));
        my = fmaf(eb, ey, fmaf(fp, by, my));
        mz = fmaf(eb, ez, fmaf(fp, bz, mz));
        rowsum += fmaxf(fabsf(f), fabsf(fp));  // the block's spectral norm
        if (P.Qs > 0) {
            const float fs = P.pn_cs * table_at(ftab + P.Q * P.nr, P.nr, xr);
            const float fsp = P.perp ? P.pn_cs * table_at(fptab + P.Q * P.nr, P.nr, xr) : 0.f;
            const float ei = (fs - fsp) * dot3(ex, ey, ez, bix, biy, biz);
            mx = fmaf(ei, ex, fmaf(fsp, bix, mx));
            my = fmaf(ei, ey, fmaf(fsp, biy, my));
            mz = fmaf(ei, ez, fmaf(fsp, biz, mz));
            rowsum += fmaxf(fabsf(fs), fabsf(fsp));
        }
    });
}

__device__ __forceinline__ void pn_stage_body(const StepParams& P, Ctrl* __restrict__ ctrl, const float4* __restrict__ pos,
                                              const int* __restrict__ nbr, const int* __restrict__ nbr_cnt,
                                              const float* __restrict__ ftab, const float* __restrict__ fptab,
                                              const PnStage& S, int blk)
{
    const int id = blk * blockDim.x + threadIdx.x;
    if (id >= P.n) return;
    const long long np = P.n_pad;
    const long long row = ctrl->step - ctrl->noise_n0;
    if (row < 0 || row >= P.T) {
        if (id == 0) atomicOr(&ctrl->err, kErrNoise);
        return;
    }
    const size_t roff = (size_t)row * 3 * np;
    const float* b1 = S.b1 + (S.b1_rows ? roff : 0);
    const float* b2 = S.b2 ? S.b2 + (S.b2_rows ? roff : 0) : nullptr;
    float* out = S.out + (S.out_rows ? roff : 0);
    const float* z = S.z + roff;
    float mx, my, mz, rowsum;
    pn_apply(P, pos, nbr, nbr_cnt, ftab, fptab, id, b1, mx, my, mz, rowsum);
    if (P.pn_cen != 0.f) {  // the interval [cen - rho, cen + rho]: (M - cen) b1
        mx = fmaf(-P.pn_cen, b1[id], mx);
        my = fmaf(-P.pn_cen, b1[np + id], my);
        mz = fmaf(-P.pn_cen, b1[2 * np + id], mz);
    }
    const float c = (S.last ? 1.0f : 2.0f) * P.pn_inv_lambda;
    const float ox = fmaf(c, mx, z[id]) - (b2 ? b2[id] : 0.f);
    const float oy = fmaf(c, my, z[np + id]) - (b2 ? b2[np + id] : 0.f);
    const float oz = fmaf(c, mz, z[2 * np + id]) - (b2 ? b2[2 * np + id] : 0.f);
    out[id] = ox;
    out[np + id] = oy;
    out[2 * np + id] = oz;
    // the symmetric bound is checked every step by Gershgorin; an interval
    // from Ritz values by the Lanczos run at each noise block
    if (S.last && !P.pn_iv && rowsum > P.pn_lambda) atomicOr(&ctrl->err, kErrPnBound);
}

// Clenshaw stage k of a degree-K evaluation: b_K = Z_K (read in place), b_k
// for K > k >= 1 in bvec[k % 3], the last stage writes F over the Z_0 row.
__host__ __device__ __forceinline__ PnStage pn_stage_args(const StepParams& P, const float* frblock, const float* zblk,
                                                 float* bvec, int K, int k)
{
    const size_t blk = (size_t)P.T * 3 * P.n_pad, vec = (size_t)3 * P.n_pad;
    auto zk = [&](int q) -> const float* { return q == 0 ? frblock : zblk + (size_t)(q - 1) * blk; };
    PnStage S{};
    S.z = zk(k);
    S.last = k == 0;
    if (k + 1 == K) { S.b1 = zk(K); S.b1_rows = 1; }
    else { S.b1 = bvec + (size_t)((k + 1) % 3) * vec; }
    if (k + 2 == K) { S.b2 = zk(K); S.b2_rows = 1; }
    else if (k + 2 < K) { S.b2 = bvec + (size_t)((k + 2) % 3) * vec; }
    if (k == 0) { S.out = const_cast<float*>(frblock); S.out_rows = 1; }
    else { S.out = bvec + (size_t)(k % 3) * vec; }
    return S;
}

__global__ void __launch_bounds__(kThreads)
    pn_stage(const StepParams P, Ctrl* __restrict__ ctrl, const float4* __restrict__ pos, const int* __restrict__ nbr,
             const int* __restrict__ nbr_cnt, const float* __restrict__ ftab, const float* __restrict__ fptab,
             const PnStage S)
{
    pn_stage_body(P, ctrl, pos, nbr, nbr_cnt, ftab, fptab, S, blockIdx.x);
}

// Stage k of every member whose degree exceeds k, over the particle tiles.
__global__ void __launch_bounds__(kThreads) b_pn_stage(const SysDesc* __restrict__ D, const Tile* __restrict__ tiles, int k)
{
    const Tile t = tiles[blockIdx.x];
    const SysDesc& d = D[t.m];
    const int K = d.P.pn_deg;
    if (k >= K) return;
    const PnStage S = pn_stage_args(d.P, d.B.frblock, d.zblk, d.bvec, K, k);
    pn_stage_body(d.P, d.B.ctrl, d.B.pos, d.B.nbr, d.B.nbr_cnt, d.B.ftab, d.B.fptab, S, t.b);
}

__global__ void __launch_bounds__(kThreads)
    pn_rowsum(const StepParams P, const float4* __restrict__ pos, const int* __restrict__ nbr,
              const int* __restrict__ nbr_cnt, const float* __restrict__ ftab, const float* __restrict__ fptab,
              unsigned* __restrict__ out)
{
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= P.n) return;
    float rowsum = 0.f;
    for_each_listed(pos[id], id, nbr, nbr_cnt[id], P.n_pad, pos, P, [&](int, float, float, float, float r2) {
        const float xr = fmaxf(sqrtf(r2), P.rc_min) * P.inv_dr;
        rowsum += fmaxf(fabsf(table_at(ftab, P.nr, xr)), P.perp ? fabsf(table_at(fptab, P.nr, xr)) : 0.f);
        if (P.Qs > 0)
            rowsum += fabsf(P.pn_cs) * fmaxf(fabsf(table_at(ftab + P.Q * P.nr, P.nr, xr)),
                                             P.perp ? fabsf(table_at(fptab + P.Q * P.nr, P.nr, xr)) : 0.f);
    });
    atomicMax(out, __float_as_uint(rowsum));  // non-negative floats order as their bits
}

// ---- extreme eigenvalues of the pair matrix by a Lanczos run ---------------
// kPnLanczosSteps steps from a fixed +-1 start vector, vectors [3][n_pad] in
// FP32 kept unnormalised (r_k, v_k = r_k / beta_k), every dot product summed
// in FP64 as per-block partials that each block of the next kernel folds in
// the same fixed order, so all blocks (and every run) see the same bits.  The
// extreme eigenvalues of the tridiagonal matrix (the Ritz values) are found
// by Sturm-sequence bisection in one thread.  ab: alpha_0 .. alpha_{K-1},
// then beta_0 .. beta_K.
__device__ __forceinline__ double block_sum_d(double v, double* red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ double fold_partials(const double* __restrict__ part, int nblk, double* red)
{
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[b];
    return block_sum_d(s, red);
}

__global__ void __launch_bounds__(kThreads) lz_start(const StepParams P, float* __restrict__ r0, double* __restrict__ part)
{
    __shared__ double red[kThreads];
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    const long long np = P.n_pad;
    double s = 0.0;
    if (id < P.n)
        for (int c = 0; c < 3; ++c) {
            const uint32_t h = (uint32_t)(c * np + id) * 0x9E3779B1u;  // Fibonacci hash: a fixed sign pattern
            r0[c * np + id] = (h >> 31) ? -1.f : 1.f;
            s += 1.0;
        }
    else if (id < np)
        for (int c = 0; c < 3; ++c) r0[c * np + id] = 0.f;
    const double t = block_sum_d(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// y = M v_k, v_k = r_k / beta_k (beta_k from the partials of |r_k|^2); partial
// sums of v_k . y.
__global__ void __launch_bounds__(kThreads)
    lz_matvec(const StepParams P, const float4* __restrict__ pos, const int* __restrict__ nbr,
              const int* __restrict__ nbr_cnt, const float* __restrict__ ftab, const float* __restrict__ fptab,
              const float* __restrict__ rk, const double* __restrict__ part_in, int nblk, float* __restrict__ y,
              double* __restrict__ part_out, double* __restrict__ ab, int k)
{
    __shared__ double red[kThreads];
    const double beta = sqrt(fold_partials(part_in, nblk, red));
    if (blockIdx.x == 0 && threadIdx.x == 0) ab[kPnLanczosSteps + k] = beta;
    const float invb = beta > 0.0 ? (float)(1.0 / beta) : 0.f;
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    const long long np = P.n_pad;
    double a = 0.0;
    if (id < P.n) {
        float mx, my, mz, rowsum;
        pn_apply(P, pos, nbr, nbr_cnt, ftab, fptab, id, rk, mx, my, mz, rowsum);
        const float yx = invb * mx, yy = invb * my, yz = invb * mz;
        y[id] = yx;
        y[np + id] = yy;
        y[2 * np + id] = yz;
        a = (double)(invb * rk[id]) * yx + (double)(invb * rk[np + id]) * yy + (double)(invb * rk[2 * np + id]) * yz;
    } else if (id < np) {
        y[id] = y[np + id] = y[2 * np + id] = 0.f;
    }
    const double t = block_sum_d(a, red);
    if (threadIdx.x == 0) part_out[blockIdx.x] = t;
}

// r_{k+1} = y - alpha_k v_k - beta_k v_{k-1}; partial sums of |r_{k+1}|^2.
__global__ void __launch_bounds__(kThreads)
    lz_update(const StepParams P, const float* __restrict__ y, const float* __restrict__ rk,
              const float* __restrict__ rkm1, const double* __restrict__ part_in, int nblk, double* __restrict__ ab,
              int k, float* __restrict__ rkp1, double* __restrict__ part_out)
{
    __shared__ double red[kThreads];
    const double alpha = fold_partials(part_in, nblk, red);
    if (blockIdx.x == 0 && threadIdx.x == 0) ab[k] = alpha;
    const double bk = ab[kPnLanczosSteps + k], bkm1 = k > 0 ? ab[kPnLanczosSteps + k - 1] : 0.0;
    const float ib = bk > 0.0 ? (float)(1.0 / bk) : 0.f, ibm = (k > 0 && bkm1 > 0.0) ? (float)(1.0 / bkm1) : 0.f;
    const float a = (float)alpha, b = (float)bk;
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    const long long np = P.n_pad;
    double s = 0.0;
    if (id < np)
        for (int c = 0; c < 3; ++c) {
            const size_t e = (size_t)c * np + id;
            float r = fmaf(-a, ib * rk[e], y[e]);
            if (k > 0) r = fmaf(-b, ibm * rkm1[e], r);
            rkp1[e] = r;
            s += (double)r * r;
        }
    const double t = block_sum_d(s, red);
    if (threadIdx.x == 0) part_out[blockIdx.x] = t;
}

// Number of eigenvalues below x of the j x j tridiagonal matrix (Sturm).
__device__ int sturm_count(const double* al, const double* be, int j, double x)
{
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < j; ++i) {
        const double off = i > 0 ? be[i] * be[i] : 0.0;
        d = al[i] - x - (i > 0 ? off / d : 0.0);
        if (d == 0.0) d = -1e-300;  // x on an eigenvalue of a leading block: count it
        cnt += d < 0.0;
    }
    return cnt;
}

// Ritz extremes into out[0] (smallest), out[1] (largest); the Krylov space
// ends at the first beta_j below 1e-6 of the spectral scale so far.  check:
// latch kErrPnBound when they leave [lo, hi].
__global__ void lz_final(const double* __restrict__ ab, double lo, double hi, int check, Ctrl* __restrict__ ctrl,
                         double* __restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double* al = ab;
    const double* be = ab + kPnLanczosSteps;  // be[i] couples rows i - 1 and i (i >= 1)
    int j = 1;
    double scale = fabs(al[0]);
    while (j < kPnLanczosSteps && be[j] > 1e-6 * scale) {
        scale = fmax(scale, fabs(al[j]) + be[j]);
        ++j;
    }
    double glo = al[0], ghi = al[0];  // Gershgorin interval of the tridiagonal matrix
    for (int i = 0; i < j; ++i) {
        const double rad = (i > 0 ? fabs(be[i]) : 0.0) + (i + 1 < j ? fabs(be[i + 1]) : 0.0);
        glo = fmin(glo, al[i] - rad);
        ghi = fmax(ghi, al[i] + rad);
    }
    double a = glo, b = ghi;  // smallest: count(x) >= 1 first at it
    for (int it = 0; it < 200 && b - a > 1e-15 * fmax(fabs(a), fabs(b)); ++it) {
        const double m = 0.5 * (a + b);
        if (sturm_count(al, be, j, m) >= 1) b = m; else a = m;
    }
    const double tmin = 0.5 * (a + b);
    a = glo;
    b = ghi;  // largest: count(x) >= j first at it
    for (int it = 0; it < 200 && b - a > 1e-15 * fmax(fabs(a), fabs(b)); ++it) {
        const double m = 0.5 * (a + b);
        if (sturm_count(al, be, j, m) >= j) b = m; else a = m;
    }
    const double tmax = 0.5 * (a + b);
    out[0] = tmin;
    out[1] = tmax;
    out[2] = (double)j;
    if (check && (tmin < lo || tmax > hi)) atomicOr(&ctrl->err, kErrPnBound);
}

}  // namespace

cudaError_t launch_batch_particles(const BatchPlan& bp, cudaStream_t st)
{
    static_assert(kBatchPartBlock == kThreads, "Clenshaw stages use the particle tiles");
    if (bp.n_part)  // pair-correlated noise of the step, stage by stage over all members
        for (int k = bp.pn_kmax - 1; k >= 0; --k) b_pn_stage<<<bp.n_part, kThreads, 0, st>>>(bp.desc, bp.part, k);
    if (bp.n_pair) {
        if (bp.pair_fast) b_pair<true><<<bp.n_pair, kPairThreads, 0, st>>>(bp.desc, bp.pair);
        else b_pair<false><<<bp.n_pair, kPairThreads, 0, st>>>(bp.desc, bp.pair);
    }
    if (bp.n_part) b_cell_assign<<<bp.n_part, kThreads, 0, st>>>(bp.desc, bp.part);
    if (bp.n_cell) b_cell_scan<<<bp.n_cell, kCellThreads, 0, st>>>(bp.desc, bp.cell);
    if (bp.n_cell) b_cell_fill<<<bp.n_cell, kCellThreads, 0, st>>>(bp.desc, bp.cell);
    if (bp.n_part) b_nbr_build<<<bp.n_part, kThreads, 0, st>>>(bp.desc, bp.part);
    if (bp.n_cf) b_cforce<<<bp.n_cf, kBatchCforceBlock, 0, st>>>(bp.desc, bp.cf);
    if (bp.n_vacf) {
        const dim3 g((unsigned)bp.n_vacf, (unsigned)((bp.vacf_no + kVacfGroup - 1) / kVacfGroup));
        b_vacf<<<g, kThreads, 0, st>>>(bp.desc, bp.vacf);
    }
    return cudaGetLastError();
}

cudaError_t launch_rebuild_decide(cudaGraphConditionalHandle h, const Ctrl* ctrl, cudaStream_t st)
{
    rebuild_decide<<<1, 1, 0, st>>>(h, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_delay(unsigned long long ns, cudaStream_t st)
{
    delay_kernel<<<1, 1, 0, st>>>(ns < 10000000ull ? ns : 10000000ull);
    return cudaGetLastError();
}

cudaError_t launch_pair_force_integrate(const StepParams& P, const ParticleBuffers& B, cudaStream_t st)
{
    const unsigned grid = (unsigned)((P.n + kPairThreads - 1) / kPairThreads);
    const bool fast = P.Q == 1 && P.Qs == 0 && !P.perp;
    auto k = fast ? pair_force_integrate<true> : pair_force_integrate<false>;
    const unsigned pgrid = fast ? (unsigned)(((long long)P.n * kPairLanes + kPairThreads - 1) / kPairThreads) : grid;
    k<<<pgrid, kPairThreads, 0, st>>>(P, B.ctrl, B.pos, B.perm, B.nbr, B.nbr_cnt, B.vel, B.fc,
                                                        B.conv, B.frblock, B.ftab, B.fptab, B.g0, B.ring,
                                                        B.pos_next,
                                                        B.vhalf, B.fd, B.disp, B.disp_build);
    return cudaGetLastError();
}

cudaError_t launch_cell_build(const StepParams& P, const ParticleBuffers& B, const float4* src, const int* gate,
                              cudaStream_t st)
{
    cell_assign<<<(P.n + kThreads - 1) / kThreads, kThreads, 0, st>>>(P, gate, src, B.cell_head, B.cell_next,
                                                                       B.cell_count);
    const unsigned chunks = (unsigned)((B.ncells + kCellThreads - 1) / kCellThreads);
    cell_scan<<<chunks, kCellThreads, 0, st>>>(gate, B.cell_count, B.ncells, B.chunk_sum, B.chunk_off,
                                               &B.ctrl->done_scan);
    cell_fill<<<chunks, kCellThreads, 0, st>>>(P, gate, B.ncells, src, B.cell_count, B.cell_head, B.cell_next,
                                               B.chunk_off, B.cell_start, B.pos_sorted);
    return cudaGetLastError();
}

cudaError_t launch_rebuild(const StepParams& P, const ParticleBuffers& B, cudaStream_t st)
{
    cudaError_t e = launch_cell_build(P, B, B.pos_next, &B.ctrl->rebuild, st);
    if (e != cudaSuccess) return e;
    nbr_build<<<(P.n + kThreads - 1) / kThreads, kThreads, 0, st>>>(P, B.ctrl, B.pos_sorted, B.cell_start, B.nbr,
                                                                     B.nbr_cnt, B.perm, B.disp, B.disp_build);
    return cudaGetLastError();
}

cudaError_t launch_cforce(const StepParams& P, const ParticleBuffers& B, int mode, cudaStream_t st)
{
    const unsigned grid = (unsigned)(((long long)P.n * kCforceLanes + kThreads - 1) / kThreads);
    const bool vac = mode && P.vacf_len > 0;
    if (vac && (P.n_os > kVacfMaxOrigins || (int)grid != B.vacf_gx)) return cudaErrorInvalidValue;
    auto k = mode ? (vac ? cforce<true, true> : cforce<true, false>) : cforce<false, false>;
    k<<<grid, kThreads, 0, st>>>(P, B.ctrl, B.pos_next, B.pos, B.perm, B.nbr, B.nbr_cnt, B.vhalf, B.vel, B.fc,
                                 B.fctab, B.vorig, B.vpartial, B.csum, B.ccnt, B.norig);
    return cudaGetLastError();
}

cudaError_t launch_vacf(const StepParams& P, const ParticleBuffers& B, cudaStream_t st)
{
    if (P.vacf_len <= 0) return cudaSuccess;
    if (P.n_os > kVacfMaxOrigins) return cudaErrorInvalidValue;
    const dim3 g((unsigned)B.vacf_gx, (unsigned)((P.n_os + kVacfGroup - 1) / kVacfGroup));
    vacf<<<g, kThreads, 0, st>>>(P, B.ctrl, B.vel, B.vorig, B.vpartial, B.csum, B.ccnt, B.norig);
    return cudaGetLastError();
}

cudaError_t launch_vacf_flush(const StepParams& P, const ParticleBuffers& B, cudaStream_t st)
{
    if (P.vacf_len <= 0) return cudaSuccess;
    vacf_flush<<<1, kThreads, 0, st>>>(P, B.ctrl, B.vpartial, B.csum, B.ccnt, B.vacf_gx);
    return cudaGetLastError();
}

cudaError_t launch_pcorr(const StepParams& P, const ParticleBuffers& B, cudaStream_t st)
{
    if (P.pc_nbins <= 0 || P.vacf_len <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::max(1, (P.n + kThreads - 1) / kThreads);
    const size_t smem = sizeof(long long) * (3 * (size_t)P.n_os * P.pc_nbins + P.pc_nbins);
    // beside the static pair queues (16 KB)
    if (smem + sizeof(PcPair) * (kThreads / 32) * kPcQueue > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(pcorr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    pcorr<<<grid, kThreads, smem, st>>>(P, B.ctrl, B.pos, B.vel, B.vorig, B.nbr, B.nbr_cnt, B.pc_step, B.pc_sa,
                                        B.pc_sc, B.pc_n);
    return cudaGetLastError();
}

cudaError_t launch_pcorr_flush(const StepParams& P, const ParticleBuffers& B, cudaStream_t st)
{
    if (P.pc_nbins <= 0 || P.vacf_len <= 0) return cudaSuccess;
    pcorr_flush<<<1, kThreads, 0, st>>>(P, B.ctrl, B.pc_step, B.pc_sa, B.pc_sc, B.pc_n);
    return cudaGetLastError();
}

cudaError_t launch_pair_noise(const StepParams& P, const ParticleBuffers& B, const float* zblk, float* bvec,
                              cudaStream_t st)
{
    const int K = P.pn_deg;
    if (K <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((P.n + kThreads - 1) / kThreads);
    for (int k = K - 1; k >= 0; --k) {
        pn_stage<<<grid, kThreads, 0, st>>>(P, B.ctrl, B.pos, B.nbr, B.nbr_cnt, B.ftab, B.fptab,
                                            pn_stage_args(P, B.frblock, zblk, bvec, K, k));
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int pn_spectrum_blocks(const StepParams& P) { return (int)((P.n_pad + kThreads - 1) / kThreads); }

cudaError_t launch_pn_spectrum(const StepParams& P, const ParticleBuffers& B, float* vec, double* part, double* ab,
                               double lo, double hi, int check, double* out, cudaStream_t st)
{
    const int nblk = pn_spectrum_blocks(P);
    const size_t vs = (size_t)3 * P.n_pad;
    float* y = vec + 3 * vs;  // r_k rotate through vec[0..2]
    double* pa = part;         // |r_k|^2 partials
    double* pb = part + nblk;  // v_k . y partials
    lz_start<<<nblk, kThreads, 0, st>>>(P, vec, pa);
    for (int k = 0; k < kPnLanczosSteps; ++k) {
        float* rk = vec + (size_t)(k % 3) * vs;
        const float* rkm1 = vec + (size_t)((k + 2) % 3) * vs;
        float* rkp1 = vec + (size_t)((k + 1) % 3) * vs;
        lz_matvec<<<nblk, kThreads, 0, st>>>(P, B.pos, B.nbr, B.nbr_cnt, B.ftab, B.fptab, rk, pa, nblk, y, pb, ab, k);
        lz_update<<<nblk, kThreads, 0, st>>>(P, y, rk, rkm1, pb, nblk, ab, k, rkp1, pa);
    }
    lz_final<<<1, 32, 0, st>>>(ab, lo, hi, check, B.ctrl, out);
    return cudaGetLastError();
}

cudaError_t launch_pn_rowsum(const StepParams& P, const ParticleBuffers& B, unsigned* out, cudaStream_t st)
{
    pn_rowsum<<<(P.n + kThreads - 1) / kThreads, kThreads, 0, st>>>(P, B.pos, B.nbr, B.nbr_cnt, B.ftab, B.fptab,
                                                                      out);
    return cudaGetLastError();
}

cudaError_t launch_pair_list(const StepParams& P, const ParticleBuffers& B, int* pairs, long long cap,
                             unsigned long long* count, cudaStream_t st)
{
    pair_list<<<(P.n + kThreads - 1) / kThreads, kThreads, 0, st>>>(P, B.pos_sorted, B.cell_start, pairs, cap, count);
    return cudaGetLastError();
}

cudaError_t launch_list_pair_list(const StepParams& P, const ParticleBuffers& B, int* pairs, long long cap,
                                  unsigned long long* count, cudaStream_t st)
{
    list_pair_list<<<(P.n + kThreads - 1) / kThreads, kThreads, 0, st>>>(P, B.pos, B.perm, B.nbr, B.nbr_cnt, pairs,
                                                                         cap, count);
    return cudaGetLastError();
}

}  // namespace gld
