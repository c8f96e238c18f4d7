// api.cu -- the C ABI of include/gld.h: context life cycle, device memory,
// step orchestration and CUDA-graph replay.
//
// One step n -> n+1 is five kernels on the context's stream:
//   hist_conv -> pair_force_integrate -> cell build (3 small kernels)
//   -> cforce (F^C_{n+1}, V_{n+1}, n += 1, and the VACF terms when enabled)
// and every T steps one noise block (wgen + fir) produces F^R for the next T
// steps.  The step counter lives on the device, so a graph holding one noise
// block and T steps is captured once and replayed for as long as the kernels
// stay the same.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "ctx.h"

using namespace gld;

namespace {

// Device-side and CUDA failures are latched (the context's device state can
// no longer be trusted); argument and ordering errors only set the message.
gld_status fail(gld_ctx* c, gld_status s, const std::string& m)
{
    if (c) {
        c->msg = m;
        const bool sticky = s == GLD_E_CUDA || s == GLD_E_NONFINITE || s == GLD_E_TIMEOUT;
        if (sticky && c->latched == GLD_OK) c->latched = s;
    }
    return s;
}

gld_status cuda_check(gld_ctx* c, cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return GLD_OK;
    return fail(c, GLD_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define GLD_TRY(expr)                          \
    do {                                       \
        gld_status s_ = (expr);                \
        if (s_ != GLD_OK) return s_;           \
    } while (0)

#define GLD_CUDA(c, expr) GLD_TRY(cuda_check((c), (expr), #expr))

void* dalloc(gld_ctx* c, size_t bytes)
{
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (c->prm.alloc) p = c->prm.alloc(bytes, c->prm.stream, c->prm.alloc_user);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (p) {
        c->allocs.push_back(p);
        c->alloc_sizes.push_back(bytes);
        c->bytes += bytes;
        cudaMemsetAsync(p, 0, bytes, c->st);
    }
    return p;
}

void dfree(gld_ctx* c, void* p)
{
    if (!p) return;
    for (size_t k = 0; k < c->allocs.size(); ++k)
        if (c->allocs[k] == p) {
            c->bytes -= c->alloc_sizes[k];
            c->allocs.erase(c->allocs.begin() + (long)k);
            c->alloc_sizes.erase(c->alloc_sizes.begin() + (long)k);
            break;
        }
    if (c->prm.free) c->prm.free(p, c->prm.stream, c->prm.alloc_user);
    else cudaFree(p);
}

template <class Tp>
Tp* alloc_n(gld_ctx* c, size_t count, bool& ok)
{
    Tp* p = (Tp*)dalloc(c, sizeof(Tp) * count);
    if (!p) ok = false;
    return p;
}

double wrap_host(double x, double L)
{
    x = std::fmod(x, L);
    if (x < 0) x += L;
    if (x >= L) x = 0.0;
    return x;
}

// Host <-> device transfers of [n][3] vectors (caller's order) stored as
// float4 in internal order.
gld_status upload_vec(gld_ctx* c, float4* dst, const double* src, bool wrap)
{
    const int n = c->P.n;
    std::vector<float4> h((size_t)c->P.n_pad, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int i = 0; i < n; ++i) {
        const size_t e = (size_t)c->int2ext[i];
        double x = src[3 * e], y = src[3 * e + 1], z = src[3 * e + 2];
        if (wrap) {
            x = wrap_host(x, c->prm.box);
            y = wrap_host(y, c->prm.box);
            z = wrap_host(z, c->prm.box);
        }
        float fx = (float)x, fy = (float)y, fz = (float)z;
        if (wrap) {  // rounding to float may land on L
            fx = fx >= c->P.box ? 0.f : fx;
            fy = fy >= c->P.box ? 0.f : fy;
            fz = fz >= c->P.box ? 0.f : fz;
        }
        h[i] = make_float4(fx, fy, fz, 0.f);
    }
    GLD_CUDA(c, cudaMemcpyAsync(dst, h.data(), sizeof(float4) * n, cudaMemcpyHostToDevice, c->st));
    GLD_CUDA(c, cudaStreamSynchronize(c->st));
    return GLD_OK;
}

gld_status download_vec(gld_ctx* c, const float4* src, double* dst)
{
    const int n = c->P.n;
    std::vector<float4> h((size_t)n);
    GLD_CUDA(c, cudaMemcpyAsync(h.data(), src, sizeof(float4) * n, cudaMemcpyDeviceToHost, c->st));
    GLD_CUDA(c, cudaStreamSynchronize(c->st));
    ctx_to_caller(c, h.data(), dst);
    return GLD_OK;
}

// [rows][3][n_pad] float planes <-> [rows][n][3] doubles.
gld_status download_planes(gld_ctx* c, const float* src, int rows, double* dst)
{
    const int n = c->P.n;
    const size_t np = c->P.n_pad;
    std::vector<float> h(rows * 3 * np);
    GLD_CUDA(c, cudaMemcpyAsync(h.data(), src, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, c->st));
    GLD_CUDA(c, cudaStreamSynchronize(c->st));
    for (int r = 0; r < rows; ++r)
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < 3; ++k) dst[((size_t)r * n + c->int2ext[i]) * 3 + k] = h[(r * 3 + k) * np + i];
    return GLD_OK;
}

gld_status sync_and_check(gld_ctx* c)
{
    GLD_CUDA(c, cudaStreamSynchronize(c->st));
    unsigned err = 0;
    GLD_CUDA(c, cudaMemcpy(&err, &c->B.ctrl->err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    return ctx_check_err(c, err);
}

void invalidate_graph(gld_ctx* c)
{
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->graph_failed = false;
    c->conv_valid_step = -1;
}

gld_status invalidate_noise(gld_ctx* c)
{
    c->noise_valid = false;
    c->conv_valid_step = -1;
    long long w[2] = {0, 1};  // {w_hi, w_lo}: w_hi < w_lo marks the W ring empty
    GLD_CUDA(c, cudaMemcpyAsync(&c->B.ctrl->w_hi, w, sizeof(w), cudaMemcpyHostToDevice, c->st));
    return GLD_OK;
}

// The white-noise ring holds the FP16 split form while the context steps
// alone with the tensor-core filter, FP32 inside a batch (the batched filter
// runs on the FP32 pipes).  A change of form clears the ring (stale values of
// the other form need not be finite read in this one, and the tensor-core
// filter multiplies the rows around its window by zero taps) and marks it
// empty, so the next block generates its whole window again; the values are
// counter-based, so nothing else changes.  Issued on stream s.
gld_status ring_form(gld_ctx* c, bool alone, cudaStream_t s)
{
    const int want = alone && c->have_wmap ? 1 : 0;
    if (c->P.wsplit == want) return GLD_OK;
    c->P.wsplit = want;
    invalidate_graph(c);
    c->noise_valid = false;
    c->conv_valid_step = -1;
    GLD_CUDA(c, cudaMemsetAsync(c->W, 0, sizeof(float) * (size_t)c->P.lw * 3 * c->P.n_pad, s));
    long long w[2] = {0, 1};  // {w_hi, w_lo}: empty
    GLD_CUDA(c, cudaMemcpyAsync(&c->B.ctrl->w_hi, w, sizeof(w), cudaMemcpyHostToDevice, s));
    return GLD_OK;
}

// Positions were replaced (pos and pos_next hold them): new lists and F^C.
gld_status rebuild_cells_and_fc(gld_ctx* c)
{
    const int one = 1;
    GLD_CUDA(c, cudaMemcpyAsync(&c->B.ctrl->rebuild, &one, sizeof(int), cudaMemcpyHostToDevice, c->st));
    GLD_CUDA(c, launch_rebuild(c->P, c->B, c->st));
    GLD_CUDA(c, launch_cforce(c->P, c->B, 0, c->st));
    return GLD_OK;
}

cudaError_t launch_noise(gld_ctx* c, cudaStream_t s)
{
    const StepParams& P = c->P;
    const CUtensorMap* wmap = c->have_wmap ? &c->wmap : nullptr;
    if (P.pn_deg <= 0)
        return launch_noise_block(P, c->B.ctrl, c->W, c->Acp, c->la, c->B.frblock, c->prm.seed, c->d_int2ext, wmap,
                                  c->num_sms, s);
    // pair-correlated noise: Z_0 .. Z_deg from one white-noise window
    cudaError_t e = launch_noise_block(P, c->B.ctrl, c->W, c->d_pntaps, c->la, c->B.frblock, c->prm.seed,
                                       c->d_int2ext, wmap, c->num_sms, s);
    for (int k = 1; k <= P.pn_deg && e == cudaSuccess; ++k)
        e = launch_noise_filter(P, c->B.ctrl, c->W, c->d_pntaps + (size_t)k * c->la,
                                c->d_zblk + (size_t)(k - 1) * P.T * 3 * P.n_pad, wmap, c->num_sms, s);
    // an interval from Ritz values: checked again at R_n of every block
    if (P.pn_iv && e == cudaSuccess)
        e = launch_pn_spectrum(P, c->B, c->d_lzv, c->d_lzpart, c->d_lzab, c->pn_lo, c->pn_hi, 1,
                               c->d_lzab + 2 * kPnLanczosSteps + 1, s);
    return e;
}

// The memory sums of step n: the history convolution, or its recursive form
// when memory modes are set.
cudaError_t launch_memory(gld_ctx* c, cudaStream_t s)
{
    if (c->P.nmodes > 0)
        return launch_modes_step(c->P, c->B.ctrl, c->B.ring, c->d_mcoef, c->d_mw, c->d_Y, c->B.conv, s);
    return launch_hist_conv(c->B.ring, c->P.hist_bf16, c->P.n_pad, c->P.m_max, c->B.ctrl, 0, c->coef, c->P.nacc,
                            c->B.conv, c->prm.kahan, s);
}

// Rebuilds the auxiliary sums of the recursive form from the ring when the
// history or the step index was replaced.
gld_status refresh_modes(gld_ctx* c)
{
    if (c->P.nmodes > 0 && c->modes_dirty) {
        GLD_CUDA(c, launch_modes_init(c->P, c->B.ctrl, c->B.ring, c->d_mz, c->d_Y, c->st));
        c->modes_dirty = false;
    }
    return GLD_OK;
}

cudaError_t launch_one_step(gld_ctx* c, cudaStream_t s)
{
    cudaError_t e = launch_memory(c, s);
    if (e != cudaSuccess) return e;
    if ((e = launch_pair_noise(c->P, c->B, c->d_zblk, c->d_bvec, s)) != cudaSuccess) return e;
    if ((e = launch_pair_force_integrate(c->P, c->B, s)) != cudaSuccess) return e;
    if ((e = launch_rebuild(c->P, c->B, s)) != cudaSuccess) return e;
    if ((e = launch_cforce(c->P, c->B, 1, s)) != cudaSuccess) return e;  // with the VACF terms
    return launch_pcorr(c->P, c->B, s);
}

// One step captured with the rebuild kernels in the body of a conditional
// (IF) node whose condition a one-thread kernel sets from ctrl->rebuild, so
// steps without a rebuild launch none of them.
// With `overlap`, the step's own convolution is not captured (the previous
// step computed it) and the next step's convolution is forked onto a second
// capture stream right after the pair kernel: it reads only the ring the pair
// kernel has just written, so it runs beside the rebuild, F^C, VACF and pair
// correlation kernels and is joined before the next pair kernel.
cudaError_t capture_fork_next(gld_ctx* c, cudaStream_t s)
{
    cudaError_t e = cudaEventRecord(c->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->cap3, c->ev_fork, 0);
    if (e == cudaSuccess)
        e = launch_hist_conv_next(c->B.ring, c->P.hist_bf16, c->P.n_pad, c->P.m_max, c->B.ctrl, c->coef, c->P.nacc,
                                  c->B.conv, c->prm.kahan, c->cap3);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->cap3);
    return e;
}

cudaError_t capture_step_gated(gld_ctx* c, cudaStream_t s, bool overlap)
{
    if (!overlap) return launch_one_step(c, s);
    cudaError_t e = launch_pair_noise(c->P, c->B, c->d_zblk, c->d_bvec, s);
    if (e == cudaSuccess) e = launch_pair_force_integrate(c->P, c->B, s);
    if (e == cudaSuccess) e = capture_fork_next(c, s);
    if (e == cudaSuccess) e = launch_rebuild(c->P, c->B, s);
    if (e == cudaSuccess) e = launch_cforce(c->P, c->B, 1, s);
    if (e == cudaSuccess) e = launch_pcorr(c->P, c->B, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_join, 0);
    return e;
}

cudaError_t capture_step_conditional(gld_ctx* c, cudaStream_t s, bool overlap)
{
    cudaError_t e = overlap ? cudaSuccess : launch_memory(c, s);
    if (e == cudaSuccess) e = launch_pair_noise(c->P, c->B, c->d_zblk, c->d_bvec, s);
    if (e == cudaSuccess) e = launch_pair_force_integrate(c->P, c->B, s);
    if (overlap && e == cudaSuccess) e = capture_fork_next(c, s);
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd);
    cudaGraphConditionalHandle h{};
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = launch_rebuild_decide(h, c->B.ctrl, s);
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd);
    cudaGraphNodeParams np{};
    cudaGraphNode_t node = nullptr;
    if (e == cudaSuccess) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeIf;
        np.conditional.size = 1;
        e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &np);
    }
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(c->cap2, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t eb = launch_rebuild(c->P, c->B, c->cap2);
        cudaGraph_t body = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(c->cap2, &body);
        e = eb != cudaSuccess ? eb : ee;
    }
    if (e == cudaSuccess) e = launch_cforce(c->P, c->B, 1, s);
    if (e == cudaSuccess) e = launch_pcorr(c->P, c->B, s);
    if (overlap && e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_join, 0);
    return e;
}

// Turns the Chebyshev form of the pair noise off and releases its buffers.
void pn_release(gld_ctx* c)
{
    for (float** p : {&c->d_pntaps, &c->d_zblk, &c->d_bvec, &c->d_lzv}) {
        dfree(c, *p);
        *p = nullptr;
    }
    for (double** p : {&c->d_lzpart, &c->d_lzab}) {
        dfree(c, *p);
        *p = nullptr;
    }
    dfree(c, c->d_rowsum);
    c->d_rowsum = nullptr;
    c->P.pn_deg = 0;
    c->P.pn_iv = 0;
    c->P.pn_cen = 0.f;
}

// ---- pair-correlated noise by a Lanczos iteration per frequency ------------
void kry_release(gld_ctx* c)
{
    auto& K = c->kry;
    for (float** p : {&K.V, &K.Y, &K.cf, &K.cosT, &K.wgt}) {
        dfree(c, *p);
        *p = nullptr;
    }
    for (double** p : {&K.part, &K.alpha, &K.beta, &K.wc}) {
        dfree(c, *p);
        *p = nullptr;
    }
    dfree(c, K.alive);
    K.alive = nullptr;
    K.M = K.Mp = K.kmax = K.window = K.Mc = 0;
    K.last_iters = 0;
    c->P.pn_kry = 0;
}

// Eigen-decomposition of a small symmetric matrix a (n x n, row-major) by
// cyclic Jacobi rotations: eigenvalues into th, eigenvectors as the columns
// of u.  Rotations stop once the off-diagonal part is below 1e-30 of the
// norm (FP64).
void jacobi_eig(int n, std::vector<double>& a, std::vector<double>& th, std::vector<double>& u)
{
    u.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) u[(size_t)i * n + i] = 1.0;
    double norm = 0.0;
    for (double x : a) norm += x * x;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += a[(size_t)p * n + q] * a[(size_t)p * n + q];
        if (off <= 1e-30 * norm) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = a[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double theta = (a[(size_t)q * n + q] - a[(size_t)p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = cs * akp - sn * akq;
                    a[(size_t)k * n + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = cs * apk - sn * aqk;
                    a[(size_t)q * n + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double ukp = u[(size_t)k * n + p], ukq = u[(size_t)k * n + q];
                    u[(size_t)k * n + p] = cs * ukp - sn * ukq;
                    u[(size_t)k * n + q] = sn * ukp + cs * ukq;
                }
            }
    }
    th.resize(n);
    for (int i = 0; i < n; ++i) th[i] = a[(size_t)i * n + i];
}

// c = |x| sqrt(H) e_1 for the j x j Lanczos matrix H (diagonal alpha,
// off-diagonal beta); *neg receives the most negative eigenvalue of H over
// its largest magnitude (a negative Ritz value means hat K_w is not positive
// semi-definite).  Negative eigenvalues contribute nothing.
void tri_sqrt_e1(int j, const double* alpha, const double* beta, double xnorm, std::vector<double>& c, double* neg)
{
    std::vector<double> a((size_t)j * j, 0.0), th, u;
    for (int p = 0; p < j; ++p) {
        a[(size_t)p * j + p] = alpha[p];
        if (p + 1 < j) a[(size_t)p * j + p + 1] = a[(size_t)(p + 1) * j + p] = beta[p];
    }
    jacobi_eig(j, a, th, u);
    double mx = 0.0, mn = 0.0;
    for (double t : th) {
        mx = std::max(mx, std::fabs(t));
        mn = std::min(mn, t);
    }
    *neg = mx > 0 ? mn / mx : 0.0;
    c.assign(j, 0.0);
    for (int i = 0; i < j; ++i) {
        const double wgt = std::sqrt(std::max(th[i], 0.0)) * u[i];  // sqrt(theta_i) (u_i)_1
        for (int p = 0; p < j; ++p) c[p] += u[(size_t)p * j + i] * wgt;
    }
    for (double& x : c) x *= xnorm;
}

// F^R of the current step by Algorithm 1, into its row of the F^R block
// (eager: host decisions between chunks of iterations).  R_0 is the
// transformed window, beta_0 = |R_0|; iteration k gives alpha_k and
// beta_{k+1} = |R_{k+1}|, and the tridiagonal matrix of dimension j has
// alpha_0 .. alpha_{j-1} on its diagonal and beta_1 .. beta_{j-1} beside it.
gld_status pair_noise_krylov(gld_ctx* c, cudaStream_t st)
{
    const StepParams& P = c->P;
    auto& K = c->kry;
    const int M = K.M, Mp = K.Mp;
    const size_t vs = 3 * (size_t)P.n_pad * Mp;
    auto R = [&](int p) { return K.V + (size_t)p * vs; };
    auto A = [&](int p) { return K.alpha + (size_t)p * Mp; };
    auto Bt = [&](int p) { return K.beta + (size_t)p * Mp; };
    GLD_CUDA(c, cudaMemsetAsync(K.alive, 1, sizeof(int) * Mp, st));  // nonzero: alive
    GLD_CUDA(c, kry_ft(P, c->B.ctrl, c->W, K.cosT, M, Mp, K.Mc, R(0), st));
    GLD_CUDA(c, kry_dot(P, R(0), R(0), Mp, K.part, Bt(0), 2, nullptr, K.alive, st));
    // the columns iterated: the cosine transforms of w < M and, with the time
    // window, the sine transforms of 1 <= w < M (columns Mc + w)
    std::vector<int> cols;
    for (int w = 0; w < M; ++w) cols.push_back(w);
    if (K.window)
        for (int w = 1; w < M; ++w) cols.push_back(K.Mc + w);
    const int NC = (int)cols.size();
    int k = 0;  // iterations done
    const int chunk = 4;
    std::vector<double> ha, hb;
    std::vector<std::vector<double>> cfin(NC);
    std::vector<int> done(NC, 0), kw(NC, 0);
    int ndone = 0;
    double worst_change = 0.0, worst_neg = 0.0;
    while (true) {
        for (int it = 0; it < chunk && k < K.kmax; ++it, ++k) {
            GLD_CUDA(c, kry_matvec(P, c->B, K.wc, Bt(k), K.alive, Mp, R(k), K.Y, K.part, A(k), st));
            GLD_CUDA(c, kry_resid(P, K.Y, R(k), k > 0 ? R(k - 1) : nullptr, A(k), Bt(k), k > 0 ? Bt(k - 1) : nullptr,
                                  K.alive, A(0), Mp, R(k + 1), K.part, Bt(k + 1), st));
        }
        ha.resize((size_t)k * Mp);
        hb.resize((size_t)(k + 1) * Mp);
        GLD_CUDA(c, cudaMemcpyAsync(ha.data(), K.alpha, sizeof(double) * ha.size(), cudaMemcpyDeviceToHost, st));
        GLD_CUDA(c, cudaMemcpyAsync(hb.data(), K.beta, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, st));
        GLD_TRY(sync_and_check(c));
        for (int ci = 0; ci < NC; ++ci) {
            if (done[ci]) continue;
            const int w = cols[ci];
            // the Krylov space of w ends at the first vanished beta (exact result)
            int j = 1;
            std::vector<double> al(k), be(std::max(k - 1, 0));
            for (int p = 0; p < k; ++p) al[p] = ha[(size_t)p * Mp + w];
            bool exhausted = false;
            for (int p = 0; p + 1 < k; ++p) {
                be[p] = hb[(size_t)(p + 1) * Mp + w];
                if (!(be[p] > 0.0)) {
                    exhausted = true;
                    break;
                }
                ++j;
            }
            if (!exhausted && j == k && !(hb[(size_t)k * Mp + w] > 0.0)) exhausted = true;
            const double xnorm = hb[w];
            std::vector<double> cj;
            double neg = 0.0;
            tri_sqrt_e1(j, al.data(), be.data(), xnorm, cj, &neg);
            worst_neg = std::min(worst_neg, neg);
            double change = 0.0, nrm = 0.0;
            if (j >= 2) {
                std::vector<double> cm;
                double neg2 = 0.0;
                tri_sqrt_e1(j - 1, al.data(), be.data(), xnorm, cm, &neg2);
                cm.resize(j, 0.0);
                for (int p = 0; p < j; ++p) {
                    change += (cj[p] - cm[p]) * (cj[p] - cm[p]);
                    nrm += cj[p] * cj[p];
                }
                change = nrm > 0 ? std::sqrt(change / nrm) : 0.0;
            } else {
                change = exhausted ? 0.0 : 1.0;
            }
            if (exhausted || change <= K.tol) {
                done[ci] = 1;
                ++ndone;
                cfin[ci] = cj;
                kw[ci] = j;
                worst_change = std::max(worst_change, exhausted ? 0.0 : change);
            } else if (k >= K.kmax) {
                cfin[ci] = cj;
                kw[ci] = j;
                worst_change = std::max(worst_change, change);
            }
        }
        if (ndone == NC || k >= K.kmax) break;
    }
    K.last_iters = *std::max_element(kw.begin(), kw.end());  // the largest Krylov dimension used
    K.last_change = worst_change;
    if (worst_neg < -1e-6) {  // beyond the rounding of FP32 vectors
        c->msg = "pair noise (Lanczos): a transformed correlation matrix is not positive semi-definite";
        if (c->latched == GLD_OK) c->latched = GLD_E_NOT_PSD;
        return GLD_E_NOT_PSD;
    }
    if (ndone < NC)
        return fail(c, GLD_E_TIMEOUT, "pair noise (Lanczos): no convergence within the iteration limit");
    // x_w = sum_p c_p v_p = sum_p (c_p / beta_p) R_p
    std::vector<float> cf((size_t)Mp * k, 0.f);
    for (int ci = 0; ci < NC; ++ci)
        for (int p = 0; p < kw[ci]; ++p) {
            const int w = cols[ci];
            const double bp = hb[(size_t)p * Mp + w];
            cf[(size_t)w * k + p] = bp > 0.0 ? (float)(cfin[ci][p] / bp) : 0.f;
        }
    GLD_CUDA(c, cudaMemcpyAsync(K.cf, cf.data(), sizeof(float) * cf.size(), cudaMemcpyHostToDevice, st));
    if (K.window) {  // every row of the block from the one window
        GLD_CUDA(c, kry_rows(P, K.V, K.cf, k, Mp, K.wgt, K.Y, c->B.frblock, st));
    } else {
        const long long row = c->host_step - c->block_start;
        GLD_CUDA(c, kry_combine(P, K.V, K.cf, k, M, Mp, c->B.frblock + (size_t)row * 3 * P.n_pad, st));
    }
    GLD_CUDA(c, cudaStreamSynchronize(st));  // cf is reused by the next step
    return GLD_OK;
}

bool capture_graph_mode(gld_ctx* c, bool conditional)
{
    // the overlapped form needs an idempotent convolution (not the recursive
    // memory form, whose kernel advances its auxiliary sums)
    bool overlap = c->P.nmodes == 0;
    if (overlap && !c->cap3 &&
        (cudaStreamCreateWithFlags(&c->cap3, cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)) {
        cudaGetLastError();
        overlap = false;
    }
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        cudaError_t e = launch_noise(c, c->cap);
        for (int t = 0; t < c->P.T && e == cudaSuccess; ++t)
            e = conditional ? capture_step_conditional(c, c->cap, overlap) : capture_step_gated(c, c->cap, overlap);
        const cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
        ok = e == cudaSuccess && e2 == cudaSuccess && g != nullptr;
    }
    if (ok) ok = cudaGraphInstantiate(&c->gexec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        c->gexec = nullptr;
        cudaGetLastError();
    }
    c->overlap_graph = ok && overlap;
    return ok;
}

bool capture_graph(gld_ctx* c)
{
    if (c->gexec) return true;
    if (c->graph_failed || c->P.pn_kry) return false;  // the Lanczos noise decides on the host every step
    // conditional rebuild first; the gated kernels are the fallback
    if (c->prm.use_graphs != 2 && capture_graph_mode(c, true)) {
        c->graph_mode = 2;
        return true;
    }
    if (capture_graph_mode(c, false)) {
        c->graph_mode = 1;
        return true;
    }
    c->graph_failed = true;
    return false;
}

int clamp_block(int) { return kMaxNoiseBlock; }  // the filter produces 64-step blocks

// Blocks of VACF partials per origin: one per 256 particles, the F^C
// kernel's grid (which accumulates them) and the batch VACF grid's width.
int vacf_blocks(int n, int) { return std::max(1, (n + 255) / 256); }

}  // namespace

namespace gld {

gld_status ctx_check_err(gld_ctx* c, unsigned err)
{
    if (err & kErrNonFinite) fail(c, GLD_E_NONFINITE, "non-finite displacement produced on the device");
    else if (err & kErrNbrOverflow) {
        c->msg = "a neighbour list exceeded its capacity (density far above the one at creation)";
        if (c->latched == GLD_OK) c->latched = GLD_E_STATE;
    }
    else if (err & kErrTimeout) fail(c, GLD_E_TIMEOUT, "a bounded device wait gave up");
    else if (err & kErrCheck) fail(c, GLD_E_CUDA, "a kernel's own bounds or alignment check failed");
    else if (err & kErrNoise) fail(c, GLD_E_CUDA, "a step ran outside its noise block");
    else if (err & kErrPnBound) {
        c->msg = "pair noise: the spectrum of the pair matrix left the interpolation interval (a Gershgorin row "
                 "sum above lambda, or a Ritz value outside [lo, hi]): set a wider one";
        if (c->latched == GLD_OK) c->latched = GLD_E_NOT_PSD;
    }
    return c->latched;
}

void ctx_to_caller(const gld_ctx* c, const float4* h, double* dst)
{
    for (int i = 0; i < c->P.n; ++i) {
        const size_t e = (size_t)c->int2ext[i];
        dst[3 * e] = h[i].x;
        dst[3 * e + 1] = h[i].y;
        dst[3 * e + 2] = h[i].z;
    }
}

void ctx_derive(const gld_params* p, StepParams& P, int& ncells)
{
    P.n = p->n;
    P.n_pad = (p->n + 31) & ~31;
    P.m_max = p->m_max;
    P.H = p->m_max - 1;
    P.Q = P.Qs = 0;
    P.nacc = 1;
    P.nr = 2;
    // Verlet lists of radius r_l = r_c + skin (r_l <= L/2), built from cells of
    // edge >= r_l (with a margin well above FP32 rounding of the coordinates),
    // at most ~8 cells per particle; fewer than 3 per side -> one cell.
    double skin = p->skin > 0 ? p->skin : 0.2 * p->r_c;
    if (p->r_c + skin > 0.5 * p->box) skin = 0.5 * p->box - p->r_c;
    const double rl = p->r_c + skin;
    int nc = (int)std::floor(p->box / rl);
    while (nc > 0 && p->box / nc < rl * (1.0 + 1e-5)) --nc;
    const int ncap = (int)std::floor(std::cbrt(8.0 * p->n));
    if (nc > ncap) nc = ncap;
    if (nc < 3) nc = 1;
    P.nc = nc;
    P.T = clamp_block(p->noise_block > 0 ? p->noise_block : kMaxNoiseBlock);
    // the white-noise ring: at least T + 2H times, in whole 32-row tiles with
    // room for a window that starts up to 31 rows before n - H
    P.lw = ((long long)P.T + 2LL * P.H + 31 + 31) / 32 * 32;
    P.box = (float)p->box;
    P.half_box = 0.5f * P.box;
    P.inv_box = 1.0f / P.box;
    P.inv_cell = (float)(nc / p->box);
    P.rc2 = (float)(p->r_c * p->r_c);
    P.rc_min = (float)p->r_c_min;
    P.inv_dr = 1.f;
    P.inv_dt = (float)(1.0 / p->dt);
    P.pos_v = (float)p->dt;
    P.pos_f = (float)(p->dt * p->dt / (2.0 * p->mass));
    P.vh_v = 1.f;
    P.vh_fc = (float)(p->dt / (2.0 * p->mass));
    P.vh_f = (float)(p->dt / p->mass);
    P.vf_fc = (float)(p->dt / (2.0 * p->mass));
    P.fc_mag = (float)(2.0 * p->A_cons / p->r_c);
    P.inv_rc = (float)(1.0 / p->r_c);
    P.rl2 = (float)(rl * rl);
    P.trig2 = (float)(0.45 * skin * 0.45 * skin);
    {
        const double expect = p->n / (p->box * p->box * p->box) * 4.18879020478639 * rl * rl * rl;
        P.maxnb = std::min(p->n, ((int)std::ceil(2.0 * expect + 32.0) + 7) & ~7);
        if (P.maxnb < 1) P.maxnb = 1;
    }
    P.hist_bf16 = p->hist_dtype == GLD_HIST_BF16;
    P.vacf_len = p->vacf_len;
    P.vacf_stride = p->vacf_stride > 0 ? p->vacf_stride : 1;
    P.n_os = p->vacf_len > 0 ? (p->vacf_len + P.vacf_stride - 1) / P.vacf_stride : 0;
    P.vacf_burnin = p->vacf_burnin < 0 ? 2LL * p->m_max : p->vacf_burnin;
    ncells = P.nc * P.nc * P.nc;
}

// Mirrors the allocations of gld_create and gld_set_kernels (each rounded to
// 256 bytes); a test compares it with the bytes a context really holds.
size_t ctx_bytes_needed(const gld_params* p, int Q, int Qs, int nr, int num_sms)
{
    StepParams P{};
    int ncells = 0;
    ctx_derive(p, P, ncells);
    const size_t np = P.n_pad, n3 = 3 * np;
    const size_t elem = P.hist_bf16 ? 2 : 4;
    const int chunks = (ncells + 511) / 512;
    const int vacf_gx = vacf_blocks(P.n, num_sms);
    const int nt = Q + Qs, nrr = nt > 0 ? nr : 2;
    const size_t sizes[] = {
        sizeof(Ctrl), 16 * np, 16 * np, 16 * np, 16 * np, 4 * (size_t)P.maxnb * np, 4 * np, 4 * np,
        16 * np, 16 * np, 16 * np, 16 * np, 16 * np, elem * n3 * P.H, 4 * (size_t)kMaxAcc * n3,
        4 * (size_t)P.T * n3, 4 * (size_t)P.lw * n3, 4 * ((size_t)ncells + 1), 4 * (size_t)ncells,
        4 * (size_t)ncells, 4 * np, 4 * (size_t)chunks, 4 * (size_t)chunks,
        16 * (size_t)std::max(P.n_os, 1) * P.n, 8 * (size_t)std::max(P.n_os, 1) * vacf_gx,
        8 * (size_t)std::max(P.vacf_len, 1), 8 * (size_t)std::max(P.vacf_len, 1), 8,
        4 * (size_t)fir_taps_len(P.H), 4 * (size_t)kMaxAcc * P.m_max, 4 * 2 * (size_t)kMaxQ,
        8 * (size_t)P.m_max, 8 * (size_t)P.m_max, 8 * (size_t)P.m_max, 8 * 2 * (size_t)P.m_max, 8 * 4, 4,
        8 * (size_t)(1 + 2 * kMaxQ) * P.m_max, 4 * np, 4 * (size_t)std::max(nt, 1) * nrr};
    size_t total = 0;
    for (size_t b : sizes) total += b == 0 ? 256 : (b + 255) & ~(size_t)255;
    return total;
}

size_t pn_bytes_needed(const gld_params* p, int K)
{
    if (K <= 0) return 0;
    StepParams P{};
    int ncells = 0;
    ctx_derive(p, P, ncells);
    const size_t sizes[] = {4 * (size_t)(K + 1) * fir_taps_len(P.H), 4 * (size_t)K * P.T * 3 * P.n_pad,
                            4 * 9 * (size_t)P.n_pad, 4};
    size_t total = 0;
    for (size_t b : sizes) total += (b + 255) & ~(size_t)255;
    return total;
}

}  // namespace gld

extern "C" {

void gld_params_default(gld_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->mass = 1.0;
    p->kT = 1.0;
    p->dt = 0.005;
    p->m_max = 2;
    p->hist_dtype = GLD_HIST_F32;
    p->vacf_stride = 1;
    p->vacf_burnin = -1;
    p->noise_block = kMaxNoiseBlock;
    p->use_graphs = 1;
}

gld_status gld_create(const gld_params* p, const double* pos, const double* vel, gld_ctx** out)
{
    if (!out) return GLD_E_INVAL;
    *out = nullptr;
    if (!p || !pos || !vel) return GLD_E_INVAL;
    if (p->use_graphs < 0 || p->use_graphs > 2) return GLD_E_INVAL;
    if (p->n < 1 || p->m_max < 2 || p->m_max > 4096 || !(p->box > 0) || !(p->mass > 0) || !(p->dt > 0) ||
        !(p->r_c > 0) || p->r_c > 0.5 * p->box || p->kT < 0 || p->r_c_min < 0 || p->skin < 0 ||
        (p->hist_dtype != GLD_HIST_F32 && p->hist_dtype != GLD_HIST_BF16) || p->vacf_len < 0 ||
        (p->vacf_len > 0 && p->vacf_stride < 1) || (p->vacf_len > 0 && p->vacf_burnin == 0) ||
        (p->vacf_len > 0 && (p->vacf_len + p->vacf_stride - 1) / p->vacf_stride > 32))
        return GLD_E_INVAL;
    gld_ctx* c = new gld_ctx();
    c->prm = *p;
    c->st = (cudaStream_t)p->stream;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap2, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return GLD_E_CUDA;
    }
    StepParams& P = c->P;
    int ncells = 0;
    ctx_derive(p, P, ncells);
    c->ring_elem = P.hist_bf16 ? 2 : 4;

    const size_t np = P.n_pad, n3 = 3 * np;
    const int nc = P.nc;
    // Internal order: the caller's, or the Morton order of the cells at R_0
    // (ties by the caller's index), so that neighbours are close in memory.
    c->int2ext.resize(p->n);
    if (p->order) {
        std::vector<char> seen(p->n, 0);
        for (int k = 0; k < p->n; ++k) {
            const int e = p->order[k];
            if (e < 0 || e >= p->n || seen[e]) {
                cudaStreamDestroy(c->cap);
                cudaStreamDestroy(c->cap2);
                delete c;
                return GLD_E_INVAL;
            }
            seen[e] = 1;
            c->int2ext[k] = e;
        }
    } else {
        auto spread = [](uint64_t v) {  // 21 bits -> every third bit
            v &= 0x1fffff;
            v = (v | v << 32) & 0x1f00000000ffffULL;
            v = (v | v << 16) & 0x1f0000ff0000ffULL;
            v = (v | v << 8) & 0x100f00f00f00f00fULL;
            v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
            v = (v | v << 2) & 0x1249249249249249ULL;
            return v;
        };
        const int g = std::max(nc, 1);
        std::vector<std::pair<uint64_t, int>> key(p->n);
        for (int e = 0; e < p->n; ++e) {
            uint64_t cc[3];
            for (int d = 0; d < 3; ++d) {
                const double x = wrap_host(pos[3 * e + d], p->box);
                long long ci = (long long)std::floor(x / p->box * g);
                ci = ci < 0 ? 0 : (ci >= g ? g - 1 : ci);
                cc[d] = (uint64_t)ci;
            }
            key[e] = {spread(cc[0]) | spread(cc[1]) << 1 | spread(cc[2]) << 2, e};
        }
        std::sort(key.begin(), key.end());
        for (int k = 0; k < p->n; ++k) c->int2ext[k] = key[k].second;
    }
    const int chunks = (ncells + 511) / 512;
    ParticleBuffers& B = c->B;
    bool ok = true;
    B.ctrl = alloc_n<Ctrl>(c, 1, ok);
    B.pos_sorted = alloc_n<float4>(c, np, ok);
    B.pos = alloc_n<float4>(c, np, ok);
    B.pos_next = alloc_n<float4>(c, np, ok);
    B.disp_build = alloc_n<float4>(c, np, ok);
    B.nbr = alloc_n<int>(c, (size_t)P.maxnb * np, ok);
    B.nbr_cnt = alloc_n<int>(c, np, ok);
    B.perm = alloc_n<int>(c, np, ok);
    B.vel = alloc_n<float4>(c, np, ok);
    B.vhalf = alloc_n<float4>(c, np, ok);
    B.fc = alloc_n<float4>(c, np, ok);
    B.fd = alloc_n<float4>(c, np, ok);
    B.disp = alloc_n<float4>(c, np, ok);
    B.ring = dalloc(c, c->ring_elem * n3 * P.H);
    if (!B.ring) ok = false;
    B.conv = alloc_n<float>(c, kMaxAcc * n3, ok);
    B.frblock = alloc_n<float>(c, (size_t)P.T * n3, ok);
    c->W = alloc_n<float>(c, (size_t)P.lw * n3, ok);
    B.ncells = ncells;
    B.cell_start = alloc_n<int>(c, ncells + 1, ok);
    B.cell_count = alloc_n<int>(c, ncells, ok);
    B.cell_head = alloc_n<int>(c, ncells, ok);
    B.cell_next = alloc_n<int>(c, np, ok);
    B.chunk_sum = alloc_n<int>(c, chunks, ok);
    B.chunk_off = alloc_n<int>(c, chunks, ok);
    B.vacf_gx = vacf_blocks(P.n, c->num_sms);
    B.vorig = alloc_n<float4>(c, (size_t)std::max(P.n_os, 1) * P.n, ok);
    B.vpartial = alloc_n<float>(c, 2 * (size_t)std::max(P.n_os, 1) * B.vacf_gx, ok);
    B.csum = alloc_n<double>(c, std::max(P.vacf_len, 1), ok);
    B.ccnt = alloc_n<long long>(c, std::max(P.vacf_len, 1), ok);
    B.norig = alloc_n<long long>(c, 1, ok);
    c->la = fir_taps_len(P.H);
    c->Acp = alloc_n<float>(c, (size_t)c->la, ok);
    c->coef = alloc_n<float>(c, (size_t)kMaxAcc * P.m_max, ok);
    c->g0 = alloc_n<float>(c, 2 * kMaxQ, ok);
    c->d_Kd = alloc_n<double>(c, P.m_max, ok);
    c->d_C = alloc_n<double>(c, P.m_max, ok);
    c->d_Chat = alloc_n<double>(c, P.m_max, ok);
    c->d_A = alloc_n<double>(c, 2 * P.m_max, ok);
    c->d_scal = alloc_n<double>(c, 4, ok);
    c->d_status = alloc_n<int>(c, 1, ok);
    c->d_in = alloc_n<double>(c, (size_t)(1 + 2 * kMaxQ) * P.m_max, ok);
    c->d_int2ext = alloc_n<int>(c, np, ok);
    B.g0 = c->g0;
    if (!ok) {
        gld_destroy(c);
        return GLD_E_NOMEM;
    }
    // tensor map of the white-noise ring for the tensor-core filter (the
    // filter runs on the FP32 pipes when it cannot be made)
    c->have_wmap = noise_filter_tc_ok(P) && make_noise_ring_map(c->W, P, &c->wmap) == cudaSuccess;
    cudaGetLastError();
    P.wsplit = c->have_wmap ? 1 : 0;  // the ring starts zeroed: valid in either form
    gld_status s = GLD_OK;
    if (cudaMemsetAsync(B.cell_head, 0xff, sizeof(int) * ncells, c->st) != cudaSuccess) s = GLD_E_CUDA;
    Ctrl h{};
    h.w_lo = 1;
    h.w_hi = 0;
    if (s == GLD_OK && cudaMemcpyAsync(B.ctrl, &h, sizeof(h), cudaMemcpyHostToDevice, c->st) != cudaSuccess) s = GLD_E_CUDA;
    const int total = P.n;
    if (s == GLD_OK && cudaMemcpyAsync(B.cell_start + ncells, &total, sizeof(int), cudaMemcpyHostToDevice, c->st) != cudaSuccess)
        s = GLD_E_CUDA;
    if (s == GLD_OK && cudaMemcpyAsync(c->d_int2ext, c->int2ext.data(), sizeof(int) * P.n, cudaMemcpyHostToDevice,
                                       c->st) != cudaSuccess)
        s = GLD_E_CUDA;
    if (s == GLD_OK) s = upload_vec(c, B.pos, pos, true);
    if (s == GLD_OK) s = upload_vec(c, B.pos_next, pos, true);
    if (s == GLD_OK) s = upload_vec(c, B.vel, vel, false);
    if (s == GLD_OK) s = rebuild_cells_and_fc(c);
    if (s == GLD_OK) s = sync_and_check(c);
    if (s != GLD_OK) {
        gld_destroy(c);
        return s;
    }
    *out = c;
    return GLD_OK;
}

gld_status gld_set_kernels(gld_ctx* c, const double* Ks, int32_t Q, const double* g, const double* f, int32_t nr,
                           double dr, const double* dKs_g, const double* dKs_f, int32_t Qs, int32_t conv)
{
    if (!c) return GLD_E_INVAL;
    if (!Ks || Q < 0 || Q > kMaxQ || Qs < 0 || Qs > kMaxQ || (Q > 0 && (!g || !f)) || (Qs > 0 && (!dKs_g || !dKs_f)) ||
        (Q + Qs > 0 && (nr < 2 || !(dr > 0))) || (conv != GLD_KCONT && conv != GLD_KDISCRETE))
        return fail(c, GLD_E_INVAL, "gld_set_kernels: invalid kernel description");
    // From here until the new kernels are in place the context has none: the
    // old tables are released below, so a failure on the way (an allocation,
    // a CUDA call, a rejected spectrum) leaves a context that refuses to step
    // rather than one whose step would read freed tables.
    c->have_kernels = false;
    c->B.ftab = nullptr;
    // the pair noise and the perpendicular factors belong to the previous
    // kernels: off, and their buffers released (stream-ordered like ftab's)
    c->P.perp = 0;
    invalidate_graph(c);
    pn_release(c);
    dfree(c, c->fptab);
    c->fptab = nullptr;
    c->B.fptab = nullptr;
    kry_release(c);
    const int M = c->P.m_max;
    std::vector<double> in((size_t)(1 + 2 * kMaxQ) * M, 0.0);
    std::memcpy(in.data(), Ks, sizeof(double) * M);
    if (Q) std::memcpy(in.data() + M, g, sizeof(double) * (size_t)Q * M);
    if (Qs) std::memcpy(in.data() + (size_t)(1 + Q) * M, dKs_g, sizeof(double) * (size_t)Qs * M);
    GLD_CUDA(c, cudaMemcpyAsync(c->d_in, in.data(), sizeof(double) * in.size(), cudaMemcpyHostToDevice, c->st));
    const int nt = Q + Qs;
    const int nrr = nt > 0 ? nr : 2;
    std::vector<float> tab((size_t)std::max(nt, 1) * nrr, 0.f);
    for (int q = 0; q < Q; ++q)
        for (int k = 0; k < nr; ++k) tab[(size_t)q * nr + k] = (float)f[(size_t)q * nr + k];
    for (int q = 0; q < Qs; ++q)
        for (int k = 0; k < nr; ++k) tab[(size_t)(Q + q) * nr + k] = (float)dKs_f[(size_t)q * nr + k];
    dfree(c, c->ftab);
    c->ftab = (float*)dalloc(c, sizeof(float) * tab.size());
    if (!c->ftab) return fail(c, GLD_E_NOMEM, "gld_set_kernels: table allocation failed");
    GLD_CUDA(c, cudaMemcpyAsync(c->ftab, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice, c->st));
    PrepArgs a{};
    a.m_max = M;
    a.Q = Q;
    a.Qs = Qs;
    a.discrete = conv == GLD_KDISCRETE;
    a.clamp = c->prm.psd_clamp;
    a.T = c->P.T;
    a.dt = c->prm.dt;
    a.kT = c->prm.kT;
    a.mass = c->prm.mass;
    a.Ks = c->d_in;
    a.g = c->d_in + M;
    a.gs = c->d_in + (size_t)(1 + Q) * M;
    a.Kd = c->d_Kd;
    a.C = c->d_C;
    a.Chat = c->d_Chat;
    a.A = c->d_A;
    a.scal = c->d_scal;
    a.status = c->d_status;
    a.coef = c->coef;
    a.g0 = c->g0;
    a.Acp = c->Acp;
    a.la = c->la;
    GLD_CUDA(c, launch_prep(a, c->st));
    double scal[4];
    int status = 0;
    c->Kd.assign(M, 0.0);
    c->A.assign(2 * M - 1, 0.0);
    GLD_CUDA(c, cudaMemcpyAsync(scal, c->d_scal, sizeof(scal), cudaMemcpyDeviceToHost, c->st));
    GLD_CUDA(c, cudaMemcpyAsync(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    GLD_CUDA(c, cudaMemcpyAsync(c->Kd.data(), c->d_Kd, sizeof(double) * M, cudaMemcpyDeviceToHost, c->st));
    GLD_CUDA(c, cudaMemcpyAsync(c->A.data(), c->d_A, sizeof(double) * (2 * M - 1), cudaMemcpyDeviceToHost, c->st));
    GLD_CUDA(c, cudaStreamSynchronize(c->st));
    c->a = scal[0];
    c->b = scal[1];
    c->spec_min = scal[2];
    c->clamped = scal[3];
    invalidate_graph(c);
    if (status != 0) {
        c->have_kernels = false;
        c->msg = "gld_set_kernels: the noise spectrum has a negative mode (not positive semi-definite)";
        return GLD_E_NOT_PSD;
    }
    StepParams& P = c->P;
    const double dt = c->prm.dt, M2 = 2.0 * c->prm.mass;
    P.Q = Q;
    P.Qs = Qs;
    P.nacc = 1 + Q + Qs;
    P.nr = nrr;
    P.inv_dr = nt > 0 ? (float)(1.0 / dr) : 1.f;
    P.pos_v = (float)(c->b * dt);
    P.pos_f = (float)(c->b * dt * dt / M2);
    P.vh_v = (float)c->a;
    P.vh_fc = (float)(c->a * dt / M2);
    P.vh_f = (float)(c->b * dt / c->prm.mass);
    P.vf_fc = (float)(dt / M2);
    c->B.ftab = c->ftab;
    // FP64 discrete weights of every accumulator (m >= 1), for the recursive form
    c->wts.assign((size_t)P.nacc * P.m_max, 0.0);
    for (int a = 0; a < P.nacc; ++a)
        for (int m = 0; m < P.m_max; ++m) {
            const double sm = in[(size_t)a * P.m_max + m];  // rows: K^s, g_1..g_Q, gs_1..gs_Qs
            c->wts[(size_t)a * P.m_max + m] = conv == GLD_KDISCRETE ? sm : (m == 0 ? 0.5 : 1.0) * dt * sm;
        }
    P.nmodes = 0;  // new kernels: back to the ring convolution until modes are set again
    P.pn_deg = 0;  // and to the self-kernel noise until the pair noise is set again
    P.perp = 0;    // and to parallel components only
    c->modes_dirty = false;
    c->have_kernels = true;
    GLD_TRY(invalidate_noise(c));
    return sync_and_check(c);
}

gld_status gld_step(gld_ctx* c, int64_t nsteps)
{
    if (!c || nsteps < 0) return GLD_E_INVAL;
    if (!c->have_kernels) return fail(c, GLD_E_STATE, "gld_step: gld_set_kernels has not succeeded");
    if (c->latched != GLD_OK) return c->latched;
    const int T = c->P.T;
    if (nsteps > 0) GLD_TRY(ring_form(c, true, c->st));
    if (nsteps > 0) GLD_TRY(refresh_modes(c));
    while (nsteps > 0) {
        if (!c->noise_valid || c->host_step >= c->noise_end) {
            if (c->prm.use_graphs && nsteps >= T && capture_graph(c)) {
                // the overlapped graph starts from the projections of its first step
                if (c->overlap_graph && c->conv_valid_step != c->host_step) GLD_CUDA(c, launch_memory(c, c->st));
                GLD_CUDA(c, cudaGraphLaunch(c->gexec, c->st));
                c->block_start = c->host_step;
                c->host_step += T;
                c->conv_valid_step = c->overlap_graph ? c->host_step : -1;
                c->noise_end = c->host_step;
                c->noise_valid = true;
                c->last_fr_row = T - 1;
                nsteps -= T;
                continue;
            }
            GLD_CUDA(c, launch_noise(c, c->st));
            c->block_start = c->host_step;
            c->noise_end = c->host_step + T;
            c->noise_valid = true;
            if (c->P.pn_kry && c->kry.window) GLD_TRY(pair_noise_krylov(c, c->st));  // the block's rows at once
        }
        if (c->P.pn_kry && !c->kry.window) GLD_TRY(pair_noise_krylov(c, c->st));
        GLD_CUDA(c, launch_one_step(c, c->st));
        c->conv_valid_step = -1;
        c->last_fr_row = c->host_step - c->block_start;
        ++c->host_step;
        --nsteps;
    }
    return GLD_OK;
}

gld_status gld_sync(gld_ctx* c)
{
    if (!c) return GLD_E_INVAL;
    return sync_and_check(c);
}

gld_status gld_vacf(gld_ctx* c, double* out, int64_t* n_origins)
{
    if (!c) return GLD_E_INVAL;
    if (c->latched == GLD_OK) GLD_CUDA(c, launch_vacf_flush(c->P, c->B, c->st));
    GLD_TRY(sync_and_check(c));
    const int L = c->P.vacf_len;
    long long no = 0;
    if (L > 0) {
        std::vector<double> s(L);
        std::vector<long long> k(L);
        GLD_CUDA(c, cudaMemcpy(s.data(), c->B.csum, sizeof(double) * L, cudaMemcpyDeviceToHost));
        GLD_CUDA(c, cudaMemcpy(k.data(), c->B.ccnt, sizeof(long long) * L, cudaMemcpyDeviceToHost));
        GLD_CUDA(c, cudaMemcpy(&no, c->B.norig, sizeof(long long), cudaMemcpyDeviceToHost));
        if (out)
            for (int l = 0; l < L; ++l) out[l] = k[l] > 0 ? s[l] / (3.0 * c->P.n * (double)k[l]) : 0.0;
    }
    if (n_origins) *n_origins = no;
    return GLD_OK;
}

gld_status gld_get_state(gld_ctx* c, double* pos, double* vel)
{
    if (!c) return GLD_E_INVAL;
    GLD_TRY(sync_and_check(c));
    if (pos) GLD_TRY(download_vec(c, c->B.pos, pos));
    if (vel) GLD_TRY(download_vec(c, c->B.vel, vel));
    return GLD_OK;
}

gld_status gld_get_array(gld_ctx* c, int32_t which, double* out)
{
    if (!c || !out) return GLD_E_INVAL;
    GLD_TRY(sync_and_check(c));
    const StepParams& P = c->P;
    const size_t np = P.n_pad;
    switch (which) {
    case GLD_ARR_POS: return download_vec(c, c->B.pos, out);
    case GLD_ARR_VEL: return download_vec(c, c->B.vel, out);
    case GLD_ARR_FC: return download_vec(c, c->B.fc, out);
    case GLD_ARR_FD: return download_vec(c, c->B.fd, out);
    case GLD_ARR_DISP: return download_vec(c, c->B.disp, out);
    case GLD_ARR_FR:
        if (c->last_fr_row < 0) return fail(c, GLD_E_STATE, "gld_get_array: no step has run");
        return download_planes(c, c->B.frblock + (size_t)c->last_fr_row * 3 * np, 1, out);
    case GLD_ARR_CONV: return download_planes(c, c->B.conv, P.nacc, out);
    case GLD_ARR_HIST: {
        const int H = P.H, n = P.n;
        std::vector<unsigned char> h(c->ring_elem * 3 * np * H);
        GLD_CUDA(c, cudaMemcpy(h.data(), c->B.ring, h.size(), cudaMemcpyDeviceToHost));
        for (int m = 1; m <= H; ++m) {
            long long slot = (c->host_step - m) % H;
            if (slot < 0) slot += H;
            for (int k = 0; k < 3; ++k)
                for (int i = 0; i < n; ++i) {
                    const size_t idx = ((size_t)slot * 3 + k) * np + i;
                    float v;
                    if (P.hist_bf16) {
                        uint16_t b16;
                        std::memcpy(&b16, h.data() + 2 * idx, 2);
                        const uint32_t w = (uint32_t)b16 << 16;
                        std::memcpy(&v, &w, 4);
                    } else {
                        std::memcpy(&v, h.data() + 4 * idx, 4);
                    }
                    out[((size_t)(m - 1) * n + c->int2ext[i]) * 3 + k] = v;
                }
        }
        return GLD_OK;
    }
    default: return fail(c, GLD_E_INVAL, "gld_get_array: unknown array");
    }
}

gld_status gld_set_array(gld_ctx* c, int32_t which, const double* in)
{
    if (c) c->conv_valid_step = -1;
    if (!c || !in) return GLD_E_INVAL;
    GLD_TRY(sync_and_check(c));
    const StepParams& P = c->P;
    switch (which) {
    case GLD_ARR_POS:
        GLD_TRY(upload_vec(c, c->B.pos, in, true));
        GLD_TRY(upload_vec(c, c->B.pos_next, in, true));
        GLD_TRY(rebuild_cells_and_fc(c));
        return sync_and_check(c);
    case GLD_ARR_VEL: return upload_vec(c, c->B.vel, in, false);
    case GLD_ARR_FC: return upload_vec(c, c->B.fc, in, false);
    case GLD_ARR_DISP: {
        // The list-rebuild criterion measures motion as disp - disp_build, so a
        // replaced displacement gets fresh lists (positions are unchanged).
        GLD_TRY(upload_vec(c, c->B.disp, in, false));
        const int one = 1, zero = 0;
        GLD_CUDA(c, cudaMemcpyAsync(&c->B.ctrl->rebuild, &one, sizeof(int), cudaMemcpyHostToDevice, c->st));
        GLD_CUDA(c, launch_rebuild(c->P, c->B, c->st));
        GLD_CUDA(c, cudaMemcpyAsync(&c->B.ctrl->rebuild, &zero, sizeof(int), cudaMemcpyHostToDevice, c->st));
        return sync_and_check(c);
    }
    case GLD_ARR_HIST: {
        const int H = P.H, n = P.n;
        const size_t np = P.n_pad;
        std::vector<unsigned char> h(c->ring_elem * 3 * np * H, 0);
        for (int m = 1; m <= H; ++m) {
            long long slot = (c->host_step - m) % H;
            if (slot < 0) slot += H;
            for (int k = 0; k < 3; ++k)
                for (int i = 0; i < n; ++i) {
                    const size_t idx = ((size_t)slot * 3 + k) * np + i;
                    const float v = (float)in[((size_t)(m - 1) * n + c->int2ext[i]) * 3 + k];
                    if (P.hist_bf16) {
                        const __nv_bfloat16 b = __float2bfloat16_rn(v);
                        std::memcpy(h.data() + 2 * idx, &b, 2);
                    } else {
                        std::memcpy(h.data() + 4 * idx, &v, 4);
                    }
                }
        }
        GLD_CUDA(c, cudaMemcpy(c->B.ring, h.data(), h.size(), cudaMemcpyHostToDevice));
        c->modes_dirty = true;
        return GLD_OK;
    }
    default: return fail(c, GLD_E_INVAL, "gld_set_array: array is read-only or unknown");
    }
}

gld_status gld_get_diag(gld_ctx* c, int64_t* out, int32_t count)
{
    if (!c || !out || count < 0) return GLD_E_INVAL;
    GLD_TRY(sync_and_check(c));
    long long rebuilds = 0;
    GLD_CUDA(c, cudaMemcpy(&rebuilds, &c->B.ctrl->rebuilds, sizeof(rebuilds), cudaMemcpyDeviceToHost));
    const int64_t v[5] = {c->graph_mode, rebuilds, c->P.maxnb, c->P.nc, c->kry.last_iters};
    for (int k = 0; k < count; ++k) out[k] = k < 5 ? v[k] : 0;
    return GLD_OK;
}

gld_status gld_get_order(gld_ctx* c, int32_t* int2ext)
{
    if (!c || !int2ext) return GLD_E_INVAL;
    std::memcpy(int2ext, c->int2ext.data(), sizeof(int32_t) * c->P.n);
    return GLD_OK;
}

gld_status gld_get_step(gld_ctx* c, int64_t* step)
{
    if (!c || !step) return GLD_E_INVAL;
    *step = c->host_step;
    return GLD_OK;
}

gld_status gld_set_step(gld_ctx* c, int64_t step)
{
    if (!c || step < 0) return GLD_E_INVAL;
    GLD_TRY(sync_and_check(c));
    c->host_step = step;
    long long s[2] = {step, step % c->P.H};
    GLD_CUDA(c, cudaMemcpyAsync(&c->B.ctrl->step, &s[0], sizeof(long long), cudaMemcpyHostToDevice, c->st));
    GLD_CUDA(c, cudaMemcpyAsync(&c->B.ctrl->hslot, &s[1], sizeof(long long), cudaMemcpyHostToDevice, c->st));
    GLD_TRY(invalidate_noise(c));
    c->last_fr_row = -1;
    c->modes_dirty = true;  // the ring's slots now stand for other times
    return sync_and_check(c);
}

gld_status gld_get_coefs(gld_ctx* c, double* Kd, double* A, double* ab, double* spec)
{
    if (!c) return GLD_E_INVAL;
    if (c->Kd.empty()) return fail(c, GLD_E_STATE, "gld_get_coefs: no kernels set");
    const int M = c->P.m_max;
    if (Kd) std::memcpy(Kd, c->Kd.data(), sizeof(double) * M);
    if (A) std::memcpy(A, c->A.data(), sizeof(double) * (2 * M - 1));
    if (ab) {
        ab[0] = c->a;
        ab[1] = c->b;
    }
    if (spec) {
        spec[0] = c->spec_min;
        spec[1] = c->clamped;
    }
    return GLD_OK;
}

gld_status gld_get_pairs(gld_ctx* c, int32_t* pairs, int64_t cap, int64_t* count)
{
    if (!c || (!pairs && cap > 0) || cap < 0) return GLD_E_INVAL;
    GLD_TRY(sync_and_check(c));
    int* d_pairs = (int*)dalloc(c, sizeof(int) * 2 * (size_t)std::max<int64_t>(cap, 1));
    unsigned long long* d_cnt = (unsigned long long*)dalloc(c, sizeof(unsigned long long));
    if (!d_pairs || !d_cnt) {
        dfree(c, d_pairs);
        dfree(c, d_cnt);
        return fail(c, GLD_E_NOMEM, "gld_get_pairs: allocation failed");
    }
    gld_status s = cuda_check(c, launch_list_pair_list(c->P, c->B, d_pairs, cap, d_cnt, c->st), "pair_list");
    unsigned long long cnt = 0;
    if (s == GLD_OK) s = cuda_check(c, cudaStreamSynchronize(c->st), "sync");
    if (s == GLD_OK) s = cuda_check(c, cudaMemcpy(&cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost), "copy");
    if (s == GLD_OK && cap > 0) {
        const size_t m = (size_t)std::min<long long>(cap, (long long)cnt);
        s = cuda_check(c, cudaMemcpy(pairs, d_pairs, sizeof(int) * 2 * m, cudaMemcpyDeviceToHost), "copy");
        for (size_t q = 0; s == GLD_OK && q < m; ++q) {  // caller's indices, i < j
            const int a = c->int2ext[pairs[2 * q]], b = c->int2ext[pairs[2 * q + 1]];
            pairs[2 * q] = std::min(a, b);
            pairs[2 * q + 1] = std::max(a, b);
        }
    }
    if (count) *count = (int64_t)cnt;
    cudaStreamSynchronize(c->st);
    dfree(c, d_pairs);
    dfree(c, d_cnt);
    return s;
}

gld_status gld_profile_steps(gld_ctx* c, int64_t nsteps, double* ms, int64_t* launches)
{
    if (!c || nsteps < 0) return GLD_E_INVAL;
    if (!c->have_kernels) return fail(c, GLD_E_STATE, "gld_profile_steps: gld_set_kernels has not succeeded");
    if (c->latched != GLD_OK) return c->latched;
    if (c->P.pn_kry)
        return fail(c, GLD_E_STATE, "gld_profile_steps: not with the Lanczos pair noise (host decisions every step)");
    // untimed steps up to the next noise-block boundary
    if (c->noise_valid && c->host_step < c->noise_end) GLD_TRY(gld_step(c, c->noise_end - c->host_step));
    GLD_TRY(ring_form(c, true, c->st));
    GLD_TRY(refresh_modes(c));
    GLD_TRY(sync_and_check(c));
    c->conv_valid_step = -1;  // the eager steps below leave no next-step projections
    const int T = c->P.T;
    const int64_t blocks = (nsteps + T - 1) / T;
    // Per noise block: a short delay kernel lets the host enqueue the whole
    // block ahead of the device, then every kernel family is bracketed by an
    // event pair, so the device times contain no host launch gaps.
    const bool pcor = c->P.vacf_len > 0 && c->P.pc_nbins > 0;
    const bool pnoise = c->P.pn_deg > 0;
    const size_t nk = 1 + (size_t)T * (4 + (pcor ? 1 : 0) + (pnoise ? 1 : 0));
    std::vector<cudaEvent_t> ev(2 * nk, nullptr);
    std::vector<int> fam(nk);
    gld_status s = GLD_OK;
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) s = fail(c, GLD_E_CUDA, "cudaEventCreate");
    double acc[GLD_PROF_N] = {0};
    int64_t cnt[GLD_PROF_N] = {0};
    for (int64_t b = 0; b < blocks && s == GLD_OK; ++b) {
        if (launch_delay(200000, c->st) != cudaSuccess) {
            s = fail(c, GLD_E_CUDA, "delay kernel");
            break;
        }
        size_t k = 0;
        auto timed = [&](int f, auto&& launch) {
            if (s != GLD_OK) return;
            fam[k] = f;
            if (cudaEventRecord(ev[2 * k], c->st) != cudaSuccess || launch() != cudaSuccess ||
                cudaEventRecord(ev[2 * k + 1], c->st) != cudaSuccess)
                s = fail(c, GLD_E_CUDA, "gld_profile_steps: launch failed");
            ++k;
        };
        timed(GLD_PROF_NOISE, [&] { return launch_noise(c, c->st); });
        c->block_start = c->host_step;
        c->noise_end = c->host_step + T;
        c->noise_valid = true;
        for (int t = 0; t < T; ++t) {
            timed(GLD_PROF_HIST, [&] {
                return launch_memory(c, c->st);
            });
            if (pnoise) timed(GLD_PROF_PNOISE, [&] { return launch_pair_noise(c->P, c->B, c->d_zblk, c->d_bvec, c->st); });
            timed(GLD_PROF_PAIR, [&] { return launch_pair_force_integrate(c->P, c->B, c->st); });
            timed(GLD_PROF_CELL, [&] { return launch_rebuild(c->P, c->B, c->st); });
            timed(GLD_PROF_CFORCE, [&] { return launch_cforce(c->P, c->B, 1, c->st); });  // with the VACF terms
            if (pcor) timed(GLD_PROF_PCORR, [&] { return launch_pcorr(c->P, c->B, c->st); });
            c->last_fr_row = t;
            ++c->host_step;
        }
        if (s == GLD_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s = fail(c, GLD_E_CUDA, "sync");
        for (size_t q = 0; q < k && s == GLD_OK; ++q) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, ev[2 * q], ev[2 * q + 1]) != cudaSuccess) {
                s = fail(c, GLD_E_CUDA, "cudaEventElapsedTime");
                break;
            }
            acc[fam[q]] += t;
            const int pd = c->P.pn_deg;
            cnt[fam[q]] += fam[q] == GLD_PROF_CELL     ? 4
                           : fam[q] == GLD_PROF_NOISE  ? 2 + pd
                           : fam[q] == GLD_PROF_PNOISE ? pd
                                                       : 1;
        }
    }
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    for (int f = 0; f < GLD_PROF_N; ++f) {
        if (ms) ms[f] += acc[f];
        if (launches) launches[f] += cnt[f];
    }
    if (s != GLD_OK) return s;
    return sync_and_check(c);
}

gld_status gld_set_conservative_table(gld_ctx* c, const double* f, int32_t nr, double dr)
{
    if (!c) return GLD_E_INVAL;
    if (nr != 0 && (nr < 2 || !f || !(dr > 0)))
        return fail(c, GLD_E_INVAL, "gld_set_conservative_table: need nr >= 2 points and dr > 0 (or nr = 0)");
    GLD_TRY(sync_and_check(c));
    StepParams& P = c->P;
    float* old = (float*)c->B.fctab;
    c->B.fctab = nullptr;
    P.fc_nr = 0;
    if (old) dfree(c, old);
    if (nr > 0) {
        std::vector<float> h((size_t)nr);
        for (int k = 0; k < nr; ++k) h[(size_t)k] = (float)f[k];
        float* d = (float*)dalloc(c, sizeof(float) * h.size());
        if (!d) return fail(c, GLD_E_NOMEM, "gld_set_conservative_table: allocation failed");
        GLD_CUDA(c, cudaMemcpyAsync(d, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, c->st));
        c->B.fctab = d;
        P.fc_nr = nr;
        P.fc_inv_dr = (float)(1.0 / dr);
    }
    invalidate_graph(c);
    GLD_CUDA(c, launch_cforce(P, c->B, 0, c->st));  // F^C_n at the current positions
    return sync_and_check(c);
}

gld_status gld_separable_terms(const double* table, int32_t nr, int32_t m, int32_t Q, double* f, double* g,
                               double* trunc)
{
    if (!table || nr < 1 || m < 1 || Q < 1 || Q > std::min(nr, m) || !f || !g) return GLD_E_INVAL;
    // Gram matrix of the smaller side, eigenvectors by cyclic Jacobi rotations
    const bool rows = nr <= m;  // G = T T^T (nr x nr) or T^T T (m x m)
    const int d = rows ? nr : m;
    auto at = [&](int k, int j) { return table[(size_t)k * m + j]; };
    std::vector<double> G((size_t)d * d, 0.0), E((size_t)d * d, 0.0);
    for (int a = 0; a < d; ++a)
        for (int b = a; b < d; ++b) {
            double acc = 0.0;
            if (rows)
                for (int j = 0; j < m; ++j) acc += at(a, j) * at(b, j);
            else
                for (int k = 0; k < nr; ++k) acc += at(k, a) * at(k, b);
            G[(size_t)a * d + b] = G[(size_t)b * d + a] = acc;
        }
    for (int a = 0; a < d; ++a) E[(size_t)a * d + a] = 1.0;
    double total = 0.0;
    for (int a = 0; a < d; ++a) total += G[(size_t)a * d + a];
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < d; ++p)
            for (int q = p + 1; q < d; ++q) off += G[(size_t)p * d + q] * G[(size_t)p * d + q];
        if (off <= 1e-30 * total * total) break;
        for (int p = 0; p < d; ++p)
            for (int q = p + 1; q < d; ++q) {
                const double apq = G[(size_t)p * d + q];
                if (apq == 0.0) continue;
                const double theta = (G[(size_t)q * d + q] - G[(size_t)p * d + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < d; ++k) {  // columns p, q
                    const double gp = G[(size_t)k * d + p], gq = G[(size_t)k * d + q];
                    G[(size_t)k * d + p] = cs * gp - sn * gq;
                    G[(size_t)k * d + q] = sn * gp + cs * gq;
                }
                for (int k = 0; k < d; ++k) {  // rows p, q
                    const double gp = G[(size_t)p * d + k], gq = G[(size_t)q * d + k];
                    G[(size_t)p * d + k] = cs * gp - sn * gq;
                    G[(size_t)q * d + k] = sn * gp + cs * gq;
                }
                for (int k = 0; k < d; ++k) {
                    const double ep = E[(size_t)k * d + p], eq = E[(size_t)k * d + q];
                    E[(size_t)k * d + p] = cs * ep - sn * eq;
                    E[(size_t)k * d + q] = sn * ep + cs * eq;
                }
            }
    }
    std::vector<int> order(d);
    for (int a = 0; a < d; ++a) order[a] = a;
    std::sort(order.begin(), order.end(),
              [&](int x, int y) { return G[(size_t)x * d + x] > G[(size_t)y * d + y]; });
    double kept = 0.0;
    for (int q = 0; q < Q; ++q) {
        const int e = order[q];
        const double lam = std::max(G[(size_t)e * d + e], 0.0), sig = std::sqrt(lam);
        kept += lam;
        // one side is the eigenvector, the other the table applied to it over sigma
        for (int k = 0; k < nr; ++k) f[(size_t)q * nr + k] = 0.0;
        for (int j = 0; j < m; ++j) g[(size_t)q * m + j] = 0.0;
        if (rows) {
            for (int k = 0; k < nr; ++k) f[(size_t)q * nr + k] = sig * E[(size_t)k * d + e];
            for (int j = 0; j < m && sig > 0; ++j) {
                double acc = 0.0;
                for (int k = 0; k < nr; ++k) acc += at(k, j) * E[(size_t)k * d + e];
                g[(size_t)q * m + j] = acc / sig;
            }
        } else {
            for (int j = 0; j < m; ++j) g[(size_t)q * m + j] = E[(size_t)j * d + e];
            for (int k = 0; k < nr; ++k) {
                double acc = 0.0;
                for (int j = 0; j < m; ++j) acc += at(k, j) * E[(size_t)j * d + e];
                f[(size_t)q * nr + k] = acc;
            }
        }
    }
    if (trunc) *trunc = total > 0 ? std::sqrt(std::max(total - kept, 0.0) / total) : 0.0;
    return GLD_OK;
}

gld_status gld_set_kernels_table(gld_ctx* c, const double* Ks, const double* Kp, int32_t nr, double dr, int32_t Q,
                                 int32_t conv, double* trunc)
{
    if (!c) return GLD_E_INVAL;
    const int M = c->P.m_max;
    if (!Kp || nr < 2 || !(dr > 0) || Q < 1 || Q > kMaxQ)
        return fail(c, GLD_E_INVAL, "gld_set_kernels_table: need a table of nr >= 2 rows and 1 <= Q <= 4");
    std::vector<double> f((size_t)Q * nr), g((size_t)Q * M);
    double tr = 0.0;
    if (gld_separable_terms(Kp, nr, M, std::min(Q, std::min(nr, M)), f.data(), g.data(), &tr) != GLD_OK)
        return fail(c, GLD_E_INVAL, "gld_set_kernels_table: invalid table");
    if (trunc) *trunc = tr;
    return gld_set_kernels(c, Ks, std::min(Q, std::min(nr, M)), g.data(), f.data(), nr, dr, nullptr, nullptr, 0, conv);
}

gld_status gld_set_perpendicular(gld_ctx* c, const double* fp, const double* fsp)
{
    if (!c) return GLD_E_INVAL;
    if (!c->have_kernels) return fail(c, GLD_E_STATE, "gld_set_perpendicular: set the kernels first");
    StepParams& P = c->P;
    GLD_TRY(sync_and_check(c));
    const int nt = P.Q + P.Qs;
    std::vector<float> tab((size_t)std::max(nt, 1) * P.nr, 0.f);
    bool any = false;
    for (int q = 0; q < P.Q && fp; ++q)
        for (int k = 0; k < P.nr; ++k) {
            tab[(size_t)q * P.nr + k] = (float)fp[(size_t)q * P.nr + k];
            any = any || fp[(size_t)q * P.nr + k] != 0.0;
        }
    for (int q = 0; q < P.Qs && fsp; ++q)
        for (int k = 0; k < P.nr; ++k) {
            tab[(size_t)(P.Q + q) * P.nr + k] = (float)fsp[(size_t)q * P.nr + k];
            any = any || fsp[(size_t)q * P.nr + k] != 0.0;
        }
    dfree(c, c->fptab);
    c->fptab = nullptr;
    c->B.fptab = nullptr;
    P.perp = 0;
    if (any) {
        c->fptab = (float*)dalloc(c, sizeof(float) * tab.size());
        if (!c->fptab) return fail(c, GLD_E_NOMEM, "gld_set_perpendicular: allocation failed");
        GLD_CUDA(c, cudaMemcpyAsync(c->fptab, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice, c->st));
        c->B.fptab = c->fptab;
        P.perp = 1;
    }
    invalidate_graph(c);
    return sync_and_check(c);
}

gld_status gld_pair_noise_filters_on(const double* ks, const double* g, int32_t m_max, double kT, double dt,
                                     double lo, double hi, int32_t degree, int32_t psd_clamp, double* taps,
                                     double* cheb_err)
{
    if (!ks || !g || !taps || m_max < 2 || degree < 1 || degree > kMaxPnDegree || !(lo < hi) || !std::isfinite(lo) ||
        !std::isfinite(hi) || !(dt > 0))
        return GLD_E_INVAL;
    const int M = m_max, K = degree, H = M - 1;
    const long long L = 2LL * M - 1;
    // the interval [cen - rad, cen + rad]; cen is exactly 0 for a symmetric one
    const double cen = 0.5 * (lo + hi), rad = 0.5 * (hi - lo);
    // transforms (Eq. FT) of the noise targets kT a_m K_m / dt (a_0 = 2) of
    // the self kernel and of the pair term's time factor, in FP64
    std::vector<double> hh(M), gh(M);
    double hmax = 0.0, worst = 0.0;
    for (int w = 0; w < M; ++w) {
        double a = 2.0 * ks[0], b = 2.0 * g[0];
        for (int m = 1; m < M; ++m) {
            const double cs = std::cos(2.0 * M_PI * (double)(((long long)w * m) % L) / (double)L);
            a += 2.0 * ks[m] * cs;
            b += 2.0 * g[m] * cs;
        }
        hh[w] = kT / dt * a;
        gh[w] = kT / dt * b;
        // h_w + g_w mu is linear in mu: its minimum over the interval is at an end
        hmax = std::max(hmax, std::fabs(hh[w]) + std::fabs(gh[w]) * std::max(std::fabs(lo), std::fabs(hi)));
        worst = std::min(worst, std::min(hh[w] + gh[w] * lo, hh[w] + gh[w] * hi));
    }
    if (worst < -1e-12 * hmax && !psd_clamp) return GLD_E_NOT_PSD;
    // Chebyshev interpolation of phi_w(x) = sqrt(h_w + g_w (cen + rad x)) on
    // [-1, 1] at degree K, its error on a fine grid, and the filter taps
    // a_k[s] = (c_0k + 2 sum_{w>=1} c_wk cos(2 pi w s / L)) / L
    auto phi = [&](int w, double x) {
        const double gm = cen == 0.0 ? gh[w] * rad * x : gh[w] * (cen + rad * x);
        return std::sqrt(std::max(hh[w] + gm, 0.0));
    };
    const int nc = K + 1;
    std::vector<double> cw((size_t)M * nc);
    double err = 0.0;
    for (int w = 0; w < M; ++w) {
        for (int k = 0; k < nc; ++k) {
            double acc = 0.0;
            for (int j = 0; j < nc; ++j) {
                const double th = M_PI * (j + 0.5) / nc;
                acc += phi(w, std::cos(th)) * std::cos(k * th);
            }
            cw[(size_t)w * nc + k] = (k == 0 ? 1.0 : 2.0) * acc / nc;
        }
        for (int t = 0; t <= 256; ++t) {
            const double x = -1.0 + 2.0 * t / 256.0, th = std::acos(std::min(1.0, std::max(-1.0, x)));
            double p = 0.0;
            for (int k = 0; k < nc; ++k) p += cw[(size_t)w * nc + k] * std::cos(k * th);
            err = std::max(err, std::fabs(p - phi(w, x)));
        }
    }
    double smax = 0.0;  // the largest square root over frequencies and the interval
    for (int w = 0; w < M; ++w) smax = std::max(smax, std::max(phi(w, 1.0), phi(w, -1.0)));
    if (cheb_err) *cheb_err = smax > 0 ? err / smax : 0.0;
    for (int k = 0; k < nc; ++k)
        for (int sg = 0; sg <= 2 * H; ++sg) {
            const long long sh = sg - H;
            double v = cw[k];
            for (int w = 1; w < M; ++w)
                v += 2.0 * cw[(size_t)w * nc + k] *
                     std::cos(2.0 * M_PI * (double)((((long long)w * sh) % L + L) % L) / (double)L);
            taps[(size_t)k * (2 * H + 1) + sg] = v / (double)L;
        }
    return GLD_OK;
}

gld_status gld_pair_noise_filters(const double* ks, const double* g, int32_t m_max, double kT, double dt,
                                  double lambda, int32_t degree, int32_t psd_clamp, double* taps, double* cheb_err)
{
    if (!(lambda > 0)) return GLD_E_INVAL;
    return gld_pair_noise_filters_on(ks, g, m_max, kT, dt, -lambda, lambda, degree, psd_clamp, taps, cheb_err);
}

namespace {

// Ritz extremes of the pair matrix are widened by this fraction of their
// spread on each side to give the interpolation interval (the extremes are
// set by the closest pairs, so they move as pairs meet: one pair at contact
// alone gives +-f(0)); an end is kept this fraction of the way from the
// spectrum to where h_w + g_w mu changes sign for some frequency.
constexpr double kPnMargin = 0.25, kPnPsdGap = 0.05;

// The transforms (Eq. FT) h_w, g_w of kT a_m K_m / dt (a_0 = 2) for the
// self kernel's and the pair term's discrete weights, FP64.
void pn_transforms(const double* ks, const double* g, int M, double kT, double dt, std::vector<double>& hh,
                   std::vector<double>& gh)
{
    const long long L = 2LL * M - 1;
    hh.assign(M, 0.0);
    gh.assign(M, 0.0);
    for (int w = 0; w < M; ++w) {
        double a = 2.0 * ks[0], b = 2.0 * g[0];
        for (int m = 1; m < M; ++m) {
            const double cs = std::cos(2.0 * M_PI * (double)(((long long)w * m) % L) / (double)L);
            a += 2.0 * ks[m] * cs;
            b += 2.0 * g[m] * cs;
        }
        hh[w] = kT / dt * a;
        gh[w] = kT / dt * b;
    }
}

// The kernel forms the Chebyshev form takes: one separable pair term and at
// most one self-difference term, whose time factor must be a multiple c of
// the pair term's (gs = c g: then every transformed matrix is
// h_w 1 + g_w (M_pair + c D_self)); c into *cs.
gld_status pn_check_form(gld_ctx* c, const char* who, int32_t degree, double* cs)
{
    const StepParams& P = c->P;
    *cs = 0.0;
    if (degree < 0 || degree > kMaxPnDegree) return fail(c, GLD_E_INVAL, std::string(who) + ": degree outside [0, 16]");
    if (degree > 0 && !c->have_kernels) return fail(c, GLD_E_STATE, std::string(who) + ": set the kernels first");
    if (degree > 0 && (P.Q != 1 || P.Qs > 1))
        return fail(c, GLD_E_INVAL,
                    std::string(who) + ": needs one separable pair term and at most one self-difference term");
    if (degree > 0 && P.Qs == 1) {
        const int M = P.m_max;
        const double* g = c->wts.data() + M;
        const double* gs = c->wts.data() + 2 * (size_t)M;
        double gg = 0.0, sg = 0.0, smax = 0.0;
        for (int m = 0; m < M; ++m) {
            gg += g[m] * g[m];
            sg += gs[m] * g[m];
            smax = std::max(smax, std::fabs(gs[m]));
        }
        const double ratio = gg > 0 ? sg / gg : 0.0;
        double dev = 0.0;
        for (int m = 0; m < M; ++m) dev = std::max(dev, std::fabs(gs[m] - ratio * g[m]));
        if (dev > 1e-9 * smax)
            return fail(c, GLD_E_INVAL,
                        std::string(who) + ": the self-difference term must have the pair term's time factor (gs = c g)");
        *cs = ratio;
    }
    return GLD_OK;
}

// Installs the Chebyshev form of degree K on the spectral interval [lo, hi]:
// the K + 1 filters, the blocks Z_1 .. Z_K and the Clenshaw vectors.
gld_status pn_install(gld_ctx* c, const char* who, int K, double lo, double hi, double* cheb_err)
{
    StepParams& P = c->P;
    const int M = P.m_max, H = M - 1;
    std::vector<double> td((size_t)(K + 1) * (2 * H + 1));
    const gld_status fs = gld_pair_noise_filters_on(c->wts.data(), c->wts.data() + M, M, c->prm.kT, c->prm.dt, lo, hi,
                                                    K, c->prm.psd_clamp, td.data(), cheb_err);
    if (fs == GLD_E_NOT_PSD)
        return fail(c, GLD_E_NOT_PSD,
                    std::string(who) + ": h_w + g_w mu < 0 for some frequency w and some mu of the spectral interval: "
                                       "positive semi-definiteness of the correlation matrices is not guaranteed "
                                       "(psd_clamp clamps)");
    if (fs != GLD_OK) return fail(c, fs, std::string(who) + ": invalid filter arguments");
    std::vector<float> taps((size_t)(K + 1) * c->la, 0.0f);
    for (int k = 0; k <= K; ++k)
        for (int sg = 0; sg <= 2 * H; ++sg) taps[(size_t)k * c->la + sg] = (float)td[(size_t)k * (2 * H + 1) + sg];
    c->d_pntaps = (float*)dalloc(c, sizeof(float) * taps.size());
    c->d_zblk = (float*)dalloc(c, sizeof(float) * (size_t)K * P.T * 3 * P.n_pad);
    c->d_bvec = (float*)dalloc(c, sizeof(float) * 3 * 3 * (size_t)P.n_pad);
    if (!c->d_pntaps || !c->d_zblk || !c->d_bvec) return fail(c, GLD_E_NOMEM, std::string(who) + ": allocation failed");
    GLD_CUDA(c, cudaMemcpyAsync(c->d_pntaps, taps.data(), sizeof(float) * taps.size(), cudaMemcpyHostToDevice, c->st));
    const double cen = 0.5 * (lo + hi), rad = 0.5 * (hi - lo);
    P.pn_deg = K;
    P.pn_cen = (float)cen;  // exactly 0 for the symmetric bound
    P.pn_lambda = (float)rad;
    P.pn_inv_lambda = (float)(1.0 / rad);
    return GLD_OK;
}

}  // namespace

gld_status gld_set_pair_noise(gld_ctx* c, int32_t degree, double* lambda, double* cheb_err)
{
    if (!c) return GLD_E_INVAL;
    StepParams& P = c->P;
    double cs_ratio = 0.0;
    GLD_TRY(pn_check_form(c, "gld_set_pair_noise", degree, &cs_ratio));
    GLD_TRY(sync_and_check(c));
    pn_release(c);
    kry_release(c);  // one form of pair noise at a time
    invalidate_graph(c);
    GLD_TRY(invalidate_noise(c));
    if (degree == 0) return sync_and_check(c);
    // the bound on the spectrum of the pair matrix: given, or 1.25 x the
    // largest Gershgorin row sum at the current positions
    double lam = lambda ? *lambda : 0.0;
    P.pn_cs = (float)cs_ratio;  // the row sums include the self-difference blocks
    if (!(lam > 0)) {
        c->d_rowsum = (unsigned*)dalloc(c, sizeof(unsigned));
        if (!c->d_rowsum) return fail(c, GLD_E_NOMEM, "gld_set_pair_noise: allocation failed");
        GLD_CUDA(c, launch_pn_rowsum(P, c->B, c->d_rowsum, c->st));
        unsigned bits = 0;
        GLD_CUDA(c, cudaMemcpyAsync(&bits, c->d_rowsum, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st));
        GLD_TRY(sync_and_check(c));
        float mx;
        std::memcpy(&mx, &bits, sizeof(float));
        lam = std::max(1.25 * (double)mx, 1e-6);
    }
    if (lambda) *lambda = lam;
    GLD_TRY(pn_install(c, "gld_set_pair_noise", degree, -lam, lam, cheb_err));
    return sync_and_check(c);
}

gld_status gld_set_pair_noise_on(gld_ctx* c, int32_t degree, double* lo, double* hi, double* cheb_err)
{
    if (!c) return GLD_E_INVAL;
    StepParams& P = c->P;
    double cs_ratio = 0.0;
    GLD_TRY(pn_check_form(c, "gld_set_pair_noise_on", degree, &cs_ratio));
    GLD_TRY(sync_and_check(c));
    pn_release(c);
    kry_release(c);
    invalidate_graph(c);
    GLD_TRY(invalidate_noise(c));
    if (degree == 0) return sync_and_check(c);
    P.pn_cs = (float)cs_ratio;
    bool ok = true;
    c->d_lzv = alloc_n<float>(c, 4 * 3 * (size_t)P.n_pad, ok);
    c->d_lzpart = alloc_n<double>(c, 2 * (size_t)pn_spectrum_blocks(P), ok);
    c->d_lzab = alloc_n<double>(c, 2 * kPnLanczosSteps + 1 + 3, ok);
    if (!ok) {
        pn_release(c);
        return fail(c, GLD_E_NOMEM, "gld_set_pair_noise_on: allocation failed");
    }
    double l = lo ? *lo : 0.0, h = hi ? *hi : 0.0;
    if (!(l < h)) {
        // Ritz extremes at the current positions, widened by kPnMargin of
        // their spread on each side
        double th[3];
        GLD_CUDA(c, launch_pn_spectrum(P, c->B, c->d_lzv, c->d_lzpart, c->d_lzab, 0.0, 0.0, 0,
                                       c->d_lzab + 2 * kPnLanczosSteps + 1, c->st));
        GLD_CUDA(c, cudaMemcpyAsync(th, c->d_lzab + 2 * kPnLanczosSteps + 1, sizeof th, cudaMemcpyDeviceToHost, c->st));
        GLD_TRY(sync_and_check(c));
        const double wd = std::max({th[1] - th[0], 1e-3 * std::max(std::fabs(th[0]), std::fabs(th[1])), 1e-12});
        l = th[0] - kPnMargin * wd;
        h = th[1] + kPnMargin * wd;
        // h_w + g_w mu >= 0 for mu >= mlo (g_w > 0) and mu <= mhi (g_w < 0)
        std::vector<double> hw, gw;
        pn_transforms(c->wts.data(), c->wts.data() + P.m_max, P.m_max, c->prm.kT, c->prm.dt, hw, gw);
        double mlo = -INFINITY, mhi = INFINITY;
        for (int w = 0; w < P.m_max; ++w) {
            if (gw[w] > 0) mlo = std::max(mlo, -hw[w] / gw[w]);
            if (gw[w] < 0) mhi = std::min(mhi, -hw[w] / gw[w]);
        }
        if (th[0] > mlo) l = std::max(l, mlo + kPnPsdGap * (th[0] - mlo));
        if (th[1] < mhi) h = std::min(h, mhi - kPnPsdGap * (mhi - th[1]));
    }
    if (!std::isfinite(l) || !std::isfinite(h)) {
        pn_release(c);
        return fail(c, GLD_E_INVAL, "gld_set_pair_noise_on: the spectral interval is not finite");
    }
    const gld_status st = pn_install(c, "gld_set_pair_noise_on", degree, l, h, cheb_err);
    if (st != GLD_OK) {
        pn_release(c);
        return st;
    }
    P.pn_iv = 1;
    c->pn_lo = l;
    c->pn_hi = h;
    if (lo) *lo = l;
    if (hi) *hi = h;
    return sync_and_check(c);
}

gld_status gld_pair_noise_spectrum(gld_ctx* c, double* out)
{
    if (!c || !out) return GLD_E_INVAL;
    if (!c->P.pn_iv || !c->d_lzab) return fail(c, GLD_E_STATE, "gld_pair_noise_spectrum: gld_set_pair_noise_on is off");
    GLD_TRY(sync_and_check(c));
    GLD_CUDA(c, cudaMemcpyAsync(out, c->d_lzab + 2 * kPnLanczosSteps + 1, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                                c->st));
    GLD_CUDA(c, cudaStreamSynchronize(c->st));
    out[3] = c->pn_lo;
    out[4] = c->pn_hi;
    return GLD_OK;
}

gld_status gld_set_pair_noise_lanczos(gld_ctx* c, double tol, int32_t kmax, int32_t window)
{
    if (!c) return GLD_E_INVAL;
    StepParams& P = c->P;
    if (tol > 0 && !c->have_kernels) return fail(c, GLD_E_STATE, "gld_set_pair_noise_lanczos: set the kernels first");
    if (tol > 0 && (kmax < 2 || kmax > 64 || !(tol < 1.0) || (window != 0 && window != 1)))
        return fail(c, GLD_E_INVAL, "gld_set_pair_noise_lanczos: need 0 < tol < 1, 2 <= kmax <= 64, window 0 or 1");
    GLD_TRY(sync_and_check(c));
    kry_release(c);
    invalidate_graph(c);
    if (!(tol > 0)) return sync_and_check(c);
    if (window && P.T != kMaxNoiseBlock)
        return fail(c, GLD_E_INVAL, "gld_set_pair_noise_lanczos: the time window needs 64-step noise blocks");
    pn_release(c);  // the Chebyshev form is replaced
    GLD_TRY(invalidate_noise(c));  // the current block's rows are regenerated
    auto& K = c->kry;
    const int M = P.m_max, Mc = (M + 31) & ~31, Mp = window ? 2 * Mc : Mc, nacc = P.nacc;
    const long long L = 2LL * M - 1;
    if (!kry_fits(P, Mp))
        return fail(c, GLD_E_INVAL, "gld_set_pair_noise_lanczos: m_max too large for the transform's shared memory");
    auto freq = [&](int col) { return col < Mc ? col : col - Mc; };  // the frequency of a column
    auto phase = [&](long long a) { return 2.0 * M_PI * (double)(a % L) / (double)L; };
    // transforms (Eq. FT) of kT a_m / dt times each discrete time factor:
    // a_w (self), g_qw (pair terms), gs_qw (self-difference terms), FP64; the
    // sine columns take their frequency's values
    std::vector<double> wc((size_t)nacc * Mp, 0.0);
    const double f0 = c->prm.kT / c->prm.dt;
    for (int a = 0; a < nacc; ++a) {
        const double* wt = c->wts.data() + (size_t)a * M;
        for (int w = 0; w < M; ++w) {
            double v = 2.0 * wt[0];
            for (int m = 1; m < M; ++m) v += 2.0 * wt[m] * std::cos(phase((long long)w * m));
            wc[(size_t)a * Mp + w] = f0 * v;
            if (window) wc[(size_t)a * Mp + Mc + w] = f0 * v;
        }
    }
    // cos (sin) of 2 pi w s / L for s = 0 .. m_max - 1: the transforms of the
    // window; columns of frequencies >= m_max zero
    std::vector<float> cosT((size_t)M * Mp, 0.f);
    for (int sg = 0; sg < M; ++sg)
        for (int col = 0; col < Mp; ++col)
            if (freq(col) < M)
                cosT[(size_t)sg * Mp + col] = (float)(col < Mc ? std::cos(phase((long long)freq(col) * sg))
                                                               : std::sin(phase((long long)freq(col) * sg)));
    // the window's row weights: (1 or 2) cos(2 pi w m / L) and 2 sin(2 pi w m / L)
    std::vector<float> wgt;
    if (window) {
        wgt.assign((size_t)Mp * kMaxNoiseBlock, 0.f);
        for (int col = 0; col < Mp; ++col) {
            const int w = freq(col);
            if (w >= M || (col >= Mc && w == 0)) continue;
            for (int m = 0; m < kMaxNoiseBlock; ++m)
                wgt[(size_t)col * kMaxNoiseBlock + m] =
                    (float)(col < Mc ? (w == 0 ? 1.0 : 2.0) * std::cos(phase((long long)w * m))
                                     : 2.0 * std::sin(phase((long long)w * m)));
        }
    }
    const size_t vs = 3 * (size_t)P.n_pad * Mp;
    bool ok = true;
    K.V = alloc_n<float>(c, (size_t)(kmax + 1) * vs, ok);
    K.Y = alloc_n<float>(c, vs, ok);
    K.cf = alloc_n<float>(c, (size_t)Mp * (kmax + 1), ok);
    K.cosT = alloc_n<float>(c, cosT.size(), ok);
    if (window) K.wgt = alloc_n<float>(c, wgt.size(), ok);
    K.part = alloc_n<double>(c, (size_t)kry_part_blocks(P) * Mp, ok);
    K.alpha = alloc_n<double>(c, (size_t)(kmax + 1) * Mp, ok);
    K.beta = alloc_n<double>(c, (size_t)(kmax + 1) * Mp, ok);
    K.wc = alloc_n<double>(c, wc.size(), ok);
    K.alive = alloc_n<int>(c, Mp, ok);
    if (!ok) {
        kry_release(c);
        return fail(c, GLD_E_NOMEM, "gld_set_pair_noise_lanczos: allocation failed");
    }
    GLD_CUDA(c, cudaMemcpyAsync(K.wc, wc.data(), sizeof(double) * wc.size(), cudaMemcpyHostToDevice, c->st));
    GLD_CUDA(c, cudaMemcpyAsync(K.cosT, cosT.data(), sizeof(float) * cosT.size(), cudaMemcpyHostToDevice, c->st));
    if (window)
        GLD_CUDA(c, cudaMemcpyAsync(K.wgt, wgt.data(), sizeof(float) * wgt.size(), cudaMemcpyHostToDevice, c->st));
    K.M = M;
    K.Mp = Mp;
    K.Mc = Mc;
    K.window = window;
    K.kmax = kmax;
    K.tol = tol;
    K.last_iters = 0;
    K.last_change = 0.0;
    P.pn_kry = 1;
    return sync_and_check(c);
}

gld_status gld_set_pair_noise_krylov(gld_ctx* c, double tol, int32_t kmax)
{
    return gld_set_pair_noise_lanczos(c, tol, kmax, 0);
}

gld_status gld_set_memory_modes(gld_ctx* c, int32_t nmodes, const double* rate, const double* omega)
{
    if (!c) return GLD_E_INVAL;
    if (!c->have_kernels) return fail(c, GLD_E_STATE, "gld_set_memory_modes: set the kernels first");
    StepParams& P = c->P;
    if (nmodes == 0) {  // back to the ring convolution
        GLD_TRY(sync_and_check(c));
        P.nmodes = 0;
        invalidate_graph(c);
        return GLD_OK;
    }
    if (nmodes < 0 || nmodes > kMaxModes || !rate || !omega)
        return fail(c, GLD_E_INVAL, "gld_set_memory_modes: 1..8 modes with rates and frequencies");
    for (int k = 0; k < nmodes; ++k)
        if (!(rate[k] > 0) || !std::isfinite(rate[k]) || !std::isfinite(omega[k]) || omega[k] < 0)
            return fail(c, GLD_E_INVAL, "gld_set_memory_modes: need rate > 0 and omega >= 0");
    const int H = P.H, M = P.m_max, na = P.nacc;
    const double dt = c->prm.dt;
    // basis functions Re z_k^m (and Im z_k^m for omega_k != 0), m = 1..H
    std::vector<std::vector<double>> cols;
    std::vector<int> col_mode, col_im;
    for (int k = 0; k < nmodes; ++k)
        for (int im = 0; im < (omega[k] != 0.0 ? 2 : 1); ++im) {
            std::vector<double> v(H);
            for (int m = 1; m <= H; ++m) {
                const double mag = std::exp(-rate[k] * dt * m), ph = omega[k] * dt * m;
                v[m - 1] = mag * (im ? std::sin(ph) : std::cos(ph));
            }
            cols.push_back(v);
            col_mode.push_back(k);
            col_im.push_back(im);
        }
    // least squares through modified Gram-Schmidt: Phi = Q R
    const int nb = (int)cols.size();
    std::vector<std::vector<double>> Qm = cols;
    std::vector<double> R((size_t)nb * nb, 0.0);
    for (int j = 0; j < nb; ++j) {
        const double n0 = std::sqrt(std::inner_product(cols[j].begin(), cols[j].end(), cols[j].begin(), 0.0));
        for (int i = 0; i < j; ++i) {
            const double r = std::inner_product(Qm[i].begin(), Qm[i].end(), Qm[j].begin(), 0.0);
            R[(size_t)i * nb + j] = r;
            for (int m = 0; m < H; ++m) Qm[j][m] -= r * Qm[i][m];
        }
        const double nj = std::sqrt(std::inner_product(Qm[j].begin(), Qm[j].end(), Qm[j].begin(), 0.0));
        if (!(nj > 1e-10 * n0)) return fail(c, GLD_E_INVAL, "gld_set_memory_modes: modes are not independent");
        R[(size_t)j * nb + j] = nj;
        for (int m = 0; m < H; ++m) Qm[j][m] /= nj;
    }
    std::vector<float2> hw((size_t)na * nmodes, make_float2(0.f, 0.f));
    double worst = 0.0;
    for (int a = 0; a < na; ++a) {
        const double* w = c->wts.data() + (size_t)a * M + 1;
        std::vector<double> x(nb, 0.0);
        for (int j = 0; j < nb; ++j) x[j] = std::inner_product(Qm[j].begin(), Qm[j].end(), w, 0.0);
        for (int j = nb - 1; j >= 0; --j) {
            for (int i = j + 1; i < nb; ++i) x[j] -= R[(size_t)j * nb + i] * x[i];
            x[j] /= R[(size_t)j * nb + j];
        }
        double wmax = 0.0, res = 0.0;
        for (int m = 0; m < H; ++m) {
            double f = 0.0;
            for (int j = 0; j < nb; ++j) f += x[j] * cols[j][m];
            res = std::max(res, std::fabs(f - w[m]));
            wmax = std::max(wmax, std::fabs(w[m]));
        }
        const double rel = wmax > 0 ? res / wmax : res;
        worst = std::max(worst, rel);
        for (int j = 0; j < nb; ++j) {
            float2& e = hw[(size_t)a * nmodes + col_mode[j]];
            (col_im[j] ? e.y : e.x) = (float)x[j];
        }
    }
    if (worst > 1e-9) {
        char buf[160];
        std::snprintf(buf, sizeof buf,
                      "gld_set_memory_modes: the kernels are not sums of these modes (relative residual %.3g)", worst);
        return fail(c, GLD_E_INVAL, buf);
    }
    std::vector<float4> hc(nmodes);
    std::vector<double> hz(2 * (size_t)nmodes);
    for (int k = 0; k < nmodes; ++k) {
        const double mag = std::exp(-rate[k] * dt), ph = omega[k] * dt;
        const double magH = std::exp(-rate[k] * dt * H), phH = omega[k] * dt * H;
        hz[2 * k] = mag * std::cos(ph);
        hz[2 * k + 1] = mag * std::sin(ph);
        hc[k] = make_float4((float)hz[2 * k], (float)hz[2 * k + 1], (float)(magH * std::cos(phH)),
                            (float)(magH * std::sin(phH)));
    }
    GLD_TRY(sync_and_check(c));
    dfree(c, c->d_mcoef);
    dfree(c, c->d_mw);
    dfree(c, c->d_Y);
    dfree(c, c->d_mz);
    c->d_mcoef = nullptr;
    c->d_mw = nullptr;
    c->d_Y = nullptr;
    c->d_mz = nullptr;
    P.nmodes = 0;
    bool ok = true;
    c->d_mcoef = alloc_n<float4>(c, (size_t)nmodes, ok);
    c->d_mw = alloc_n<float2>(c, hw.size(), ok);
    c->d_Y = alloc_n<float2>(c, (size_t)nmodes * 3 * P.n_pad, ok);
    c->d_mz = alloc_n<double>(c, hz.size(), ok);
    if (!ok) return fail(c, GLD_E_NOMEM, "gld_set_memory_modes: allocation failed");
    GLD_CUDA(c, cudaMemcpyAsync(c->d_mcoef, hc.data(), sizeof(float4) * hc.size(), cudaMemcpyHostToDevice, c->st));
    GLD_CUDA(c, cudaMemcpyAsync(c->d_mw, hw.data(), sizeof(float2) * hw.size(), cudaMemcpyHostToDevice, c->st));
    GLD_CUDA(c, cudaMemcpyAsync(c->d_mz, hz.data(), sizeof(double) * hz.size(), cudaMemcpyHostToDevice, c->st));
    P.nmodes = nmodes;
    c->modes_dirty = true;  // the sums are built from the ring before the next step
    invalidate_graph(c);
    return sync_and_check(c);
}

gld_status gld_set_pair_correlation(gld_ctx* c, int32_t nbins, double r_max)
{
    if (!c) return GLD_E_INVAL;
    StepParams& P = c->P;
    if (P.vacf_len <= 0) return fail(c, GLD_E_INVAL, "gld_set_pair_correlation: the VACF (vacf_len > 0) is off");
    if (nbins < 1 || !(r_max > 0) || r_max > c->prm.r_c)
        return fail(c, GLD_E_INVAL, "gld_set_pair_correlation: need nbins >= 1 and 0 < r_max <= r_c");
    if ((long long)P.n_os * nbins > kPcMaxOriginBins)
        return fail(c, GLD_E_INVAL, "gld_set_pair_correlation: origins in flight x bins exceeds 2048");
    GLD_TRY(sync_and_check(c));
    dfree(c, c->B.pc_step);
    dfree(c, c->B.pc_sa);
    dfree(c, c->B.pc_sc);
    dfree(c, c->B.pc_n);
    c->B.pc_step = nullptr;
    c->B.pc_sa = c->B.pc_sc = nullptr;
    c->B.pc_n = nullptr;
    P.pc_nbins = 0;
    bool ok = true;
    const size_t cells = (size_t)P.vacf_len * nbins;
    c->B.pc_step = alloc_n<long long>(c, 2 * 3 * (size_t)P.n_os * nbins, ok);
    c->B.pc_sa = alloc_n<double>(c, cells, ok);
    c->B.pc_sc = alloc_n<double>(c, cells, ok);
    c->B.pc_n = alloc_n<long long>(c, cells, ok);
    if (!ok) return fail(c, GLD_E_NOMEM, "gld_set_pair_correlation: allocation failed");
    P.pc_nbins = nbins;
    P.pc_rmax2 = (float)(r_max * r_max);
    P.pc_inv_dr = (float)(nbins / r_max);
    const int zero[2] = {0, 0};  // no sums pending from an earlier setting
    GLD_CUDA(c, cudaMemcpyAsync(&c->B.ctrl->pc_pending, zero, sizeof(int), cudaMemcpyHostToDevice, c->st));
    GLD_CUDA(c, cudaMemcpyAsync(&c->B.ctrl->pc_pv_nact, zero, sizeof(int), cudaMemcpyHostToDevice, c->st));
    invalidate_graph(c);  // the step now has one more kernel
    return sync_and_check(c);
}

gld_status gld_pair_correlation(gld_ctx* c, double* ca, double* cc, int64_t* counts)
{
    if (!c) return GLD_E_INVAL;
    const StepParams& P = c->P;
    if (P.pc_nbins <= 0) return fail(c, GLD_E_STATE, "gld_pair_correlation: not enabled");
    if (c->latched == GLD_OK) GLD_CUDA(c, launch_pcorr_flush(P, c->B, c->st));
    GLD_TRY(sync_and_check(c));
    const size_t cells = (size_t)P.vacf_len * P.pc_nbins;
    std::vector<double> sa(cells), sc(cells);
    std::vector<long long> sn(cells);
    GLD_CUDA(c, cudaMemcpy(sa.data(), c->B.pc_sa, sizeof(double) * cells, cudaMemcpyDeviceToHost));
    GLD_CUDA(c, cudaMemcpy(sc.data(), c->B.pc_sc, sizeof(double) * cells, cudaMemcpyDeviceToHost));
    GLD_CUDA(c, cudaMemcpy(sn.data(), c->B.pc_n, sizeof(long long) * cells, cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < cells; ++k) {
        if (ca) ca[k] = sn[k] > 0 ? sa[k] / (2.0 * (double)sn[k]) : 0.0;
        if (cc) cc[k] = sn[k] > 0 ? sc[k] / (2.0 * (double)sn[k]) : 0.0;
        if (counts) counts[k] = sn[k];
    }
    return GLD_OK;
}

// Checkpoint of the observables.  Layout of the blob (native byte order):
// header, VACF sums [L] f64, counts [L] i64, origins so far (i64), origin
// velocities [n_os][n][4] f32 in the caller's particle order, then, when the
// pair correlations are on, their sums a and c [L][nbins] f64 and counts
// [L][nbins] i64.  Pending per-step partials are folded in first (the same
// additions, in the same order, as the next VACF launch would make).
namespace {
struct ObsHeader {
    uint64_t magic;
    int32_t version, n, vacf_len, vacf_stride, n_os, pc_nbins;
    int64_t vacf_burnin, step;
};
constexpr uint64_t kObsMagic = 0x31534256444C47ull;  // "GLDVBS1"

size_t obs_bytes(const StepParams& P)
{
    const size_t L = (size_t)std::max(P.vacf_len, 0), cells = L * (size_t)std::max(P.pc_nbins, 0);
    return sizeof(ObsHeader) + 16 * L + 8 + 16 * (size_t)P.n_os * P.n + 24 * cells;
}
}  // namespace

gld_status gld_save_observables(gld_ctx* c, void* buf, int64_t cap, int64_t* size)
{
    if (!c || !size || cap < 0) return GLD_E_INVAL;
    const StepParams& P = c->P;
    const size_t need = obs_bytes(P);
    *size = (int64_t)need;
    if (!buf) return GLD_OK;
    if ((size_t)cap < need) return fail(c, GLD_E_INVAL, "gld_save_observables: buffer smaller than *size");
    if (c->latched == GLD_OK && P.vacf_len > 0) GLD_CUDA(c, launch_vacf_flush(P, c->B, c->st));
    if (c->latched == GLD_OK && P.pc_nbins > 0) GLD_CUDA(c, launch_pcorr_flush(P, c->B, c->st));
    GLD_TRY(sync_and_check(c));
    unsigned char* o = (unsigned char*)buf;
    ObsHeader h{kObsMagic, 1, P.n, P.vacf_len, P.vacf_stride, P.n_os, P.pc_nbins, P.vacf_burnin, c->host_step};
    std::memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    const size_t L = (size_t)std::max(P.vacf_len, 0);
    if (L > 0) {
        GLD_CUDA(c, cudaMemcpy(o, c->B.csum, 8 * L, cudaMemcpyDeviceToHost));
        GLD_CUDA(c, cudaMemcpy(o + 8 * L, c->B.ccnt, 8 * L, cudaMemcpyDeviceToHost));
        GLD_CUDA(c, cudaMemcpy(o + 16 * L, c->B.norig, 8, cudaMemcpyDeviceToHost));
    } else {
        std::memset(o + 16 * L, 0, 8);
    }
    o += 16 * L + 8;
    if (P.n_os > 0) {
        std::vector<float4> v((size_t)P.n_os * P.n);
        GLD_CUDA(c, cudaMemcpy(v.data(), c->B.vorig, sizeof(float4) * v.size(), cudaMemcpyDeviceToHost));
        float4* dst = (float4*)o;  // caller's order
        for (int q = 0; q < P.n_os; ++q)
            for (int i = 0; i < P.n; ++i) std::memcpy(dst + (size_t)q * P.n + c->int2ext[i], &v[(size_t)q * P.n + i], 16);
        o += 16 * v.size();
    }
    if (P.pc_nbins > 0) {
        const size_t cells = L * P.pc_nbins;
        GLD_CUDA(c, cudaMemcpy(o, c->B.pc_sa, 8 * cells, cudaMemcpyDeviceToHost));
        GLD_CUDA(c, cudaMemcpy(o + 8 * cells, c->B.pc_sc, 8 * cells, cudaMemcpyDeviceToHost));
        GLD_CUDA(c, cudaMemcpy(o + 16 * cells, c->B.pc_n, 8 * cells, cudaMemcpyDeviceToHost));
    }
    return GLD_OK;
}

gld_status gld_load_observables(gld_ctx* c, const void* buf, int64_t size)
{
    if (!c || !buf || size < (int64_t)sizeof(ObsHeader)) return GLD_E_INVAL;
    const StepParams& P = c->P;
    ObsHeader h{};
    std::memcpy(&h, buf, sizeof(h));
    if (h.magic != kObsMagic || h.version != 1 || (size_t)size != obs_bytes(P) || h.n != P.n ||
        h.vacf_len != P.vacf_len || h.vacf_stride != P.vacf_stride || h.n_os != P.n_os ||
        h.pc_nbins != P.pc_nbins || h.vacf_burnin != P.vacf_burnin)
        return fail(c, GLD_E_INVAL, "gld_load_observables: the blob belongs to another configuration");
    if (h.step != c->host_step)
        return fail(c, GLD_E_STATE, "gld_load_observables: set the step index of the checkpoint first");
    GLD_TRY(sync_and_check(c));
    const unsigned char* o = (const unsigned char*)buf + sizeof(h);
    const size_t L = (size_t)std::max(P.vacf_len, 0);
    if (L > 0) {
        GLD_CUDA(c, cudaMemcpy(c->B.csum, o, 8 * L, cudaMemcpyHostToDevice));
        GLD_CUDA(c, cudaMemcpy(c->B.ccnt, o + 8 * L, 8 * L, cudaMemcpyHostToDevice));
        GLD_CUDA(c, cudaMemcpy(c->B.norig, o + 16 * L, 8, cudaMemcpyHostToDevice));
    }
    o += 16 * L + 8;
    if (P.n_os > 0) {
        std::vector<float4> v((size_t)P.n_os * P.n);
        const float4* src = (const float4*)o;
        for (int q = 0; q < P.n_os; ++q)
            for (int i = 0; i < P.n; ++i) std::memcpy(&v[(size_t)q * P.n + i], src + (size_t)q * P.n + c->int2ext[i], 16);
        GLD_CUDA(c, cudaMemcpy(c->B.vorig, v.data(), sizeof(float4) * v.size(), cudaMemcpyHostToDevice));
        o += 16 * v.size();
    }
    if (P.pc_nbins > 0) {
        const size_t cells = L * P.pc_nbins;
        GLD_CUDA(c, cudaMemcpy(c->B.pc_sa, o, 8 * cells, cudaMemcpyHostToDevice));
        GLD_CUDA(c, cudaMemcpy(c->B.pc_sc, o + 8 * cells, 8 * cells, cudaMemcpyHostToDevice));
        GLD_CUDA(c, cudaMemcpy(c->B.pc_n, o + 16 * cells, 8 * cells, cudaMemcpyHostToDevice));
        GLD_CUDA(c, cudaMemsetAsync(c->B.pc_step, 0, sizeof(long long) * 2 * 3 * (size_t)P.n_os * P.pc_nbins, c->st));
    }
    // nothing pending from before the checkpoint
    const int zero = 0;
    GLD_CUDA(c, cudaMemcpyAsync(&c->B.ctrl->vacf_pending, &zero, sizeof(int), cudaMemcpyHostToDevice, c->st));
    GLD_CUDA(c, cudaMemcpyAsync(&c->B.ctrl->pv_nact, &zero, sizeof(int), cudaMemcpyHostToDevice, c->st));
    GLD_CUDA(c, cudaMemcpyAsync(&c->B.ctrl->pc_pending, &zero, sizeof(int), cudaMemcpyHostToDevice, c->st));
    GLD_CUDA(c, cudaMemcpyAsync(&c->B.ctrl->pc_pv_nact, &zero, sizeof(int), cudaMemcpyHostToDevice, c->st));
    return sync_and_check(c);
}

const char* gld_last_error(const gld_ctx* c) { return c ? c->msg.c_str() : "null context"; }

gld_status gld_destroy(gld_ctx* c)
{
    if (!c) return GLD_E_INVAL;
    if (c->st || c->cap) cudaStreamSynchronize(c->st);
    invalidate_graph(c);
    for (void* p : c->allocs) {
        if (c->prm.free) c->prm.free(p, c->prm.stream, c->prm.alloc_user);
        else cudaFree(p);
    }
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->cap2) cudaStreamDestroy(c->cap2);
    if (c->cap3) cudaStreamDestroy(c->cap3);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    delete c;
    return GLD_OK;
}

gld_status gld_get_bytes(gld_ctx* c, int64_t* bytes)
{
    if (!c || !bytes) return GLD_E_INVAL;
    *bytes = (int64_t)c->bytes;
    return GLD_OK;
}

gld_status gld_bytes_needed(const gld_params* p, int32_t Q, int32_t Qs, int32_t nr, int64_t* bytes)
{
    if (!p || !bytes || p->n < 1 || p->m_max < 2 || !(p->box > 0) || !(p->r_c > 0) || Q < 0 || Qs < 0) return GLD_E_INVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GLD_E_CUDA;
    *bytes = (int64_t)ctx_bytes_needed(p, Q, Qs, nr, sms);
    return GLD_OK;
}

gld_status gld_philox_dev(const uint32_t* ctr, const uint32_t key[2], uint32_t* out, int64_t n, void* stream)
{
    if (!key || n < 0 || (n > 0 && (!ctr || !out))) return GLD_E_INVAL;
    return launch_philox(ctr, key[0], key[1], out, n, (cudaStream_t)stream) == cudaSuccess ? GLD_OK : GLD_E_CUDA;
}

gld_status gld_gauss3_dev(uint64_t seed, const uint32_t* particle, const int64_t* time, uint32_t stream_id,
                          float* out, int64_t n, void* stream)
{
    if (n < 0 || (n > 0 && (!particle || !time || !out))) return GLD_E_INVAL;
    return launch_gauss3((uint32_t)seed, (uint32_t)(seed >> 32), particle, (const long long*)time, stream_id, out, n,
                         (cudaStream_t)stream) == cudaSuccess
               ? GLD_OK
               : GLD_E_CUDA;
}

gld_status gld_hist_conv_dev(const void* ring, int32_t bf16, int32_t n_pad, int32_t m_max, int64_t step,
                             const float* coef, int32_t nacc, float* out, int32_t kahan, void* stream)
{
    if (!ring || !coef || !out || n_pad <= 0 || n_pad % 32 || m_max < 2 || nacc < 1 || nacc > kMaxAcc ||
        ((uintptr_t)ring & 15) || ((uintptr_t)out & 15))
        return GLD_E_INVAL;
    return launch_hist_conv(ring, bf16, n_pad, m_max, nullptr, step, coef, nacc, out, kahan, (cudaStream_t)stream) ==
                   cudaSuccess
               ? GLD_OK
               : GLD_E_CUDA;
}

// ---- batches of independent systems ----------------------------------------


namespace {

gld_status bfail(gld_batch* b, gld_status s, const std::string& m)
{
    if (b) b->msg = m;
    return s;
}

// Executable graphs are destroyed only after their last launch finished.
void batch_reap(gld_batch* b, bool all)
{
    size_t keep = 0;
    for (auto& r : b->retired) {
        if (all || cudaEventQuery(r.second) == cudaSuccess) {
            if (all) cudaEventSynchronize(r.second);
            cudaGraphExecDestroy(r.first);
            cudaEventDestroy(r.second);
        } else {
            b->retired[keep++] = r;
        }
    }
    b->retired.resize(keep);
}

void batch_drop_graph(gld_batch* b)
{
    if (b->gexec) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventRecord(e, b->st) == cudaSuccess) {
            b->retired.push_back({b->gexec, e});
        } else {  // cannot track it: wait
            if (e) cudaEventDestroy(e);
            cudaStreamSynchronize(b->st);
            cudaGraphExecDestroy(b->gexec);
        }
    }
    b->gexec = nullptr;
    batch_reap(b, false);
}

// Convolution schedules: 0 tiles of 256 columns, longest memories first;
// 1 tiles of 128 columns, longest first; 2 tiles of 256 in member order;
// 3 one CTA of 256 per member (block-per-replica).
void conv_tiles(const std::vector<gld_ctx*>& ms, int schedule, std::vector<Tile>& out, int* block)
{
    *block = schedule == 1 ? 128 : 256;
    std::vector<int> idx(ms.size());
    for (size_t k = 0; k < ms.size(); ++k) idx[k] = (int)k;
    if (schedule == 0 || schedule == 1)
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return ms[a]->P.H > ms[b]->P.H; });
    for (int m : idx) {
        const long long cols = 3LL * ms[m]->P.n_pad / (ms[m]->P.hist_bf16 ? 8 : 4);
        const int nb = schedule == 3 ? 1 : (int)((cols + *block - 1) / *block);
        for (int b = 0; b < nb; ++b) out.push_back(Tile{m, b, nb, 0});
    }
}

gld_status batch_plan(gld_batch* b, int schedule)
{
    const auto& ms = b->members;
    std::vector<SysDesc> desc(ms.size());
    std::vector<Tile> pair, part, cell, vacf, conv, fir, cf;
    BatchPlan& P = b->plan;
    P = BatchPlan{};
    P.pair_fast = 1;
    for (const gld_ctx* c : ms) P.pair_fast &= (c->P.Q == 1 && c->P.Qs == 0 && !c->P.perp) ? 1 : 0;
    const int pair_per_block = P.pair_fast ? kBatchPairBlock / kBatchPairLanes : kBatchPairBlock;
    for (size_t m = 0; m < ms.size(); ++m) {
        gld_ctx* c = ms[m];
        SysDesc& d = desc[m];
        d.P = c->P;
        d.P.wsplit = 0;  // the batched filter reads the FP32 ring
        d.B = c->B;
        d.coef = c->coef;
        d.W = c->W;
        d.taps = c->P.pn_deg > 0 ? c->d_pntaps : c->Acp;  // row 0 of the pair-noise filters
        d.ntaps = fir_taps_len(c->P.H);
        d.pntaps = c->d_pntaps;
        d.zblk = c->d_zblk;
        d.bvec = c->d_bvec;
        d.pn_la = c->la;
        P.pn_kmax = std::max(P.pn_kmax, c->P.pn_deg);
        d.k0 = (uint32_t)c->prm.seed;
        d.k1 = (uint32_t)(c->prm.seed >> 32);
        d.int2ext = c->d_int2ext;
        d.nb_pair = (c->P.n + pair_per_block - 1) / pair_per_block;
        d.nb_part = (c->P.n + kBatchPartBlock - 1) / kBatchPartBlock;
        d.nb_cf = (int)(((long long)c->P.n * kBatchCforceLanes + kBatchCforceBlock - 1) / kBatchCforceBlock);
        d.nb_cell = (c->B.ncells + kBatchCellChunk - 1) / kBatchCellChunk;
        d.nb_vacf = c->P.vacf_len > 0 ? c->B.vacf_gx : 0;
        d.nb_conv = 0;
        d.nb_fir = (int)((3LL * c->P.n_pad + kBatchFirStreams - 1) / kBatchFirStreams);
        for (int k = 0; k < d.nb_pair; ++k) pair.push_back(Tile{(int)m, k, d.nb_pair, 0});
        for (int k = 0; k < d.nb_part; ++k) part.push_back(Tile{(int)m, k, d.nb_part, 0});
        for (int k = 0; k < d.nb_cf; ++k) cf.push_back(Tile{(int)m, k, d.nb_cf, 0});
        for (int k = 0; k < d.nb_cell; ++k) cell.push_back(Tile{(int)m, k, d.nb_cell, 0});
        for (int k = 0; k < d.nb_vacf; ++k) vacf.push_back(Tile{(int)m, k, d.nb_vacf, 0});
        for (int k = 0; k < d.nb_fir; ++k) fir.push_back(Tile{(int)m, k, d.nb_fir, 0});
        P.max_H = std::max(P.max_H, c->P.H);
        P.max_n = std::max(P.max_n, c->P.n);
        P.max_ntaps = std::max(P.max_ntaps, d.ntaps);
        P.vacf_no = std::max(P.vacf_no, c->P.n_os);
    }
    conv_tiles(ms, schedule < 0 ? 0 : schedule, conv, &P.conv_block);

    if (!ms.empty()) {
        P.nacc = ms[0]->P.nacc;
        P.bf16 = ms[0]->P.hist_bf16;
        P.kahan = ms[0]->prm.kahan;
    }
    std::vector<Tile> all;
    auto append = [&](std::vector<Tile>& v, int* n) {
        *n = (int)v.size();
        const size_t off = all.size();
        all.insert(all.end(), v.begin(), v.end());
        return off;
    };
    const size_t o_pair = append(pair, &P.n_pair), o_part = append(part, &P.n_part), o_cell = append(cell, &P.n_cell),
                 o_vacf = append(vacf, &P.n_vacf), o_conv = append(conv, &P.n_conv), o_fir = append(fir, &P.n_fir),
                 o_cf = append(cf, &P.n_cf);
    b->snap = desc;
    // One upload of descriptors and tiles through pinned staging, ordered on
    // the batch's stream after the blocks already queued (which keep reading
    // the previous plan until they finish); no host synchronisation.
    const size_t desc_bytes = (sizeof(SysDesc) * desc.size() + 255) & ~(size_t)255;
    const size_t bytes = desc_bytes + sizeof(Tile) * all.size();
    if (bytes > b->plan_cap) {
        if (b->d_plan) cudaFreeAsync(b->d_plan, b->st);
        b->d_plan = nullptr;
        b->plan_cap = std::max(bytes, 2 * b->plan_cap);
        if (cudaMallocAsync((void**)&b->d_plan, b->plan_cap, b->st) != cudaSuccess) {
            b->plan_cap = 0;
            return bfail(b, GLD_E_NOMEM, "batch plan allocation");
        }
    }
    const int k = b->stage_k ^= 1;
    if (b->stage_ev[k] && cudaEventSynchronize(b->stage_ev[k]) != cudaSuccess)
        return bfail(b, GLD_E_CUDA, "batch plan staging");
    if (bytes > b->stage_cap[k]) {
        if (b->h_stage[k]) cudaFreeHost(b->h_stage[k]);
        b->h_stage[k] = nullptr;
        b->stage_cap[k] = std::max(bytes, 2 * b->stage_cap[k]);
        if (cudaHostAlloc((void**)&b->h_stage[k], b->stage_cap[k], cudaHostAllocDefault) != cudaSuccess) {
            b->stage_cap[k] = 0;
            return bfail(b, GLD_E_NOMEM, "batch plan staging allocation");
        }
    }
    if (!b->stage_ev[k] && cudaEventCreateWithFlags(&b->stage_ev[k], cudaEventDisableTiming) != cudaSuccess)
        return bfail(b, GLD_E_CUDA, "batch plan event");
    std::memcpy(b->h_stage[k], desc.data(), sizeof(SysDesc) * desc.size());
    std::memcpy(b->h_stage[k] + desc_bytes, all.data(), sizeof(Tile) * all.size());
    if (cudaMemcpyAsync(b->d_plan, b->h_stage[k], bytes, cudaMemcpyHostToDevice, b->st) != cudaSuccess ||
        cudaEventRecord(b->stage_ev[k], b->st) != cudaSuccess)
        return bfail(b, GLD_E_CUDA, "batch plan upload");
    const Tile* t0 = (const Tile*)(b->d_plan + desc_bytes);
    P.desc = (const SysDesc*)b->d_plan;
    P.pair = t0 + o_pair;
    P.part = t0 + o_part;
    P.cell = t0 + o_cell;
    P.vacf = t0 + o_vacf;
    P.conv = t0 + o_conv;
    P.fir = t0 + o_fir;
    P.cf = t0 + o_cf;
    return GLD_OK;
}

cudaError_t batch_launch_block(gld_batch* b, cudaStream_t s)
{
    cudaError_t e = launch_batch_noise(b->plan, s);
    for (int t = 0; t < kMaxNoiseBlock && e == cudaSuccess; ++t) {
        e = launch_batch_conv(b->plan, s);
        if (e == cudaSuccess) e = launch_batch_particles(b->plan, s);
    }
    return e;
}

// Times each convolution schedule on the current composition (the
// convolution only reads the rings and rewrites the projections, so repeating
// it leaves the state unchanged) and keeps the fastest.
gld_status batch_autotune(gld_batch* b)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bfail(b, GLD_E_CUDA, "autotune events");
    int best = 0;
    float best_ms = 1e30f;
    for (int sc = 0; sc < 4; ++sc) {
        GLD_TRY(batch_plan(b, sc));
        float ms = 0.f;
        bool ok = launch_batch_conv(b->plan, b->st) == cudaSuccess && cudaEventRecord(e0, b->st) == cudaSuccess;
        for (int r = 0; r < 5 && ok; ++r) ok = launch_batch_conv(b->plan, b->st) == cudaSuccess;
        ok = ok && cudaEventRecord(e1, b->st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
             cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        if (!ok) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return bfail(b, GLD_E_CUDA, "autotune launch");
        }
        b->schedule_ms[sc] = ms / 5.0;
        if (ms < best_ms) {
            best_ms = ms;
            best = sc;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->schedule = best;
    return batch_plan(b, best);
}

gld_status batch_prepare(gld_batch* b)
{
    if (!b->dirty) return GLD_OK;
    batch_drop_graph(b);
    long long cols = 0;
    for (const gld_ctx* c : b->members) cols += 3LL * c->P.n_pad / (c->P.hist_bf16 ? 8 : 4);
    if (b->tuning == 1 && b->schedule >= 0 && cols <= 2 * b->tuned_cols && 2 * cols >= b->tuned_cols) {
        GLD_TRY(batch_plan(b, b->schedule));
    } else {
        GLD_TRY(batch_autotune(b));
        b->tuned_cols = cols;
    }
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        const cudaError_t e = batch_launch_block(b, b->cap);
        const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
        ok = e == cudaSuccess && e2 == cudaSuccess && g;
    }
    if (ok) ok = cudaGraphInstantiate(&b->gexec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        cudaGetLastError();
        b->gexec = nullptr;  // eager launches below
    }
    b->dirty = false;
    return GLD_OK;
}

}  // namespace

gld_status gld_batch_create(void* stream, gld_batch** out)
{
    if (!out) return GLD_E_INVAL;
    gld_batch* b = new gld_batch();
    b->st = (cudaStream_t)stream;
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return GLD_E_CUDA;
    }
    *out = b;
    return GLD_OK;
}

gld_status gld_batch_add(gld_batch* b, gld_ctx* c)
{
    if (!b || !c) return GLD_E_INVAL;
    if (!c->have_kernels) return bfail(b, GLD_E_STATE, "gld_batch_add: the member has no kernels set");
    if (c->st != b->st) return bfail(b, GLD_E_INVAL, "gld_batch_add: the member must use the batch's stream");
    if (c->P.T != kMaxNoiseBlock) return bfail(b, GLD_E_INVAL, "gld_batch_add: the member's noise block must be 64");
    if (c->P.pc_nbins > 0 || c->P.nmodes > 0 || c->P.pn_iv || c->P.pn_kry)
        return bfail(b, GLD_E_INVAL,
                     "gld_batch_add: pair correlations, memory modes, and pair noise on an estimated interval or by "
                     "Lanczos iterations are single-context features");
    if (c->noise_valid && c->host_step != c->noise_end)
        return bfail(b, GLD_E_STATE, "gld_batch_add: the member is inside a noise block (step a multiple of 64)");
    for (gld_ctx* m : b->members)
        if (m == c) return bfail(b, GLD_E_INVAL, "gld_batch_add: already a member");
    if (!b->members.empty()) {
        const gld_ctx* f = b->members[0];
        if (f->P.nacc != c->P.nacc || f->P.hist_bf16 != c->P.hist_bf16 || f->prm.kahan != c->prm.kahan)
            return bfail(b, GLD_E_INVAL, "gld_batch_add: members must share kernel terms, history type and Kahan");
    }
    b->members.push_back(c);
    b->dirty = true;
    return GLD_OK;
}

gld_status gld_batch_remove(gld_batch* b, gld_ctx* c)
{
    if (!b || !c) return GLD_E_INVAL;
    for (size_t k = 0; k < b->members.size(); ++k)
        if (b->members[k] == c) {
            b->members.erase(b->members.begin() + (long)k);
            b->dirty = true;
            return GLD_OK;
        }
    return bfail(b, GLD_E_INVAL, "gld_batch_remove: not a member");
}

gld_status gld_batch_step(gld_batch* b, int64_t nsteps)
{
    if (!b || nsteps < 0) return GLD_E_INVAL;
    if (nsteps % kMaxNoiseBlock) return bfail(b, GLD_E_INVAL, "gld_batch_step: steps must be a multiple of 64");
    if (b->members.empty() || nsteps == 0) return GLD_OK;
    for (gld_ctx* c : b->members) {
        if (c->latched != GLD_OK) return bfail(b, c->latched, "gld_batch_step: a member has a latched error");
        if (!c->have_kernels) return bfail(b, GLD_E_STATE, "gld_batch_step: a member has no kernels set");
        if (c->noise_valid && c->host_step != c->noise_end)
            return bfail(b, GLD_E_STATE, "gld_batch_step: a member left its noise-block boundary");
    }
    for (gld_ctx* c : b->members) {
        const gld_status st = ring_form(c, false, b->st);
        if (st != GLD_OK) return bfail(b, st, "gld_batch_step: the white-noise ring of a member");
    }
    for (size_t m = 0; m < b->members.size() && !b->dirty; ++m)  // kernels reset since the plan
        if (m >= b->snap.size() || std::memcmp(&b->snap[m].P, &b->members[m]->P, sizeof(StepParams)) != 0 ||
            std::memcmp(&b->snap[m].B, &b->members[m]->B, sizeof(ParticleBuffers)) != 0 ||
            b->snap[m].coef != b->members[m]->coef || b->snap[m].pntaps != b->members[m]->d_pntaps ||
            b->snap[m].zblk != b->members[m]->d_zblk || b->snap[m].bvec != b->members[m]->d_bvec)
            b->dirty = true;
    GLD_TRY(batch_prepare(b));
    for (int64_t k = 0; k < nsteps; k += kMaxNoiseBlock) {
        const cudaError_t e = b->gexec ? cudaGraphLaunch(b->gexec, b->st) : batch_launch_block(b, b->st);
        if (e != cudaSuccess) return bfail(b, GLD_E_CUDA, std::string("gld_batch_step: ") + cudaGetErrorString(e));
        for (gld_ctx* c : b->members) {
            c->conv_valid_step = -1;
            c->block_start = c->host_step;
            c->host_step += kMaxNoiseBlock;
            c->noise_end = c->host_step;
            c->noise_valid = true;
            c->last_fr_row = kMaxNoiseBlock - 1;
        }
    }
    return GLD_OK;
}

gld_status gld_batch_sync(gld_batch* b)
{
    if (!b) return GLD_E_INVAL;
    if (cudaStreamSynchronize(b->st) != cudaSuccess) return bfail(b, GLD_E_CUDA, "gld_batch_sync");
    gld_status s = GLD_OK;
    for (gld_ctx* c : b->members) {
        const gld_status t = sync_and_check(c);
        if (s == GLD_OK) s = t;
    }
    return s;
}

gld_status gld_batch_info(gld_batch* b, int32_t* members, int32_t* schedule, double* schedule_ms)
{
    if (!b) return GLD_E_INVAL;
    if (members) *members = (int32_t)b->members.size();
    if (schedule) *schedule = b->schedule;
    if (schedule_ms)
        for (int k = 0; k < 4; ++k) schedule_ms[k] = b->schedule_ms[k];
    return GLD_OK;
}

gld_status gld_batch_set_tuning(gld_batch* b, int32_t policy)
{
    if (!b || policy < 0 || policy > 1) return GLD_E_INVAL;
    b->tuning = policy;
    return GLD_OK;
}

const char* gld_batch_last_error(const gld_batch* b) { return b ? b->msg.c_str() : "null batch"; }

gld_status gld_batch_destroy(gld_batch* b)
{
    if (!b) return GLD_E_INVAL;
    cudaStreamSynchronize(b->st);
    batch_drop_graph(b);
    batch_reap(b, true);
    if (b->d_plan) cudaFreeAsync(b->d_plan, b->st);
    cudaStreamSynchronize(b->st);
    for (int k = 0; k < 2; ++k) {
        if (b->h_stage[k]) cudaFreeHost(b->h_stage[k]);
        if (b->stage_ev[k]) cudaEventDestroy(b->stage_ev[k]);
    }
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return GLD_OK;
}

}  // extern "C"
