// launch.h -- host-side launchers of the GLD kernels (one per kernel family),
// shared by the translation units of the library.  All return the CUDA error
// of the launch.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "gld_internal.cuh"

namespace gld {

// History convolution (k_history.cu).  ctrl != nullptr: the step is read on
// the device; otherwise `step` is used.
cudaError_t launch_hist_conv(const void* ring, int bf16, int n_pad, int m_max, const Ctrl* ctrl,
                             long long step, const float* coef, int nacc, float* out, int kahan,
                             cudaStream_t st);

// The convolution of the step after the current one (its index read from
// ctrl->conv_step, written by the pair kernel), so that it can run beside the
// current step's F^C and VACF kernels.
cudaError_t launch_hist_conv_next(const void* ring, int bf16, int n_pad, int m_max, const Ctrl* ctrl,
                                  const float* coef, int nacc, float* out, int kahan, cudaStream_t st);

// Particle kernels (k_particles.cu).
struct ParticleBuffers {
    Ctrl* ctrl;
    float4 *pos, *pos_next;      // R_n and R_{n+1} by particle id
    float4 *pos_sorted;          // cell-ordered copy with the id in w (last build)
    float4 *vel, *vhalf, *fc, *fd, *disp, *disp_build;
    int *nbr, *nbr_cnt, *perm;   // neighbour lists [maxnb][n_pad] in build order
    void* ring;
    float* conv;
    float* frblock;
    const float* ftab;
    const float* fptab;   // perpendicular factors [Q + Qs][nr] (StepParams::perp) or null
    const float* fctab;   // tabulated -dU/dr (StepParams::fc_nr rows) or null
    const float* g0;
    int *cell_start, *cell_count, *cell_head, *cell_next, *chunk_sum, *chunk_off;
    int ncells;
    // VACF
    float4* vorig;
    float* vpartial;      // per-block VACF partials [2][n_os][vacf_gx] (two steps)
    double* csum;
    long long* ccnt;
    long long* norig;
    int vacf_gx;
    // pair correlations: per-step fixed-point sums [2][n_os][nbins][3] (a, c,
    // count) and the FP64 sums [vacf_len][nbins] with their counts
    long long* pc_step;
    double *pc_sa, *pc_sc;
    long long* pc_n;
};

cudaError_t launch_pair_force_integrate(const StepParams& P, const ParticleBuffers& B, cudaStream_t st);
// One thread idles for ns nanoseconds (at most 10 ms) on the device.
cudaError_t launch_delay(unsigned long long ns, cudaStream_t st);
// Cell list of the positions `src`; skipped on the device when gate != nullptr
// and *gate == 0.
cudaError_t launch_cell_build(const StepParams& P, const ParticleBuffers& B, const float4* src, const int* gate,
                              cudaStream_t st);
// Cell list and neighbour lists at R_{n+1} (pos_next), when ctrl->rebuild != 0.
cudaError_t launch_rebuild(const StepParams& P, const ParticleBuffers& B, cudaStream_t st);
// Inside a captured graph: sets conditional handle h to (ctrl->rebuild != 0).
cudaError_t launch_rebuild_decide(cudaGraphConditionalHandle h, const Ctrl* ctrl, cudaStream_t st);
// mode 0: F^C only (initialisation); mode 1: F^C_{n+1}, V_{n+1}, step += 1.
// Both copy pos_next into pos and clear ctrl->rebuild.
cudaError_t launch_cforce(const StepParams& P, const ParticleBuffers& B, int mode, cudaStream_t st);
cudaError_t launch_vacf(const StepParams& P, const ParticleBuffers& B, cudaStream_t st);
// Adds the last VACF launch's partials to the FP64 sums (before reading them).
cudaError_t launch_vacf_flush(const StepParams& P, const ParticleBuffers& B, cudaStream_t st);
// Distance-binned pair correlations at the current step (after vacf), and the
// fold of the last launch's sums before they are read.
cudaError_t launch_pcorr(const StepParams& P, const ParticleBuffers& B, cudaStream_t st);
cudaError_t launch_pcorr_flush(const StepParams& P, const ParticleBuffers& B, cudaStream_t st);
// Pair-correlated noise of step n: F = sum_k T_k(M / lambda) Z_k by Clenshaw's
// recurrence (pn_deg neighbour sweeps); Z_0 rows are frblock's, Z_k (k >= 1)
// rows of zblk[k - 1]; bvec holds three vectors [3][n_pad]; F replaces the
// Z_0 row of step n in frblock.
cudaError_t launch_pair_noise(const StepParams& P, const ParticleBuffers& B, const float* zblk, float* bvec,
                              cudaStream_t st);
// Extreme eigenvalues of the pair matrix M (as the Clenshaw sweeps apply it)
// by kPnLanczosSteps Lanczos steps: vec holds four vectors [3][n_pad], part
// 2 x ceil(n_pad / 256) doubles, ab 2 kPnLanczosSteps + 1 doubles; out[0],
// out[1] the smallest and largest Ritz values, out[2] the Krylov dimension
// used.  check: latch kErrPnBound when they leave [lo, hi].
cudaError_t launch_pn_spectrum(const StepParams& P, const ParticleBuffers& B, float* vec, double* part, double* ab,
                               double lo, double hi, int check, double* out, cudaStream_t st);
int pn_spectrum_blocks(const StepParams& P);
// Pair-correlated noise by Algorithm 1 (k_pn_krylov.cu): vectors [3 n_pad][Mp]
// (frequency fastest), Lanczos vectors unnormalised (R_k, v_k = R_k / beta_k).
// kry_ft: the transformed white-noise window of step ctrl->step into V0
// (cosT[s][w] = cos(2 pi w s / (2 m_max - 1)), s < m_max, zero columns for
// w >= M; with the time window, columns Mc + w the sine transform); kry_dot: per-frequency a.b folded into out (mode 0), or the
// square roots (2; 1 also marks exhausted Krylov spaces in alive, relative
// to ref); kry_matvec: Z = hat K_w R_k / beta_k for every w (wc: a_w, g_qw,
// gs_qw rows) and alpha_k; kry_resid: R_{k+1} = Z - alpha_k v_k - beta_k
// v_{k-1} and beta_{k+1} (fold mode 1); kry_combine: out[I] = (sum_w c_w
// sum_p cf[w][p] R_p[I][w]) / (2 m_max - 1).  part: kry_part_blocks x Mp
// doubles.  kry_fits: the transform's and the sweep's shared memory fit.
bool kry_fits(const StepParams& P, int Mp);
int kry_part_blocks(const StepParams& P);
cudaError_t kry_ft(const StepParams& P, const Ctrl* ctrl, const float* W, const float* cosT, int M, int Mp, int Mc,
                   float* V0, cudaStream_t st);
// The time window: out[m][I] (m < 64, the block's rows) = (1/L) sum_c
// wgt[c][m] sum_p cf[c][p] R_p[I][c]; Y is scratch [3 n_pad][Mp].
cudaError_t kry_rows(const StepParams& P, const float* V, const float* cf, int kp, int Mp, const float* wgt, float* Y,
                     float* out, cudaStream_t st);
cudaError_t kry_fold(const double* part, int nblk, int Mp, double* out, int mode, const double* ref, int* alive,
                     cudaStream_t st);
cudaError_t kry_dot(const StepParams& P, const float* a, const float* b, int Mp, double* part, double* out, int mode,
                    const double* ref, int* alive, cudaStream_t st);
cudaError_t kry_matvec(const StepParams& P, const ParticleBuffers& B, const double* wc, const double* beta_k,
                       const int* alive, int Mp, const float* R, float* Z, double* part, double* alpha_k,
                       cudaStream_t st);
cudaError_t kry_resid(const StepParams& P, const float* Z, const float* Rk, const float* Rkm1, const double* alpha_k,
                      const double* beta_k, const double* beta_km1, int* alive, const double* ref, int Mp,
                      float* Rkp1, double* part, double* beta_kp1, cudaStream_t st);
cudaError_t kry_combine(const StepParams& P, const float* V, const float* cf, int kp, int M, int Mp, float* out,
                        cudaStream_t st);
// Largest Gershgorin row sum sum_j |f(r_ij)| of the pair matrix at the
// current positions (as the bit pattern of a non-negative float).
cudaError_t launch_pn_rowsum(const StepParams& P, const ParticleBuffers& B, unsigned* out, cudaStream_t st);
// Pairs from a fresh cell traversal of pos_sorted / cell_start.
cudaError_t launch_pair_list(const StepParams& P, const ParticleBuffers& B, int* pairs,
                             long long cap, unsigned long long* count, cudaStream_t st);
// Pairs the force kernels use (neighbour lists at R_n).
cudaError_t launch_list_pair_list(const StepParams& P, const ParticleBuffers& B, int* pairs,
                                  long long cap, unsigned long long* count, cudaStream_t st);

// ---- batches of independent systems -------------------------------------
// Every member keeps its own buffers; one launch per kernel family covers all
// members through a tile list of (member, block within member).  Members share
// the accumulator count, history type and compensation; block counts per
// member drive the per-member last-block logic.
struct SysDesc {
    StepParams P;
    ParticleBuffers B;
    const float* coef;       // convolution coefficients [nacc][m_max]
    float* W;                // white-noise ring
    const float* taps;       // FP32 filter taps
    int ntaps;
    uint32_t k0, k1;         // Philox key
    const int* int2ext;
    int nb_pair, nb_part, nb_cell, nb_vacf, nb_conv, nb_fir, nb_cf;
    // pair-correlated noise (Chebyshev form, P.pn_deg > 0): taps
    // [pn_deg + 1][pn_la] (row 0 is `taps`), the blocks Z_1 .. Z_deg and three
    // Clenshaw vectors [3][n_pad]
    const float* pntaps;
    float* zblk;
    float* bvec;
    int pn_la;
};
struct Tile {
    int m, b;   // member, block within member
    int nb, r;  // blocks of the member in this schedule (convolution), unused
};
struct BatchPlan {
    const SysDesc* desc;
    const Tile *pair, *part, *cell, *vacf, *conv, *fir, *cf;
    int n_pair, n_part, n_cell, n_vacf, n_conv, n_fir, n_cf;
    int max_H, max_n, max_ntaps, nacc, bf16, kahan, vacf_no;
    int conv_block;  // threads per convolution tile (128 or 256)
    int pair_fast;   // every member has one pair term and no self-difference term
    int pn_kmax;     // the largest Chebyshev degree of the members' pair noise (0: none)
};
cudaError_t launch_batch_conv(const BatchPlan& bp, cudaStream_t st);      // k_history.cu
cudaError_t launch_batch_particles(const BatchPlan& bp, cudaStream_t st); // k_particles.cu
cudaError_t launch_batch_noise(const BatchPlan& bp, cudaStream_t st);     // k_noise.cu
// Block sizes of the tile schedules.
constexpr int kBatchPairLanes = 1;    // lanes per particle of the one-term pair kernel
constexpr int kBatchCforceLanes = 1;  // lanes per particle of the F^C kernel
constexpr int kBatchCforceBlock = 128; // threads per F^C tile of a batch
constexpr int kBatchPairBlock = 128, kBatchPartBlock = 256, kBatchCellChunk = 512, kBatchConvCols = 256,
              kBatchFirStreams = 32, kBatchVacfBlock = 256;

// Memory sums in auxiliary-variable form (k_modes.cu): coef[k] = {Re z, Im z,
// Re z^H, Im z^H}, w[a * nmodes + k] = {x_ak, y_ak}, Y[nmodes][3 n_pad].
cudaError_t launch_modes_step(const StepParams& P, const Ctrl* ctrl, const void* ring, const float4* coef,
                              const float2* w, float2* Y, float* conv, cudaStream_t st);
cudaError_t launch_modes_init(const StepParams& P, const Ctrl* ctrl, const void* ring, const double* zd, float2* Y,
                              cudaStream_t st);

// Noise and kernel preparation (k_noise.cu).
struct PrepArgs {
    int m_max, Q, Qs, discrete, clamp, T;
    double dt, kT, mass;
    const double* Ks;   // [m_max]
    const double* g;    // [Q][m_max]
    const double* gs;   // [Qs][m_max]
    double* Kd;         // [m_max] discrete K^s
    double* C;          // [m_max]
    double* Chat;       // [m_max]
    double* A;          // [2 m_max - 1]
    double* scal;       // [4]: a, b, min mode, clamped mass
    int* status;        // 0 or -3
    float* coef;        // [1+Q+Qs][m_max] discrete weights for the convolution
    float* g0;          // [Q+Qs] discrete m = 0 weights
    float* Acp;         // [la] FP32 filter taps A_{sigma-H}, zero padded
    int la;
};
cudaError_t launch_prep(const PrepArgs& a, cudaStream_t st);
int fir_copy_len(int T, int H);
// Padded length of the FP32 tap array (2H + 1 rounded up to 16).
int fir_taps_len(int H);

// int2ext maps the internal index to the caller's index, which keys the noise.
// With P.wsplit the ring holds the FP16 split of the white noise and the
// filter runs on the tensor cores (wmap: the ring's tensor map,
// make_noise_ring_map; required); else the ring is FP32 and the filter runs
// on the FP32 pipes.
cudaError_t launch_noise_block(const StepParams& P, Ctrl* ctrl, float* W, const float* Acp, int la,
                               float* frblock, unsigned long long seed, const int* int2ext,
                               const CUtensorMap* wmap, int num_sms, cudaStream_t st);
// One more moving-average pass over the white noise already in the ring of
// the current block (after launch_noise_block): out[t] = sum_s taps W.
cudaError_t launch_noise_filter(const StepParams& P, Ctrl* ctrl, const float* W, const float* taps, float* out,
                                const CUtensorMap* wmap, int num_sms, cudaStream_t st);
// Tensor-core filter (k_noise_tc.cu): whether it serves these parameters
// (64-step blocks, a ring of 32-row tiles, taps that fit shared memory), the
// tensor map of the split ring (FP16 planes hi [lw][3 n_pad], then lo) in
// boxes of 32 rows x 64 streams with 128-byte swizzle, and the launch.
bool noise_filter_tc_ok(const StepParams& P);
cudaError_t make_noise_ring_map(void* W, const StepParams& P, CUtensorMap* map);
cudaError_t launch_noise_filter_tc(const StepParams& P, Ctrl* ctrl, const CUtensorMap* wmap, const float* taps,
                                   float* out, int num_sms, cudaStream_t st);
cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out, long long n,
                          cudaStream_t st);
cudaError_t launch_gauss3(uint32_t k0, uint32_t k1, const uint32_t* particle, const long long* time,
                          uint32_t stream_id, float* out, long long n, cudaStream_t st);

}  // namespace gld
