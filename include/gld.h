/*
 * gld.h -- C ABI of the GB300 (sm_103a) integrator for discretized generalized
 * Langevin dynamics (GLD), after Jung, Hanke & Schmid, "Generalized Langevin
 * dynamics: Construction and numerical integration of non-Markovian
 * particle-based models" (arXiv:1808.00270).
 *
 * One GLD step (Sec. II B, Eq. GLD_integrator) on N particles in a cubic
 * periodic box:
 *   R_{n+1} = R_n + b dt V_n + b dt^2/(2M) (F^C_n + F^D_n + F^R_n)
 *   V_{n+1} = a V_n + dt/(2M) (a F^C_n + F^C_{n+1}) + b dt/M (F^D_n + F^R_n)
 * with b = [1 + dt K^s_0/(2M)]^-1, a = b [1 - dt K^s_0/(2M)] (Eq. aa-bb); the
 * conservative soft repulsion F^C over a cell list; the dissipative memory
 * force F^D of Eq. dissipative_force2, evaluated from a device-resident ring
 * of the last m_max-1 displacements dR_{n-m}; and the colored random force
 * F^R_n = sum_{s=-(m_max-1)}^{m_max-1} A_s W_{n+s} of Eq. noise_production
 * built from counter-based Philox4x32-10 Gaussians, with A_s derived from the
 * self kernel by the Fourier route of Sec. II C.
 *
 * Conventions shared by every call:
 *   - All pointers passed to gld_create / gld_set_kernels / gld_get_* /
 *     gld_set_* / gld_vacf / gld_pair_correlation and the host-only helpers
 *     gld_separable_terms / gld_pair_noise_filters are HOST pointers owned by
 *     the caller; the library copies from or into them and keeps no
 *     reference.  Arrays of particle vectors are row-major [n][3] doubles;
 *     tables are row-major as written ([rows][columns]).
 *   - The library owns all device memory of a context.  It allocates through
 *     gld_params.alloc / .free when given (e.g. a framework's caching
 *     allocator), else with cudaMalloc / cudaFree.
 *   - Work is queued on gld_params.stream (a cudaStream_t; NULL = legacy
 *     default stream).  gld_step returns without waiting; errors raised on the
 *     device are latched and returned by the next synchronizing call
 *     (gld_sync, gld_vacf, gld_get_*).  gld_last_error gives a message.
 *   - No call is thread-safe against another call on the same context.
 *
 * Entry points whose names end in _dev take DEVICE pointers allocated by the
 * caller, run one kernel on the given stream and return without waiting.
 */
#ifndef GLD_H
#define GLD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gld_ctx gld_ctx;

typedef enum {
    GLD_OK = 0,
    GLD_E_INVAL = -1,     /* bad argument or parameter combination            */
    GLD_E_NOMEM = -2,     /* device allocation failed                         */
    GLD_E_NOT_PSD = -3,   /* noise spectrum has a negative mode (Sec. II B)   */
    GLD_E_CUDA = -4,      /* a CUDA runtime call or launch failed             */
    GLD_E_NONFINITE = -5, /* a non-finite displacement was produced           */
    GLD_E_TIMEOUT = -6,   /* a bounded wait gave up (device, or gld_server_drain) */
    GLD_E_STATE = -7,     /* call out of order (e.g. gld_step before kernels) */
    GLD_E_CANCELLED = -8  /* a served request was cancelled                   */
} gld_status;

enum { GLD_HIST_F32 = 0, GLD_HIST_BF16 = 1 };
enum { GLD_KCONT = 0, GLD_KDISCRETE = 1 };

/* Optional device allocator: returns a pointer to at least `bytes` bytes of
 * device memory usable on `stream`, or NULL. */
typedef void* (*gld_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*gld_free_fn)(void* ptr, void* stream, void* user);

typedef struct gld_params {
    int32_t n;           /* particles, >= 1                                        */
    double box;          /* edge L of the cubic periodic box (Sec. II A, App. B)   */
    double mass;         /* particle mass M                                         */
    double kT;           /* k_B T of the fluctuation-dissipation theorem, Eq. FDT   */
    double dt;           /* time step                                               */
    int32_t m_max;       /* memory cutoff: K_m for m < m_max (Eq. k-discrete), >= 2 */
    double r_c;          /* spatial cutoff of F^C and pair kernels, 0 < r_c <= L/2  */
    double r_c_min;      /* kernels evaluated at max(r, r_c_min) (Sec. III B)       */
    double A_cons;       /* soft repulsion U(r) = A (1 - r/r_c)^2 for r < r_c        */
    double skin;         /* Verlet-list skin (0: 0.2 r_c); lists hold r < r_c + skin */
    uint64_t seed;       /* Philox key of the white noise W                         */
    int32_t hist_dtype;  /* GLD_HIST_F32 (default) or GLD_HIST_BF16 ring storage    */
    int32_t kahan;       /* 1: compensated summation over the m_max-1 history terms */
    int32_t vacf_len;    /* VACF lags kept (0 = no VACF)                             */
    int32_t vacf_stride; /* steps between VACF time origins (>= 1); at most 32      */
                         /* origins in flight: ceil(vacf_len / vacf_stride) <= 32   */
    int64_t vacf_burnin; /* first origin time, >= 1 (samples follow steps); < 0
                          * selects 2 m_max                                    */
    int32_t noise_block; /* steps of F^R produced per noise launch (0 = 64)          */
    int32_t psd_clamp;   /* 1: clamp negative noise modes to 0 instead of failing    */
    int32_t use_graphs;  /* 1 (default): replay steps from a captured CUDA graph
                          * whose list rebuild is a conditional node; 2: the same
                          * graph with device-gated rebuild kernels instead (every
                          * node a plain kernel, e.g. for per-kernel profilers);
                          * 0: launch every kernel from the host              */
    const int32_t* order; /* optional [n]: internal storage order (see gld_get_order) */
    void* stream;        /* cudaStream_t for all work of this context                */
    gld_alloc_fn alloc;  /* optional device allocator (NULL: cudaMalloc)             */
    gld_free_fn free;
    void* alloc_user;
} gld_params;

/* Fills *p with defaults (kT = 1, mass = 1, r_c_min = 0, skin = 0 (auto), F32
 * history, no Kahan, vacf_stride = 1, vacf_burnin = -1, noise_block = 64,
 * graphs on).  Neighbour sums use Verlet lists of radius r_c + skin, rebuilt on
 * the device whenever a particle has moved more than 0.45 skin since the last
 * build; the r < r_c test is applied exactly at every use, so results do not
 * depend on the skin.  A list longer than its capacity (set from the density
 * at creation) latches GLD_E_STATE. */
void gld_params_default(gld_params* p);

/* Creates a context on the current CUDA device.  pos and vel are [n][3]
 * host arrays (positions are wrapped into [0, L)).  Computes F^C_0 at R_0.
 * The displacement history starts at zero (cold start).  Returns GLD_E_INVAL
 * for n < 1, m_max < 2, r_c > L/2, non-positive L, M, dt, or an unknown
 * hist_dtype; GLD_E_NOMEM if device memory runs out. */
gld_status gld_create(const gld_params* p, const double* pos, const double* vel, gld_ctx** out);

/* Sets the memory kernels (Sec. II A, Eqs. GLD_basic, GLD_basic2, parallel
 * components only; Sec. II B, Eq. k-discrete) and derives everything the
 * step needs, in FP64 on the device:
 *   Ks[m_max]        self kernel K^s.  With GLD_KCONT these are continuous
 *                    samples K^s(m dt); the discrete weights are
 *                    K_m = dt K(m dt) for m >= 1 and K_0 = dt K(0)/2.
 *                    With GLD_KDISCRETE they are the K_m themselves.
 *   Q, g[Q][m_max], f[Q][nr]
 *                    pair kernel K^p_m(r) = sum_q f_q(r) g_q[m] (parallel
 *                    component, acting through e e^T); g converted like Ks;
 *                    f tabulated on r = k dr, k < nr, linear interpolation,
 *                    constant past the last entry.  Q = 0 disables it.
 *   dKs_g[Qs][m_max], dKs_f[Qs][nr], Qs
 *                    neighbour contribution to the self kernel dK^s_m(r), same
 *                    representation.  Qs = 0 (pointers may be NULL) disables it.
 * Then: noise target C_m = kT a_m K^s_m / dt (Eq. FDT_discretized, a_0 = 2),
 * its length-(2 m_max - 1) transform (Eq. FT), A_s = inverse transform of
 * sqrt(hat C) (Sec. II C), and a, b (Eq. aa-bb).  Returns GLD_E_NOT_PSD if a
 * mode of hat C is negative (beyond 1e-12 of the largest) unless psd_clamp;
 * GLD_E_INVAL for Q or Qs outside [0, 4] or nr < 2 / dr <= 0 with Q+Qs > 0.
 * Synchronizes the stream. */
gld_status gld_set_kernels(gld_ctx* ctx, const double* Ks, int32_t Q, const double* g,
                           const double* f, int32_t nr, double dr, const double* dKs_g,
                           const double* dKs_f, int32_t Qs, int32_t kernel_convention);

/* Queues nsteps GLD steps (>= 0) on the context's stream; returns without
 * waiting.  GLD_E_STATE if no kernels are set. */
gld_status gld_step(gld_ctx* ctx, int64_t nsteps);

/* Waits for the context's stream; returns the first latched error. */
gld_status gld_sync(gld_ctx* ctx);

/* Velocity autocorrelation (Sec. III A, self part of C^a), per Cartesian
 * component: out[tau] = < V_x(t0 + tau) V_x(t0) > averaged over particles,
 * components and time origins t0 = burnin + k vacf_stride, accumulated in
 * FP64 on the device.  out has vacf_len entries; *n_origins (may be NULL)
 * receives the number of origins so far.  Synchronizes. */
gld_status gld_vacf(gld_ctx* ctx, double* out, int64_t* n_origins);

/* Current wrapped positions and velocities, [n][3] each (either may be NULL).
 * Synchronizes. */
gld_status gld_get_state(gld_ctx* ctx, double* pos, double* vel);

/* Arrays that can be read (and, where marked, written) for checks and
 * checkpoints.  Sizes: [n][3] unless stated. */
enum {
    GLD_ARR_POS = 0,  /* R_n, wrapped (rw; writing rebuilds cells and F^C)        */
    GLD_ARR_VEL = 1,  /* V_n (rw)                                                 */
    GLD_ARR_FC = 2,   /* F^C_n (rw)                                               */
    GLD_ARR_FD = 3,   /* F^D of the last completed step (r)                       */
    GLD_ARR_FR = 4,   /* F^R of the last completed step (r)                       */
    GLD_ARR_DISP = 5, /* unwrapped displacement since creation, sum of dR (rw)    */
    GLD_ARR_HIST = 6, /* [m_max-1][n][3]: entry m-1 holds dR_{n-m} (rw)           */
    GLD_ARR_CONV = 7  /* [1+Q+Qs][n][3]: history projections as last computed (r):
                       * of the last step, or of the next one after a
                       * replayed graph block, which computes them early */
};
gld_status gld_get_array(gld_ctx* ctx, int32_t which, double* out);
gld_status gld_set_array(gld_ctx* ctx, int32_t which, const double* in);

/* Internally particles are stored in the Morton order of their cells at
 * creation, so that neighbours sit close in memory; every array of this API
 * is in the caller's order and the noise of a particle depends only on the
 * caller's index.  Summation orders inside the library follow the internal
 * order, so a checkpoint resumes bit for bit when the new context is created
 * with the same order: int2ext[k] (length n) receives the caller's index of
 * the particle stored at position k; pass it as gld_params.order. */
gld_status gld_get_order(gld_ctx* ctx, int32_t* int2ext);

/* Diagnostics, out[count] (count <= 5 filled): {graph form of gld_step (0: not
 * captured yet, 1: rebuild kernels gated on the device, 2: rebuild in a
 * conditional graph node), neighbour-list builds so far, list capacity per
 * particle, cells per box edge, the largest Krylov dimension any frequency
 * used in the last step's pair-correlated noise (gld_set_pair_noise_krylov;
 * 0 when off)}.
 * Synchronizes. */
gld_status gld_get_diag(gld_ctx* ctx, int64_t* out, int32_t count);

/* Step counter n (the time index of R_n) and its setter (n >= 0, else
 * GLD_E_INVAL); setting it invalidates the noise window, which is rebuilt
 * from the counters. */
gld_status gld_get_step(gld_ctx* ctx, int64_t* step);
gld_status gld_set_step(gld_ctx* ctx, int64_t step);

/* FP64 results of gld_set_kernels: Kd[m_max] discrete K^s_m, A[2 m_max - 1]
 * noise coefficients A_s at s + m_max - 1, ab[2] = {a, b}, spec[2] = {min
 * mode of hat C, clamped negative mass}.  Any pointer may be NULL. */
gld_status gld_get_coefs(gld_ctx* ctx, double* Kd, double* A, double* ab, double* spec);

/* Pairs (i < j) with |R_i - R_j| < r_c found by the cell-list traversal that
 * the force kernels use, at the current positions.  The distance test is
 * single precision with this exact order: d = x_i - x_j; if d > L/2 then
 * d -= L, else if d < -L/2 then d += L; r2 = (dx*dx + dy*dy) + dz*dz without
 * fused multiply-add; pair if r2 < float(r_c^2).  pairs is [cap][2] int32;
 * *count receives the total (may exceed cap).  Synchronizes. */
gld_status gld_get_pairs(gld_ctx* ctx, int32_t* pairs, int64_t cap, int64_t* count);

/* Runs at least nsteps steps (rounded up to whole noise blocks, after untimed
 * steps up to the next block boundary) with every kernel family bracketed by
 * CUDA events on the context's stream; each block starts with a 0.2 ms idle
 * kernel so that the host enqueues the block ahead of the device and the
 * event pairs time device work only.  Adds each family's device time in
 * milliseconds to ms[GLD_PROF_N] and its launch count to launches[GLD_PROF_N]
 * (either may be NULL).  Advances the simulation like gld_step.
 * Synchronizes. */
enum {
    GLD_PROF_NOISE = 0,  /* white-noise generation + moving average (per block) */
    GLD_PROF_HIST = 1,   /* history convolution                               */
    GLD_PROF_PAIR = 2,   /* F^D, position update, history write               */
    GLD_PROF_CELL = 3,   /* cell + neighbour-list rebuild (4 kernels, gated)  */
    GLD_PROF_CFORCE = 4, /* F^C_{n+1}, velocity update and the VACF terms     */
    GLD_PROF_VACF = 5,   /* velocity autocorrelation in batches only (single  */
                         /* contexts accumulate it inside the F^C kernel: 0)  */
    GLD_PROF_PCORR = 6,  /* distance-binned pair correlations (when enabled)  */
    GLD_PROF_PNOISE = 7, /* Clenshaw sweeps of the pair-correlated noise      */
    GLD_PROF_N = 8
};
gld_status gld_profile_steps(gld_ctx* ctx, int64_t nsteps, double* ms, int64_t* launches);

/* Tabulated conservative force (the form iterative Boltzmann inversion gives,
 * Sec. III): F^C_ij = f(r_ij) e_ij with f = -dU/dr sampled on r = k dr,
 * k < nr, linear between samples and constant past the last (pairs are taken
 * within r_c).  Replaces the soft repulsion A (1 - r/r_c)^2; nr = 0 returns to
 * it.  F^C is recomputed at the current positions.  Synchronizes. */
gld_status gld_set_conservative_table(gld_ctx* ctx, const double* f, int32_t nr, double dr);
/* A general, not separable, pair kernel given as samples Kp[k][m] =
 * K^p(k dr, m dt) (k < nr, m < m_max; the parallel component of Eq.
 * dissipative_force2): its best rank-Q approximation (SVD in FP64, 1 <= Q <= 4)
 * becomes Q separable terms f_q(r) g_q[m], set with gld_set_kernels together
 * with the self kernel Ks (kernel_convention as there).  *trunc receives the
 * relative Frobenius norm of the discarded part (NULL allowed). */
gld_status gld_set_kernels_table(gld_ctx* ctx, const double* Ks, const double* Kp, int32_t nr, double dr,
                                 int32_t Q, int32_t kernel_convention, double* trunc);
/* The separation itself, on the host (no device needed): f[Q][nr], g[Q][m]
 * with table ~ sum_q f_q g_q^T, f_q carrying the singular value; *trunc as
 * above.  GLD_E_INVAL unless 1 <= Q <= min(nr, m). */
gld_status gld_separable_terms(const double* table, int32_t nr, int32_t m, int32_t Q, double* f, double* g,
                               double* trunc);

/* Perpendicular components of the pair and self-difference kernels (Sec.
 * II A: each two-particle tensor is K_par(r) e e^T + K_perp(r) (1 - e e^T)):
 * fp[Q][nr] and fsp[Qs][nr] are the perpendicular radial factors of the terms
 * set by gld_set_kernels, sharing their time factors g_q, gs_q and r grid
 * (NULL or all zero: none; gld_set_kernels clears them).  They enter F^D and,
 * when set, the pair-correlated noise.  Synchronizes. */
gld_status gld_set_perpendicular(gld_ctx* ctx, const double* fp, const double* fsp);

/* Pair-correlated random force (Sec. II C, Eqs. stochastic_force2,
 * correlation_matrix, noise_ansatz; the matrix square root that Algorithm 1
 * applies by a Lanczos iteration per frequency), under the time-scale
 * separation remarked on after Algorithm 1 (kernels at the current R_n).  With
 * one separable pair term f(r) g(t) the transformed correlation matrices are
 * hat K_w = h_w 1 + g_w M, M the pair matrix with blocks f(r_ij) e_ij e_ij^T
 * (+ fp(r_ij) (1 - e_ij e_ij^T) with perpendicular factors),
 * so every sqrt(hat K_w) is one function of M: it is replaced by its
 * Chebyshev interpolant of `degree` (1..16) on [-lambda, lambda], giving
 * F_n = sum_k T_k(M / lambda) Z_k with Z_k moving averages of the same white
 * noise (degree + 1 filters per 64-step block, `degree` neighbour sweeps per
 * step).  *lambda: in, a bound on the spectrum of M (<= 0 or NULL: 1.25 x
 * the largest Gershgorin row sum at the current positions); out, the bound
 * used.  Every step checks the Gershgorin bound and latches GLD_E_NOT_PSD if
 * a row sum exceeds lambda.  *cheb_err: the largest interpolation error
 * relative to the largest square root (NULL allowed).  Needs Q = 1 and
 * Qs <= 1, a self-difference term having the pair term's time factor
 * (gs = c g: its blocks c fs(r) e e^T join M on the diagonal; GLD_E_INVAL
 * otherwise); GLD_E_NOT_PSD if h_w < |g_w| lambda for some w (positive
 * semi-definiteness not guaranteed) unless psd_clamp.  degree = 0 returns to
 * the self-kernel noise; gld_set_kernels does too.  Such a context can join a
 * batch: its K + 1 filters run in the batch's noise block and its Clenshaw
 * sweeps as batch launches over the members' particle tiles (the batch uses
 * the FP32-pipe filter, so a member's F^R differs from the context alone by
 * FP32 rounding).  Synchronizes. */
gld_status gld_set_pair_noise(gld_ctx* ctx, int32_t degree, double* lambda, double* cheb_err);
/* The filters of gld_set_pair_noise, on the host (no device needed): from the
 * discrete weights ks[m_max] of the self kernel and g[m_max] of the pair
 * term's time factor (K_0 already halved, as gld_set_kernels derives them),
 * taps[(degree + 1)][2 m_max - 1]: Z_k = sum_s taps[k][s + m_max - 1]
 * W_{n+s}, so that F_n = sum_k T_k(M / lambda) Z_k.  *cheb_err as there.
 * GLD_E_NOT_PSD if h_w < |g_w| lambda for some w and !psd_clamp;
 * GLD_E_INVAL for m_max < 2, degree outside [1, 16], lambda <= 0, dt <= 0. */
gld_status gld_pair_noise_filters(const double* ks, const double* g, int32_t m_max, double kT, double dt,
                                  double lambda, int32_t degree, int32_t psd_clamp, double* taps, double* cheb_err);
/* The same on an interval [lo, hi] holding the spectrum of M (lo < hi,
 * finite): F_n = sum_k T_k((M - c) / rho) Z_k, c = (lo + hi) / 2,
 * rho = (hi - lo) / 2; GLD_E_NOT_PSD if h_w + g_w mu < 0 at mu = lo or hi for
 * some w and !psd_clamp (h_w + g_w mu is linear in mu).  gld_pair_noise_filters
 * is this with [-lambda, lambda], bit for bit. */
gld_status gld_pair_noise_filters_on(const double* ks, const double* g, int32_t m_max, double kT, double dt,
                                     double lo, double hi, int32_t degree, int32_t psd_clamp, double* taps,
                                     double* cheb_err);
/* The Chebyshev form of gld_set_pair_noise on an interval [lo, hi] of the
 * spectrum of M rather than a symmetric Gershgorin bound.  The positive
 * semi-definiteness of hat K_w = h_w 1 + g_w M only needs h_w + g_w mu >= 0
 * on the actual eigenvalues mu; a Gershgorin bound overestimates them (for
 * the workloads' pair kernel f = 2 (1 - r/r_c)^2 at density 0.1 it gives 8.2
 * where the spectrum is [-2.4, 3.8]) and so refuses kernels that are
 * positive definite.  *lo, *hi: in, the interval (used when *lo < *hi); else
 * (or NULL) it is estimated by 32 Lanczos steps on M at the current
 * positions (FP32 vectors, FP64 sums, Sturm bisection of the tridiagonal
 * matrix) and the Ritz extremes widened by 25 % of their spread on each side
 * (the extremes are set by the closest pairs and move as pairs meet), each
 * end kept 5 % of the way from the spectrum to where h_w + g_w mu changes
 * sign for some w; out, the interval used.  Ritz values approach the extremes from inside, so
 * the estimate is not a bound: at every 64-step noise block the same Lanczos
 * run is repeated on the device (inside the captured step graph) and
 * GLD_E_NOT_PSD latches when a Ritz extreme leaves [lo, hi].  Otherwise as
 * gld_set_pair_noise (kernel forms, degree, psd_clamp, *cheb_err, exclusions);
 * it replaces either other form of pair noise.  Synchronizes. */
gld_status gld_set_pair_noise_on(gld_ctx* ctx, int32_t degree, double* lo, double* hi, double* cheb_err);
/* out[5]: the smallest and largest Ritz values of the last Lanczos run of
 * gld_set_pair_noise_on, the Krylov dimension it used, and the interval
 * [lo, hi].  GLD_E_STATE when that form is off.  Synchronizes. */
gld_status gld_pair_noise_spectrum(gld_ctx* ctx, double* out);

/* Pair-correlated random force by Algorithm 1 of Sec. II C: every step, for
 * each frequency w = 0 .. m_max - 1, a Lanczos iteration on the transformed
 * correlation matrix hat K_w (the right-hand side of Eq. stochastic_force2 at
 * the current configuration, the time-scale separation remarked on after
 * Algorithm 1) from the transformed white-noise window hat W_w, stopped when
 * the relative change of |hat W_w| V sqrt(H) e_1 between iterations falls to
 * tol (Algorithm 1's Delta; the vectors are FP32, so tol of 1e-6 .. 1e-4 is
 * meaningful), at most kmax iterations; F_n = (x_0 + 2
 * sum_{w>=1} x_w) / (2 m_max - 1).  It takes every kernel form (any Q, Qs <= 4
 * with time factors of their own, perpendicular factors, r_c,min) and needs
 * only that each hat K_w is positive semi-definite at the configuration; a
 * Ritz value below -1e-6 of the largest latches GLD_E_NOT_PSD, no
 * convergence within kmax
 * GLD_E_TIMEOUT.  It replaces the Chebyshev form of gld_set_pair_noise (and
 * the reverse).  Cost per step: kmax neighbour sweeps over all m_max
 * frequencies at most, with the host deciding between chunks of four
 * iterations, so steps run without graphs; device memory (kmax + 2) x 3 n_pad
 * x m_max floats.  tol <= 0 turns it off; 0 < tol < 1, 2 <= kmax <= 64, else
 * GLD_E_INVAL; GLD_E_STATE before kernels are set.  Single contexts only (not
 * in a batch); gld_profile_steps refuses it.  A new gld_set_kernels turns it
 * off.  Synchronizes. */
gld_status gld_set_pair_noise_krylov(gld_ctx* ctx, double tol, int32_t kmax);
/* gld_set_pair_noise_krylov with a choice of window: 0 as there (Algorithm 1
 * every step); 1 the time window of the remark after Algorithm 1 -- with the
 * kernels held at the configuration of a 64-step noise block's first step,
 * one Lanczos iteration per frequency on both the cosine and the sine
 * transform of that step's white-noise window gives hat F_w, and the whole
 * inverse transform gives F at all 64 steps of the block:
 *   F_{n0+m} = (X^c_0 + 2 sum_{w>=1} (X^c_w cos(2 pi w m / L) + X^s_w sin(2 pi w m / L))) / L.
 * Within a block the forces have the covariance of Eq. noise_ansatz exactly
 * (the periodic images of a lag below 64 fall beyond m_max); across blocks
 * they come from different windows.  Twice the vectors of window 0, once per
 * block instead of every step.  Needs 64-step noise blocks (GLD_E_INVAL
 * otherwise); else as gld_set_pair_noise_krylov.  Synchronizes. */
gld_status gld_set_pair_noise_lanczos(gld_ctx* ctx, double tol, int32_t kmax, int32_t window);

/* Memory sums in auxiliary-variable form (App. C discusses auxiliary-variable
 * expansions as the alternative to a stored history).  When every kernel
 * given to gld_set_kernels is, for m >= 1, a combination of the modes
 *   z_k^m = exp((-rate_k + i omega_k) m dt)   (real and imaginary parts),
 * the projections S, P, Ps of Eq. dissipative_force2 are carried as
 * per-particle sums Y_k(n) = sum_{m=1}^{m_max-1} z_k^m dR_{n-m}, updated in
 * O(1) per step as Y_k(n+1) = z_k (dR_n + Y_k(n) - z_k^{m_max-1} dR_{n-m_max+1}):
 * the same truncated convolution without streaming the ring every step (the
 * ring still holds the term that leaves the window).  The combination
 * coefficients are fitted in FP64 to the discrete weights; GLD_E_INVAL when
 * the relative residual exceeds 1e-9 (the kernels are not sums of these
 * modes), rate_k <= 0, omega_k < 0 or nmodes > 8.  Sums are FP32 (the Kahan
 * option does not apply).  The sums are rebuilt from the ring before the next
 * step (and after gld_set_step or a history write).  nmodes = 0, or a new
 * gld_set_kernels, returns to the ring convolution.  Single contexts only:
 * such a context cannot join a batch.  Synchronizes. */
gld_status gld_set_memory_modes(gld_ctx* ctx, int32_t nmodes, const double* rate, const double* omega);

/* Distance-binned velocity auto- and cross-correlations of pairs (Sec. III A,
 * the functions C^a(R,t) and C^c(R,t) from which the paper reconstructs the
 * pair memory kernels), sampled with the VACF's origins: for every unordered
 * pair i < j with r_ij(t) < r_max in bins of width r_max/nbins (distance at
 * the later time t), with e = (R_i - R_j)/r_ij(t) and the velocity components
 * along e,
 *   C^a(bin, lag) = < v_i(t) v_i(t0) + v_j(t) v_j(t0) > / 2,
 *   C^c(bin, lag) = < v_i(t) v_j(t0) + v_j(t) v_i(t0) > / 2,  lag = t - t0,
 * averaged over the pairs and origins of the bin.  Needs vacf_len > 0 and
 * 0 < r_max <= r_c; origins in flight x nbins <= 2048 (else GLD_E_INVAL).
 * Per-step sums are kept in 2^-28 fixed point (order-independent, so results
 * are reproducible bit for bit), accumulated in FP64.  Setting it again
 * clears the sums; contexts with it cannot join a batch. */
gld_status gld_set_pair_correlation(gld_ctx* ctx, int32_t nbins, double r_max);
/* ca, cc [vacf_len][nbins] (0 where the bin saw no pair), counts [vacf_len]
 * [nbins] pair samples; any pointer may be NULL.  Synchronizes. */
gld_status gld_pair_correlation(gld_ctx* ctx, double* ca, double* cc, int64_t* counts);

/* Checkpoint of the observables (Sec. III A: the VACF and the pair
 * correlations C^a, C^c accumulate over time origins, so a resumed run needs
 * their sums and the velocities of the origins still in flight).  The blob
 * holds the VACF sums, counts and origin count, the origin velocities (in
 * the caller's particle order) and, when enabled, the pair-correlation sums;
 * partials not yet added are added first.  gld_save_observables: *size
 * receives the blob's byte size; with buf != NULL (cap >= *size, else
 * GLD_E_INVAL) it is written.  gld_load_observables restores a blob into a
 * context of the same n, VACF settings and pair-correlation bins (else
 * GLD_E_INVAL) whose step index is the checkpoint's (gld_set_step first; else
 * GLD_E_STATE).  With the rest of the state restored through gld_set_array
 * and the same particle order, the resumed VACF and pair correlations are
 * those of the uninterrupted run bit for bit.  Both synchronize; the caller
 * owns buf. */
gld_status gld_save_observables(gld_ctx* ctx, void* buf, int64_t cap, int64_t* size);
gld_status gld_load_observables(gld_ctx* ctx, const void* buf, int64_t size);

/* Device bytes the context holds (all of its buffers, 256-byte granules). */
gld_status gld_get_bytes(gld_ctx* ctx, int64_t* bytes);
/* Device bytes a context with these parameters will hold after gld_create
 * and a gld_set_kernels with Q pair terms, Qs self-difference terms and nr
 * table points: exactly what gld_get_bytes then reports.  Needs a current
 * device (the VACF partial sums scale with its SM count); no device memory
 * is touched.  The history ring is (m_max-1)*3*n_pad*{4,2} bytes of it, the
 * white-noise window (64 + 2(m_max-1))*3*n_pad*4 bytes. */
gld_status gld_bytes_needed(const gld_params* params, int32_t Q, int32_t Qs, int32_t nr, int64_t* bytes);

const char* gld_last_error(const gld_ctx* ctx);
gld_status gld_destroy(gld_ctx* ctx);

/* ---- batches of independent systems -------------------------------------
 * Many GLD systems of different sizes, densities and memory lengths stepped
 * together: every kernel family runs as ONE launch over a tile list of
 * (member, block) for all members, and a 64-step block of the whole batch is
 * one captured CUDA graph.  Members remain ordinary contexts (their arrays,
 * VACF and state are read through the gld_* calls above); a member must have
 * its kernels set, use the batch's stream, sit at a 64-step boundary, and
 * share the number of kernel terms, the history type and compensation with
 * the other members.  A member's kernels, tables and parameters are read when
 * it joins: change them only while it is out of the batch.  Results of a
 * member do not depend on the other members.  Members may carry the
 * pair-correlated noise of gld_set_pair_noise (not the interval form of
 * gld_set_pair_noise_on, whose check runs a Lanczos iteration per member,
 * nor gld_set_pair_noise_krylov: GLD_E_INVAL); pair correlations and memory
 * modes are single-context features.
 * The convolution's tile schedule is picked by timing four candidates on the
 * current composition (256- or 128-column tiles, longest memory first, member
 * order, or one block per member). */
typedef struct gld_batch gld_batch;
gld_status gld_batch_create(void* stream, gld_batch** out);
gld_status gld_batch_add(gld_batch* batch, gld_ctx* member);
gld_status gld_batch_remove(gld_batch* batch, gld_ctx* member);
/* Steps every member by nsteps (a multiple of 64); returns without waiting. */
gld_status gld_batch_step(gld_batch* batch, int64_t nsteps);
/* Waits, then returns the first latched error of the members. */
gld_status gld_batch_sync(gld_batch* batch);
/* members, chosen convolution schedule (-1 before the first step), and the
 * timed milliseconds of the four schedules; pointers may be NULL. */
gld_status gld_batch_info(gld_batch* batch, int32_t* members, int32_t* schedule, double* schedule_ms);
/* policy 0 (default): re-time the schedules whenever the members change;
 * 1: re-time only when the total number of convolution columns has moved by
 * more than 2x since the last timing (for batches that change every block). */
gld_status gld_batch_set_tuning(gld_batch* batch, int32_t policy);
const char* gld_batch_last_error(const gld_batch* batch);
/* Frees the batch; the members stay valid. */
gld_status gld_batch_destroy(gld_batch* batch);

/* ---- serving: continuous batching of simulation requests ----------------
 * A request is a whole simulation (system, kernels, number of steps) whose
 * result is its VACF (and, on request, its final state).  Requests that have
 * arrived are admitted in arrival order while the device bytes of their
 * systems (gld_bytes_needed) fit the server's budget and a member slot is
 * free; a request that does not fit waits (no overtaking), one larger than
 * the whole budget fails with GLD_E_NOMEM.  Admitted systems live on the
 * device until they finish and are stepped together as one batch in 64-step
 * blocks (gld_batch_*); the composition changes at block boundaries while
 * the next block is already queued, so admission, retirement and result
 * read-back overlap the device work.  Steps beyond the last whole block run
 * alone on the server's stream.  A request's result does not depend on the
 * other requests.  Not thread-safe: one thread drives a server. */
typedef struct gld_server gld_server;
typedef struct {
    int64_t hbm_budget;   /* device bytes for admitted systems; 0: 85% of the free memory at creation */
    int32_t max_members;  /* systems stepped together at most; 0: no limit */
    int32_t in_flight;    /* blocks queued ahead of the device (default 2) */
    int32_t tuning;       /* gld_batch_set_tuning policy of the batch (default 1) */
    void* stream;         /* cudaStream_t of the batched work; NULL: the server creates one */
} gld_server_params;
typedef struct {
    gld_params params;    /* the system; stream, alloc, free, order and use_graphs are the server's */
    const double* pos;    /* [n][3], copied at submission */
    const double* vel;    /* [n][3] */
    const double* Ks;     /* kernels as for gld_set_kernels, copied at submission */
    int32_t Q;
    const double* g;
    const double* f;
    int32_t nr;
    double dr;
    const double* dKs_g;
    const double* dKs_f;
    int32_t Qs;
    int32_t kernel_convention;
    int64_t steps;        /* steps to run (>= 0) */
    double arrival;       /* server clock (s) before which it is not admitted; non-decreasing */
    int32_t keep_state;   /* also return the final positions and velocities */
    int32_t pair_noise;   /* Chebyshev degree of the pair-correlated random force (as gld_set_pair_noise on
                             the Gershgorin bound at the initial positions, admission counting its bytes);
                             0: self noise only.  A kernel form it does not take fails the request. */
} gld_request;
enum {  /* gld_server_stats slots */
    GLD_SRV_QUEUED = 0, GLD_SRV_ACTIVE = 1, GLD_SRV_RETIRING = 2, GLD_SRV_DONE = 3, GLD_SRV_FAILED = 4,
    GLD_SRV_BLOCKS = 5, GLD_SRV_PARTICLE_STEPS = 6, GLD_SRV_BYTES = 7, GLD_SRV_BYTES_PEAK = 8,
    GLD_SRV_MEMBERS_PEAK = 9, GLD_SRV_BUDGET = 10, GLD_SRV_N = 11
};
void gld_server_params_default(gld_server_params* params);
gld_status gld_server_create(const gld_server_params* params, gld_server** out);
/* Queues a request (inputs copied); *id numbers requests from 0. */
gld_status gld_server_submit(gld_server* server, const gld_request* request, int64_t* id);
/* One scheduling round: collects finished results, admits arrived requests,
 * queues one 64-step block of the batch (waiting only while `in_flight`
 * blocks are ahead of the device).  *active: systems in the batch. */
gld_status gld_server_pump(gld_server* server, int32_t* active);
/* Pumps until every submitted request has finished (timeout_s <= 0: none). */
gld_status gld_server_drain(gld_server* server, double timeout_s);
/* Seconds since the server was created (the clock of arrivals and results). */
gld_status gld_server_clock(const gld_server* server, double* t);
/* Result of request id: vacf[vacf_len], *n_origins, pos/vel [n][3] (only
 * with keep_state; else pass NULL), times[3] = {arrival, admission, done}
 * (-1 where not reached; filled whatever the status).  GLD_E_STATE while it
 * has not finished; the request's error if it failed.  Any pointer may be NULL. */
gld_status gld_server_result(gld_server* server, int64_t id, double* vacf, int64_t* n_origins, double* pos,
                             double* vel, double* times);
/* Cancels request id: a queued request is dropped, an admitted one leaves the
 * batch at once and its system is freed once the device has finished the
 * blocks already queued for it.  Its result then reports GLD_E_CANCELLED.
 * GLD_E_STATE if it has already finished or is being read back. */
gld_status gld_server_cancel(gld_server* server, int64_t id);
/* out[k] for the GLD_SRV_* slots k < count. */
gld_status gld_server_stats(gld_server* server, int64_t* out, int32_t count);
const char* gld_server_last_error(const gld_server* server);
/* Waits for the device, frees every system and the server. */
gld_status gld_server_destroy(gld_server* server);

/* ---- single kernels on caller-owned device memory ----------------------- */

/* Philox4x32-10 (Salmon et al., SC'11) on n counters: ctr [n][4] uint32,
 * key[2] (host), out [n][4] uint32. */
gld_status gld_philox_dev(const uint32_t* ctr, const uint32_t key[2], uint32_t* out, int64_t n,
                          void* stream);

/* White noise W_{i,k}: for item j, particle[j] and time[j] give the counter
 * (particle, (time + 2^62) low word, high word, stream_id); out [n][3] float.
 * u = ((x >> 9) + 1/2) 2^-23 (exact in FP32); Box-Muller on words (0,1) gives x, y and on
 * (2,3) gives z (Sec. II C requires uncorrelated unit Gaussians). */
gld_status gld_gauss3_dev(uint64_t seed, const uint32_t* particle, const int64_t* time,
                          uint32_t stream_id, float* out, int64_t n, void* stream);

/* History convolution of Eq. dissipative_force2 for every particle and
 * component (the memory-bound step):
 *   out[a][c][i] = sum_{m=1}^{m_max-1} coef[a][m] dR_{i,c,step-m}
 * ring: [m_max-1][3][n_pad] (float, or bf16 when bf16 != 0); dR_k is at slot
 * k mod (m_max-1).  coef: [nacc][m_max] float; out: [nacc][3][n_pad] float.
 * n_pad must be a multiple of 32 and the pointers 16-byte aligned; nacc in
 * [1, 9].  kahan != 0 uses compensated sums. */
gld_status gld_hist_conv_dev(const void* ring, int32_t bf16, int32_t n_pad, int32_t m_max,
                             int64_t step, const float* coef, int32_t nacc, float* out,
                             int32_t kahan, void* stream);

/* ---- neighbour pairs without device allocation ---------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory (code running while another library
 * captures the stream into a graph, allocation-free real-time loops, hosts
 * whose device memory belongs to a framework with a fixed budget).
 *
 * Same pairs as gld_get_pairs, from caller-owned device memory: pos4 is
 * [n][4] float (x, y, z, unused; 16-byte aligned) inside [0, box); pairs is
 * [cap][2] int32 (i < j, in no particular order); *count (device) receives the
 * total, which may exceed cap.  Runs on `stream` and returns without waiting.
 * Its scratch is one static device array of about 4.3 MB that every GPU
 * loading the library keeps until exit; no cudaMalloc, cudaFree or
 * allocating library routine is called.  The first call on a device looks
 * the array's address up (cudaGetSymbolAddress with that device current);
 * make that first call before any stream capture.  All calls share the
 * array: calls that overlap on the GPU (other streams, other threads) race.
 * GLD_E_INVAL for n < 1, n > GLD_NOALLOC_MAX_N, r_c > box/2, a misaligned
 * pos4, or NULL outputs. */
#define GLD_NOALLOC_MAX_N 65536
gld_status gld_pairs_noalloc(const float* pos4, int32_t n, double box, double r_c, int32_t* pairs,
                             int64_t cap, unsigned long long* count, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GLD_H */
