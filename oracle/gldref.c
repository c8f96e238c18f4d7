/*
 * gldref.c -- FP64 CPU oracle for the discretized generalized Langevin dynamics
 * (GLD) time step of Jung, Hanke & Schmid, "Generalized Langevin dynamics:
 * Construction and numerical integration of non-Markovian particle-based
 * models" (arXiv:1808.00270).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test-suite, the smoke check of the
 * package entry point and the CPU-baseline leg of the benchmark may build,
 * load or run it.  It shares no code, header, table or constant generator with
 * the CUDA library; the Philox generator below is written from its published
 * definition (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11).
 *
 * Every quantity is double precision.  Each function names the passage of the
 * paper it follows:
 *   Sec. II A   model: memory tensor = self part K^s + sum_k dK^s(R_ik), pair
 *               part K^p(R_ij); only the component parallel to e_ij is kept,
 *               K^s isotropic (Eqs. GLD_basic, GLD_basic2 and the parallel /
 *               perpendicular decomposition that follows them).
 *   Sec. II B   discrete kernels K_m (Eq. k-discrete), discrete FDT with
 *               a_0 = 2, a_m = 1 (Eq. FDT_discretized), the integrator
 *               (Eq. GLD_integrator), its factors a, b (Eq. aa-bb), the
 *               dissipative force (Eq. dissipative_force2) and the random
 *               force correlations (Eq. stochastic_force2).
 *   Sec. II C   moving-average noise F_n = sum_s A_s W_{n+s}
 *               (Eqs. noise_ansatz, noise_production) with A_s obtained from
 *               the length-(2 m_max - 1) Fourier transform (Eq. FT), the
 *               self-kernel-only case named at the end of that section.
 *   App. A      derivation of the integrator; position update uses b.
 *   Sec. III A  velocity autocorrelation (the self part of C^a) and the
 *               distance-binned auto and cross correlations C^a(R,t), C^c(R,t)
 *               (velocity components along e_ij at the later time t, pairs
 *               binned by their distance at t).
 *
 * Readings of the paper that this file takes:
 *   - position update uses b V_n (App. A) and not a V_n (Sec. II B);
 *   - kernels given as continuous samples K(m dt) become K_m = dt K(m dt),
 *     K_0 = dt K(0) / 2 (trapezoid weights of the delta comb, consistent with
 *     a_0 = 2), unless the caller passes discrete K_m directly;
 *   - the noise is generated from the self kernel only (Sec. II C, last
 *     remark) unless the caller supplies F^R for the step (the
 *     pair-correlated noise of Algorithm 1, evaluated by pairnoise.py);
 *   - the inverse transform for A_s uses 1/(2 m_max - 1);
 *   - history and noise before t = 0: Delta R = 0, W from the same counters.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846264338327950288

/* OR_PLANT selects a deliberately wrong variant of this oracle, built only by
 * the test that checks that the pins catch such mistakes (0 = correct):
 *   1 K_0 not halved          2 position update with a instead of b
 *   3 sign of the pair history term flipped
 *   4 inverse transform scaled by 1/m_max   5 history read one step late
 *   6 a_0 = 1 in the noise target           7 V_i in place of V_j at m = 0
 *   8 sign of F^C flipped                  9 auto and cross pair terms swapped
 *  10 pair-kernel table read at the lower row, not interpolated
 *  (11 and 12 are planted in pairnoise.py; this file builds unchanged)
 *  13 perpendicular pair terms without the projection 1 - e e^T
 *  14 pairs closer than r_c,min dropped instead of clamped
 *  15 perpendicular factors read at the unclamped distance
 *  16 the clamped distance used for the unit vector e as well
 *  (17 is planted in pairnoise.py) */
#ifndef OR_PLANT
#define OR_PLANT 0
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 bit      */
/* multiplications; the key is bumped by the Weyl constants between rounds.  */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter of the white noise W_{i,k}: (particle, time+2^62 low, high, stream).
 * Key: the 64-bit seed split into two words.  Uniform u = ((x>>9)+1/2) 2^-23
 * lies strictly inside (0,1) and is exact in single precision as well, so
 * every implementation sees the same u.  Box-Muller on (x0,x1) gives the x
 * and y components, on (x2,x3) the z component. */
static double u01(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

void or_gauss3(uint64_t seed, uint32_t particle, int64_t time, uint32_t stream, double z[3])
{
    uint64_t t = (uint64_t)(time + ((int64_t)1 << 62));
    uint32_t ctr[4] = { particle, (uint32_t)t, (uint32_t)(t >> 32), stream };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    double r01 = sqrt(-2.0 * log(u01(x[0])));
    double r23 = sqrt(-2.0 * log(u01(x[2])));
    z[0] = r01 * cos(2.0 * OR_PI * u01(x[1]));
    z[1] = r01 * sin(2.0 * OR_PI * u01(x[1]));
    z[2] = r23 * cos(2.0 * OR_PI * u01(x[3]));
}

/* ------------------------------------------------------------------------ */
/* Kernel preparation (Sec. II B, Eqs. k-discrete, FDT_discretized, aa-bb;  */
/* Sec. II C, Eqs. noise_ansatz, noise_production, FT).                     */
/* ------------------------------------------------------------------------ */
/* Continuous samples -> discrete weights of Eq. k-discrete. */
static void discretize(const double* samples, int m_max, double dt, int discrete, double* out)
{
    for (int m = 0; m < m_max; ++m) {
        if (discrete) out[m] = samples[m];
        else out[m] = (m == 0) ? (OR_PLANT == 1 ? 1.0 : 0.5) * dt * samples[0] : dt * samples[m];
    }
}

/* cos(2 pi w m / L) with the integer product reduced mod L first. */
static double cos_frac(int64_t w, int64_t m, int64_t L)
{
    int64_t r = (w * m) % L;
    if (r < 0) r += L;
    return cos(2.0 * OR_PI * (double)r / (double)L);
}

/* Noise coefficients A_s, s = -(m_max-1) .. m_max-1 (stored at s + m_max - 1)
 * from the target correlation C_m = kT a_m K_m / dt of Eq. stochastic_force2
 * (self part).  Returns 0, or -3 if a Fourier mode is negative (the noise
 * correlation matrix is then not positive semi-definite, Sec. II B end). */
int or_noise_coefs(int m_max, double kT, double dt, const double* Kd, int clamp,
                   double* C, double* Chat, double* A, double* clamped_mass)
{
    const int64_t L = 2 * (int64_t)m_max - 1;
    for (int m = 0; m < m_max; ++m) C[m] = kT * (m == 0 ? (OR_PLANT == 6 ? 1.0 : 2.0) : 1.0) * Kd[m] / dt;
    double cmax = 0.0;
    for (int w = 0; w < m_max; ++w) {
        /* Eq. FT with K_{-m} = K_m: the transform is real. */
        double s = C[0];
        for (int m = 1; m < m_max; ++m) s += 2.0 * C[m] * cos_frac(w, m, L);
        Chat[w] = s;
        if (fabs(s) > cmax) cmax = fabs(s);
    }
    int status = 0;
    double mass = 0.0;
    double Ahat[m_max > 0 ? m_max : 1];
    for (int w = 0; w < m_max; ++w) {
        double c = Chat[w];
        if (c < 0.0) {
            if (c < -1e-12 * cmax && !clamp) status = -3;
            mass += -c * (w == 0 ? 1.0 : 2.0);
            c = 0.0;
        }
        Ahat[w] = sqrt(c);          /* hat A = sqrt(hat K), Sec. II C */
    }
    for (int s = -(m_max - 1); s <= m_max - 1; ++s) {
        double v = Ahat[0];
        for (int w = 1; w < m_max; ++w) v += 2.0 * Ahat[w] * cos_frac(w, s, L);
        A[s + m_max - 1] = v / (OR_PLANT == 4 ? (double)m_max : (double)L);
    }
    if (clamped_mass) *clamped_mass = mass / (double)L;
    return status;
}

/* Eq. aa-bb for isotropic K^s_0: b = 1/(1 + dt K_0/2M), a = b (1 - dt K_0/2M). */
void or_integrator_factors(double K0, double dt, double mass, double* a, double* b)
{
    double c = dt * K0 / (2.0 * mass);
    *b = 1.0 / (1.0 + c);
    *a = *b * (1.0 - c);
}

/* ------------------------------------------------------------------------ */
/* Geometry: minimum image in a cubic periodic box, neighbour sets.         */
/* ------------------------------------------------------------------------ */
static double min_image(double d, double L) { return d - L * nearbyint(d / L); }

static double wrap(double x, double L)
{
    if (x < 0.0) x += L;
    else if (x >= L) x -= L;
    if (x >= L) x = 0.0;
    return x;
}

/* All pairs (i<j) with |R_i - R_j| < rc by brute force, FP64.  Returns the
 * number of pairs (writes at most cap). */
int64_t or_pairs_brute(const double* pos, int n, double L, double rc, int32_t* pairs, int64_t cap)
{
    int64_t np = 0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double dx = min_image(pos[3 * i] - pos[3 * j], L);
            double dy = min_image(pos[3 * i + 1] - pos[3 * j + 1], L);
            double dz = min_image(pos[3 * i + 2] - pos[3 * j + 2], L);
            if (dx * dx + dy * dy + dz * dz < rc * rc) {
                if (np < cap) { pairs[2 * np] = i; pairs[2 * np + 1] = j; }
                ++np;
            }
        }
    return np;
}

/* The same in single precision with a fixed operation order: d = x_i - x_j;
 * one periodic correction against L/2; r^2 = (dx*dx + dy*dy) + dz*dz, no
 * fused multiply-add; r^2 < rc2.  This is the distance test the CUDA path
 * states in its header; a pair set computed here from the same FP32
 * positions must equal the GPU's bit for bit. */
int64_t or_pairs_brute_f32(const float* pos, int n, float L, float rc2, int32_t* pairs, int64_t cap)
{
    const float half = 0.5f * L;
    int64_t np = 0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            volatile float d[3];
            for (int c = 0; c < 3; ++c) {
                float v = pos[3 * i + c] - pos[3 * j + c];
                if (v > half) v = v - L;
                else if (v < -half) v = v + L;
                d[c] = v;
            }
            volatile float xx = d[0] * d[0];
            volatile float yy = d[1] * d[1];
            volatile float zz = d[2] * d[2];
            volatile float s = xx + yy;
            volatile float r2 = s + zz;
            if (r2 < rc2) {
                if (np < cap) { pairs[2 * np] = i; pairs[2 * np + 1] = j; }
                ++np;
            }
        }
    return np;
}

/* Neighbour lists through a cell list of cell edge >= rc (Sec. II C: the
 * method iterates over neighbours within the cutoff).  nb_start[n+1], nb[]
 * hold for every i all j != i with r_ij < rc, sorted by j. */
typedef struct {
    int64_t* start;
    int32_t* list;
    int64_t cap;
} or_nblist;

static int cmp_i32(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

static void build_neighbors(const double* pos, int n, double L, double rc, or_nblist* nl)
{
    int nc = (int)floor(L / (rc * 1.001));
    /* at most about 8 cells per particle: larger cells are still correct */
    int ncap = (int)floor(cbrt(8.0 * (n > 0 ? n : 1)));
    if (nc > ncap) nc = ncap;
    if (nc < 3) nc = 1;
    int64_t ncell = (int64_t)nc * nc * nc;
    int32_t* head = (int32_t*)malloc(sizeof(int32_t) * ncell);
    int32_t* next = (int32_t*)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    int32_t* cell = (int32_t*)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    for (int i = n - 1; i >= 0; --i) {
        int cx = (int)floor(pos[3 * i] / L * nc), cy = (int)floor(pos[3 * i + 1] / L * nc),
            cz = (int)floor(pos[3 * i + 2] / L * nc);
        cx = cx < 0 ? 0 : (cx >= nc ? nc - 1 : cx);
        cy = cy < 0 ? 0 : (cy >= nc ? nc - 1 : cy);
        cz = cz < 0 ? 0 : (cz >= nc ? nc - 1 : cz);
        int c = (cz * nc + cy) * nc + cx;
        cell[i] = c;
        next[i] = head[c];
        head[c] = i;
    }
    int32_t* cnt = (int32_t*)calloc(n > 0 ? n : 1, sizeof(int32_t));
    const int span = nc == 1 ? 0 : 1;
    /* pass 1: count; pass 2: fill */
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            nl->start[0] = 0;
            for (int i = 0; i < n; ++i) nl->start[i + 1] = nl->start[i] + cnt[i];
            if (nl->start[n] > nl->cap) {
                nl->cap = nl->start[n] * 2 + 16;
                nl->list = (int32_t*)realloc(nl->list, sizeof(int32_t) * nl->cap);
            }
        }
#pragma omp parallel for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            int c = cell[i];
            int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
            int k = 0;
            for (int oz = -span; oz <= span; ++oz)
                for (int oy = -span; oy <= span; ++oy)
                    for (int ox = -span; ox <= span; ++ox) {
                        int nx = (cx + ox + nc) % nc, ny = (cy + oy + nc) % nc, nz = (cz + oz + nc) % nc;
                        for (int j = head[(nz * nc + ny) * nc + nx]; j >= 0; j = next[j]) {
                            if (j == i) continue;
                            double dx = min_image(pos[3 * i] - pos[3 * j], L);
                            double dy = min_image(pos[3 * i + 1] - pos[3 * j + 1], L);
                            double dz = min_image(pos[3 * i + 2] - pos[3 * j + 2], L);
                            if (dx * dx + dy * dy + dz * dz < rc * rc) {
                                if (pass == 1) nl->list[nl->start[i] + k] = j;
                                ++k;
                            }
                        }
                    }
            if (pass == 0) cnt[i] = k;
            else qsort(nl->list + nl->start[i], (size_t)k, sizeof(int32_t), cmp_i32);
        }
    }
    free(cnt);
    free(head);
    free(next);
    free(cell);
}

/* Pairs (i<j) from the cell-list neighbour lists, for comparison with the
 * brute-force search. */
int64_t or_pairs_cells(const double* pos, int n, double L, double rc, int32_t* pairs, int64_t cap)
{
    or_nblist nl;
    nl.start = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    nl.cap = 16;
    nl.list = (int32_t*)malloc(sizeof(int32_t) * nl.cap);
    build_neighbors(pos, n, L, rc, &nl);
    int64_t np = 0;
    for (int i = 0; i < n; ++i)
        for (int64_t k = nl.start[i]; k < nl.start[i + 1]; ++k) {
            int j = nl.list[k];
            if (j > i) {
                if (np < cap) { pairs[2 * np] = i; pairs[2 * np + 1] = j; }
                ++np;
            }
        }
    free(nl.start);
    free(nl.list);
    return np;
}

/* ------------------------------------------------------------------------ */
/* The simulated system.                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n, m_max, Q, Qs, nr, have_kernels, clamp;
    double L, mass, kT, dt, rc, rc_min, A_cons, dr;
    uint64_t seed;
    int vacf_len, vacf_stride;
    int64_t vacf_burnin;
    /* discrete kernels (Eq. k-discrete) */
    double *Kd, *gd, *f, *gsd, *fs;
    /* perpendicular radial factors of the same terms (Sec. II A: the part
     * acting through 1 - e e^T), sharing g_q, gs_q and the r grid; NULL: 0 */
    double *fp, *fsp;
    double *C, *Chat, *A, clamped_mass;
    double a, b;
    /* state at step `step`: R_n, V_n, F^C_n, ring of Delta R_{n-1..n-m_max+1} */
    int64_t step;
    double *pos, *vel, *fc, *fd, *fr, *disp, *hist;
    /* cache of white noise W_{i,k}, slot k mod (2 m_max - 1) */
    double* W;
    int64_t* wtime;
    /* velocity autocorrelation */
    double *vorig, *csum;
    int64_t *ccnt, n_origins;
    int n_os;
    /* distance-binned auto- and cross-correlations C^a(R,t), C^c(R,t) (Sec.
     * III A): sums [vacf_len][pc_nbins] over unordered pairs and origins */
    int pc_nbins;
    double pc_rmax;
    double *pc_a, *pc_c;
    int64_t* pc_n;
    /* tabulated conservative force magnitude f(r) on r = k fc_dr (0 rows: the
     * soft repulsion) */
    double* fct;
    int fc_nr;
    double fc_dr;
    /* a general pair-kernel table: discrete weights kpt[k][m] of K^p_m(r_k),
     * r_k = k kp_dr, linear in r between rows (0 rows: the separable terms) */
    double* kpt;
    int kp_nr;
    double kp_dr;
    /* F^R supplied by the caller for the next step only (the pair-correlated
     * noise of Algorithm 1 is evaluated outside this file) */
    double* fr_ovr;
    int fr_ovr_on;
    or_nblist nl;
} or_sys;

static void conservative_forces(or_sys* s);

static double* zalloc(size_t count) { return (double*)calloc(count > 0 ? count : 1, sizeof(double)); }

or_sys* or_create(int n, double L, double mass, double kT, double dt, int m_max, double rc,
                  double rc_min, double A_cons, uint64_t seed, int vacf_len, int vacf_stride,
                  int64_t vacf_burnin, const double* pos, const double* vel)
{
    /* VACF samples are taken after each step: the first origin is t = 1 */
    if (n < 0 || m_max < 2 || !(L > 0) || !(rc > 0) || rc > 0.5 * L || !(mass > 0) || !(dt > 0) ||
        (vacf_len > 0 && vacf_burnin < 1))
        return NULL;
    or_sys* s = (or_sys*)calloc(1, sizeof(or_sys));
    s->n = n; s->L = L; s->mass = mass; s->kT = kT; s->dt = dt; s->m_max = m_max;
    s->rc = rc; s->rc_min = rc_min; s->A_cons = A_cons; s->seed = seed;
    s->vacf_len = vacf_len > 0 ? vacf_len : 0;
    s->vacf_stride = vacf_stride > 0 ? vacf_stride : 1;
    s->vacf_burnin = vacf_burnin;
    size_t n3 = (size_t)3 * n;
    s->pos = zalloc(n3); s->vel = zalloc(n3); s->fc = zalloc(n3); s->fd = zalloc(n3);
    s->fr = zalloc(n3); s->disp = zalloc(n3);
    s->hist = zalloc(n3 * (m_max - 1));
    s->W = zalloc(n3 * (2 * m_max - 1));
    s->wtime = (int64_t*)malloc(sizeof(int64_t) * (2 * m_max - 1));
    for (int k = 0; k < 2 * m_max - 1; ++k) s->wtime[k] = INT64_MIN;
    for (size_t k = 0; k < n3; ++k) { s->pos[k] = wrap(pos[k], L); s->vel[k] = vel[k]; }
    s->n_os = s->vacf_len > 0 ? (s->vacf_len + s->vacf_stride - 1) / s->vacf_stride : 0;
    s->vorig = zalloc(n3 * (s->n_os > 0 ? s->n_os : 1));
    s->csum = zalloc(s->vacf_len > 0 ? s->vacf_len : 1);
    s->ccnt = (int64_t*)calloc(s->vacf_len > 0 ? s->vacf_len : 1, sizeof(int64_t));
    s->nl.start = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    s->nl.cap = 16;
    s->nl.list = (int32_t*)malloc(sizeof(int32_t) * s->nl.cap);
    conservative_forces(s); /* F^C_0 and the neighbour lists at R_0 */
    return s;
}

void or_destroy(or_sys* s)
{
    if (!s) return;
    double* arrs[] = { s->Kd, s->gd, s->f, s->gsd, s->fs, s->C, s->Chat, s->A, s->pos, s->vel,
                       s->fc, s->fd, s->fr, s->disp, s->hist, s->W, s->vorig, s->csum, s->pc_a, s->pc_c,
                       s->fct, s->kpt, s->fr_ovr, s->fp, s->fsp };
    for (size_t k = 0; k < sizeof(arrs) / sizeof(arrs[0]); ++k) free(arrs[k]);
    free(s->wtime); free(s->ccnt); free(s->nl.start); free(s->nl.list); free(s->pc_n);
    free(s);
}

/* Tabulated radial factor on r = k dr, linear interpolation; constant past the
 * last entry. */
static double table_at(const double* t, int nr, double dr, double r)
{
    double x = r / dr;
    if (x <= 0.0) return t[0];
    int k = (int)floor(x);
    if (k >= nr - 1) return t[nr - 1];
    double w = x - k;
    return t[k] * (1.0 - w) + t[k + 1] * w;
}

/* Pair kernels are given as K^p_m(r) = sum_q f_q(r) g_q[m] and
 * dK^s_m(r) = sum_q fs_q(r) gs_q[m] (parallel components, Sec. II A). */
int or_set_kernels(or_sys* s, const double* Ks, int Q, const double* g, const double* f, int nr,
                   double dr, int Qs, const double* gs, const double* fs, int discrete, int clamp)
{
    int M = s->m_max;
    if (Q < 0 || Qs < 0 || Q > 8 || Qs > 8 || (Q + Qs > 0 && (nr < 2 || !(dr > 0)))) return -1;
    free(s->Kd); free(s->gd); free(s->f); free(s->gsd); free(s->fs);
    free(s->fp); free(s->fsp);
    s->fp = s->fsp = NULL;
    free(s->C); free(s->Chat); free(s->A);
    s->Q = Q; s->Qs = Qs; s->nr = nr; s->dr = dr; s->clamp = clamp;
    s->Kd = zalloc(M); s->gd = zalloc((size_t)Q * M); s->f = zalloc((size_t)Q * nr);
    s->gsd = zalloc((size_t)Qs * M); s->fs = zalloc((size_t)Qs * nr);
    s->C = zalloc(M); s->Chat = zalloc(M); s->A = zalloc(2 * M - 1);
    discretize(Ks, M, s->dt, discrete, s->Kd);
    for (int q = 0; q < Q; ++q) {
        discretize(g + (size_t)q * M, M, s->dt, discrete, s->gd + (size_t)q * M);
        memcpy(s->f + (size_t)q * nr, f + (size_t)q * nr, sizeof(double) * nr);
    }
    for (int q = 0; q < Qs; ++q) {
        discretize(gs + (size_t)q * M, M, s->dt, discrete, s->gsd + (size_t)q * M);
        memcpy(s->fs + (size_t)q * nr, fs + (size_t)q * nr, sizeof(double) * nr);
    }
    or_integrator_factors(s->Kd[0], s->dt, s->mass, &s->a, &s->b);
    int st = or_noise_coefs(M, s->kT, s->dt, s->Kd, clamp, s->C, s->Chat, s->A, &s->clamped_mass);
    s->have_kernels = (st == 0);
    return st;
}

/* Perpendicular radial factors fp[Q][nr], fsp[Qs][nr] of the terms set by
 * or_set_kernels (either may be NULL: zero): K^p_m(r) = sum_q g_q[m]
 * (f_q(r) e e^T + fp_q(r) (1 - e e^T)), likewise dK^s with gs_q, fsp_q. */
int or_set_perp(or_sys* s, const double* fp, const double* fsp)
{
    if (!s->have_kernels) return -7;
    free(s->fp); free(s->fsp);
    s->fp = s->fsp = NULL;
    if (fp && s->Q > 0) {
        s->fp = zalloc((size_t)s->Q * s->nr);
        memcpy(s->fp, fp, sizeof(double) * (size_t)s->Q * s->nr);
    }
    if (fsp && s->Qs > 0) {
        s->fsp = zalloc((size_t)s->Qs * s->nr);
        memcpy(s->fsp, fsp, sizeof(double) * (size_t)s->Qs * s->nr);
    }
    return 0;
}

/* -dU/dr on r = k dr, k < nr (nr = 0: back to the soft repulsion); F^C is
 * recomputed at the current positions. */
int or_set_fc_table(or_sys* s, const double* f, int nr, double dr)
{
    if (nr < 0 || (nr > 0 && (nr < 2 || !(dr > 0) || !f))) return -1;
    free(s->fct);
    s->fct = NULL;
    s->fc_nr = nr;
    s->fc_dr = dr;
    if (nr > 0) {
        s->fct = zalloc((size_t)nr);
        memcpy(s->fct, f, sizeof(double) * nr);
    }
    conservative_forces(s);
    return 0;
}

/* A general (not separable) pair kernel: samples Kp[k][m] of K^p(r_k, m)
 * (continuous samples or discrete weights as for or_set_kernels), added to
 * the separable terms (set Q = 0 to use the table alone); the self kernel and
 * the noise are set by or_set_kernels as before (call this after it). */
int or_set_pair_table(or_sys* s, const double* Kp, int nr, double dr, int discrete)
{
    const int M = s->m_max;
    if (nr < 0 || (nr > 0 && (nr < 2 || !(dr > 0) || !Kp))) return -1;
    free(s->kpt);
    s->kpt = NULL;
    s->kp_nr = nr;
    s->kp_dr = dr;
    if (nr > 0) {
        s->kpt = zalloc((size_t)nr * M);
        for (int k = 0; k < nr; ++k) discretize(Kp + (size_t)k * M, M, s->dt, discrete, s->kpt + (size_t)k * M);
    }
    return 0;
}

static void ensure_noise(or_sys* s, int64_t n)
{
    const int M = s->m_max, LW = 2 * M - 1;
    for (int64_t k = n - (M - 1); k <= n + (M - 1); ++k) {
        int slot = (int)(((k % LW) + LW) % LW);
        if (s->wtime[slot] == k) continue;
        double* w = s->W + (size_t)slot * 3 * s->n;
#pragma omp parallel for schedule(static)
        for (int i = 0; i < s->n; ++i) or_gauss3(s->seed, (uint32_t)i, k, 0u, w + 3 * i);
        s->wtime[slot] = k;
    }
}

static const double* W_at(const or_sys* s, int64_t k)
{
    const int LW = 2 * s->m_max - 1;
    return s->W + (size_t)(((k % LW) + LW) % LW) * 3 * s->n;
}

/* Delta R_{i,k} of the history ring (zero before the first step). */
static const double* dR_at(const or_sys* s, int64_t k)
{
    const int H = s->m_max - 1;
    return s->hist + (size_t)(((k % H) + H) % H) * 3 * s->n;
}

/* F^C_i = sum_j -dU/dr e_ij with U = A (1 - r/rc)^2, or with -dU/dr = f(r)
 * read from a table (the form iterative Boltzmann inversion produces), at the
 * current positions. */
static void conservative_forces(or_sys* s)
{
    build_neighbors(s->pos, s->n, s->L, s->rc, &s->nl);
    const double L = s->L, rc = s->rc, A = s->A_cons;
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < s->n; ++i) {
        double F[3] = { 0, 0, 0 };
        for (int64_t k = s->nl.start[i]; k < s->nl.start[i + 1]; ++k) {
            int j = s->nl.list[k];
            double d[3];
            for (int c = 0; c < 3; ++c) d[c] = min_image(s->pos[3 * i + c] - s->pos[3 * j + c], L);
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double mag = s->fc_nr > 0 ? table_at(s->fct, s->fc_nr, s->fc_dr, r)
                                      : (OR_PLANT == 8 ? -2.0 : 2.0) * A / rc * (1.0 - r / rc);
            for (int c = 0; c < 3; ++c) F[c] += mag * d[c] / r;
        }
        for (int c = 0; c < 3; ++c) s->fc[3 * i + c] = F[c];
    }
}

/* Dissipative force of particle i at step n, Eq. dissipative_force2, taken
 * term by term from its definition (double loop over neighbours and memory
 * index; no projection shortcut):
 *   F^D_i = - sum_j [ K^p_0(R_ij) V_j + dK^s_0(R_ij) V_i ]
 *           - (1/dt) sum_{m=1}^{m_max-1} { sum_j K^p_m(R_ij) dR_{j,n-m}
 *                 + ( K^s_m + sum_k dK^s_m(R_ik) ) dR_{i,n-m} }
 * with K(R) = K_par(|R|) e e^T and |R| clamped below at rc_min. */
static void dissipative_force_i(const or_sys* s, int i, const int32_t* nb, int64_t nnb, double F[3])
{
    const int M = s->m_max, Q = s->Q, Qs = s->Qs;
    const int64_t n = s->step;
    F[0] = F[1] = F[2] = 0.0;
    for (int64_t k = 0; k < nnb; ++k) {
        int j = nb[k];
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = min_image(s->pos[3 * i + c] - s->pos[3 * j + c], s->L);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double rt = r < s->rc_min ? s->rc_min : r;
        if (OR_PLANT == 14 && r < s->rc_min) continue;
        const double re = OR_PLANT == 16 ? rt : r;
        double e[3] = { d[0] / re, d[1] / re, d[2] / re };
        double fq[8], fsq[8], fpq[8], fspq[8]; /* radial factors f_q, fs_q and their
                                                  perpendicular parts (Q, Qs <= 8) */
        for (int q = 0; q < Q; ++q) {
            fq[q] = table_at(s->f + (size_t)q * s->nr, s->nr, s->dr, rt);
            fpq[q] = s->fp ? table_at(s->fp + (size_t)q * s->nr, s->nr, s->dr, OR_PLANT == 15 ? r : rt) : 0.0;
        }
        for (int q = 0; q < Qs; ++q) {
            fsq[q] = table_at(s->fs + (size_t)q * s->nr, s->nr, s->dr, rt);
            fspq[q] = s->fsp ? table_at(s->fsp + (size_t)q * s->nr, s->nr, s->dr, OR_PLANT == 15 ? r : rt) : 0.0;
        }
        /* rows and weight of a general table at rt (the interpolation of table_at) */
        int kr0 = 0, kr1 = 0;
        double kw = 0.0;
        if (s->kp_nr > 0) {
            const double x = rt / s->kp_dr;
            kr0 = x <= 0.0 ? 0 : (int)floor(x);
            if (kr0 >= s->kp_nr - 1) { kr0 = kr1 = s->kp_nr - 1; }
            else { kr1 = kr0 + 1; kw = (x <= 0.0 || OR_PLANT == 10) ? 0.0 : x - kr0; }
        }
        for (int m = 0; m < M; ++m) {
            /* K^p_m(r) = sum_q f_q(r) g_q[m] (or the general table),
             * dK^s_m(r) = sum_q fs_q(r) gs_q[m] */
            double kp = 0.0, kds = 0.0, kpp = 0.0, kdsp = 0.0;
            if (s->kp_nr > 0)
                kp = s->kpt[(size_t)kr0 * M + m] * (1.0 - kw) + s->kpt[(size_t)kr1 * M + m] * kw;
            for (int q = 0; q < Q; ++q) kp += fq[q] * s->gd[(size_t)q * M + m];
            for (int q = 0; q < Qs; ++q) kds += fsq[q] * s->gsd[(size_t)q * M + m];
            for (int q = 0; q < Q; ++q) kpp += fpq[q] * s->gd[(size_t)q * M + m];
            for (int q = 0; q < Qs; ++q) kdsp += fspq[q] * s->gsd[(size_t)q * M + m];
            const double *xj, *xi;
            double scale;
            if (m == 0) { xj = s->vel + 3 * (OR_PLANT == 7 ? i : j); xi = s->vel + 3 * i; scale = 1.0; }
            else {
                int64_t k = n - m + (OR_PLANT == 5 ? 1 : 0);
                xj = dR_at(s, k) + 3 * j; xi = dR_at(s, k) + 3 * i; scale = 1.0 / s->dt;
            }
            if (m > 0 && OR_PLANT == 3) kp = -kp;
            double pj = e[0] * xj[0] + e[1] * xj[1] + e[2] * xj[2];
            double pi = e[0] * xi[0] + e[1] * xi[1] + e[2] * xi[2];
            /* parallel parts through e e^T, perpendicular ones through 1 - e e^T */
            for (int c = 0; c < 3; ++c) {
                const double xjp = OR_PLANT == 13 ? xj[c] : xj[c] - pj * e[c];
                const double xip = OR_PLANT == 13 ? xi[c] : xi[c] - pi * e[c];
                F[c] -= scale * ((kp * pj + kds * pi) * e[c] + kpp * xjp + kdsp * xip);
            }
        }
    }
    for (int m = 1; m < M; ++m) {
        const double* xi = dR_at(s, n - m + (OR_PLANT == 5 ? 1 : 0)) + 3 * i;
        for (int c = 0; c < 3; ++c) F[c] -= s->Kd[m] * xi[c] / s->dt;
    }
}

/* F^R_i,n = sum_{s=-(m_max-1)}^{m_max-1} A_s W_{i,n+s}, Eq. noise_production
 * for the self kernel.  With direct != 0 the W are drawn here instead of
 * being read from the cache of the full-system step. */
static void random_force_i(const or_sys* s, int i, double F[3], int direct)
{
    const int M = s->m_max;
    F[0] = F[1] = F[2] = 0.0;
    for (int sh = -(M - 1); sh <= M - 1; ++sh) {
        double wd[3];
        const double* w = wd;
        if (direct) or_gauss3(s->seed, (uint32_t)i, s->step + sh, 0u, wd);
        else w = W_at(s, s->step + sh) + 3 * i;
        double A = s->A[sh + M - 1];
        for (int c = 0; c < 3; ++c) F[c] += A * w[c];
    }
}

static void paircorr_sample(or_sys* s, int64_t o_now);

static void vacf_sample(or_sys* s)
{
    /* V at time t = step (after the step that produced it). */
    if (s->vacf_len <= 0) return;
    int64_t t = s->step;
    if (t < s->vacf_burnin) return;
    const size_t n3 = (size_t)3 * s->n;
    int64_t rel = t - s->vacf_burnin;
    int64_t o_now = rel / s->vacf_stride;
    if (rel % s->vacf_stride == 0) {
        memcpy(s->vorig + (size_t)(o_now % s->n_os) * n3, s->vel, sizeof(double) * n3);
        s->n_origins++;
    }
    paircorr_sample(s, o_now);
    for (int64_t o = o_now; o >= 0 && o > o_now - s->n_os; --o) {
        int64_t t0 = s->vacf_burnin + o * s->vacf_stride;
        int64_t lag = t - t0;
        if (lag < 0 || lag >= s->vacf_len) continue;
        const double* v0 = s->vorig + (size_t)(o % s->n_os) * n3;
        double acc = 0.0;
        for (size_t k = 0; k < n3; ++k) acc += s->vel[k] * v0[k];
        s->csum[lag] += acc;
        s->ccnt[lag] += 1;
    }
}

/* The pair part of the sample at time t = step: for every unordered pair
 * i < j with r_ij(t) < r_max (distance at time t, bins of width r_max/nbins)
 * and every active origin t0, with e = (R_i - R_j)/r at time t and the
 * velocity components along e,
 *   a = v_i(t) v_i(t0) + v_j(t) v_j(t0),   c = v_i(t) v_j(t0) + v_j(t) v_i(t0).
 * C^a, C^c are the sums over i, j != i of these terms divided by twice the
 * number of ordered pairs: per bin and lag, sum over unordered pairs / (2 n). */
static void paircorr_sample(or_sys* s, int64_t o_now)
{
    if (s->pc_nbins <= 0) return;
    const size_t n3 = (size_t)3 * s->n;
    const double dr = s->pc_rmax / s->pc_nbins;
    for (int i = 0; i < s->n; ++i) {
        for (int64_t k = s->nl.start[i]; k < s->nl.start[i + 1]; ++k) {
            const int j = s->nl.list[k];
            if (j <= i) continue;
            double d[3], r2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                d[c] = min_image(s->pos[3 * i + c] - s->pos[3 * j + c], s->L);
                r2 += d[c] * d[c];
            }
            const double r = sqrt(r2);
            if (!(r < s->pc_rmax)) continue;
            int b = (int)(r / dr);
            if (b >= s->pc_nbins) b = s->pc_nbins - 1;
            double vit = 0.0, vjt = 0.0;
            for (int c = 0; c < 3; ++c) {
                vit += s->vel[3 * i + c] * d[c] / r;
                vjt += s->vel[3 * j + c] * d[c] / r;
            }
            for (int64_t o = o_now; o >= 0 && o > o_now - s->n_os; --o) {
                const int64_t lag = s->step - (s->vacf_burnin + o * s->vacf_stride);
                if (lag < 0 || lag >= s->vacf_len) continue;
                const double* v0 = s->vorig + (size_t)(o % s->n_os) * n3;
                double vi0 = 0.0, vj0 = 0.0;
                for (int c = 0; c < 3; ++c) {
                    vi0 += v0[3 * i + c] * d[c] / r;
                    vj0 += v0[3 * j + c] * d[c] / r;
                }
                const size_t at = (size_t)lag * s->pc_nbins + b;
                const double ta = vit * vi0 + vjt * vj0, tc = vit * vj0 + vjt * vi0;
                s->pc_a[at] += OR_PLANT == 9 ? tc : ta;
                s->pc_c[at] += OR_PLANT == 9 ? ta : tc;
                s->pc_n[at] += 1;
            }
        }
    }
}

int or_set_paircorr(or_sys* s, int nbins, double rmax)
{
    if (s->vacf_len <= 0 || nbins < 1 || !(rmax > 0) || rmax > s->rc) return -1;
    free(s->pc_a); free(s->pc_c); free(s->pc_n);
    const size_t cnt = (size_t)s->vacf_len * nbins;
    s->pc_nbins = nbins;
    s->pc_rmax = rmax;
    s->pc_a = zalloc(cnt);
    s->pc_c = zalloc(cnt);
    s->pc_n = (int64_t*)calloc(cnt, sizeof(int64_t));
    return 0;
}

/* ca, cc [vacf_len][nbins] (0 where no pair was seen), counts of pair samples. */
void or_get_paircorr(const or_sys* s, double* ca, double* cc, int64_t* counts)
{
    const size_t cnt = (size_t)s->vacf_len * s->pc_nbins;
    for (size_t k = 0; k < cnt; ++k) {
        ca[k] = s->pc_n[k] > 0 ? s->pc_a[k] / (2.0 * (double)s->pc_n[k]) : 0.0;
        cc[k] = s->pc_n[k] > 0 ? s->pc_c[k] / (2.0 * (double)s->pc_n[k]) : 0.0;
        counts[k] = s->pc_n[k];
    }
}

/* One step n -> n+1 of Eq. GLD_integrator:
 *   R_{n+1} = R_n + b dt V_n + b dt^2/(2M) (F^C_n + F^D_n + F^R_n)
 *   V_{n+1} = a V_n + dt/(2M) (a F^C_n + F^C_{n+1}) + b dt/M (F^D_n + F^R_n) */
int or_step(or_sys* s, int64_t nsteps)
{
    if (!s->have_kernels) return -7;
    const int n = s->n;
    const double dt = s->dt, M = s->mass, a = s->a, b = s->b;
    double* vhalf = zalloc((size_t)3 * n);
    for (int64_t it = 0; it < nsteps; ++it) {
        /* neighbours at R_n: the lists built with F^C_n are still current */
        ensure_noise(s, s->step);
        double* dRnew = (double*)dR_at(s, s->step); /* slot of dR_{n-m_max+1}, read below first */
        double* dRtmp = zalloc((size_t)3 * n);
#pragma omp parallel for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            double FD[3], FR[3];
            dissipative_force_i(s, i, s->nl.list + s->nl.start[i], s->nl.start[i + 1] - s->nl.start[i], FD);
            if (s->fr_ovr_on) for (int c = 0; c < 3; ++c) FR[c] = s->fr_ovr[3 * i + c];
            else random_force_i(s, i, FR, 0);
            for (int c = 0; c < 3; ++c) {
                double v = s->vel[3 * i + c];
                double Ft = s->fc[3 * i + c] + FD[c] + FR[c];
                dRtmp[3 * i + c] = (OR_PLANT == 2 ? a : b) * dt * v + b * dt * dt / (2.0 * M) * Ft;
                vhalf[3 * i + c] = a * v + dt / (2.0 * M) * a * s->fc[3 * i + c] + b * dt / M * (FD[c] + FR[c]);
                s->fd[3 * i + c] = FD[c];
                s->fr[3 * i + c] = FR[c];
            }
        }
        for (int i = 0; i < 3 * n; ++i) {
            dRnew[i] = dRtmp[i];
            s->disp[i] += dRtmp[i];
            s->pos[i] = wrap(s->pos[i] + dRtmp[i], s->L);
        }
        free(dRtmp);
        s->fr_ovr_on = 0;
        conservative_forces(s); /* F^C_{n+1} at R_{n+1}; rebuilds the lists */
        for (int i = 0; i < 3 * n; ++i) s->vel[i] = vhalf[i] + dt / (2.0 * M) * s->fc[i];
        s->step++;
        vacf_sample(s);
    }
    free(vhalf);
    return 0;
}

/* The white noise of the window of step n: out[s + m_max - 1][i][c] =
 * W_{i,n+s}, s = -(m_max-1) .. m_max-1 (the counters of or_gauss3). */
void or_white_window(const or_sys* s, int64_t n, double* out)
{
    const int M = s->m_max;
#pragma omp parallel for schedule(static)
    for (int sh = -(M - 1); sh <= M - 1; ++sh)
        for (int i = 0; i < s->n; ++i)
            or_gauss3(s->seed, (uint32_t)i, n + sh, 0u, out + ((size_t)(sh + M - 1) * s->n + i) * 3);
}

/* Uses fr[i][c] as F^R of the next step (one step only). */
void or_set_fr_override(or_sys* s, const double* fr)
{
    if (!s->fr_ovr) s->fr_ovr = zalloc((size_t)3 * s->n);
    memcpy(s->fr_ovr, fr, sizeof(double) * 3 * (size_t)s->n);
    s->fr_ovr_on = 1;
}

/* Forces of the coming step n for a subset of particles (neighbours by
 * brute force), without advancing the state. */
void or_forces_subset(or_sys* s, const int32_t* idx, int count, double* fd, double* fr)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < count; ++k) {
        int i = idx[k];
        int32_t* nb = (int32_t*)malloc(sizeof(int32_t) * 64);
        int64_t cap = 64, nn = 0;
        for (int j = 0; j < s->n; ++j) {
            if (j == i) continue;
            double r2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                double d = min_image(s->pos[3 * i + c] - s->pos[3 * j + c], s->L);
                r2 += d * d;
            }
            if (r2 < s->rc * s->rc) {
                if (nn == cap) { cap *= 2; nb = (int32_t*)realloc(nb, sizeof(int32_t) * cap); }
                nb[nn++] = j;
            }
        }
        dissipative_force_i(s, i, nb, nn, fd + 3 * k);
        random_force_i(s, i, fr + 3 * k, 1);
        free(nb);
    }
}

/* ---- accessors ---------------------------------------------------------- */
enum { OR_POS = 0, OR_VEL = 1, OR_FC = 2, OR_FD = 3, OR_FR = 4, OR_DISP = 5, OR_HIST = 6 };

static double* arr(or_sys* s, int which)
{
    switch (which) {
    case OR_POS: return s->pos;
    case OR_VEL: return s->vel;
    case OR_FC: return s->fc;
    case OR_FD: return s->fd;
    case OR_FR: return s->fr;
    case OR_DISP: return s->disp;
    default: return NULL;
    }
}

/* HIST is exchanged as [m-1][n][3] holding dR_{n-m}, m = 1 .. m_max-1. */
int or_get(or_sys* s, int which, double* out)
{
    size_t n3 = (size_t)3 * s->n;
    if (which == OR_HIST) {
        for (int m = 1; m < s->m_max; ++m) memcpy(out + (m - 1) * n3, dR_at(s, s->step - m), sizeof(double) * n3);
        return 0;
    }
    double* p = arr(s, which);
    if (!p) return -1;
    memcpy(out, p, sizeof(double) * n3);
    return 0;
}

int or_set(or_sys* s, int which, const double* in)
{
    size_t n3 = (size_t)3 * s->n;
    if (which == OR_HIST) {
        for (int m = 1; m < s->m_max; ++m) memcpy((double*)dR_at(s, s->step - m), in + (m - 1) * n3, sizeof(double) * n3);
        return 0;
    }
    double* p = arr(s, which);
    if (!p) return -1;
    memcpy(p, in, sizeof(double) * n3);
    if (which == OR_POS) {
        for (size_t k = 0; k < n3; ++k) p[k] = wrap(p[k], s->L);
        build_neighbors(s->pos, s->n, s->L, s->rc, &s->nl);
    }
    return 0;
}

/* Moves the step counter; the history ring is addressed relative to it, so
 * callers set the step before the history. */
void or_set_step(or_sys* s, int64_t step) { s->step = step; }
int64_t or_get_step(const or_sys* s) { return s->step; }
void or_recompute_fc(or_sys* s) { conservative_forces(s); }

void or_get_coefs(const or_sys* s, double* Kd, double* A, double* C, double* Chat, double* ab, double* clamped)
{
    int M = s->m_max;
    if (Kd) memcpy(Kd, s->Kd, sizeof(double) * M);
    if (A) memcpy(A, s->A, sizeof(double) * (2 * M - 1));
    if (C) memcpy(C, s->C, sizeof(double) * M);
    if (Chat) memcpy(Chat, s->Chat, sizeof(double) * M);
    if (ab) { ab[0] = s->a; ab[1] = s->b; }
    if (clamped) *clamped = s->clamped_mass;
}

/* C(tau) per Cartesian component: <V_x(t0+tau) V_x(t0)>, averaged over
 * particles, components and origins. */
int64_t or_get_vacf(const or_sys* s, double* out)
{
    for (int l = 0; l < s->vacf_len; ++l)
        out[l] = s->ccnt[l] > 0 ? s->csum[l] / (3.0 * s->n * (double)s->ccnt[l]) : 0.0;
    return s->n_origins;
}

void or_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int or_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
