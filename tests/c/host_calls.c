/* Plain-C client of the library's host-only entry points (no device needed):
 * checks that include/gld.h is valid C and that a C program links and calls
 * through the ABI.  Prints "ok" and exits 0 on success. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "gld.h"

int main(void)
{
    /* a rank-two table: f_a(r) g_a(m) + f_b(r) g_b(m) */
    enum { NR = 6, M = 9 };
    double table[NR * M], f[2 * NR], g[2 * M], trunc = -1.0;
    for (int k = 0; k < NR; ++k)
        for (int m = 0; m < M; ++m)
            table[k * M + m] = (1.0 + k) * exp(-0.3 * m) + 0.5 * sin(0.7 * k) * cos(0.4 * m);
    if (gld_separable_terms(table, NR, M, 2, f, g, &trunc) != GLD_OK) return 1;
    double err = 0.0;
    for (int k = 0; k < NR; ++k)
        for (int m = 0; m < M; ++m) {
            const double v = f[k] * g[m] + f[NR + k] * g[M + m];
            err = fmax(err, fabs(v - table[k * M + m]));
        }
    if (!(err < 1e-10 && trunc < 1e-6)) {
        printf("separable terms: err %g trunc %g\n", err, trunc);
        return 2;
    }
    if (gld_separable_terms(table, NR, M, 0, f, g, &trunc) != GLD_E_INVAL) return 3;
    /* pair-noise filters: white self kernel (only K_0), no pair term: the
     * degree-0 taps are sqrt(2 kT K_0 / dt) at s = 0 and zero elsewhere */
    double ks[4] = {0.5, 0.0, 0.0, 0.0}, gp[4] = {0.0, 0.0, 0.0, 0.0}, taps[2 * 7], cheb = -1.0;
    if (gld_pair_noise_filters(ks, gp, 4, 1.0, 0.01, 1.0, 1, 0, taps, &cheb) != GLD_OK) return 4;
    const double a0 = sqrt(2.0 * 1.0 * 0.5 / 0.01);
    for (int s = 0; s < 7; ++s) {
        const double want = s == 3 ? a0 : 0.0;
        if (fabs(taps[s] - want) > 1e-12 * a0 || fabs(taps[7 + s]) > 1e-12 * a0) {
            printf("filters: tap %d = %g %g\n", s, taps[s], taps[7 + s]);
            return 5;
        }
    }
    printf("ok\n");
    return 0;
}
