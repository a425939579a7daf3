/*
 * Direct space-time history sum of the MOT-JVIE (Eq. PnMOT), term by term.
 *
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle (see oracle/__init__.py).  Nothing
 * in the product path loads this file; it shares no code with the CUDA library.
 *
 *     P_{n-1}(m) = sum_{l=1}^{min(ell, n-1)} Z_l J_{n-l}  at voxel m,
 *     Z_l(m, s)  = delta_ms (T(l)/eps_m + delta_l) I - chi_m G_l(r_m - r_s)
 *
 * (Eq. Z with the reading S(F) = grad div A - c^-2 d_t^2 A + F; the FIR taps delta_l
 * of Sec. 6.1 add to the identity coefficient; T is the quadratic B-spline on
 * (-dt, 2 dt), so T(0) = T(dt) = 1/2 and T(l dt) = 0 for l >= 2.)
 *
 * Plain loops: for every target voxel, every source voxel and every lag whose element
 * is nonzero at that offset, the 3x3 block times the source's current.  The element
 * table is the oracle's own octant table G[l][c][|dz|][|dy|][|dx|] (components xx, yy,
 * zz, xy, xz, yz); other octants follow from parity (diagonal components even in every
 * d_i, the (a, b) component odd in d_a and in d_b).  Lags where every component at an
 * offset is zero are skipped: they contribute exactly nothing.
 *
 * Layouts: voxel m = u + U (v + V w); J[k][m][b] holds J_{k+1} (J_1 first), b = x, y, z.
 */
#include <stdlib.h>

static double T_at_lag(int l) { return (l == 0 || l == 1) ? 0.5 : 0.0; }

/* first and last lag with a nonzero component, per octant offset (hi < lo: none) */
static void lag_range(int noff, int nlag, const double* G, int* lo, int* hi) {
    for (int o = 0; o < noff; ++o) {
        lo[o] = nlag;
        hi[o] = -1;
        for (int l = 0; l < nlag; ++l) {
            int any = 0;
            for (int c = 0; c < 6; ++c)
                if (G[((long long)l * 6 + c) * noff + o] != 0.0) any = 1;
            if (any) {
                if (l < lo[o]) lo[o] = l;
                hi[o] = l;
            }
        }
    }
}

/*
 * P_{n-1} at the voxels tgt[0..ntgt) from the sources src[0..nsrc) (voxels whose
 * current may be nonzero), for the step n (1-based; J_1 .. J_{n-1} are read).
 *  U, V, W    grid; nlag = ell + 1 lags 0..ell in G
 *  eps        [M] relative permittivities
 *  taps       delta_0 .. delta_{ntaps-1} (may be NULL when ntaps = 0)
 *  P          [ntgt][3] output
 * Returns 0, or -1 if a scratch allocation failed.
 */
int oracle_history(int U, int V, int W, int nlag, const double* G, const double* eps,
                   const double* taps, int ntaps, int nsrc, const int* src, int ntgt,
                   const int* tgt, int n, const double* J, double* P) {
    const int noff = U * V * W;
    const long long M = noff;
    int* lo = (int*)malloc(sizeof(int) * noff);
    int* hi = (int*)malloc(sizeof(int) * noff);
    if (!lo || !hi) {
        free(lo);
        free(hi);
        return -1;
    }
    lag_range(noff, nlag, G, lo, hi);
    const int lmax = (n - 1 < nlag - 1) ? n - 1 : nlag - 1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < ntgt; ++i) {
        const int m = tgt[i];
        const int mu = m % U, mv = (m / U) % V, mw = m / (U * V);
        const double chi = (eps[m] - 1.0) / eps[m];
        double acc[3] = {0.0, 0.0, 0.0};
        /* identity part: (T(l)/eps_m + delta_l) J_{n-l}(m) */
        for (int l = 1; l <= lmax; ++l) {
            const double coef = T_at_lag(l) / eps[m] + (l < ntaps ? taps[l] : 0.0);
            const double* j = J + ((long long)(n - l - 1) * M + m) * 3;
            for (int b = 0; b < 3; ++b) acc[b] += coef * j[b];
        }
        /* interaction part: -chi_m sum_s G_l(r_m - r_s) J_{n-l}(s) */
        double g[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < nsrc; ++k) {
            const int s = src[k];
            const int du = mu - s % U, dv = mv - (s / U) % V, dw = mw - s / (U * V);
            const int o = (abs(dw) * V + abs(dv)) * U + abs(du);
            /* sign(d_i), 0 at d_i = 0: an off-diagonal component vanishes there */
            const double sx = (du > 0) - (du < 0), sy = (dv > 0) - (dv < 0),
                         sz = (dw > 0) - (dw < 0);
            const int l0 = lo[o] > 1 ? lo[o] : 1;
            const int l1 = hi[o] < lmax ? hi[o] : lmax;
            for (int l = l0; l <= l1; ++l) {
                const double* gl = G + (long long)l * 6 * noff + o;
                const double xx = gl[0], yy = gl[noff], zz = gl[2 * noff];
                const double xy = gl[3 * noff] * sx * sy;
                const double xz = gl[4 * noff] * sx * sz;
                const double yz = gl[5 * noff] * sy * sz;
                const double* j = J + ((long long)(n - l - 1) * M + s) * 3;
                g[0] += xx * j[0] + xy * j[1] + xz * j[2];
                g[1] += xy * j[0] + yy * j[1] + yz * j[2];
                g[2] += xz * j[0] + yz * j[1] + zz * j[2];
            }
        }
        for (int b = 0; b < 3; ++b) P[(long long)i * 3 + b] = acc[b] - chi * g[b];
    }
    free(lo);
    free(hi);
    return 0;
}
