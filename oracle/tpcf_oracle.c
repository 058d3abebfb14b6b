/*
 * Plain FP64 CPU oracle of the anisotropic 3PCF estimator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke() and the
 * benchmark's CPU-baseline / reference leg may load this library.  It shares no
 * code, header, table or constant with the CUDA path.
 *
 * What it computes, in the paper's order (Sec. 4.2, "3PCF estimator"):
 *   - a linked-list cell partition of the catalogue and a pair cut at r_max
 *     (Sec. 4.1 describes the linked list used for the pair counts);
 *   - for every primary x_i and every secondary j in radial bin b
 *     (step function phi of Eq. alm):
 *         a_l^m[b](x_i) = sum_j w_j Y_l^m(r_hat_ij),   Y orthonormal (Eq. alm),
 *     for all l <= l_max and m = -l..l, with the line of sight fixed along z
 *     (Sec. 4.1), or, with los_mode 1, along the direction from an observer to
 *     the primary (a varying line of sight, the survey generalisation);
 *   - the local product of Eq. measured_mult, kept for m = m' (common LOS),
 *     with the second coefficient conjugated, summed over primaries with the
 *     primary weight (average over x, Sec. 4.2):
 *         NNN^m_{l1 l2}[b1][b2] = sum_i w_i ( a_{l1}^m[b1] conj(a_{l2}^m[b2])
 *                                   - delta_{b1 b2} sum_j w_j^2 Y_{l1}^m conj(Y_{l2}^m) ),
 *     the subtracted term removing the degenerate j = k "triangles";
 *   - integer pair counts and integer triplet counts
 *         T[b1][b2] = sum_i n_{b1}(i) (n_{b2}(i) - delta_{b1 b2}).
 *   The TripoSH projection (Eq. slep2sugy) and the normaliser are done by the
 *   Python side of the oracle (oracle/oracle.py) with wigner3j() below.
 *
 * Conventions (readings of points the paper leaves open):
 *   - positions are uint32 fixed point (one unit = L / 2^32); the separation is
 *     the exact integer difference (minimum image modulo 2^32 in periodic
 *     boxes) and r^2 is an exact unsigned 64-bit integer;
 *   - bin edges r_b = r_min + ((r_max - r_min) * b) / n_b in FP64, the
 *     fixed-point edge s_b = (r_b * 2^32) / L in FP64, and the exact integer
 *     edge E_b = ceil(s_b^2); a pair is in bin b iff E_b <= r^2 < E_{b+1}
 *     (half-open bins);
 *   - in periodic mode with analytic randoms, a_0^0[b] is offset by the
 *     expected monopole of the other points, c_b = (W - 1) / L^3 * V_b * Y_0^0.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORA_PI 3.14159265358979323846

/* ------------------------------------------------------------------ edges */

/* Exact ceil(s^2) for a finite double s >= 0, using s = mant * 2^e. */
static uint64_t ceil_square(double s)
{
    if (!(s > 0.0)) return 0;
    int e;
    double fr = frexp(s, &e);                       /* s = fr * 2^e, fr in [0.5, 1) */
    uint64_t mant = (uint64_t)ldexp(fr, 53);        /* exact: fr has 53 bits */
    e -= 53;                                        /* s = mant * 2^e */
    unsigned __int128 m2 = (unsigned __int128)mant * mant;   /* s^2 = m2 * 2^(2e) */
    int sh = -2 * e;
    if (sh <= 0) return (uint64_t)(m2 << (-sh));
    if (sh >= 127) return 1;                        /* 0 < s^2 < 1 */
    unsigned __int128 one = 1;
    unsigned __int128 q = m2 >> sh;
    if (m2 & ((one << sh) - 1)) q += 1;
    return (uint64_t)q;
}

void ora_edges(double r_min, double r_max, int n_bins, double box, uint64_t *E, double *r_edges)
{
    for (int b = 0; b <= n_bins; ++b) {
        double r = r_min + ((r_max - r_min) * (double)b) / (double)n_bins;
        double s = (r * 4294967296.0) / box;
        E[b] = ceil_square(s);
        if (r_edges) r_edges[b] = r;
    }
}

/* ---------------------------------------------------------- 3j (Racah) */

static double fact(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

/* Wigner 3j symbol (j1 j2 j3; m1 m2 m3) for integer arguments, Racah's formula. */
double ora_wigner3j(int j1, int j2, int j3, int m1, int m2, int m3)
{
    if (m1 + m2 + m3 != 0) return 0.0;
    if (j1 < 0 || j2 < 0 || j3 < 0) return 0.0;
    if (j3 < abs(j1 - j2) || j3 > j1 + j2) return 0.0;
    if (abs(m1) > j1 || abs(m2) > j2 || abs(m3) > j3) return 0.0;
    double tri = fact(j1 + j2 - j3) * fact(j1 - j2 + j3) * fact(-j1 + j2 + j3) / fact(j1 + j2 + j3 + 1);
    double pre = sqrt(tri * fact(j1 + m1) * fact(j1 - m1) * fact(j2 + m2) * fact(j2 - m2)
                      * fact(j3 + m3) * fact(j3 - m3));
    int kmin = 0;
    if (j2 - j3 - m1 > kmin) kmin = j2 - j3 - m1;
    if (j1 - j3 + m2 > kmin) kmin = j1 - j3 + m2;
    int kmax = j1 + j2 - j3;
    if (j1 - m1 < kmax) kmax = j1 - m1;
    if (j2 + m2 < kmax) kmax = j2 + m2;
    double sum = 0.0;
    for (int k = kmin; k <= kmax; ++k) {
        double den = fact(k) * fact(j3 - j2 + k + m1) * fact(j3 - j1 + k - m2)
                   * fact(j1 + j2 - j3 - k) * fact(j1 - k - m1) * fact(j2 - k + m2);
        sum += ((k & 1) ? -1.0 : 1.0) / den;
    }
    int ph = j1 - j2 - m3;
    double sign = (ph % 2 == 0) ? 1.0 : -1.0;
    return sign * pre * sum;
}

/* ------------------------------------------------- spherical harmonics */

/* Orthonormal complex Y_l^m(theta, phi) for all l <= lmax, m = -l..l, stored
 * at index l*l + l + m.  P_l^m carries the Condon-Shortley phase and comes from
 * the standard associated-Legendre recurrences; negative m use
 * Y_l^{-m} = (-1)^m conj(Y_l^m). */
void ora_ylm(double x, double y, double z, int lmax, cplx *Y)
{
    double ct = z;
    if (ct > 1.0) ct = 1.0;
    if (ct < -1.0) ct = -1.0;
    double theta = acos(ct);
    double phi = atan2(y, x);
    double cth = cos(theta), sth = sin(theta);
    double P[16][16];
    for (int m = 0; m <= lmax; ++m) {
        /* P_m^m = (-1)^m (2m-1)!! sin^m(theta) */
        double pmm = 1.0;
        for (int i = 1; i <= m; ++i) pmm *= -(2.0 * i - 1.0) * sth;
        P[m][m] = pmm;
        if (m + 1 <= lmax) P[m + 1][m] = cth * (2.0 * m + 1.0) * pmm;
        for (int l = m + 2; l <= lmax; ++l)
            P[l][m] = (cth * (2.0 * l - 1.0) * P[l - 1][m] - (double)(l + m - 1) * P[l - 2][m]) / (double)(l - m);
    }
    for (int l = 0; l <= lmax; ++l) {
        for (int m = 0; m <= l; ++m) {
            double nrm = sqrt((2.0 * l + 1.0) / (4.0 * ORA_PI) * fact(l - m) / fact(l + m));
            cplx v = nrm * P[l][m] * cexp(I * (double)m * phi);
            Y[l * l + l + m] = v;
            if (m > 0) Y[l * l + l - m] = ((m & 1) ? -1.0 : 1.0) * conj(v);
        }
    }
}

/* ------------------------------------------------------------ estimator */

typedef struct {
    double r_min, r_max;
    int32_t n_bins, l_max;
    int32_t periodic;
    int32_t remove_self;
    double box;
    double offset_weight;   /* periodic analytic randoms: W of the catalogue; < 0: no offset */
    int32_t los_mode;       /* 0: line of sight z for every primary; 1: from the observer */
    double observer[3];     /* observer position in fixed-point units (los_mode 1) */
} ora_cfg;

static int cell_of(uint32_t u, int nc) { return (int)(((uint64_t)u * (uint64_t)nc) >> 32); }

/* The field's points act both as primaries (those listed in prim, or all) and
 * as secondaries.  Outputs (all accumulated with +=, caller zeroes them):
 *   nnn_re/nnn_im [2L+1][L+1][L+1][nb][nb]   (m index m + l_max, L = l_max)
 *   pair_counts [nb], trip_counts [nb][nb]
 *   alm_re/alm_im [n_prim][nb][(L+1)^2] and cnt [n_prim][nb] per listed primary (optional).
 * Returns 0 on success, -1 on bad arguments. */
int ora_run(const ora_cfg *c, const uint32_t *xyz, const double *w, int64_t n,
            const int64_t *prim, int64_t n_prim,
            double *nnn_re, double *nnn_im, int64_t *pair_counts, int64_t *trip_counts,
            double *alm_re, double *alm_im, int32_t *cnt_out, int nthreads)
{
    const int nb = c->n_bins, L = c->l_max;
    if (nb < 1 || L < 0 || L > 12 || n < 0 || !(c->r_max > c->r_min) || !(c->r_min > 0.0)
        || !(2.0 * c->r_max < c->box)) return -1;
    const int nlm = (L + 1) * (L + 1);
    const int nm = 2 * L + 1;
    uint64_t E[257];
    double redge[257];
    if (nb > 256) return -1;
    ora_edges(c->r_min, c->r_max, nb, c->box, E, redge);

    /* periodic analytic offset c_b = (W - 1)/L^3 * V_b * Y_0^0 */
    double *cb = (double *)calloc((size_t)nb, sizeof(double));
    if (c->offset_weight >= 0.0) {
        double nbar = (c->offset_weight - 1.0) / (c->box * c->box * c->box);
        for (int b = 0; b < nb; ++b) {
            double vb = 4.0 * ORA_PI / 3.0 * (pow(redge[b + 1], 3) - pow(redge[b], 3));
            cb[b] = nbar * vb / sqrt(4.0 * ORA_PI);
        }
    }

    /* linked-list cells of side >= r_max */
    int nc = (int)floor(c->box / c->r_max);
    if (nc < 1) nc = 1;
    int64_t ncell = (int64_t)nc * nc * nc;
    int64_t *head = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));
    int64_t *next = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t q = 0; q < ncell; ++q) head[q] = -1;
    for (int64_t j = n - 1; j >= 0; --j) {
        int64_t q = ((int64_t)cell_of(xyz[3 * j + 2], nc) * nc + cell_of(xyz[3 * j + 1], nc)) * nc
                    + cell_of(xyz[3 * j + 0], nc);
        next[j] = head[q];
        head[q] = j;
    }
    /* distinct neighbour cell offsets along one axis */
    int offs[3], noff = 0;
    for (int d = -1; d <= 1; ++d) {
        if (c->periodic) {
            int dup = 0;
            for (int k = 0; k < noff; ++k)
                if (((offs[k] % nc) + nc) % nc == ((d % nc) + nc) % nc) dup = 1;
            if (dup) continue;
        }
        offs[noff++] = d;
    }

    const size_t nnn_sz = (size_t)nm * (L + 1) * (L + 1) * nb * nb;
    int nthr = 1;
#ifdef _OPENMP
    if (nthreads > 0) nthr = nthreads; else nthr = omp_get_max_threads();
#endif
    cplx *part = (cplx *)calloc((size_t)nthr * nnn_sz, sizeof(cplx));
    int64_t *ppart = (int64_t *)calloc((size_t)nthr * nb, sizeof(int64_t));
    int64_t *tpart = (int64_t *)calloc((size_t)nthr * nb * nb, sizeof(int64_t));
    const int64_t np = prim ? n_prim : n;

#pragma omp parallel num_threads(nthr)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        cplx *acc = part + (size_t)tid * nnn_sz;
        int64_t *pc = ppart + (size_t)tid * nb;
        int64_t *tc = tpart + (size_t)tid * nb * nb;
        cplx *a = (cplx *)malloc((size_t)nb * nlm * sizeof(cplx));
        /* self[b][l1][l2][m + L] = sum_j w_j^2 Y_{l1}^m conj(Y_{l2}^m) */
        cplx *self = (cplx *)malloc((size_t)nb * (L + 1) * (L + 1) * nm * sizeof(cplx));
        int64_t *cnt = (int64_t *)malloc((size_t)nb * sizeof(int64_t));
        cplx Y[169];

#pragma omp for schedule(static)
        for (int64_t ip = 0; ip < np; ++ip) {
            const int64_t i = prim ? prim[ip] : ip;
            memset(a, 0, (size_t)nb * nlm * sizeof(cplx));
            memset(self, 0, (size_t)nb * (L + 1) * (L + 1) * nm * sizeof(cplx));
            memset(cnt, 0, (size_t)nb * sizeof(int64_t));
            const uint32_t ux = xyz[3 * i], uy = xyz[3 * i + 1], uz = xyz[3 * i + 2];
            const int cx = cell_of(ux, nc), cy = cell_of(uy, nc), cz = cell_of(uz, nc);
            /* varying line of sight: n_i = (x_i - observer) / |x_i - observer| at polar
             * angle th and azimuth ph; separations are turned by R_y(-th) R_z(-ph),
             * which takes n_i to z, before their harmonics are taken */
            double cth = 1.0, sth = 0.0, cph = 1.0, sph = 0.0;
            if (c->los_mode == 1) {
                const double nx = (double)ux - c->observer[0], ny = (double)uy - c->observer[1],
                             nz = (double)uz - c->observer[2];
                const double nr = sqrt(nx * nx + ny * ny + nz * nz);
                if (nr > 0.0) {   /* a primary at the observer keeps z */
                    const double th = acos(nz / nr), ph = atan2(ny, nx);
                    cth = cos(th); sth = sin(th); cph = cos(ph); sph = sin(ph);
                }
            }
            for (int oz = 0; oz < noff; ++oz)
            for (int oy = 0; oy < noff; ++oy)
            for (int ox = 0; ox < noff; ++ox) {
                int qx = cx + offs[ox], qy = cy + offs[oy], qz = cz + offs[oz];
                if (c->periodic) {
                    qx = (qx % nc + nc) % nc; qy = (qy % nc + nc) % nc; qz = (qz % nc + nc) % nc;
                } else if (qx < 0 || qy < 0 || qz < 0 || qx >= nc || qy >= nc || qz >= nc) {
                    continue;
                }
                for (int64_t j = head[((int64_t)qz * nc + qy) * nc + qx]; j >= 0; j = next[j]) {
                    if (j == i) continue;
                    int64_t dx, dy, dz;
                    if (c->periodic) {
                        dx = (int32_t)(xyz[3 * j] - ux);
                        dy = (int32_t)(xyz[3 * j + 1] - uy);
                        dz = (int32_t)(xyz[3 * j + 2] - uz);
                    } else {
                        dx = (int64_t)xyz[3 * j] - (int64_t)ux;
                        dy = (int64_t)xyz[3 * j + 1] - (int64_t)uy;
                        dz = (int64_t)xyz[3 * j + 2] - (int64_t)uz;
                    }
                    /* r_max < L/2, so an axis separation of 2^31 units or more is
                     * out of range; this also keeps every square below 2^62. */
                    if (llabs(dx) >= 2147483648LL || llabs(dy) >= 2147483648LL || llabs(dz) >= 2147483648LL)
                        continue;
                    uint64_t r2 = (uint64_t)(dx * dx) + (uint64_t)(dy * dy) + (uint64_t)(dz * dz);
                    if (r2 < E[0] || r2 >= E[nb]) continue;
                    int b = 0;
                    while (b + 1 < nb && r2 >= E[b + 1]) ++b;
                    double r = sqrt((double)dx * dx + (double)dy * dy + (double)dz * dz);
                    double vx = (double)dx / r, vy = (double)dy / r, vz = (double)dz / r;
                    if (c->los_mode == 1) {
                        const double x1 = cph * vx + sph * vy, y1 = -sph * vx + cph * vy;
                        vx = cth * x1 - sth * vz;
                        vz = sth * x1 + cth * vz;
                        vy = y1;
                    }
                    ora_ylm(vx, vy, vz, L, Y);
                    const double wj = w[j];
                    cplx *ab = a + (size_t)b * nlm;
                    for (int k = 0; k < nlm; ++k) ab[k] += wj * Y[k];
                    cplx *sb = self + (size_t)b * (L + 1) * (L + 1) * nm;
                    for (int l1 = 0; l1 <= L; ++l1)
                    for (int l2 = 0; l2 <= L; ++l2) {
                        int mm = l1 < l2 ? l1 : l2;
                        for (int m = -mm; m <= mm; ++m)
                            sb[((size_t)l1 * (L + 1) + l2) * nm + m + L] +=
                                wj * wj * Y[l1 * l1 + l1 + m] * conj(Y[l2 * l2 + l2 + m]);
                    }
                    cnt[b] += 1;
                }
            }
            if (c->offset_weight >= 0.0)
                for (int b = 0; b < nb; ++b) a[(size_t)b * nlm] -= cb[b];

            const double wi = w[i];
            for (int m = -L; m <= L; ++m) {
                int am = abs(m);
                for (int l1 = am; l1 <= L; ++l1)
                for (int l2 = am; l2 <= L; ++l2)
                for (int b1 = 0; b1 < nb; ++b1)
                for (int b2 = 0; b2 < nb; ++b2) {
                    cplx v = a[(size_t)b1 * nlm + l1 * l1 + l1 + m] * conj(a[(size_t)b2 * nlm + l2 * l2 + l2 + m]);
                    if (b1 == b2 && c->remove_self)
                        v -= self[(((size_t)b1 * (L + 1) + l1) * (L + 1) + l2) * nm + m + L];
                    acc[((((size_t)(m + L) * (L + 1) + l1) * (L + 1) + l2) * nb + b1) * nb + b2] += wi * v;
                }
            }
            for (int b1 = 0; b1 < nb; ++b1) {
                pc[b1] += cnt[b1];
                for (int b2 = 0; b2 < nb; ++b2)
                    tc[b1 * nb + b2] += cnt[b1] * (cnt[b2] - (b1 == b2 ? 1 : 0));
            }
            if (alm_re) {
                for (int b = 0; b < nb; ++b)
                    for (int k = 0; k < nlm; ++k) {
                        alm_re[((size_t)ip * nb + b) * nlm + k] = creal(a[(size_t)b * nlm + k]);
                        alm_im[((size_t)ip * nb + b) * nlm + k] = cimag(a[(size_t)b * nlm + k]);
                    }
            }
            if (cnt_out)
                for (int b = 0; b < nb; ++b) cnt_out[(size_t)ip * nb + b] = (int32_t)cnt[b];
        }
        free(a);
        free(self);
        free(cnt);
    }
    /* fixed-order reduction over threads; with the static schedule every thread
     * sums a fixed contiguous block of primaries in order, so for a given thread
     * count the FP64 result is the same from run to run */
    for (int t = 0; t < nthr; ++t) {
        const cplx *p = part + (size_t)t * nnn_sz;
        for (size_t k = 0; k < nnn_sz; ++k) {
            nnn_re[k] += creal(p[k]);
            nnn_im[k] += cimag(p[k]);
        }
        for (int b = 0; b < nb; ++b) pair_counts[b] += ppart[(size_t)t * nb + b];
        for (int b = 0; b < nb * nb; ++b) trip_counts[b] += tpart[(size_t)t * nb * nb + b];
    }
    free(part); free(ppart); free(tpart);
    free(head); free(next); free(cb);
    return 0;
}

int ora_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
