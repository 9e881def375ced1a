/*
 * FP64 CPU reference for plane-wave receive beamforming.
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg are the only callers.  The product library
 * never links, loads or calls this file, and this file uses nothing of the
 * product library: no header, no table, no helper is shared.
 *
 * What it computes (per pixel p = (x_p, z_p), plane-wave angle theta,
 * receive element i at (x_i, 0); all in double precision):
 *
 *   Receive delay, Eq. (1) of the paper (Sec. II-B-1).  The printed delay is
 *   the monostatic round trip 2*fs/c*|r_i - r_p|; for a plane-wave transmit
 *   the transmit leg is the wavefront's travel time to the pixel, so the
 *   fractional sample index is
 *       n = (x_p sin(theta) + z_p cos(theta) + sqrt((x_p - x_i)^2 + z_p^2)) * (fs / c)
 *   with t = 0 when the wavefront crosses the array centre.
 *
 *   Interpolation: k = floor(n), alpha = n - k,
 *       v = (1 - alpha) u_i[k] + alpha u_i[k + 1]   if 0 <= k <= Ns - 2, else 0.
 *
 *   Apodization (Eq. (1)'s w_i[p]): boxcar of F-number F, channel i is
 *   active iff |x_p - x_i| <= z_p / (2 F)  (w = 1 inside, 0 outside).
 *
 *   Combiners, per angle over active channels:
 *     DAS (Eq. (1)):     S1 = sum v
 *     DMAS (signed square root, pairwise products):
 *                        s_i = sign(v) sqrt|v|,  T1 = sum s,  T2 = sum s^2,
 *                        y = (T1^2 - T2) / 2   (= sum_{i<j} s_i s_j)
 *     coherence factor:  Su2 = sum v^2, M = number of active channels
 *   Compounding over angles:
 *     DAS  = sum_theta S1
 *     DMAS = sum_theta y
 *     CF   = (DAS^2 / (M_tot * sum_theta Su2)) * DAS   (0 if the denominator is 0)
 *
 *   pDAS (Eq. (2)-(3), Sec. II-B-2; oracle_beamform_pdas): per angle the
 *   p-th root of every active delayed sample keeps its sign, the roots are
 *   summed and the sum is raised to the p-th power, again keeping its sign:
 *       yt = sum sign(v) |v|^(1/p),   y = sign(yt) |yt|^p,
 *   compounded coherently over angles like DMAS: pDAS = sum_theta y.
 *
 *   IQ-DAS and BB-DMAS (Sec. II-B-1, Eq. (4); oracle_beamform_iq): the
 *   channel records come in as complex baseband IQ_i[k] (demodulated by the
 *   caller).  The delayed baseband sample is interpolated linearly like the
 *   RF one, IQ(n) = (1 - alpha) IQ[k] + alpha IQ[k + 1] (0 outside the record),
 *   and the carrier phase of the delay is restored:
 *       s_i = IQ(n) exp(+j 2 pi f0 n / fs).
 *   IQ-DAS:  Y = sum_theta sum_active s_i, image |Y|.
 *   BB-DMAS: s^_i = sqrt|s_i| exp(j arg s_i) (0 for s_i = 0); per angle
 *            y = ((1/M) sum_active s^_i)^2 with M the channels inside the
 *            aperture; Y = sum_theta y, image |Y|.
 *
 * The floating-point expressions above are evaluated exactly as written (no
 * contraction into fused multiply-adds: built with -ffp-contract=off), so
 * every discrete decision (aperture membership, record bounds) is the
 * double-precision decision of those expressions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <omp.h>

/* Inclusive linspace [lo, hi] of n points, element j (n == 1 gives lo). */
static double grid_coord(double lo, double hi, int32_t n, int32_t j)
{
    if (n == 1)
        return lo;
    return lo + (double)j * ((hi - lo) / (double)(n - 1));
}

/* Delay + linear interpolation of one channel for one pixel and one angle.
 * Returns 1 when the channel is inside the F-number aperture (whatever the
 * record bounds), 0 otherwise.  *v receives the interpolated sample, 0 when
 * the channel is inactive or the delay falls outside the record.  *inrec
 * tells whether 0 <= floor(n) <= Ns - 2. */
static int channel_sample(const int16_t *u, int32_t ns, double xp, double zp, double xi,
                          double st, double ct, double kappa, double fnum, double *v,
                          int *inrec)
{
    *v = 0.0;
    *inrec = 0;
    if (!(fabs(xp - xi) <= zp / (2.0 * fnum)))
        return 0;
    double tx = xp * st + zp * ct;
    double dx = xp - xi;
    double rx = sqrt(dx * dx + zp * zp);
    double n = (tx + rx) * kappa;
    double k = floor(n);
    if (k >= 0.0 && k <= (double)(ns - 2)) {
        long kk = (long)k;
        double alpha = n - k;
        *v = (1.0 - alpha) * (double)u[kk] + alpha * (double)u[kk + 1];
        *inrec = 1;
    }
    return 1;
}

static double signed_sqrt(double v)
{
    if (v > 0.0)
        return sqrt(v);
    if (v < 0.0)
        return -sqrt(-v);
    return 0.0;
}

/* Per-channel delayed samples of one pixel: v[a*N + i], aperture flag and
 * record flag per (angle, channel).  Used by the tests that check the
 * combiners against brute force. */
int oracle_delayed_samples(const int16_t *rf, int32_t na, int32_t ne, int32_t ns,
                           const double *x_elem, const double *theta, int32_t nx, int32_t nz,
                           double x0, double x1, double z0, double z1, int32_t ix, int32_t iz,
                           double fs, double c, double fnum, double *v, uint8_t *active,
                           uint8_t *inrec)
{
    if (ix < 0 || ix >= nx || iz < 0 || iz >= nz)
        return -1;
    double xp = grid_coord(x0, x1, nx, ix);
    double zp = grid_coord(z0, z1, nz, iz);
    double kappa = fs / c;
    for (int32_t a = 0; a < na; ++a) {
        double st = sin(theta[a]), ct = cos(theta[a]);
        for (int32_t i = 0; i < ne; ++i) {
            const int16_t *u = rf + ((size_t)a * ne + i) * (size_t)ns;
            int rec;
            active[a * ne + i] = (uint8_t)channel_sample(u, ns, xp, zp, x_elem[i], st, ct, kappa,
                                                         fnum, &v[a * ne + i], &rec);
            inrec[a * ne + i] = (uint8_t)rec;
        }
    }
    return 0;
}

/* One pixel through all angles and channels. */
static void beamform_pixel(const int16_t *rf, int32_t na, int32_t ne, int32_t ns,
                           const double *x_elem, const double *st, const double *ct, double xp,
                           double zp, double kappa, double fnum, double *das, double *dmas,
                           double *cf, int32_t *m_tot)
{
    double s1_tot = 0.0, su2_tot = 0.0, y_dmas = 0.0;
    int32_t m = 0;
    for (int32_t a = 0; a < na; ++a) {
        double s1 = 0.0, t1 = 0.0, t2 = 0.0;
        for (int32_t i = 0; i < ne; ++i) {
            const int16_t *u = rf + ((size_t)a * ne + i) * (size_t)ns;
            double v;
            int rec;
            if (!channel_sample(u, ns, xp, zp, x_elem[i], st[a], ct[a], kappa, fnum, &v, &rec))
                continue;
            m += 1;
            double s = signed_sqrt(v);
            s1 += v;
            t1 += s;
            t2 += s * s;
            su2_tot += v * v;
        }
        s1_tot += s1;
        y_dmas += 0.5 * (t1 * t1 - t2);
    }
    double den = (double)m * su2_tot;
    *das = s1_tot;
    *dmas = y_dmas;
    *cf = den > 0.0 ? (s1_tot * s1_tot / den) * s1_tot : 0.0;
    *m_tot = m;
}

/* Beamform a list of pixels (linear index ix * nz + iz), or the whole grid
 * when pix == NULL (outputs are then [nx][nz], z fastest).  Any output
 * pointer may be NULL.  threads <= 0 uses the OpenMP default. */
int oracle_beamform(const int16_t *rf, int32_t na, int32_t ne, int32_t ns, const double *x_elem,
                    const double *theta, int32_t nx, int32_t nz, double x0, double x1, double z0,
                    double z1, double fs, double c, double fnum, const int64_t *pix, int64_t npix,
                    double *das, double *dmas, double *cf, int32_t *m_tot, int32_t threads)
{
    if (na <= 0 || ne <= 0 || ns < 2 || nx <= 0 || nz <= 0 || fnum <= 0.0)
        return -1;
    double *st = (double *)malloc(sizeof(double) * (size_t)na);
    double *ct = (double *)malloc(sizeof(double) * (size_t)na);
    if (!st || !ct) {
        free(st);
        free(ct);
        return -2;
    }
    for (int32_t a = 0; a < na; ++a) {
        st[a] = sin(theta[a]);
        ct[a] = cos(theta[a]);
    }
    double kappa = fs / c;
    int64_t total = pix ? npix : (int64_t)nx * nz;
    int nt = threads > 0 ? threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
    for (int64_t q = 0; q < total; ++q) {
        int64_t lin = pix ? pix[q] : q;
        int32_t ix = (int32_t)(lin / nz), iz = (int32_t)(lin % nz);
        double xp = grid_coord(x0, x1, nx, ix);
        double zp = grid_coord(z0, z1, nz, iz);
        double d, m2, f;
        int32_t m;
        beamform_pixel(rf, na, ne, ns, x_elem, st, ct, xp, zp, kappa, fnum, &d, &m2, &f, &m);
        if (das)
            das[q] = d;
        if (dmas)
            dmas[q] = m2;
        if (cf)
            cf[q] = f;
        if (m_tot)
            m_tot[q] = m;
    }
    free(st);
    free(ct);
    return 0;
}

/* sign(v) |v|^e with sign(0) = 0. */
static double signed_pow(double v, double e)
{
    if (v > 0.0)
        return pow(v, e);
    if (v < 0.0)
        return -pow(-v, e);
    return 0.0;
}

/* pDAS image (Eq. (2)-(3)) of a pixel list or the whole grid, p >= 1. */
int oracle_beamform_pdas(const int16_t *rf, int32_t na, int32_t ne, int32_t ns,
                         const double *x_elem, const double *theta, int32_t nx, int32_t nz,
                         double x0, double x1, double z0, double z1, double fs, double c,
                         double fnum, double p, const int64_t *pix, int64_t npix, double *out,
                         int32_t threads)
{
    if (na <= 0 || ne <= 0 || ns < 2 || nx <= 0 || nz <= 0 || fnum <= 0.0 || !(p >= 1.0))
        return -1;
    double kappa = fs / c;
    int64_t total = pix ? npix : (int64_t)nx * nz;
    int nt = threads > 0 ? threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
    for (int64_t q = 0; q < total; ++q) {
        int64_t lin = pix ? pix[q] : q;
        int32_t ix = (int32_t)(lin / nz), iz = (int32_t)(lin % nz);
        double xp = grid_coord(x0, x1, nx, ix);
        double zp = grid_coord(z0, z1, nz, iz);
        double y = 0.0;
        for (int32_t a = 0; a < na; ++a) {
            double st = sin(theta[a]), ct = cos(theta[a]);
            double yt = 0.0;
            for (int32_t i = 0; i < ne; ++i) {
                const int16_t *u = rf + ((size_t)a * ne + i) * (size_t)ns;
                double v;
                int rec;
                if (channel_sample(u, ns, xp, zp, x_elem[i], st, ct, kappa, fnum, &v, &rec))
                    yt += signed_pow(v, 1.0 / p);
            }
            y += signed_pow(yt, p);
        }
        out[q] = y;
    }
    return 0;
}

/* |IQ-DAS| and |BB-DMAS| images from complex baseband records
 * iq_re / iq_im [A][N][Ns] (either output may be NULL). */
int oracle_beamform_iq(const double *iq_re, const double *iq_im, int32_t na, int32_t ne,
                       int32_t ns, const double *x_elem, const double *theta, int32_t nx,
                       int32_t nz, double x0, double x1, double z0, double z1, double fs, double c,
                       double fnum, double f0, const int64_t *pix, int64_t npix, double *iqdas,
                       double *bbdmas, int32_t threads)
{
    if (na <= 0 || ne <= 0 || ns < 2 || nx <= 0 || nz <= 0 || fnum <= 0.0)
        return -1;
    const double two_pi = 6.283185307179586476925286766559;
    double kappa = fs / c;
    int64_t total = pix ? npix : (int64_t)nx * nz;
    int nt = threads > 0 ? threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
    for (int64_t q = 0; q < total; ++q) {
        int64_t lin = pix ? pix[q] : q;
        int32_t ix = (int32_t)(lin / nz), iz = (int32_t)(lin % nz);
        double xp = grid_coord(x0, x1, nx, ix);
        double zp = grid_coord(z0, z1, nz, iz);
        double y1r = 0.0, y1i = 0.0, y2r = 0.0, y2i = 0.0;
        for (int32_t a = 0; a < na; ++a) {
            double st = sin(theta[a]), ct = cos(theta[a]);
            double tr = 0.0, ti = 0.0;
            int32_t m = 0;
            for (int32_t i = 0; i < ne; ++i) {
                double xi = x_elem[i];
                if (!(fabs(xp - xi) <= zp / (2.0 * fnum)))
                    continue;
                m += 1;
                double tx = xp * st + zp * ct;
                double dx = xp - xi;
                double rx = sqrt(dx * dx + zp * zp);
                double n = (tx + rx) * kappa;
                double k = floor(n);
                if (!(k >= 0.0 && k <= (double)(ns - 2)))
                    continue;
                size_t o = ((size_t)a * ne + i) * (size_t)ns + (size_t)k;
                double alpha = n - k;
                double br = (1.0 - alpha) * iq_re[o] + alpha * iq_re[o + 1];
                double bi = (1.0 - alpha) * iq_im[o] + alpha * iq_im[o + 1];
                double ph = two_pi * f0 * n / fs;
                double cr = cos(ph), ci = sin(ph);
                double sr = br * cr - bi * ci, si = br * ci + bi * cr;
                y1r += sr;
                y1i += si;
                double mag = sqrt(sr * sr + si * si);
                if (mag > 0.0) {
                    double w = 1.0 / sqrt(mag);
                    tr += sr * w;
                    ti += si * w;
                }
            }
            if (m > 0) {
                double ur = tr / (double)m, ui = ti / (double)m;
                y2r += ur * ur - ui * ui;
                y2i += 2.0 * ur * ui;
            }
        }
        if (iqdas)
            iqdas[q] = sqrt(y1r * y1r + y1i * y1i);
        if (bbdmas)
            bbdmas[q] = sqrt(y2r * y2r + y2i * y2i);
    }
    return 0;
}

/* Threads an oracle_beamform call with threads <= 0 uses. */
int32_t oracle_max_threads(void) { return (int32_t)omp_get_max_threads(); }
