// Host-side resident tables of the beamformer, built once per handle (geometry)
// and once per (handle, sample count, angle set, precision) (transmit tables).
//
// Every discrete decision of the method is taken here, in double precision,
// with the expressions include/bf.h defines (this file is compiled with
// -ffp-contract=off so that no multiply-add is fused): which channels are
// inside the F-number aperture of a pixel (Eq. (1)'s w_i[p], read as an
// inclusive boxcar) and which delayed samples fall inside the record.  The
// GPU then only does the per-pixel arithmetic, in FP32.
#include "bf_tables.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <thread>

namespace bfi {

double grid_coord(double lo, double hi, int n, int j)
{
    if (n == 1)
        return lo;
    return lo + (double)j * ((hi - lo) / (double)(n - 1));
}

// Fractional sample index of Eq. (1) with the plane-wave transmit leg.
static inline double sample_index(double xp, double zp, double xi, double st, double ct,
                                  double kappa)
{
    double tx = xp * st + zp * ct;
    double dx = xp - xi;
    double rx = std::sqrt(dx * dx + zp * zp);
    return (tx + rx) * kappa;
}

static inline bool in_aperture(double xp, double zp, double xi, double fnum)
{
    return std::fabs(xp - xi) <= zp / (2.0 * fnum);
}

// First index in [lo, hi] where the monotone (false ... true) predicate holds,
// hi + 1 if nowhere.
template <class P>
static int first_true(int lo, int hi, P pred)
{
    int a = lo, b = hi + 1;
    while (a < b) {
        int m = a + (b - a) / 2;
        if (pred(m))
            b = m;
        else
            a = m + 1;
    }
    return a;
}

template <class F>
static void parallel_for(int n, F fn)
{
    unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    int nt = (int)std::min<unsigned>(hw, (unsigned)std::max(1, n / 16));
    if (nt <= 1) {
        for (int i = 0; i < n; ++i)
            fn(i);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            for (int i = t; i < n; i += nt)
                fn(i);
        });
    for (auto &x : th)
        x.join();
}

void geometry_tables(const GeomHost &g, GeometryHost &out)
{
    const double kappa = g.fs / g.c;
    out.ap_first.assign((size_t)g.nx * g.ne, g.nz);
    out.apcnt.assign((size_t)g.nx * g.nz, 0);
    const int nxp = pad_cols(g.nx);
    out.rowZ.resize(g.nz);
    out.dx2.assign((size_t)g.ne * nxp, 0.0f);
    for (int iz = 0; iz < g.nz; ++iz)
        out.rowZ[iz] = (float)(kappa * grid_coord(g.z0, g.z1, g.nz, iz));
    parallel_for(g.nx, [&](int ix) {
        const double xp = grid_coord(g.x0, g.x1, g.nx, ix);
        std::vector<int> hist(g.nz + 1, 0);
        for (int i = 0; i < g.ne; ++i) {
            const double xi = g.xe[i];
            double d = kappa * (xp - xi);
            out.dx2[(size_t)i * nxp + ix] = std::max((float)(d * d), 1e-30f);  // keeps sqrt off 0
            int t = first_true(0, g.nz - 1, [&](int iz) {
                return in_aperture(xp, grid_coord(g.z0, g.z1, g.nz, iz), xi, g.fnum);
            });
            out.ap_first[(size_t)ix * g.ne + i] = t;
            hist[t] += 1;
        }
        int run = 0;
        for (int iz = 0; iz < g.nz; ++iz) {
            run += hist[iz];
            out.apcnt[(size_t)ix * g.nz + iz] = (uint16_t)run;
        }
    });
}

void angle_tables(const GeomHost &g, const GeometryHost &geo, int ns,
                  const std::vector<double> &angles, int prec, int rows_per_thread,
                  int stage_bytes, PlanHost &out)
{
    const double kappa = g.fs / g.c;
    const int na = (int)angles.size();
    const int nxp = pad_cols(g.nx);
    out.colK.resize((size_t)na * g.nx);
    out.colF.resize((size_t)na * g.nx);
    out.rowK.resize((size_t)na * g.nz);
    out.rowF.resize((size_t)na * g.nz);
    // An empty row range is (-1, -1): row -1 never exists, and the kernel's
    // test (row - first) <= (last - first) in unsigned arithmetic stays exact.
    out.valid.assign((size_t)na * g.ne * nxp * 2, -1);
    double smax = 0.0;
    for (int a = 0; a < na; ++a) {
        const double st = std::sin(angles[a]), ct = std::cos(angles[a]);
        smax = std::max(smax, std::fabs(st));
        for (int ix = 0; ix < g.nx; ++ix) {
            double v = kappa * (grid_coord(g.x0, g.x1, g.nx, ix) * st);
            double k = std::nearbyint(v);
            out.colK[(size_t)a * g.nx + ix] = (int)k;
            out.colF[(size_t)a * g.nx + ix] = (float)(v - k);
        }
        for (int iz = 0; iz < g.nz; ++iz) {
            double v = kappa * (grid_coord(g.z0, g.z1, g.nz, iz) * (1.0 + ct));
            double k = std::nearbyint(v);
            out.rowK[(size_t)a * g.nz + iz] = (int)k;
            out.rowF[(size_t)a * g.nz + iz] = (float)(v - k);
        }
    }
    // Rows of each (angle, column, channel) whose sample counts: inside the
    // aperture and 0 <= floor(n) <= ns - 2.  All three predicates are
    // monotone in the row index (z_p grows with it, n grows with z_p).
    const double kmax = (double)(ns - 2);
    parallel_for(na * g.nx, [&](int t) {
        const int a = t / g.nx, ix = t % g.nx;
        const double st = std::sin(angles[a]), ct = std::cos(angles[a]);
        const double xp = grid_coord(g.x0, g.x1, g.nx, ix);
        auto n_at = [&](int iz, double xi) {
            return sample_index(xp, grid_coord(g.z0, g.z1, g.nz, iz), xi, st, ct, kappa);
        };
        for (int i = 0; i < g.ne; ++i) {
            const double xi = g.xe[i];
            int lo = geo.ap_first[(size_t)ix * g.ne + i];
            int hi = g.nz - 1;
            if (lo <= hi && !(std::floor(n_at(lo, xi)) >= 0.0))
                lo = first_true(lo, hi, [&](int iz) { return std::floor(n_at(iz, xi)) >= 0.0; });
            if (lo <= hi && !(std::floor(n_at(hi, xi)) <= kmax))
                hi = first_true(lo, hi, [&](int iz) { return !(std::floor(n_at(iz, xi)) <= kmax); }) - 1;
            if (lo > hi) {
                lo = -1;
                hi = -1;
            }
            size_t o = (((size_t)a * g.ne + i) * nxp + ix) * 2;
            out.valid[o] = lo;
            out.valid[o + 1] = hi;
        }
    });
    // Window of sample pairs one tile needs per channel, over the pixels that
    // count it: the delay grows by at most (1 + cos) kappa dz <= 2 kappa dz per
    // row and by at most (|sin| + 1 / sqrt(1 + 4 F^2)) kappa dx per column (the
    // transmit leg's slope, plus the receive leg's slope |x_p - x_i| /
    // sqrt((x_p - x_i)^2 + z_p^2) inside the aperture |x_p - x_i| <= z_p / (2 F)).
    // Two counted pixels of a tile are joined by a row-then-column or
    // column-then-row path inside the aperture (the aperture widens with
    // depth), so the spread adds up along it.  The planner checks every window
    // against wmax (an error, never a silent clamp).
    const int align = 16 / pair_bytes(prec);
    const double dz = g.nz > 1 ? (g.z1 - g.z0) / (double)(g.nz - 1) : 0.0;
    const double dx = g.nx > 1 ? (g.x1 - g.x0) / (double)(g.nx - 1) : 0.0;
    const int rows = std::min(tile_rows(rows_per_thread), g.nz) - 1;
    const int cols = std::min(kTileCols, g.nx) - 1;
    const double rx_slope = 1.0 / std::sqrt(1.0 + 4.0 * g.fnum * g.fnum);
    double spread = 2.0 * kappa * dz * rows + (smax + rx_slope) * kappa * dx * cols;
    int span = (int)std::ceil(spread) + 1 + 4 + align;
    // Box widths are whole multiples of 128 bytes, so every shared-memory
    // destination of a tensor copy (channel stride wmax, box offsets) stays
    // 128-byte aligned; start coordinates are 16-byte aligned (align pairs).
    const int box_align = 128 / pair_bytes(prec);
    const int maxbox = max_box_pairs(prec);
    int nb = (span + maxbox - 1) / maxbox;
    int box = (span + nb - 1) / nb;
    box = (box + box_align - 1) / box_align * box_align;
    out.box = box;
    out.wmax = nb * box;
    out.nsp = (ns + kPadL + 7) / 8 * 8;
    out.rows = rows_per_thread;
    out.align = align;
    int grp = stage_bytes / (out.wmax * pair_bytes(prec) + kTileCols * 12);
    // at most 16 channels per stage on 32- and 64-row tiles (three stages: more
    // leaves one CTA per SM), up to kMaxGroup on 16-row tiles (two stages)
    const int cap = rows_per_thread == 2 ? kMaxGroup : 16;
    out.group = std::max(1, std::min(cap, std::min(grp, g.ne)));
}

void bandpass_bins(int nz, double z0, double z1, double c, double f0, int &lo, int &hi)
{
    lo = 1;
    hi = 0;
    if (nz < 2)
        return;
    const double L = (double)nz;
    const double dz = (z1 - z0) / (double)(nz - 1);
    bool found = false;
    for (int k = 1; k <= nz / 2; ++k) {
        double f = (double)k * c / (2.0 * L * dz);
        if (f >= f0 && f <= 3.0 * f0) {
            if (!found) {
                lo = k;
                found = true;
            }
            hi = k;
        }
    }
}

void fk_mapping_tables(int ne, int nt, int nk, double pitch, double dz,
                       const std::vector<double> &sc, bool stolt, std::vector<int> &i0,
                       std::vector<float> &aw)
{
    (void)ne;
    const int na = (int)sc.size() / 2, half = nt / 2;
    const size_t npts = (size_t)half * nk;
    i0.assign((size_t)na * npts, -1);
    aw.assign((size_t)na * npts * 2, 0.0f);
    // lateral bin m in units of temporal bins: X = m_s (nt dz / (nk pitch))
    const double r = (double)nt * dz / ((double)nk * pitch);
    for (int a = 0; a < na; ++a) {
        const double st = sc[2 * a], ct = sc[2 * a + 1];
        const double bet = std::sqrt(1.0 + ct - 0.5 * st * st);  // Stolt: depth scale
        parallel_for(half, [&](int qi) {
            const double Q = (double)(qi + 1);
            for (int m = 0; m < nk; ++m) {
                const double X = (double)(m < nk / 2 ? m : m - nk) * r;
                double pos, w;
                bool ok;
                if (!stolt) {
                    // exact plane-wave mapping k = (Kx^2 + Kz^2) / (2 (Kx sin + Kz cos))
                    const double den = X * st + Q * ct;
                    const double num = X * X + Q * Q;
                    pos = num / den;
                    w = (Q * den - 0.5 * num * ct) / (den * den);
                    ok = den > 0.0 && std::fabs(2.0 * X - pos * st) <= pos && pos >= 0.0 &&
                         pos < (double)half;
                } else {
                    // Stolt's mapping of the exploding reflector at velocity c / bet,
                    // sheared and scaled back onto the native grid
                    const double Qp = (Q - st * X) / bet;
                    const double rad = std::sqrt(X * X + Qp * Qp);
                    pos = (2.0 / bet) * rad;
                    w = Qp / (bet * bet * rad);
                    ok = Qp > 0.0 && pos >= 0.0 && pos < (double)half;
                }
                if (!ok)
                    continue;
                const double fl = std::floor(pos);
                const size_t t = (size_t)a * npts + (size_t)qi * nk + m;
                i0[t] = (int)fl;
                aw[2 * t] = (float)(pos - fl);
                aw[2 * t + 1] = (float)w;
            }
        });
    }
}

static void fft_inplace(std::vector<std::complex<double>> &a)
{
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1)
            j ^= bit;
        j ^= bit;
        if (i < j)
            std::swap(a[i], a[j]);
    }
    const double pi = 3.14159265358979323846;
    for (size_t len = 2; len <= n; len <<= 1) {
        for (size_t i = 0; i < n; i += len)
            for (size_t j = 0; j < len / 2; ++j) {
                double ang = -2.0 * pi * (double)j / (double)len;
                std::complex<double> w(std::cos(ang), std::sin(ang));
                std::complex<double> u = a[i + j], v = a[i + j + len / 2] * w;
                a[i + j] = u + v;
                a[i + j + len / 2] = u - v;
            }
    }
}

void envelope_tables(int nz, EnvHost &out)
{
    const double pi = 3.14159265358979323846;
    out.nz = nz;
    const bool pow2 = (nz & (nz - 1)) == 0;
    int m = 1;
    if (pow2)
        m = nz;
    else
        while (m < 2 * nz - 1)
            m <<= 1;
    out.fft_m = m;
    out.bluestein = pow2 ? 0 : 1;
    out.tw.resize((size_t)m * 2);
    for (int k = 0; k < m; ++k) {
        double ang = -2.0 * pi * (double)k / (double)m;
        out.tw[2 * k] = (float)std::cos(ang);
        out.tw[2 * k + 1] = (float)std::sin(ang);
    }
    out.chirp.clear();
    out.bhat.clear();
    if (!pow2) {
        std::vector<std::complex<double>> w(nz), b(m, 0.0);
        for (int n = 0; n < nz; ++n) {
            long long r = ((long long)n * n) % (2LL * nz);
            double ang = pi * (double)r / (double)nz;
            w[n] = std::complex<double>(std::cos(ang), std::sin(ang));
        }
        for (int n = 0; n < nz; ++n) {
            b[n] = w[n];
            if (n > 0)
                b[m - n] = w[n];
        }
        fft_inplace(b);
        out.chirp.resize(2 * nz);
        out.bhat.resize(2 * m);
        for (int n = 0; n < nz; ++n) {
            out.chirp[2 * n] = (float)w[n].real();
            out.chirp[2 * n + 1] = (float)w[n].imag();
        }
        for (int k = 0; k < m; ++k) {
            out.bhat[2 * k] = (float)b[k].real();
            out.bhat[2 * k + 1] = (float)b[k].imag();
        }
    }
}

}  // namespace bfi
